// C ABI of the learned warm start: a convolutional encoder-decoder that maps
// an observation C to an initial guess X_0 = C + net(C) and log(lambda),
// trained on the GPU by its own forward and backward kernels (k_nn.cu).
//
//   e1 = relu(conv(C; 3 -> c))         e2 = relu(conv_s2(e1; c -> 2c))
//   e3 = relu(conv_s2(e2; 2c -> 4c))   e4 = relu(conv_s2(e3; 4c -> 4c))
//   d3 = relu(conv(up(e4); 4c -> 4c)) + e3
//   d2 = relu(conv(up(d3); 4c -> 2c)) + e2
//   d1 = relu(conv(up(d2); 2c -> c)) + e1
//   X_0 = C + conv(d1; c -> 3),  log(lambda) = w . mean_pixels(e4) + b
//
// 3x3 convolutions, zero padding 1, stride-2 outputs centred on even
// pixels, nearest x2 up-sampling.  Parameters are FP32 masters with a BF16
// copy for the tensor-core products; accumulation is FP32.  The flat
// parameter order is, per layer e1..e4, d3, d2, d1, out: weights
// (c_out, 3, 3, c_in) then biases; then the head's weights and bias.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "nn_internal.cuh"
#include "rtg_internal.cuh"

namespace {

using namespace rtg;

rtg_status nfail(rtg_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  rtg::record_error(buf);
  return st;
}

#define NCK(call)                                                                           \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return nfail(RTG_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
#define NRK(call)                    \
  do {                               \
    rtg_status s_ = (call);          \
    if (s_ != RTG_OK) return s_;     \
  } while (0)

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
  Buf() = default;
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  ~Buf() {
    if (p) cudaFree(p);
  }
  rtg_status ensure(size_t b) {
    if (b <= bytes && p) return RTG_OK;
    if (p) {
      cudaDeviceSynchronize();
      cudaFree(p);
      p = nullptr;
      bytes = 0;
    }
    if (cudaMalloc(&p, b) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return nfail(RTG_ERR_ALLOC, "cudaMalloc(%zu bytes) failed", b);
    }
    bytes = b;
    return RTG_OK;
  }
  template <typename T>
  T* as() const { return static_cast<T*>(p); }
};

struct Layer {
  int cin, cout, stride;
  int64_t w, b;   // offsets in the flat parameter array
};

enum { E1 = 0, E2, E3, E4, D3, D2, D1, OUT, NLAYER };

}  // namespace

struct rtg_warmstart {
  int device = 0;
  int base = 32;
  Layer L[NLAYER];
  int64_t head_w = 0, head_b = 0, nparams = 0;
  Buf P, Pb, G, Mo, Vo;    // FP32 params, BF16 copy, gradients, Adam moments
  int adam_t = 0;
  // activations and their gradients, sized for the last (N, H, W)
  int N = 0, H = 0, W = 0;
  Buf act, grad, col, dA, part, dzf, dzb, z, small;
  float *x0, *e1, *e2, *e3, *e4, *u4, *r3, *d3, *u3, *r2, *d2, *u2, *r1, *d1, *zo, *g, *loglam;
  float *gd1, *gu2, *gd2, *gu3, *gd3, *gu4, *ge4, *ge3, *ge2, *ge1, *gtmp, *dout, *dll;
  double* loss;
};

namespace {

void layout(rtg_warmstart* ws) {
  const int c = ws->base;
  const int cin[NLAYER] = {3, c, 2 * c, 4 * c, 4 * c, 4 * c, 2 * c, c};
  const int cout[NLAYER] = {c, 2 * c, 4 * c, 4 * c, 4 * c, 2 * c, c, 3};
  const int st[NLAYER] = {1, 2, 2, 2, 1, 1, 1, 1};
  int64_t off = 0;
  for (int l = 0; l < NLAYER; ++l) {
    ws->L[l] = Layer{cin[l], cout[l], st[l], off, off + int64_t(cout[l]) * 9 * cin[l]};
    off = ws->L[l].b + cout[l];
  }
  ws->head_w = off;
  ws->head_b = off + 4 * c;
  ws->nparams = off + 4 * c + 1;
}

// Grows the activation / gradient / workspace buffers for (N, H, W).
rtg_status shape_buffers(rtg_warmstart* ws, int N, int H, int W) {
  if (N == ws->N && H == ws->H && W == ws->W) return RTG_OK;
  const int c = ws->base;
  const int64_t p1 = int64_t(N) * H * W, p2 = p1 / 4, p4 = p1 / 16, p8 = p1 / 64;
  // activation sizes in floats (order matters: pointers are carved in this order)
  const int64_t sz[] = {p1 * 3, p1 * c, p2 * 2 * c, p4 * 4 * c, p8 * 4 * c, p4 * 4 * c, p4 * 4 * c, p4 * 4 * c,
                        p2 * 4 * c, p2 * 2 * c, p2 * 2 * c, p1 * 2 * c, p1 * c, p1 * c, p1 * 3,
                        int64_t(N) * 4 * c, int64_t(N)};
  float** ptr[] = {&ws->x0, &ws->e1, &ws->e2, &ws->e3, &ws->e4, &ws->u4, &ws->r3, &ws->d3, &ws->u3, &ws->r2,
                   &ws->d2, &ws->u2, &ws->r1, &ws->d1, &ws->zo, &ws->g, &ws->loglam};
  int64_t tot = 0;
  for (int64_t v : sz) tot += (v + 63) / 64 * 64;
  NRK(ws->act.ensure(size_t(tot) * 4));
  int64_t o = 0;
  for (size_t i = 0; i < sizeof(sz) / sizeof(sz[0]); ++i) {
    *ptr[i] = ws->act.as<float>() + o;
    o += (sz[i] + 63) / 64 * 64;
  }
  const int64_t gs[] = {p1 * c, p1 * 2 * c, p2 * 2 * c, p2 * 4 * c, p4 * 4 * c, p4 * 4 * c, p8 * 4 * c,
                        p4 * 4 * c, p2 * 2 * c, p1 * c, p1 * 2 * c, p1 * 3, int64_t(N)};
  float** gp[] = {&ws->gd1, &ws->gu2, &ws->gd2, &ws->gu3, &ws->gd3, &ws->gu4, &ws->ge4, &ws->ge3, &ws->ge2,
                  &ws->ge1, &ws->gtmp, &ws->dout, &ws->dll};
  tot = 0;
  for (int64_t v : gs) tot += (v + 63) / 64 * 64;
  NRK(ws->grad.ensure(size_t(tot) * 4));
  o = 0;
  for (size_t i = 0; i < sizeof(gs) / sizeof(gs[0]); ++i) {
    *gp[i] = ws->grad.as<float>() + o;
    o += (gs[i] + 63) / 64 * 64;
  }
  // largest im2col (rows x 9 c_in) and GEMM output over the layers
  int64_t mk = 0, mn = 0;
  const int hs[NLAYER] = {H, H / 2, H / 4, H / 8, H / 4, H / 2, H, H};
  const int wsz[NLAYER] = {W, W / 2, W / 4, W / 8, W / 4, W / 2, W, W};
  for (int l = 0; l < NLAYER; ++l) {
    const int64_t M = int64_t(N) * hs[l] * wsz[l];
    mk = std::max<int64_t>(mk, M * 9 * ws->L[l].cin);
    mn = std::max<int64_t>(mn, M * ws->L[l].cout);
  }
  mk = std::max<int64_t>(mk, int64_t(N) * 32 * 4 * c);   // dA also holds the pooling partial sums
  NRK(ws->col.ensure(size_t(mk) * 2));
  NRK(ws->dA.ensure(size_t(mk) * 4));
  NRK(ws->z.ensure(size_t(mn) * 4));
  NRK(ws->dzf.ensure(size_t(mn) * 4));
  NRK(ws->dzb.ensure(size_t(mn) * 2));
  NRK(ws->part.ensure(size_t(64) * 4 * ws->base * 9 * 4 * ws->base * 4 + 1024));
  NRK(ws->small.ensure(64));
  ws->loss = ws->small.as<double>();
  ws->N = N;
  ws->H = H;
  ws->W = W;
  return RTG_OK;
}

const float* Bf(const rtg_warmstart* ws, int l) { return ws->P.as<float>() + ws->L[l].b; }
const __nv_bfloat16* Wb(const rtg_warmstart* ws, int l) { return ws->Pb.as<__nv_bfloat16>() + ws->L[l].w; }

// Backward of layer l: dy is the gradient of its output (after the ReLU when
// mask != null); x its input (N, h, w, cin).  Writes the parameter gradients
// and, if dx != null, the input gradient.
rtg_status conv_bwd(rtg_warmstart* ws, int l, const float* x, int h, int w, const float* dy, const float* mask,
                    float* dx, cudaStream_t s) {
  const Layer& L = ws->L[l];
  const int ho = h / L.stride, wo = w / L.stride;
  const int M = ws->N * ho * wo, K = 9 * L.cin;
  NCK(nn::mask_grad(dy, mask, ws->dzf.as<float>(), ws->dzb.as<__nv_bfloat16>(), int64_t(M) * L.cout, s));
  float* G = ws->G.as<float>();
  NCK(nn::colsum(ws->dzf.as<float>(), G + L.b, M, L.cout, s));
  NCK(nn::im2col(x, ws->col.as<__nv_bfloat16>(), ws->N, h, w, L.cin, L.stride, s));
  int splits = M / 2048;
  if (splits < 1) splits = 1;
  if (splits > 64) splits = 64;
  NCK(nn::gemm(true, false, ws->dzb.as<__nv_bfloat16>(), ws->col.as<__nv_bfloat16>(), G + L.w, nullptr, L.cout, K,
               M, L.cout, K, splits, ws->part.as<float>(), s));
  if (dx != nullptr) {
    NCK(nn::gemm(false, false, ws->dzb.as<__nv_bfloat16>(), Wb(ws, l), ws->dA.as<float>(), nullptr, M, K, L.cout,
                 L.cout, K, 1, nullptr, s));
    NCK(nn::col2im(ws->dA.as<float>(), dx, ws->N, h, w, L.cin, L.stride, s));
  }
  return RTG_OK;
}

// One forward layer through the implicit-GEMM kernel: r = relu(conv(x) + b)
// (when r), out = r + skip (skip may be null); the output layer has no ReLU.
// up: x is the half-resolution tensor, read through its x2 up-sampling.
rtg_status layer_fwd(rtg_warmstart* ws, int l, const float* x, int h, int w, bool up, float* r, const float* skip,
                     float* out, cudaStream_t s) {
  const Layer& L = ws->L[l];
  NCK(nn::conv_fwd(x, Wb(ws, l), Bf(ws, l), r, skip, out, ws->N, h, w, L.cin, L.stride, L.cout, l != OUT, up,
                   ws->dA.as<float>(), int64_t(ws->dA.bytes / 4), s));
  return RTG_OK;
}

// training: the up-sampled decoder inputs are materialised (the backward
// pass reads them); inference reads them through the convolution's gather.
rtg_status forward(rtg_warmstart* ws, const float* C, float* X0, float* loglam_out, bool training, cudaStream_t s) {
  const int N = ws->N, H = ws->H, W = ws->W, c = ws->base;
  NCK(nn::to_nhwc(C, ws->x0, N, H, W, 3, s));
  NRK(layer_fwd(ws, E1, ws->x0, H, W, false, nullptr, nullptr, ws->e1, s));
  NRK(layer_fwd(ws, E2, ws->e1, H, W, false, nullptr, nullptr, ws->e2, s));
  NRK(layer_fwd(ws, E3, ws->e2, H / 2, W / 2, false, nullptr, nullptr, ws->e3, s));
  NRK(layer_fwd(ws, E4, ws->e3, H / 4, W / 4, false, nullptr, nullptr, ws->e4, s));
  if (training) {
    NCK(nn::up2(ws->e4, ws->u4, N, H / 8, W / 8, 4 * c, s));
    NRK(layer_fwd(ws, D3, ws->u4, H / 4, W / 4, false, ws->r3, ws->e3, ws->d3, s));
    NCK(nn::up2(ws->d3, ws->u3, N, H / 4, W / 4, 4 * c, s));
    NRK(layer_fwd(ws, D2, ws->u3, H / 2, W / 2, false, ws->r2, ws->e2, ws->d2, s));
    NCK(nn::up2(ws->d2, ws->u2, N, H / 2, W / 2, 2 * c, s));
    NRK(layer_fwd(ws, D1, ws->u2, H, W, false, ws->r1, ws->e1, ws->d1, s));
  } else {
    NRK(layer_fwd(ws, D3, ws->e4, H / 4, W / 4, true, nullptr, ws->e3, ws->d3, s));
    NRK(layer_fwd(ws, D2, ws->d3, H / 2, W / 2, true, nullptr, ws->e2, ws->d2, s));
    NRK(layer_fwd(ws, D1, ws->d2, H, W, true, nullptr, ws->e1, ws->d1, s));
  }
  NRK(layer_fwd(ws, OUT, ws->d1, H, W, false, nullptr, nullptr, ws->zo, s));
  NCK(nn::from_nhwc_add(ws->zo, C, X0, N, H, W, 3, s));
  const float* Pf = ws->P.as<float>();
  NCK(nn::pool_head(ws->e4, Pf + ws->head_w, Pf + ws->head_b, ws->g, loglam_out, ws->dA.as<float>(), N,
                    (H / 8) * (W / 8), 4 * c, s));
  return RTG_OK;
}

rtg_status backward(rtg_warmstart* ws, cudaStream_t s) {
  const int N = ws->N, H = ws->H, W = ws->W, c = ws->base;
  const int64_t p1 = int64_t(N) * H * W, p2 = p1 / 4, p4 = p1 / 16;
  float* G = ws->G.as<float>();
  // out (no ReLU): input d1
  NRK(conv_bwd(ws, OUT, ws->d1, H, W, ws->dout, nullptr, ws->gd1, s));
  // d1 = relu(conv(u2)) + e1
  NRK(conv_bwd(ws, D1, ws->u2, H, W, ws->gd1, ws->r1, ws->gu2, s));
  NCK(nn::up2_back(ws->gu2, ws->gd2, N, H / 2, W / 2, 2 * c, false, s));
  // d2 = relu(conv(u3)) + e2
  NRK(conv_bwd(ws, D2, ws->u3, H / 2, W / 2, ws->gd2, ws->r2, ws->gu3, s));
  NCK(nn::up2_back(ws->gu3, ws->gd3, N, H / 4, W / 4, 4 * c, false, s));
  // d3 = relu(conv(u4)) + e3
  NRK(conv_bwd(ws, D3, ws->u4, H / 4, W / 4, ws->gd3, ws->r3, ws->gu4, s));
  NCK(nn::up2_back(ws->gu4, ws->ge4, N, H / 8, W / 8, 4 * c, false, s));
  // lambda head
  const float* Pf = ws->P.as<float>();
  NCK(nn::head_back(ws->g, ws->dll, Pf + ws->head_w, G + ws->head_w, G + ws->head_b, ws->ge4, N,
                    (H / 8) * (W / 8), 4 * c, s));
  // encoder: each e_k feeds the next level and a skip sum
  NRK(conv_bwd(ws, E4, ws->e3, H / 4, W / 4, ws->ge4, ws->e4, ws->gtmp, s));
  NCK(nn::add(ws->gd3, ws->gtmp, ws->ge3, p4 * 4 * c, s));
  NRK(conv_bwd(ws, E3, ws->e2, H / 2, W / 2, ws->ge3, ws->e3, ws->gtmp, s));
  NCK(nn::add(ws->gd2, ws->gtmp, ws->ge2, p2 * 2 * c, s));
  NRK(conv_bwd(ws, E2, ws->e1, H, W, ws->ge2, ws->e2, ws->gtmp, s));
  NCK(nn::add(ws->gd1, ws->gtmp, ws->ge1, p1 * c, s));
  NRK(conv_bwd(ws, E1, ws->x0, H, W, ws->ge1, ws->e1, nullptr, s));
  return RTG_OK;
}

rtg_status check_batch(rtg_warmstart* ws, int n, int I1, int I2) {
  if (ws == nullptr) return nfail(RTG_ERR_INVALID_ARG, "warm-start handle is NULL");
  if (n < 1 || n > 1024) return nfail(RTG_ERR_INVALID_ARG, "n_img=%d not in 1..1024", n);
  if (I1 < 8 || I2 < 8 || I1 % 8 || I2 % 8)
    return nfail(RTG_ERR_INVALID_ARG, "image sides must be multiples of 8 (got %d x %d)", I1, I2);
  return shape_buffers(ws, n, I2, I1);
}

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int d) {
    cudaGetDevice(&prev);
    cudaSetDevice(d);
  }
  ~DevGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" {

rtg_status rtg_ws_create(int32_t device, int32_t base, const float* params, rtg_ws* out) {
  if (out == nullptr) return nfail(RTG_ERR_INVALID_ARG, "out is NULL");
  if (base < 4 || base > 64 || base % 4) return nfail(RTG_ERR_INVALID_ARG, "base=%d must be a multiple of 4 in 4..64", base);
  if (params == nullptr) return nfail(RTG_ERR_INVALID_ARG, "params is NULL (initial values come from the caller)");
  DevGuard dg(device);
  auto* ws = new rtg_warmstart();
  ws->device = device;
  ws->base = base;
  layout(ws);
  const size_t n = size_t(ws->nparams);
  rtg_status st = RTG_OK;
  if ((st = ws->P.ensure(n * 4)) != RTG_OK || (st = ws->Pb.ensure(n * 2)) != RTG_OK ||
      (st = ws->G.ensure(n * 4)) != RTG_OK || (st = ws->Mo.ensure(n * 4)) != RTG_OK ||
      (st = ws->Vo.ensure(n * 4)) != RTG_OK) {
    delete ws;
    return st;
  }
  cudaMemcpy(ws->P.p, params, n * 4, cudaMemcpyHostToDevice);
  cudaMemset(ws->G.p, 0, n * 4);
  cudaMemset(ws->Mo.p, 0, n * 4);
  cudaMemset(ws->Vo.p, 0, n * 4);
  if (nn::to_bf16(ws->P.as<float>(), ws->Pb.as<__nv_bfloat16>(), ws->nparams, nullptr) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    delete ws;
    return nfail(RTG_ERR_CUDA, "warm-start parameter upload failed");
  }
  *out = ws;
  return RTG_OK;
}

rtg_status rtg_ws_destroy(rtg_ws ws) {
  if (ws == nullptr) return RTG_OK;
  DevGuard dg(ws->device);
  cudaDeviceSynchronize();
  delete ws;
  return RTG_OK;
}

int64_t rtg_ws_num_params(rtg_ws ws) { return ws ? ws->nparams : -1; }

rtg_status rtg_ws_get(rtg_ws ws, float* params, float* grads) {
  if (ws == nullptr) return nfail(RTG_ERR_INVALID_ARG, "warm-start handle is NULL");
  DevGuard dg(ws->device);
  if (params) NCK(cudaMemcpy(params, ws->P.p, size_t(ws->nparams) * 4, cudaMemcpyDeviceToHost));
  if (grads) NCK(cudaMemcpy(grads, ws->G.p, size_t(ws->nparams) * 4, cudaMemcpyDeviceToHost));
  return RTG_OK;
}

rtg_status rtg_ws_predict(rtg_ws ws, int32_t n_img, int32_t I1, int32_t I2, const float* C, float* X0,
                          float* loglam, rtg_stream stream) {
  if (ws == nullptr) return nfail(RTG_ERR_INVALID_ARG, "warm-start handle is NULL");
  DevGuard dg(ws->device);
  NRK(check_batch(ws, n_img, I1, I2));
  if (C == nullptr || X0 == nullptr || loglam == nullptr) return nfail(RTG_ERR_INVALID_ARG, "NULL argument");
  return forward(ws, C, X0, loglam, false, reinterpret_cast<cudaStream_t>(stream));
}

rtg_status rtg_ws_train_step(rtg_ws ws, int32_t n_img, int32_t I1, int32_t I2, const float* C, const float* Xstar,
                             const float* logmu, float lr, float* X0_scratch, double* loss_out,
                             rtg_stream stream) {
  if (ws == nullptr) return nfail(RTG_ERR_INVALID_ARG, "warm-start handle is NULL");
  DevGuard dg(ws->device);
  NRK(check_batch(ws, n_img, I1, I2));
  if (C == nullptr || Xstar == nullptr || logmu == nullptr || X0_scratch == nullptr)
    return nfail(RTG_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  NRK(forward(ws, C, X0_scratch, ws->loglam, true, s));
  NCK(nn::loss(X0_scratch, Xstar, ws->loglam, logmu, ws->dout, ws->dll, ws->loss, ws->N, ws->H, ws->W, 3, s));
  NRK(backward(ws, s));
  if (lr > 0.f) {
    ws->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, float(ws->adam_t)), c2 = 1.f - powf(b2, float(ws->adam_t));
    NCK(nn::adam(ws->P.as<float>(), ws->G.as<float>(), ws->Mo.as<float>(), ws->Vo.as<float>(),
                 ws->Pb.as<__nv_bfloat16>(), ws->nparams, lr, b1, b2, 1e-8f, c1, c2, s));
  }
  if (loss_out) {
    NCK(cudaMemcpyAsync(loss_out, ws->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    NCK(cudaStreamSynchronize(s));
  }
  return RTG_OK;
}

rtg_status rtg_nn_conv3x3(int32_t device, int32_t N, int32_t H, int32_t W, int32_t cin, int32_t cout,
                          int32_t stride, const float* x, const float* w, const float* b, float* y,
                          const float* dy, float* dx, float* dw, float* db, rtg_stream stream) {
  if (N < 1 || H < 1 || W < 1 || cin < 1 || cout < 1 || (stride != 1 && stride != 2) || H % stride || W % stride)
    return nfail(RTG_ERR_INVALID_ARG, "bad convolution shape");
  if (x == nullptr || w == nullptr) return nfail(RTG_ERR_INVALID_ARG, "x and w must not be NULL");
  if (dy == nullptr && y == nullptr) return nfail(RTG_ERR_INVALID_ARG, "give y (forward) or dy (backward)");
  DevGuard dg(device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int ho = H / stride, wo = W / stride;
  const int M = N * ho * wo, K = 9 * cin;
  Buf wb, col, zf, zb, dA, part;
  NRK(wb.ensure(size_t(cout) * K * 2));
  NRK(col.ensure(size_t(M) * K * 2));
  NCK(nn::to_bf16(w, wb.as<__nv_bfloat16>(), int64_t(cout) * K, s));
  NCK(nn::im2col(x, col.as<__nv_bfloat16>(), N, H, W, cin, stride, s));
  if (y != nullptr)
    NCK(nn::conv_fwd(x, wb.as<__nv_bfloat16>(), b, nullptr, nullptr, y, N, H, W, cin, stride, cout, false, false,
                     nullptr, 0, s));
  if (dy != nullptr) {
    NRK(zf.ensure(size_t(M) * cout * 4));
    NRK(zb.ensure(size_t(M) * cout * 2));
    NCK(nn::mask_grad(dy, nullptr, zf.as<float>(), zb.as<__nv_bfloat16>(), int64_t(M) * cout, s));
    if (db != nullptr) NCK(nn::colsum(zf.as<float>(), db, M, cout, s));
    if (dw != nullptr) {
      int splits = M / 2048;
      splits = splits < 1 ? 1 : (splits > 64 ? 64 : splits);
      NRK(part.ensure(size_t(splits) * cout * K * 4 + 64));
      NCK(nn::gemm(true, false, zb.as<__nv_bfloat16>(), col.as<__nv_bfloat16>(), dw, nullptr, cout, K, M, cout, K,
                   splits, part.as<float>(), s));
    }
    if (dx != nullptr) {
      NRK(dA.ensure(size_t(M) * K * 4));
      NCK(nn::gemm(false, false, zb.as<__nv_bfloat16>(), wb.as<__nv_bfloat16>(), dA.as<float>(), nullptr, M, K,
                   cout, cout, K, 1, nullptr, s));
      NCK(nn::col2im(dA.as<float>(), dx, N, H, W, cin, stride, s));
    }
  }
  NCK(cudaStreamSynchronize(s));
  return RTG_OK;
}

}  // extern "C"
