// Kernels of the learned warm start (a convolutional encoder-decoder that
// predicts X_0 and log(lambda) from C).  Activations are FP32 and channels
// last (N, H, W, C); 3x3 convolutions with zero padding 1 run on BF16
// tensor cores with FP32 accumulation: forward as an implicit GEMM that
// gathers its patches from the activations, backward as im2col + GEMM
// (data gradient through the transposed product, weight gradient as a
// split-K product over the pixels).  Everything else (ReLU masks,
// nearest up-sampling, skip sums, pooling, the lambda head, the loss and
// Adam) is elementwise or a small reduction.
#include <cuda_bf16.h>

#include "nn_internal.cuh"

namespace rtg {
namespace nn {

// ------------------------------------------------------------------ GEMM
// C[M x N] (FP32) = A[M x K] * B[K x N] (+ bias[n]) with BF16 operands.
//   A_CM = false: A row-major (element (m, k) at A[m * lda + k])
//   A_CM = true : A stored as its transpose (element (m, k) at A[k * lda + m])
//   B_T  = true : B stored as N x K row-major (element (k, n) at B[n * ldb + k])
//   B_T  = false: B row-major K x N (element (k, n) at B[k * ldb + n])
// CTA tile 64 x 64, K step 32, four warps of 32 x 32 (2 x 4 m16n8k16 tiles).
// gridDim.z splits K; slice z writes C + z * M * N (summed by the caller).
constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8;

__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <bool A_CM, bool B_T>
__global__ void __launch_bounds__(128)
k_gemm_bf16(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B,
            float* __restrict__ C, const float* __restrict__ bias, int M, int N, int K, int lda,
            int ldb, int kchunk) {
  __shared__ __align__(16) __nv_bfloat16 As[GBM][GBK + GPAD];   // [m][k]
  __shared__ __align__(16) __nv_bfloat16 Bs[GBN][GBK + GPAD];   // [n][k]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  for (int k0 = kbeg; k0 < kend; k0 += GBK) {
    // stage the tiles (bounds-checked, zero filled)
    for (int e = tid; e < GBM * GBK; e += 128) {
      int m, k;
      if (A_CM) { m = e % GBM; k = e / GBM; } else { k = e % GBK; m = e / GBK; }
      const int gm = m0 + m, gk = k0 + k;
      __nv_bfloat16 v = zero;
      if (gm < M && gk < kend) v = A_CM ? A[static_cast<int64_t>(gk) * lda + gm] : A[static_cast<int64_t>(gm) * lda + gk];
      As[m][k] = v;
    }
    for (int e = tid; e < GBN * GBK; e += 128) {
      int n, k;
      if (B_T) { k = e % GBK; n = e / GBK; } else { n = e % GBN; k = e / GBN; }
      const int gn = n0 + n, gk = k0 + k;
      __nv_bfloat16 v = zero;
      if (gn < N && gk < kend) v = B_T ? B[static_cast<int64_t>(gn) * ldb + gk] : B[static_cast<int64_t>(gk) * ldb + gn];
      Bs[n][k] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; kk += 16) {
      uint32_t af[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r = wm + mt * 16 + gid;
        af[mt][0] = *reinterpret_cast<const uint32_t*>(&As[r][kk + tig * 2]);
        af[mt][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + tig * 2]);
        af[mt][2] = *reinterpret_cast<const uint32_t*>(&As[r][kk + tig * 2 + 8]);
        af[mt][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + tig * 2 + 8]);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int cidx = wn + nt * 8 + gid;
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&Bs[cidx][kk + tig * 2]);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&Bs[cidx][kk + tig * 2 + 8]);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) mma16816(acc[mt][nt], af[mt], b0, b1);
      }
    }
    __syncthreads();
  }
  float* Cz = C + static_cast<int64_t>(blockIdx.z) * M * N;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = m0 + wm + mt * 16 + gid + h * 8;
        const int c = n0 + wn + nt * 8 + tig * 2;
        if (r >= M) continue;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (c + q >= N) continue;
          float v = acc[mt][nt][2 * h + q];
          if (bias != nullptr && blockIdx.z == 0) v += bias[c + q];
          Cz[static_cast<int64_t>(r) * N + c + q] = v;
        }
      }
}

// out[i] = sum over the split slices of part[z * len + i]
__global__ void k_sum_slices(const float* __restrict__ part, float* __restrict__ out, int64_t len, int nz) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < len;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float v = 0.f;
    for (int z = 0; z < nz; ++z) v += part[static_cast<int64_t>(z) * len + i];
    out[i] = v;
  }
}

static unsigned grid_of(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  return static_cast<unsigned>(b < 1 ? 1 : b);
}

cudaError_t gemm(bool a_cm, bool b_t, const __nv_bfloat16* A, const __nv_bfloat16* B, float* C,
                 const float* bias, int M, int N, int K, int lda, int ldb, int splits, float* part,
                 cudaStream_t s) {
  if (splits < 1) splits = 1;
  int kchunk = (K + splits - 1) / splits;
  kchunk = ((kchunk + GBK - 1) / GBK) * GBK;
  splits = (K + kchunk - 1) / kchunk;
  float* dst = splits > 1 ? part : C;
  dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM, splits);
  if (!a_cm && b_t) k_gemm_bf16<false, true><<<grid, 128, 0, s>>>(A, B, dst, bias, M, N, K, lda, ldb, kchunk);
  else if (!a_cm && !b_t) k_gemm_bf16<false, false><<<grid, 128, 0, s>>>(A, B, dst, bias, M, N, K, lda, ldb, kchunk);
  else if (a_cm && !b_t) k_gemm_bf16<true, false><<<grid, 128, 0, s>>>(A, B, dst, bias, M, N, K, lda, ldb, kchunk);
  else return cudaErrorInvalidValue;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  k_sum_slices<<<grid_of(int64_t(M) * N), 256, 0, s>>>(part, C, int64_t(M) * N, splits);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ implicit-GEMM convolution
// Forward 3x3 convolution without a materialised im2col: the A tile (128
// output pixels x 32 of the 9 c_in patch entries) is gathered from the
// channels-last input while the previous tile is multiplied.  When
// c_in % 32 == 0 a 32-wide K slice is one tap and 32 consecutive channels,
// i.e. 8 float4 per pixel; otherwise (the 3-channel input layer) entries are
// gathered one by one.  Weights (c_out x K, BF16) come in 16-byte pieces
// when K % 8 == 0.  The epilogue adds the bias, applies the ReLU and the skip
// sum and stores FP32: r = act(acc + b) (optional), out = r + skip.
// Eight warps; warp w owns output rows 16w..16w+15 and all BN channels.
constexpr int CBM = 128, CBK = 32, CPAD = 8;

// up = 1: x holds the half-resolution tensor (H/2 x W/2) and the layer
// reads its nearest x2 up-sampling without materialising it.  gridDim.z > 1
// splits K: slice z writes its raw sums to part + z * M * cout and the
// epilogue runs in k_conv_split_epilogue.
template <int BN>
__global__ void __launch_bounds__(256, BN <= 64 ? 3 : 2)
k_conv_fwd(const float* __restrict__ x, const __nv_bfloat16* __restrict__ wt, const float* __restrict__ bias,
           float* __restrict__ rout, const float* __restrict__ skip, float* __restrict__ out, int N, int H, int W,
           int C, int stride, int cout, int relu, int up, int kchunk, float* __restrict__ part) {
  __shared__ __align__(16) __nv_bfloat16 As[2][CBM][CBK + CPAD];
  __shared__ __align__(16) __nv_bfloat16 Bs[2][BN][CBK + CPAD];
  constexpr int NB = (BN * 4 + 255) / 256;   // 16-byte weight pieces per thread
  const int Ho = H / stride, Wo = W / stride;
  const int M = N * Ho * Wo, Kfull = 9 * C;
  const int kbeg = blockIdx.z * kchunk;
  const int K = min(Kfull, kbeg + kchunk);   // this slice covers [kbeg, K)
  const int Hs = up ? H / 2 : H, Ws = up ? W / 2 : W, sh = up ? 1 : 0;   // stored input grid
  const int m0 = blockIdx.x * CBM, n0 = blockIdx.y * BN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, gid = lane >> 2, tig = lane & 3;
  const bool fastA = (C % 32) == 0;
  const bool fastB = (Kfull % 8) == 0;
  float4 ra[4];
  float rs[16];
  uint4 rb[NB];
  auto load_tiles = [&](int k0) {
    if (fastA) {
      const int tap = k0 / C, c0 = k0 - tap * C, ky = tap / 3, kx = tap - ky * 3;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = tid + q * 256, row = e >> 3, piece = e & 7;
        const int m = m0 + row;
        ra[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m < M) {
          const int j = m % Wo, i = (m / Wo) % Ho, n = m / (Wo * Ho);
          const int yy = stride * i + ky - 1, xx = stride * j + kx - 1;
          if (yy >= 0 && yy < H && xx >= 0 && xx < W)
            ra[q] = *reinterpret_cast<const float4*>(
                x + ((static_cast<int64_t>(n) * Hs + (yy >> sh)) * Ws + (xx >> sh)) * C + c0 + piece * 4);
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int e = tid + q * 256, row = e >> 5, kk = e & 31;
        const int m = m0 + row, k = k0 + kk;
        rs[q] = 0.f;
        if (m < M && k < K) {
          const int c = k % C, t = k / C, kx = t % 3, ky = t / 3;
          const int j = m % Wo, i = (m / Wo) % Ho, n = m / (Wo * Ho);
          const int yy = stride * i + ky - 1, xx = stride * j + kx - 1;
          if (yy >= 0 && yy < H && xx >= 0 && xx < W)
            rs[q] = x[((static_cast<int64_t>(n) * Hs + (yy >> sh)) * Ws + (xx >> sh)) * C + c];
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int e = tid + q * 256, row = e >> 2, piece = e & 3;
      rb[q] = make_uint4(0u, 0u, 0u, 0u);
      if (row < BN && n0 + row < cout) {
        const int k = k0 + piece * 8;
        if (fastB && k + 8 <= K) {
          rb[q] = *reinterpret_cast<const uint4*>(wt + static_cast<int64_t>(n0 + row) * Kfull + k);
        } else {
          __nv_bfloat16 t8[8];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            t8[u] = (k + u < K) ? wt[static_cast<int64_t>(n0 + row) * Kfull + k + u] : __float2bfloat16(0.f);
          rb[q] = *reinterpret_cast<const uint4*>(t8);
        }
      }
    }
  };
  auto store_tiles = [&](int buf) {
    if (fastA) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = tid + q * 256, row = e >> 3, piece = e & 7;
        __nv_bfloat162 h0 = __floats2bfloat162_rn(ra[q].x, ra[q].y);
        __nv_bfloat162 h1 = __floats2bfloat162_rn(ra[q].z, ra[q].w);
        uint2 v;
        v.x = *reinterpret_cast<uint32_t*>(&h0);
        v.y = *reinterpret_cast<uint32_t*>(&h1);
        *reinterpret_cast<uint2*>(&As[buf][row][piece * 4]) = v;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int e = tid + q * 256, row = e >> 5, kk = e & 31;
        As[buf][row][kk] = __float2bfloat16(rs[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int e = tid + q * 256, row = e >> 2, piece = e & 3;
      if (row < BN) *reinterpret_cast<uint4*>(&Bs[buf][row][piece * 8]) = rb[q];
    }
  };
  float acc[BN / 8][4];
#pragma unroll
  for (int a = 0; a < BN / 8; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;
  load_tiles(kbeg);
  store_tiles(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = kbeg; k0 < K; k0 += CBK) {
    const bool more = k0 + CBK < K;
    if (more) load_tiles(k0 + CBK);   // in flight during the products
#pragma unroll
    for (int kk = 0; kk < CBK; kk += 16) {
      uint32_t af[4];
      const int r = warp * 16 + gid;
      af[0] = *reinterpret_cast<const uint32_t*>(&As[buf][r][kk + tig * 2]);
      af[1] = *reinterpret_cast<const uint32_t*>(&As[buf][r + 8][kk + tig * 2]);
      af[2] = *reinterpret_cast<const uint32_t*>(&As[buf][r][kk + tig * 2 + 8]);
      af[3] = *reinterpret_cast<const uint32_t*>(&As[buf][r + 8][kk + tig * 2 + 8]);
#pragma unroll
      for (int nt = 0; nt < BN / 8; ++nt) {
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&Bs[buf][nt * 8 + gid][kk + tig * 2]);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&Bs[buf][nt * 8 + gid][kk + tig * 2 + 8]);
        mma16816(acc[nt], af, b0, b1);
      }
    }
    if (more) {
      store_tiles(buf ^ 1);   // the other buffer: nobody reads it during this step
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int nt = 0; nt < BN / 8; ++nt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = m0 + warp * 16 + gid + h * 8;
      if (m >= M) continue;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int c = n0 + nt * 8 + tig * 2 + q;
        if (c >= cout) continue;
        if (gridDim.z > 1) {
          part[(static_cast<int64_t>(blockIdx.z) * M + m) * cout + c] = acc[nt][2 * h + q];
          continue;
        }
        float v = acc[nt][2 * h + q] + (bias ? bias[c] : 0.f);
        if (relu) v = fmaxf(v, 0.f);
        const int64_t o = static_cast<int64_t>(m) * cout + c;
        if (rout != nullptr) rout[o] = v;
        if (out != nullptr) out[o] = skip ? v + skip[o] : v;
      }
    }
}

// Epilogue of a K-split convolution: sum the slices in order, then bias,
// activation and skip as in k_conv_fwd.
__global__ void k_conv_split_epilogue(const float* __restrict__ part, const float* __restrict__ bias,
                                      float* __restrict__ rout, const float* __restrict__ skip,
                                      float* __restrict__ out, int64_t MC, int cout, int nz, int relu) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < MC;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float v = 0.f;
    for (int z = 0; z < nz; ++z) v += part[static_cast<int64_t>(z) * MC + i];
    v += bias ? bias[i % cout] : 0.f;
    if (relu) v = fmaxf(v, 0.f);
    if (rout != nullptr) rout[i] = v;
    if (out != nullptr) out[i] = skip ? v + skip[i] : v;
  }
}

cudaError_t conv_fwd(const float* x, const __nv_bfloat16* w, const float* bias, float* r, const float* skip,
                     float* out, int N, int H, int W, int C, int stride, int cout, bool relu, bool up,
                     float* part, int64_t part_floats, cudaStream_t s) {
  const int M = N * (H / stride) * (W / stride);
  const int K = 9 * C;
  const int bn = cout <= 8 ? 8 : (cout <= 32 ? 32 : (cout <= 64 ? 64 : 128));
  const int mtiles = (M + CBM - 1) / CBM, ntiles = (cout + bn - 1) / bn;
  // split K (in whole 32-wide steps) when the tiles alone leave SMs idle
  int splits = 1;
  if (part != nullptr && mtiles * ntiles < 152) {
    splits = (304 + mtiles * ntiles - 1) / (mtiles * ntiles);
    const int ksteps = (K + CBK - 1) / CBK;
    if (splits > ksteps / 2) splits = ksteps / 2 > 1 ? ksteps / 2 : 1;
    while (splits > 1 && int64_t(splits) * M * cout > part_floats) --splits;
  }
  int kchunk = (K + splits - 1) / splits;
  kchunk = ((kchunk + CBK - 1) / CBK) * CBK;
  splits = (K + kchunk - 1) / kchunk;
  dim3 grid(mtiles, ntiles, splits);
  const int rl = relu ? 1 : 0, u = up ? 1 : 0;
#define RTG_CONV_CASE(B_)                                                                                   \
  if (bn == B_)                                                                                             \
    k_conv_fwd<B_><<<grid, 256, 0, s>>>(x, w, bias, r, skip, out, N, H, W, C, stride, cout, rl, u, kchunk, part);
  RTG_CONV_CASE(8) RTG_CONV_CASE(32) RTG_CONV_CASE(64) RTG_CONV_CASE(128)
#undef RTG_CONV_CASE
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  const int64_t MC = int64_t(M) * cout;
  k_conv_split_epilogue<<<grid_of(MC), 256, 0, s>>>(part, bias, r, skip, out, MC, cout, splits, rl);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ im2col / col2im
// A[m, k], m = (n, i, j) over output pixels, k = (ky, kx, c): x[n, s i + ky - 1, s j + kx - 1, c]
__global__ void k_im2col(const float* __restrict__ x, __nv_bfloat16* __restrict__ A, int N, int H, int W,
                         int C, int stride, int Ho, int Wo) {
  const int64_t K = 9LL * C;
  const int64_t total = static_cast<int64_t>(N) * Ho * Wo * K;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t m = e / K;
    const int k = static_cast<int>(e - m * K);
    const int c = k % C, t = k / C, kx = t % 3, ky = t / 3;
    const int j = static_cast<int>(m % Wo);
    const int i = static_cast<int>((m / Wo) % Ho);
    const int n = static_cast<int>(m / (static_cast<int64_t>(Wo) * Ho));
    const int y = stride * i + ky - 1, xx = stride * j + kx - 1;
    float v = 0.f;
    if (y >= 0 && y < H && xx >= 0 && xx < W) v = x[((static_cast<int64_t>(n) * H + y) * W + xx) * C + c];
    A[e] = __float2bfloat16(v);
  }
}

// dx[n, y, x, c] = sum over (ky, kx) with y = s i + ky - 1, x = s j + kx - 1 of dA[(n, i, j), (ky, kx, c)]
__global__ void k_col2im(const float* __restrict__ dA, float* __restrict__ dx, int N, int H, int W, int C,
                         int stride, int Ho, int Wo) {
  const int64_t total = static_cast<int64_t>(N) * H * W * C;
  const int64_t K = 9LL * C;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(e % C);
    const int xx = static_cast<int>((e / C) % W);
    const int y = static_cast<int>((e / (static_cast<int64_t>(C) * W)) % H);
    const int n = static_cast<int>(e / (static_cast<int64_t>(C) * W * H));
    float v = 0.f;
    for (int ky = 0; ky < 3; ++ky) {
      const int yi = y + 1 - ky;
      if (yi < 0 || yi % stride != 0) continue;
      const int i = yi / stride;
      if (i >= Ho) continue;
      for (int kx = 0; kx < 3; ++kx) {
        const int xj = xx + 1 - kx;
        if (xj < 0 || xj % stride != 0) continue;
        const int j = xj / stride;
        if (j >= Wo) continue;
        const int64_t m = (static_cast<int64_t>(n) * Ho + i) * Wo + j;
        v += dA[m * K + (ky * 3 + kx) * C + c];
      }
    }
    dx[e] = v;
  }
}

cudaError_t im2col(const float* x, __nv_bfloat16* A, int N, int H, int W, int C, int stride, cudaStream_t s) {
  const int Ho = H / stride, Wo = W / stride;
  k_im2col<<<grid_of(int64_t(N) * Ho * Wo * 9 * C), 256, 0, s>>>(x, A, N, H, W, C, stride, Ho, Wo);
  return cudaGetLastError();
}

cudaError_t col2im(const float* dA, float* dx, int N, int H, int W, int C, int stride, cudaStream_t s) {
  k_col2im<<<grid_of(int64_t(N) * H * W * C), 256, 0, s>>>(dA, dx, N, H, W, C, stride, H / stride, W / stride);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ elementwise
// r = relu(z); out = r + skip (skip may be null: out = r; out may alias z)
__global__ void k_relu_skip(const float* __restrict__ z, float* r, const float* skip, float* out, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float v = fmaxf(z[i], 0.f);
    if (r != nullptr) r[i] = v;
    if (out != nullptr) out[i] = v + (skip ? skip[i] : 0.f);
  }
}

// dz = dy * (mask > 0) (mask null: dz = dy), in FP32 and BF16
__global__ void k_mask_grad(const float* __restrict__ dy, const float* __restrict__ mask, float* dz,
                            __nv_bfloat16* dzb, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float v = (mask == nullptr || mask[i] > 0.f) ? dy[i] : 0.f;
    dz[i] = v;
    dzb[i] = __float2bfloat16(v);
  }
}

// db[c] = sum over rows of dz[r, c] (one block per column chunk, fixed order)
__global__ void k_colsum(const float* __restrict__ dz, float* __restrict__ db, int64_t rows, int cols) {
  const int c = blockIdx.x;
  __shared__ float red[256];
  float v = 0.f;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) v += dz[r * cols + c];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[c] = red[0];
}

__global__ void k_up2(const float* __restrict__ x, float* __restrict__ y, int N, int H, int W, int C) {
  const int64_t total = static_cast<int64_t>(N) * 2 * H * 2 * W * C;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(e % C);
    const int xx = static_cast<int>((e / C) % (2 * W));
    const int yy = static_cast<int>((e / (static_cast<int64_t>(C) * 2 * W)) % (2 * H));
    const int n = static_cast<int>(e / (static_cast<int64_t>(C) * 4 * W * H));
    y[e] = x[((static_cast<int64_t>(n) * H + yy / 2) * W + xx / 2) * C + c];
  }
}

// dx[n, i, j, c] = sum of the four dy entries it was copied to; dx += (accumulate) when acc
__global__ void k_up2_back(const float* __restrict__ dy, float* __restrict__ dx, int N, int H, int W, int C,
                           int acc) {
  const int64_t total = static_cast<int64_t>(N) * H * W * C;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(e % C);
    const int j = static_cast<int>((e / C) % W);
    const int i = static_cast<int>((e / (static_cast<int64_t>(C) * W)) % H);
    const int n = static_cast<int>(e / (static_cast<int64_t>(C) * W * H));
    const int64_t W2 = 2LL * W;
    const int64_t b = ((static_cast<int64_t>(n) * 2 * H + 2 * i) * W2 + 2 * j) * C + c;
    const float v = (dy[b] + dy[b + C]) + (dy[b + W2 * C] + dy[b + W2 * C + C]);
    dx[e] = acc ? dx[e] + v : v;
  }
}

__global__ void k_add(const float* a, const float* b, float* out, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[i] = a[i] + b[i];
}

// solver layout (per image x fastest, then y, then channel) <-> channels last
__global__ void k_to_nhwc(const float* __restrict__ src, float* __restrict__ dst, int N, int H, int W, int C) {
  const int64_t total = static_cast<int64_t>(N) * H * W * C;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int x = static_cast<int>(e % W);
    const int y = static_cast<int>((e / W) % H);
    const int c = static_cast<int>((e / (static_cast<int64_t>(W) * H)) % C);
    const int n = static_cast<int>(e / (static_cast<int64_t>(W) * H * C));
    dst[((static_cast<int64_t>(n) * H + y) * W + x) * C + c] = src[e];
  }
}

// dst (solver layout) = base (solver layout) + src (channels last)
__global__ void k_from_nhwc_add(const float* __restrict__ src, const float* __restrict__ base,
                                float* __restrict__ dst, int N, int H, int W, int C) {
  const int64_t total = static_cast<int64_t>(N) * H * W * C;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int x = static_cast<int>(e % W);
    const int y = static_cast<int>((e / W) % H);
    const int c = static_cast<int>((e / (static_cast<int64_t>(W) * H)) % C);
    const int n = static_cast<int>(e / (static_cast<int64_t>(W) * H * C));
    dst[e] = base[e] + src[((static_cast<int64_t>(n) * H + y) * W + x) * C + c];
  }
}

// g[n, c] = mean over pixels of e[n, ., ., c] in two fixed-order stages:
// block (n, b) sums the pixels of slice b for every channel (consecutive
// threads read consecutive channels), then one block per image adds the
// slices and applies the head loglam[n] = w . g[n] + b.
constexpr int POOL_SLICES = 32;
__global__ void k_pool_part(const float* __restrict__ e, float* __restrict__ part, int HW, int C) {
  const int n = blockIdx.x, b = blockIdx.y;
  const int p0 = static_cast<int>((static_cast<int64_t>(HW) * b) / POOL_SLICES);
  const int p1 = static_cast<int>((static_cast<int64_t>(HW) * (b + 1)) / POOL_SLICES);
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    float v = 0.f;
    for (int p = p0; p < p1; ++p) v += e[(static_cast<int64_t>(n) * HW + p) * C + c];
    part[(static_cast<int64_t>(n) * POOL_SLICES + b) * C + c] = v;
  }
}

__global__ void k_pool_head(const float* __restrict__ part, const float* __restrict__ w, const float* __restrict__ b,
                            float* __restrict__ g, float* __restrict__ loglam, int HW, int C) {
  const int n = blockIdx.x;
  __shared__ float red[256];
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    float v = 0.f;
    for (int s2 = 0; s2 < POOL_SLICES; ++s2) v += part[(static_cast<int64_t>(n) * POOL_SLICES + s2) * C + c];
    g[static_cast<int64_t>(n) * C + c] = v / HW;
  }
  __syncthreads();
  float v = 0.f;
  for (int c = threadIdx.x; c < C; c += blockDim.x) v += w[c] * g[static_cast<int64_t>(n) * C + c];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) loglam[n] = red[0] + b[0];
}

// Loss of the batch (one block, fixed order) and the output gradients:
// per image ||X0 - X*||^2 / ||X*||^2 + (loglam - logmu)^2, averaged;
// dout = 2 (X0 - X*) / (||X*||^2 N) (channels last), dloglam = 2 (loglam - logmu) / N.
// X0 and X* in solver layout; out_nhwc is the network output in channels last.
__global__ void k_loss(const float* __restrict__ X0, const float* __restrict__ Xs, const float* __restrict__ loglam,
                       const float* __restrict__ logmu, float* __restrict__ dout, float* __restrict__ dloglam,
                       double* __restrict__ loss, int N, int H, int W, int C) {
  __shared__ double red[2][256];
  __shared__ double inv[1024];
  const int64_t per = static_cast<int64_t>(H) * W * C;
  double total = 0.0;
  for (int n = 0; n < N; ++n) {
    double a = 0.0, bsum = 0.0;
    for (int64_t e = threadIdx.x; e < per; e += blockDim.x) {
      const double d = static_cast<double>(X0[n * per + e]) - Xs[n * per + e];
      a += d * d;
      bsum += static_cast<double>(Xs[n * per + e]) * Xs[n * per + e];
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = bsum;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        red[0][threadIdx.x] += red[0][threadIdx.x + o];
        red[1][threadIdx.x] += red[1][threadIdx.x + o];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double dl = static_cast<double>(loglam[n]) - logmu[n];
      total += red[0][0] / red[1][0] + dl * dl;
      if (n < 1024) inv[n] = 2.0 / (red[1][0] * N);
      dloglam[n] = static_cast<float>(2.0 * dl / N);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = total / N;
  for (int n = 0; n < N; ++n) {
    const double f = inv[n < 1024 ? n : 1023];
    for (int64_t e = threadIdx.x; e < per; e += blockDim.x) {
      const int x = static_cast<int>(e % W);
      const int y = static_cast<int>((e / W) % H);
      const int c = static_cast<int>(e / (static_cast<int64_t>(W) * H));
      dout[((static_cast<int64_t>(n) * H + y) * W + x) * C + c] =
          static_cast<float>(f * (static_cast<double>(X0[n * per + e]) - Xs[n * per + e]));
    }
  }
}

// Lambda head backward: dw[c] = sum_n g[n, c] dloglam[n], db = sum_n dloglam[n];
// de[n, p, c] += dloglam[n] w[c] / HW
__global__ void k_head_back(const float* __restrict__ g, const float* __restrict__ dll, const float* __restrict__ w,
                            float* __restrict__ dw, float* __restrict__ db, int N, int C) {
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    float v = 0.f;
    for (int n = 0; n < N; ++n) v += g[static_cast<int64_t>(n) * C + c] * dll[n];
    dw[c] = v;
  }
  if (threadIdx.x == 0) {
    float v = 0.f;
    for (int n = 0; n < N; ++n) v += dll[n];
    db[0] = v;
  }
}

__global__ void k_head_back_spread(const float* __restrict__ dll, const float* __restrict__ w, float* __restrict__ de,
                                   int N, int HW, int C) {
  const int64_t total = static_cast<int64_t>(N) * HW * C;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(e % C);
    const int n = static_cast<int>(e / (static_cast<int64_t>(HW) * C));
    de[e] += dll[n] * w[c] / HW;
  }
}

// Adam on the FP32 master weights; the BF16 copy used by the GEMMs follows.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       __nv_bfloat16* __restrict__ pb, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float w = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = w;
    if (pb != nullptr) pb[i] = __float2bfloat16(w);
  }
}

__global__ void k_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

#define NN_EW(kernel, n, ...)                                 \
  do {                                                        \
    kernel<<<grid_of(n), 256, 0, s>>>(__VA_ARGS__);           \
    return cudaGetLastError();                                \
  } while (0)

cudaError_t relu_skip(const float* z, float* r, const float* skip, float* out, int64_t n, cudaStream_t s) {
  NN_EW(k_relu_skip, n, z, r, skip, out, n);
}
cudaError_t mask_grad(const float* dy, const float* mask, float* dz, __nv_bfloat16* dzb, int64_t n, cudaStream_t s) {
  NN_EW(k_mask_grad, n, dy, mask, dz, dzb, n);
}
cudaError_t colsum(const float* dz, float* db, int64_t rows, int cols, cudaStream_t s) {
  k_colsum<<<cols, 256, 0, s>>>(dz, db, rows, cols);
  return cudaGetLastError();
}
cudaError_t up2(const float* x, float* y, int N, int H, int W, int C, cudaStream_t s) {
  NN_EW(k_up2, int64_t(N) * 4 * H * W * C, x, y, N, H, W, C);
}
cudaError_t up2_back(const float* dy, float* dx, int N, int H, int W, int C, bool acc, cudaStream_t s) {
  NN_EW(k_up2_back, int64_t(N) * H * W * C, dy, dx, N, H, W, C, acc ? 1 : 0);
}
cudaError_t add(const float* a, const float* b, float* out, int64_t n, cudaStream_t s) {
  NN_EW(k_add, n, a, b, out, n);
}
cudaError_t to_nhwc(const float* src, float* dst, int N, int H, int W, int C, cudaStream_t s) {
  NN_EW(k_to_nhwc, int64_t(N) * H * W * C, src, dst, N, H, W, C);
}
cudaError_t from_nhwc_add(const float* src, const float* base, float* dst, int N, int H, int W, int C,
                          cudaStream_t s) {
  NN_EW(k_from_nhwc_add, int64_t(N) * H * W * C, src, base, dst, N, H, W, C);
}
cudaError_t pool_head(const float* e, const float* w, const float* b, float* g, float* loglam, float* part, int N,
                      int HW, int C, cudaStream_t s) {
  k_pool_part<<<dim3(N, POOL_SLICES), 128, 0, s>>>(e, part, HW, C);
  k_pool_head<<<N, 256, 0, s>>>(part, w, b, g, loglam, HW, C);
  return cudaGetLastError();
}
cudaError_t loss(const float* X0, const float* Xs, const float* loglam, const float* logmu, float* dout,
                 float* dloglam, double* out, int N, int H, int W, int C, cudaStream_t s) {
  k_loss<<<1, 256, 0, s>>>(X0, Xs, loglam, logmu, dout, dloglam, out, N, H, W, C);
  return cudaGetLastError();
}
cudaError_t head_back(const float* g, const float* dll, const float* w, float* dw, float* db, float* de, int N,
                      int HW, int C, cudaStream_t s) {
  k_head_back<<<1, 256, 0, s>>>(g, dll, w, dw, db, N, C);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  NN_EW(k_head_back_spread, int64_t(N) * HW * C, dll, w, de, N, HW, C);
}
cudaError_t adam(float* p, const float* g, float* m, float* v, __nv_bfloat16* pb, int64_t n, float lr, float b1,
                 float b2, float eps, float c1, float c2, cudaStream_t s) {
  NN_EW(k_adam, n, p, g, m, v, pb, n, lr, b1, b2, eps, c1, c2);
}
cudaError_t to_bf16(const float* x, __nv_bfloat16* y, int64_t n, cudaStream_t s) {
  NN_EW(k_to_bf16, n, x, y, n);
}

}  // namespace nn
}  // namespace rtg
