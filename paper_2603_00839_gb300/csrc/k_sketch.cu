// Mode-wise Rademacher sketch S(X) = X x_1 Theta_1 x_2 ... x_d Theta_d
// (Section 3, the global tensor sketching operator; Section 3.1).
//
// Each sketched mode k is one contraction of the current tensor, viewed as
// (L, I_k, R) column-major: Y(l, q, r) = sum_i Theta_k(q, i) X(l, i, r).
// Theta_k is held as packed sign bits, so every product is an exact
// sign flip; the scale prod_k 1/sqrt(s_k) is applied once, by the last
// contraction.  Intermediates live in two scratch tensors.
#include "rtg_internal.cuh"

namespace rtg {

// Y(l, q, r) = scale * sum_i (-1)^bit(q, i) X(l, i, r)
template <typename T>
__global__ void k_sketch_mode(PtrRef Xr, T* __restrict__ Y, int64_t L, int64_t I, int64_t R,
                              int64_t s, const uint32_t* __restrict__ bits, int wpr, T scale,
                              const int* stop) {
  if (stop != nullptr && *stop) return;
  const T* __restrict__ X = Xr.get<const T>();
  const int64_t total = L * s * R;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total;
       o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = o % L;
    const int64_t q = (o / L) % s;
    const int64_t r = o / (L * s);
    const T* xp = X + l + L * I * r;
    const uint32_t* brow = bits + q * wpr;
    T acc = 0;
    for (int w = 0; w < wpr; ++w) {
      const uint32_t b = __ldg(brow + w);
      const int64_t i0 = static_cast<int64_t>(w) * 32;
      const int cnt = (I - i0) < 32 ? static_cast<int>(I - i0) : 32;
      for (int u = 0; u < cnt; ++u) {
        const T x = xp[L * (i0 + u)];
        acc += ((b >> u) & 1u) ? -x : x;
      }
    }
    Y[o] = acc * scale;
  }
}

template <typename T>
__global__ void k_copy_scale(PtrRef Xr, T* __restrict__ Y, int64_t n, const int* stop) {
  if (stop != nullptr && *stop) return;
  const T* X = Xr.get<const T>();
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n;
       o += (int64_t)gridDim.x * blockDim.x)
    Y[o] = X[o];
}

static unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  return static_cast<unsigned>(b < 1 ? 1 : b);
}

template <typename T>
static cudaError_t sketch_t(const SketchPlan& sp, const uint32_t* bits, PtrRef X, T* SX, T* tmp0,
                           T* tmp1, const int* stop, cudaStream_t s) {
  int64_t cur[kMaxOrder];
  int64_t n = 1;
  for (int k = 0; k < sp.order; ++k) {
    cur[k] = sp.dims[k];
    n *= sp.dims[k];
  }
  int modes[kMaxOrder], nm = 0;
  for (int k = 0; k < sp.order; ++k)
    if (sp.sketched[k]) modes[nm++] = k;
  if (nm == 0) {     // no sketched mode: S = identity
    k_copy_scale<T><<<grid_for(n), 256, 0, s>>>(X, SX, n, stop);
    return cudaGetLastError();
  }
  PtrRef src = X;
  for (int t = 0; t < nm; ++t) {
    const int k = modes[t];
    int64_t L = 1, R = 1;
    for (int u = 0; u < k; ++u) L *= cur[u];
    for (int u = k + 1; u < sp.order; ++u) R *= cur[u];
    const int64_t I = cur[k], sk = sp.sdims[k];
    const bool last = (t == nm - 1);
    T* dst = last ? SX : ((t % 2 == 0) ? tmp0 : tmp1);
    const T scale = last ? static_cast<T>(sp.scale) : static_cast<T>(1);
    k_sketch_mode<T><<<grid_for(L * sk * R), 256, 0, s>>>(src, dst, L, I, R, sk,
                                                          bits + sp.word_off[k], sp.wpr[k], scale,
                                                          stop);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cur[k] = sk;
    src = ref(dst);
  }
  return cudaSuccess;
}

int sketch_launches(const SketchPlan& sp) {
  int nm = 0;
  for (int k = 0; k < sp.order; ++k) nm += sp.sketched[k] ? 1 : 0;
  return nm == 0 ? 1 : nm;
}

cudaError_t launch_sketch(const SketchPlan& sp, int dtype, const uint32_t* bits, PtrRef X,
                          void* SX, void* tmp0, void* tmp1, const int* stop, cudaStream_t s) {
  if (dtype == RTG_F64)
    return sketch_t<double>(sp, bits, X, static_cast<double*>(SX), static_cast<double*>(tmp0),
                            static_cast<double*>(tmp1), stop, s);
  return sketch_t<float>(sp, bits, X, static_cast<float*>(SX), static_cast<float*>(tmp0),
                         static_cast<float*>(tmp1), stop, s);
}

}  // namespace rtg
