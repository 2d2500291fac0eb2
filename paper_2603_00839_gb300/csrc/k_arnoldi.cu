// Sketched global Arnoldi step (Section 4.3; algorithm "Block GMRES via
// Sketched Einstein Product"): Gram-Schmidt in the sketch space against the
// stored sketched basis Q = [S(V_0) .. S(V_j)], the full-space basis update,
// and the Givens update of the Hessenberg least-squares residual (Eq. 11S).
//
// The paper orthogonalises with modified Gram-Schmidt, recomputing the
// sketch of W after every subtraction.  Because S is linear,
// S(W - h V_i) = S(W) - h S(V_i), so the whole process can run on the
// sketch s = S(Phi V_j): classical Gram-Schmidt with one
// re-orthogonalisation pass (h = h1 + h2), equal to MGS in exact
// arithmetic.  h_{j+1,j} = ||s - Q h||, taken as sqrt(||s'||^2 - ||h2||^2)
// with s' = s - Q h1 (Q has orthonormal columns).  The full-space
// update then applies the total h once:
//   V_{j+1} = (W - sum_i h_i V_i) / h_{j+1,j},  Q_{j+1} = (s' - Q h2) / h_{j+1,j}.
//
// Reductions: each CTA reduces its slice (data-type partials, warp
// shuffles, FP64 across warps) into a row of `part`; the last CTA to finish
// (atomic ticket) sums the rows in FP64 and runs the scalar epilogue.
// Nothing waits on another CTA.
#include "gs_common.cuh"

namespace rtg {

constexpr int GS_THREADS = 256;
constexpr int GS_ITEMS = 8;

// Blocks of the Gram-Schmidt passes: about 1024 sketch entries each (at
// most GS_THREADS * GS_ITEMS), so the last block has few rows to combine.
int gs_grid(int64_t d) {
  int64_t g = (d + GS_THREADS * GS_ITEMS - 1) / (GS_THREADS * GS_ITEMS);
  int64_t want = (d + 1023) / 1024;
  if (want > 152) want = 152;
  if (g < want) g = want;
  return static_cast<int>(g < 1 ? 1 : g);
}

// pass 0: start (norm of the summed sketch -> beta); 1: h1 = Q^T S and
// ||S||^2 (S summed from the chain's partial sketches); 2: S <- S - Q h1,
// h2 = Q^T S, ||S||^2, then the step epilogue.
template <typename T>
__global__ void __launch_bounds__(GS_THREADS) k_gs_pass(Work w, int pass, StepOpts o) {
  Ctl* ctl = w.ctl;
  if (ctl->stop) return;
  const int J = ctl->j;
  const int ncols = (pass == 0) ? 0 : J + 1;
  const int d = w.d;
  T* S = static_cast<T*>(w.S);
  const T* Q = static_cast<const T*>(w.Q);
  __shared__ T coef[kMaxK + 1];
  __shared__ double red[GS_MAXW][kMaxK + 2];
  __shared__ double tot[kMaxK + 2];
  __shared__ int am_last;
  if (pass == 2)
    for (int i = threadIdx.x; i < ncols; i += GS_THREADS) coef[i] = static_cast<T>(w.h1[i]);
  __syncthreads();

  const int64_t chunk = (d + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = (lo + chunk < d) ? lo + chunk : d;
  T sv[GS_ITEMS];
  int64_t ix[GS_ITEMS];
  int cnt = 0;
#pragma unroll
  for (int k = 0; k < GS_ITEMS; ++k) {
    ix[k] = lo + threadIdx.x + static_cast<int64_t>(k) * GS_THREADS;
    if (ix[k] < hi) cnt = k + 1;
  }
  if (pass == 2) {
#pragma unroll
    for (int k = 0; k < GS_ITEMS; ++k) {
      if (k >= cnt) break;
      T v = S[ix[k]];
      for (int i = 0; i < ncols; ++i) v -= coef[i] * Q[static_cast<int64_t>(i) * d + ix[k]];
      sv[k] = v;
      S[ix[k]] = v;
    }
  } else {
    // sum the partial sketches of the contraction chain into S
    const T* P = static_cast<const T*>(w.Spart);
#pragma unroll
    for (int k = 0; k < GS_ITEMS; ++k) {
      if (k >= cnt) break;
      T v = 0;
      for (int p = 0; p < w.nparts; ++p) v += P[static_cast<int64_t>(p) * d + ix[k]];
      S[ix[k]] = v;
      sv[k] = v;
    }
  }
  block_partials<T, GS_ITEMS>(w, sv, ix, cnt, ncols, red);
  if (!last_block_combine(w, ncols, tot, &am_last)) return;
  if (threadIdx.x == 0) gs_finish(w, pass, o, tot, ncols);
}

// V_0 = src / beta, Q_0 = S / beta
template <typename T>
__global__ void k_start_scale(Work w, PtrRef srcr) {
  const Ctl* ctl = w.ctl;
  if (ctl->stop) return;
  const T* src = srcr.get<const T>();
  const T inv = static_cast<T>(1.0 / ctl->beta);
  T* V = static_cast<T*>(w.V);
  T* Q = static_cast<T*>(w.Q);
  const T* S = static_cast<const T*>(w.S);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (sizeof(T) == 4 && (w.n % 4) == 0 && (reinterpret_cast<uintptr_t>(src) % 16) == 0) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* v4 = reinterpret_cast<float4*>(V);
    const float fi = static_cast<float>(inv);
    for (int64_t o = t0; o < w.n / 4; o += stride) {
      float4 x = s4[o];
      x.x *= fi; x.y *= fi; x.z *= fi; x.w *= fi;
      v4[o] = x;
    }
  } else {
    for (int64_t o = t0; o < w.n; o += stride) V[o] = src[o] * inv;
  }
  for (int64_t o = t0; o < w.d; o += stride) Q[o] = S[o] * inv;
}

// V_{j} = (W - sum_{i<j} h_i V_i) / h_{j,j-1};  Q_{j} = (S - sum_{i<j} h2_i Q_i) / h_{j,j-1}
// FP32 tensors move as float4; four basis vectors are in flight per iteration.
template <typename T>
__global__ void k_update(Work w, StepOpts o) {
  Ctl* ctl = w.ctl;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // hard cap on the device-controlled loop: never more than m+1 bodies
    const int loops = ++ctl->loops;
    if (loops > w.m) {
      ctl->stop = 1;
      if (o.use_cond && loops > w.m + 1 && ctl->status == 0) ctl->status = RTG_ERR_TIMEOUT;
      set_cond(o, 0);
    }
  }
  if (ctl->skip_update || ctl->j == 0) return;
  const int jj = ctl->j;
  __shared__ T hs[kMaxK + 1], h2s[kMaxK + 1];
  const int ld = w.m + 1;
  for (int i = threadIdx.x; i < jj; i += blockDim.x) {
    hs[i] = static_cast<T>(w.H[static_cast<int64_t>(ld) * (jj - 1) + i]);
    h2s[i] = static_cast<T>(w.h2[i]);
  }
  __syncthreads();
  const T inv = static_cast<T>(1.0 / ctl->hnext);
  T* V = static_cast<T*>(w.V);
  T* Q = static_cast<T*>(w.Q);
  const T* W = static_cast<const T*>(w.W);
  const T* S = static_cast<const T*>(w.S);
  const int64_t n = w.n, d = w.d;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (sizeof(T) == 4 && (n % 4) == 0) {
    const int64_t n4 = n / 4;
    const float4* W4 = reinterpret_cast<const float4*>(W);
    const float4* V4 = reinterpret_cast<const float4*>(V);
    float4* out = reinterpret_cast<float4*>(V) + static_cast<int64_t>(jj) * n4;
    for (int64_t e = t0; e < n4; e += stride) {
      float4 acc = W4[e];
      int i = 0;
      for (; i + 4 <= jj; i += 4) {
        const float4 a = V4[static_cast<int64_t>(i) * n4 + e];
        const float4 b = V4[static_cast<int64_t>(i + 1) * n4 + e];
        const float4 c = V4[static_cast<int64_t>(i + 2) * n4 + e];
        const float4 dd = V4[static_cast<int64_t>(i + 3) * n4 + e];
        const float h0 = hs[i], h1 = hs[i + 1], h2 = hs[i + 2], h3 = hs[i + 3];
        acc.x -= h0 * a.x; acc.y -= h0 * a.y; acc.z -= h0 * a.z; acc.w -= h0 * a.w;
        acc.x -= h1 * b.x; acc.y -= h1 * b.y; acc.z -= h1 * b.z; acc.w -= h1 * b.w;
        acc.x -= h2 * c.x; acc.y -= h2 * c.y; acc.z -= h2 * c.z; acc.w -= h2 * c.w;
        acc.x -= h3 * dd.x; acc.y -= h3 * dd.y; acc.z -= h3 * dd.z; acc.w -= h3 * dd.w;
      }
      for (; i < jj; ++i) {
        const float4 a = V4[static_cast<int64_t>(i) * n4 + e];
        const float h0 = hs[i];
        acc.x -= h0 * a.x; acc.y -= h0 * a.y; acc.z -= h0 * a.z; acc.w -= h0 * a.w;
      }
      const float fi = static_cast<float>(inv);
      acc.x *= fi; acc.y *= fi; acc.z *= fi; acc.w *= fi;
      out[e] = acc;
    }
  } else {
    for (int64_t e = t0; e < n; e += stride) {
      T v = W[e];
      for (int i = 0; i < jj; ++i) v -= hs[i] * V[static_cast<int64_t>(i) * n + e];
      V[static_cast<int64_t>(jj) * n + e] = v * inv;
    }
  }
  for (int64_t e = t0; e < d; e += stride) {
    T v = S[e];
    for (int i = 0; i < jj; ++i) v -= h2s[i] * Q[static_cast<int64_t>(i) * d + e];
    Q[static_cast<int64_t>(jj) * d + e] = v * inv;
  }
}

__global__ void k_reset(Ctl* ctl, int new_cycle) {
  ctl->j = 0;
  ctl->stop = 0;
  ctl->breakdown = 0;
  ctl->converged = 0;
  ctl->skip_update = 0;
  ctl->pre2 = 0.0;
  ctl->hnext = 0.0;
  ctl->loops = 0;
  if (new_cycle) {
    ctl->cycle += 1;
  } else {
    ctl->status = 0;
    ctl->iters_total = 0;
    ctl->cycle = 0;
    ctl->beta0 = 0.0;
    ctl->beta = 0.0;
    ctl->rho = 1.0;
    ctl->mu = 0.0;
  }
}

static unsigned ew_grid(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return static_cast<unsigned>(b < 1 ? 1 : b);
}

cudaError_t launch_reset(const Work& w, int new_cycle, cudaStream_t s) {
  k_reset<<<1, 1, 0, s>>>(w.ctl, new_cycle);
  return cudaGetLastError();
}

cudaError_t launch_start(const Work& w, PtrRef src, const StepOpts& o, bool fused, cudaStream_t s) {
  const int g = gs_grid(w.d);
  if (w.dtype == RTG_F64) {
    if (!fused) k_gs_pass<double><<<g, GS_THREADS, 0, s>>>(w, 0, o);
    k_start_scale<double><<<ew_grid(w.n), 256, 0, s>>>(w, src);
  } else {
    if (!fused) k_gs_pass<float><<<g, GS_THREADS, 0, s>>>(w, 0, o);
    k_start_scale<float><<<ew_grid(w.n / 4 + 1), 256, 0, s>>>(w, src);
  }
  return cudaGetLastError();
}

cudaError_t launch_pass1(const Work& w, cudaStream_t s) {
  StepOpts o{};
  const int g = gs_grid(w.d);
  if (w.dtype == RTG_F64) k_gs_pass<double><<<g, GS_THREADS, 0, s>>>(w, 1, o);
  else k_gs_pass<float><<<g, GS_THREADS, 0, s>>>(w, 1, o);
  return cudaGetLastError();
}

cudaError_t launch_pass2(const Work& w, const StepOpts& o, cudaStream_t s) {
  const int g = gs_grid(w.d);
  if (w.dtype == RTG_F64) k_gs_pass<double><<<g, GS_THREADS, 0, s>>>(w, 2, o);
  else k_gs_pass<float><<<g, GS_THREADS, 0, s>>>(w, 2, o);
  return cudaGetLastError();
}

cudaError_t launch_update(const Work& w, const StepOpts& o, cudaStream_t s) {
  if (w.dtype == RTG_F64) k_update<double><<<ew_grid(w.n), 256, 0, s>>>(w, o);
  else k_update<float><<<ew_grid(w.n / 4 + 1), 256, 0, s>>>(w, o);
  return cudaGetLastError();
}

}  // namespace rtg
