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
#include "rtg_internal.cuh"

namespace rtg {

constexpr int GS_THREADS = 256;
constexpr int GS_ITEMS = 8;
constexpr int GS_WARPS = GS_THREADS / 32;

int gs_grid(int64_t d) {
  int64_t g = (d + GS_THREADS * GS_ITEMS - 1) / (GS_THREADS * GS_ITEMS);
  int64_t want = (d + GS_THREADS - 1) / GS_THREADS;
  if (want > 152) want = 152;
  if (g < want) g = want;
  return static_cast<int>(g < 1 ? 1 : g);
}

template <typename A>
__device__ __forceinline__ A warp_sum(A v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void set_cond(const StepOpts& o, int keep_going) {
  if (o.use_cond) cudaGraphSetConditional(static_cast<cudaGraphConditionalHandle>(o.cond),
                                          keep_going ? 1u : 0u);
}

// Givens update of column c = J of the rotated Hessenberg (Eq. 11S):
// rotations 0..J-1 applied to R(:, J), a new rotation zeroes R(J+1, J),
// g is rotated; |g[J+1]| is the least-squares residual.
__device__ void givens_column(const Work& w, int J) {
  const int ld = w.m + 1;
  double* Rc = w.R + static_cast<int64_t>(ld) * J;
  const double* Hc = w.H + static_cast<int64_t>(ld) * J;
  for (int i = 0; i <= J + 1; ++i) Rc[i] = Hc[i];
  for (int i = 0; i < J; ++i) {
    const double a = Rc[i], b = Rc[i + 1];
    Rc[i] = w.cs[i] * a + w.sn[i] * b;
    Rc[i + 1] = -w.sn[i] * a + w.cs[i] * b;
  }
  const double a = Rc[J], b = Rc[J + 1];
  const double den = hypot(a, b);
  double c = 1.0, s = 0.0;
  if (den != 0.0) {
    c = a / den;
    s = b / den;
  }
  Rc[J] = den;
  Rc[J + 1] = 0.0;
  w.cs[J] = c;
  w.sn[J] = s;
  const double gJ = w.g[J];
  w.g[J + 1] = -s * gJ;
  w.g[J] = c * gJ;
}

// pass 0: start (norm of S -> beta); 1: h1 = Q^T S and ||S||^2;
// 2: S <- S - Q h1, h2 = Q^T S, ||S||^2, then the step epilogue.
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
  __shared__ double red[GS_WARPS][kMaxK + 2];
  __shared__ int am_last;
  if (pass == 2)
    for (int i = threadIdx.x; i < ncols; i += GS_THREADS) coef[i] = static_cast<T>(w.h1[i]);
  __syncthreads();

  const int64_t chunk = (d + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = (lo + chunk < d) ? lo + chunk : d;
  T sv[GS_ITEMS];
#pragma unroll
  for (int k = 0; k < GS_ITEMS; ++k) {
    const int64_t e = lo + threadIdx.x + static_cast<int64_t>(k) * GS_THREADS;
    sv[k] = (e < hi) ? S[e] : static_cast<T>(0);
  }
  if (pass == 2) {
#pragma unroll
    for (int k = 0; k < GS_ITEMS; ++k) {
      const int64_t e = lo + threadIdx.x + static_cast<int64_t>(k) * GS_THREADS;
      if (e < hi) {
        T v = sv[k];
        for (int i = 0; i < ncols; ++i) v -= coef[i] * Q[static_cast<int64_t>(i) * d + e];
        sv[k] = v;
        S[e] = v;
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = 0; i <= ncols; ++i) {            // column ncols is the squared norm
    T p = 0;
#pragma unroll
    for (int k = 0; k < GS_ITEMS; ++k) {
      const int64_t e = lo + threadIdx.x + static_cast<int64_t>(k) * GS_THREADS;
      if (e < hi) p += sv[k] * ((i < ncols) ? Q[static_cast<int64_t>(i) * d + e] : sv[k]);
    }
    p = warp_sum(p);
    if (lane == 0) red[warp][i] = static_cast<double>(p);
  }
  __syncthreads();
  const int rowlen = w.m + 2;
  for (int i = threadIdx.x; i <= ncols; i += GS_THREADS) {
    double acc = 0.0;
#pragma unroll
    for (int u = 0; u < GS_WARPS; ++u) acc += red[u][i];
    w.part[static_cast<int64_t>(blockIdx.x) * rowlen + i] = acc;
  }
  __threadfence();
  __syncthreads();
  // self-wrapping ticket: the counter returns to 0 after the last block
  if (threadIdx.x == 0) am_last = (atomicInc(w.counter, gridDim.x - 1) == gridDim.x - 1);
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  __shared__ double tot[kMaxK + 2];
  for (int i = threadIdx.x; i <= ncols; i += GS_THREADS) {
    double acc = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) acc += __ldcg(w.part + static_cast<int64_t>(b) * rowlen + i);
    tot[i] = acc;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double tol = o.desc_tol ? *o.desc_tol : o.tol;
  const double bd_tol = o.desc_bd_tol ? *o.desc_bd_tol : o.bd_tol;

  if (pass == 0) {                                        // beta = ||R_0||_Theta
    const double beta = sqrt(tot[0]);
    if (!isfinite(beta)) {
      ctl->status = RTG_ERR_NONFINITE;
      ctl->stop = 1;
    } else if (beta == 0.0) {
      ctl->converged = 1;
      ctl->stop = 1;
    } else {
      ctl->beta = beta;
      if (ctl->cycle == 0) ctl->beta0 = beta;
      w.g[0] = beta;
      ctl->rho = beta / ctl->beta0;
      if (ctl->rho <= tol && ctl->cycle > 0) {
        ctl->converged = 1;
        ctl->stop = 1;
      }
      if (w.m == 0) ctl->stop = 1;
    }
    set_cond(o, !ctl->stop);
    return;
  }
  if (pass == 1) {
    for (int i = 0; i < ncols; ++i) w.h1[i] = tot[i];
    ctl->pre2 = tot[ncols];
    return;
  }
  // pass 2: finish the step
  double hh = 0.0;
  const int ld = w.m + 1;
  double* Hc = w.H + static_cast<int64_t>(ld) * J;
  bool finite = true;
  for (int i = 0; i < ncols; ++i) {
    w.h2[i] = tot[i];
    hh += tot[i] * tot[i];
    const double h = w.h1[i] + tot[i];
    Hc[i] = h;
    finite = finite && isfinite(h);
  }
  double hn2 = tot[ncols] - hh;
  double hn = sqrt(hn2 > 0.0 ? hn2 : 0.0);
  finite = finite && isfinite(hn) && isfinite(ctl->pre2);
  const bool breakdown = finite && (hn <= bd_tol * sqrt(ctl->pre2));
  Hc[J + 1] = breakdown ? 0.0 : hn;
  for (int i = J + 2; i < ld; ++i) Hc[i] = 0.0;
  givens_column(w, J);
  const double rho = fabs(w.g[J + 1]) / ctl->beta0;
  ctl->rho = rho;
  w.rho_hist[ctl->iters_total] = rho;
  ctl->iters_total += 1;
  ctl->hnext = hn;
  ctl->j = J + 1;
  if (!finite) ctl->status = RTG_ERR_NONFINITE;
  if (breakdown) ctl->breakdown = 1;
  const bool conv = finite && rho <= tol;
  if (conv || breakdown) ctl->converged = 1;
  const bool stop = !finite || breakdown || conv || (J + 1 >= w.m);
  ctl->stop = stop ? 1 : 0;
  ctl->skip_update = (!finite || breakdown || (o.solve_mode && stop)) ? 1 : 0;
  set_cond(o, !stop);
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
  const int64_t tot = w.n + w.d;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < tot;
       o += (int64_t)gridDim.x * blockDim.x) {
    if (o < w.n) V[o] = src[o] * inv;
    else Q[o - w.n] = S[o - w.n] * inv;
  }
}

// V_{j} = (W - sum_{i<j} h_i V_i) / h_{j,j-1};  Q_{j} = (S - sum_{i<j} h2_i Q_i) / h_{j,j-1}
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
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n + d;
       o += (int64_t)gridDim.x * blockDim.x) {
    if (o < n) {
      T v = W[o];
      for (int i = 0; i < jj; ++i) v -= hs[i] * V[static_cast<int64_t>(i) * n + o];
      V[static_cast<int64_t>(jj) * n + o] = v * inv;
    } else {
      const int64_t e = o - n;
      T v = S[e];
      for (int i = 0; i < jj; ++i) v -= h2s[i] * Q[static_cast<int64_t>(i) * d + e];
      Q[static_cast<int64_t>(jj) * d + e] = v * inv;
    }
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

cudaError_t launch_start(const Work& w, PtrRef src, const StepOpts& o, cudaStream_t s) {
  const int g = gs_grid(w.d);
  if (w.dtype == RTG_F64) {
    k_gs_pass<double><<<g, GS_THREADS, 0, s>>>(w, 0, o);
    k_start_scale<double><<<ew_grid(w.n + w.d), 256, 0, s>>>(w, src);
  } else {
    k_gs_pass<float><<<g, GS_THREADS, 0, s>>>(w, 0, o);
    k_start_scale<float><<<ew_grid(w.n + w.d), 256, 0, s>>>(w, src);
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
  if (w.dtype == RTG_F64) k_update<double><<<ew_grid(w.n + w.d), 256, 0, s>>>(w, o);
  else k_update<float><<<ew_grid(w.n + w.d), 256, 0, s>>>(w, o);
  return cudaGetLastError();
}

}  // namespace rtg
