// Device helpers shared by the kernels that finish a sketched Gram-Schmidt
// reduction (the sketch kernel fuses the first pass; k_arnoldi.cu holds
// the others): block partial dot products with the stored sketched basis,
// the last-block combine, the Givens update of Eq. 11S and the scalar
// epilogue of each pass (Section 4.3; the Block GMRES algorithm's steps).
#pragma once

#include "rtg_internal.cuh"

namespace rtg {

constexpr int GS_MAXW = 8;   // warps per block of the reducing kernels (256 threads)

template <typename A>
__device__ __forceinline__ A warp_sum(A v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void set_cond(const StepOpts& o, int keep_going) {
  if (o.use_cond)
    cudaGraphSetConditional(static_cast<cudaGraphConditionalHandle>(o.cond), keep_going ? 1u : 0u);
}

// Givens update of column J of the rotated Hessenberg (Eq. 11S):
// rotations 0..J-1 applied to R(:, J), a new rotation zeroes R(J+1, J),
// g is rotated; |g[J+1]| is the least-squares residual.
__device__ inline void givens_column(const Work& w, int J) {
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

// Per-block partial sums: column i < ncols is sum_e Q_i[e] * v[e] over the
// entries this block holds, column ncols is sum_e v[e]^2.  Each thread
// passes up to ITEMS entries (vals, idx; cnt valid).  Data-type products
// and warp sums, FP64 across warps.  Writes row blockIdx.x of w.part.
// red: shared scratch [GS_MAXW][kMaxK + 2].
template <typename T, int ITEMS>
__device__ void block_partials(const Work& w, const T* vals, const int64_t* idx, int cnt, int ncols,
                               double (*red)[kMaxK + 2]) {
  const T* Q = static_cast<const T*>(w.Q);
  const int64_t d = w.d;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i <= ncols; ++i) {
    T p = 0;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k)
      if (k < cnt) p += vals[k] * ((i < ncols) ? Q[static_cast<int64_t>(i) * d + idx[k]] : vals[k]);
    p = warp_sum(p);
    if (lane == 0) red[warp][i] = static_cast<double>(p);
  }
  __syncthreads();
  const int rowlen = w.m + 2;
  for (int i = threadIdx.x; i <= ncols; i += blockDim.x) {
    double acc = 0.0;
    for (int u = 0; u < nw; ++u) acc += red[u][i];
    w.part[static_cast<int64_t>(blockIdx.x + gridDim.x * blockIdx.y) * rowlen + i] = acc;
  }
}

// Ticket: returns true in every thread of the last block to finish, after
// tot[0..ncols] holds the sum of all blocks' rows (one warp per column,
// lanes striding over rows).  The counter wraps back to zero by itself.
__device__ inline bool last_block_combine(const Work& w, int ncols, double* tot, int* am_last) {
  __threadfence();
  __syncthreads();
  const unsigned nblk = gridDim.x * gridDim.y;
  if (threadIdx.x == 0) *am_last = (atomicInc(w.counter, nblk - 1) == nblk - 1);
  __syncthreads();
  if (!*am_last) return false;
  __threadfence();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int rowlen = w.m + 2;
  for (int i = warp; i <= ncols; i += nw) {
    double a0 = 0.0, a1 = 0.0;
    unsigned b = lane;
    for (; b + 32 < nblk; b += 64) {
      a0 += __ldcg(w.part + static_cast<int64_t>(b) * rowlen + i);
      a1 += __ldcg(w.part + static_cast<int64_t>(b + 32) * rowlen + i);
    }
    if (b < nblk) a0 += __ldcg(w.part + static_cast<int64_t>(b) * rowlen + i);
    a0 = warp_sum(a0 + a1);
    if (lane == 0) tot[i] = a0;
  }
  __syncthreads();
  return true;
}

// Scalar epilogue (one thread).  pass 0: beta = ||R_0||_Theta; pass 1:
// h1 and ||S(W)||^2; pass 2: h = h1 + h2, h_{j+1,j}, breakdown test,
// Givens, rho_j and the stop rule.
__device__ inline void gs_finish(const Work& w, int pass, const StepOpts& o, const double* tot,
                                 int ncols) {
  Ctl* ctl = w.ctl;
  const int J = ctl->j;
  const double tol = o.desc_tol ? *o.desc_tol : o.tol;
  const double bd_tol = o.desc_bd_tol ? *o.desc_bd_tol : o.bd_tol;
  if (pass == 0) {
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
  const double hn2 = tot[ncols] - hh;
  const double hn = sqrt(hn2 > 0.0 ? hn2 : 0.0);
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

}  // namespace rtg
