// Reduced solves and solution assembly of RTG-GMRES.
//
// The Givens QR of the step kernels already holds Hbar_k = Omega^T [R; 0]
// and Omega^T beta e1 = g, so
//   ||beta e1 - Hbar y||^2 + mu ||y||^2 = ||g_{0:k} - R y||^2 + g_k^2 + mu ||y||^2.
// Projected Tikhonov (Eq. 12S) is solved in the stacked form of Eq. 13,
// min || [R; sqrt(mu) I] y - [g_{0:k}; 0] ||, by Householder reflections
// that use the structure (column j touches row j of R and rows 0..j of the
// sqrt(mu) I block), then back substitution.  GCV (Section 3, "Parameter
// selection via GCV"): the numerator is ||Hbar y_mu - beta e1||^2; the
// trace is tr(I - Hbar (Hbar^T Hbar + mu I)^{-1} Hbar^T) = 1 + mu ||R_mu^{-1}||_F^2
// (k+1 minus k plus mu tr((R_mu^T R_mu)^{-1})).  One CTA per candidate mu;
// the last CTA to finish picks the smallest GCV (ties: the larger mu).
// Everything here is FP64.
#include "gs_common.cuh"
#include "queue.cuh"

namespace rtg {

// Four warps per candidate mu.  An FP64 warp instruction occupies its SM
// sub-partition's FP64 unit for about 64 cycles on this GPU, so the cost of
// this kernel is the number of FP64 warp instructions each sub-partition
// issues: the work of every step is spread over all 128 lanes (rows and
// columns at once), and the scalars of a reflection are computed by every
// warp at the same time instead of being broadcast.
constexpr int TK_THREADS = 128;
constexpr int TK_WARPS = TK_THREADS / 32;

__device__ __forceinline__ double tk_block_sum(double v, double* wsum) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
  __syncthreads();
  const double t = (wsum[0] + wsum[1]) + (wsum[2] + wsum[3]);
  __syncthreads();
  return t;
}

// Back substitution y = U^{-1} b for an upper-triangular k x k U (leading
// dimension ldu) with precomputed reciprocal pivots rinv (0 for a zero
// pivot: y_i = 0, the smallest-norm least-squares choice on that
// direction), run by one warp; b is overwritten.
__device__ void back_subst(const double* U, int ldu, const double* rinv, double* b, double* y,
                           int k) {
  const int lane = threadIdx.x & 31;
  for (int i = k - 1; i >= 0; --i) {
    __syncwarp();
    const double yi = b[i] * rinv[i];
    if (lane == 0) y[i] = yi;
    for (int t = lane; t < i; t += 32) b[t] -= U[t + static_cast<int64_t>(ldu) * i] * yi;
  }
  __syncwarp();
}

// mode 0: least squares (mu = 0); 1: fixed mu = lambda; 2: GCV over the grid.
// Working set per CTA (tk_scratch_doubles(m) doubles): T and B, both
// (m+1) x (m+1) with row stride m+1, then y and rinv.  T holds R (becoming
// R_mu) with g_{0:k} as column k; B holds the sqrt(mu) I block with its
// right-hand side (0) as column k, and after the factorisation the
// inverse R_mu^{-1} is built in it.  With in_smem the working set is the
// CTA's dynamic shared memory, else the per-CTA global scratch.
__global__ void __launch_bounds__(TK_THREADS)
k_tikhonov(Work w0, const SolveDesc* desc0, int mode, double* scratch0, int in_smem, const int* gate) {
  const int64_t bo = bidx(w0.b).off;
  const Work w = w0.at(bo);
  const SolveDesc* desc = bsh(desc0, bo);
  double* scratch = bsh(scratch0, bo);
  Ctl* ctl = w.ctl;
  gate = bsh(gate, bo);
  if (gate != nullptr && *gate) return;
  // a GCV plan whose descriptor carries lambda > 0 (the learned warm start's
  // prediction) solves with that fixed mu on its first block
  if (mode == 2 && desc->lambda > 0.0) {
    if (blockIdx.x != 0) return;
    mode = 1;
  }
  const int k = ctl->j;
  const int m = w.m, ld = m + 1;
  __shared__ double red[TK_WARPS][kMaxK + 1];   // per-warp partial dot products of a step
  __shared__ double sp[TK_WARPS];               // per-warp partial squares of the next column
  __shared__ double wsum[TK_WARPS];
  __shared__ int am_last;
  extern __shared__ __align__(16) double tk_smem[];
  if (k == 0) {
    if (threadIdx.x == 0 && blockIdx.x == 0) ctl->mu = (mode == 1) ? desc->lambda : 0.0;
    return;
  }
  const double mu = (mode == 0) ? 0.0 : (mode == 1 ? desc->lambda : desc->mu_grid[blockIdx.x]);
  const int lm = m + 1;
  double* T = in_smem ? tk_smem : scratch + static_cast<int64_t>(blockIdx.x) * tk_scratch_doubles(m);
  double* Bm = T + lm * lm;
  double* y = Bm + lm * lm;
  double* rinv = y + lm;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double smu = sqrt(mu);
  for (int idx = tid; idx < k * (k + 1); idx += TK_THREADS) {
    const int col = idx / k, i = idx - col * k;
    T[i + lm * col] = (col == k) ? w.g[i] : (i <= col ? w.R[i + static_cast<int64_t>(ld) * col] : 0.0);
    Bm[i + lm * col] = (i == col) ? smu : 0.0;
  }
  if (tid < TK_WARPS) sp[tid] = 0.0;
  __syncthreads();
  if (mode != 0) {
    // Householder on column j: rows {j of T} U {0..j of B}; row j of B is
    // still sqrt(mu), rows 0..j-1 were filled by the earlier reflections.
    for (int j = 0; j < k; ++j) {
      const int nc = k - j;   // columns j+1 .. k (k: the right-hand side)
      // a warp covers cw column slots and 32/cw row stripes
      const int cw = nc >= 32 ? 32 : 1 << (32 - __clz(nc - 1));
      const int nst = TK_WARPS * (32 / cw);
      const int st = warp * (32 / cw) + lane / cw;
      const int cs = lane % cw;
      const double sigma = ((sp[0] + sp[1]) + (sp[2] + sp[3])) + smu * smu;
      const double alpha = T[j + lm * j];
      const double nrm = sqrt(alpha * alpha + sigma);
      const bool refl = nrm != 0.0 && sigma != 0.0;
      const double sgn = (alpha >= 0.0) ? 1.0 : -1.0;
      const double v0 = alpha + sgn * nrm;
      const double tau = refl ? 2.0 / (v0 * v0 + sigma) : 0.0;
      if (refl) {   // v . column, per stripe, then over the warp's stripes
        for (int c0 = 0; c0 < nc; c0 += cw) {
          const int c = c0 + cs, col = j + 1 + c;
          double a = 0.0;
          if (c < nc) {
            if (st == 0) a = v0 * T[j + lm * col];
            for (int i = st; i <= j; i += nst) a = fma(Bm[i + lm * j], Bm[i + lm * col], a);
          }
          for (int o = cw; o < 32; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
          if (lane < cw && c < nc) red[warp][c] = a;
        }
      }
      __syncthreads();
      double s2 = 0.0;   // squares of the updated column j+1 (slot 0) over this thread's rows
      for (int c0 = 0; c0 < nc; c0 += cw) {
        const int c = c0 + cs, col = j + 1 + c;
        if (c >= nc) continue;
        double wv = 0.0;
        if (refl) {
          wv = tau * ((red[0][c] + red[1][c]) + (red[2][c] + red[3][c]));
          if (st == 0) T[j + lm * col] -= wv * v0;
        }
        for (int i = st; i <= j; i += nst) {
          double bv = Bm[i + lm * col];
          if (refl) {
            bv = fma(-wv, Bm[i + lm * j], bv);
            Bm[i + lm * col] = bv;
          }
          if (c == 0) s2 = fma(bv, bv, s2);
        }
      }
      for (int o = cw; o < 32; o <<= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      if (lane == 0) sp[warp] = s2;
      if (tid == 0 && refl) T[j + lm * j] = -sgn * nrm;
      __syncthreads();
    }
  }
  for (int i = tid; i < k; i += TK_THREADS) {
    const double piv = T[i + lm * i];
    rinv[i] = (piv != 0.0) ? 1.0 / piv : 0.0;
  }
  __syncthreads();
  if (warp == 0) back_subst(T, lm, rinv, T + lm * k, y, k);
  __syncthreads();
  // residual ||g_{0:k} - R y||^2 + g_k^2 with the unregularised R
  double part = 0.0;
  for (int i = tid; i < k; i += TK_THREADS) {
    double r0 = w.g[i], r1 = 0.0;
    int jj = i;
    for (; jj + 1 < k; jj += 2) {
      r0 -= w.R[i + static_cast<int64_t>(ld) * jj] * y[jj];
      r1 -= w.R[i + static_cast<int64_t>(ld) * (jj + 1)] * y[jj + 1];
    }
    if (jj < k) r0 -= w.R[i + static_cast<int64_t>(ld) * jj] * y[jj];
    const double r = r0 + r1;
    part += r * r;
  }
  const double res2 = tk_block_sum(part, wsum) + w.g[k] * w.g[k];
  if (mode == 2) {
    // ||Z||_F^2 with Z = R_mu^{-1}: right-looking substitution on W = I
    // (stored in B), rows of Z from the last up.  Row l of Z is
    // W[l, l:] / R_mu[l,l]; with the columns of R_mu above the diagonal
    // pre-scaled by the pivot's reciprocal, each update of W is one FMA.
    for (int idx = tid; idx < k * k; idx += TK_THREADS) {
      const int col = idx / k, i = idx - col * k;
      Bm[i + lm * col] = (i == col) ? 1.0 : 0.0;
      if (i < col) T[i + lm * col] *= rinv[col];
    }
    __syncthreads();
    double inv2 = 0.0;
    for (int l = k - 1; l >= 0; --l) {
      const int nc = k - l;
      const double rl = rinv[l];
      for (int idx = tid; idx < (l + 1) * nc; idx += TK_THREADS) {
        const int i = idx / nc, col = l + (idx - i * nc);
        const double wl = Bm[l + lm * col];
        if (i == l) {
          const double z = wl * rl;
          inv2 = fma(z, z, inv2);
        } else {
          Bm[i + lm * col] = fma(-T[i + lm * l], wl, Bm[i + lm * col]);
        }
      }
      __syncthreads();
    }
    const double trace = 1.0 + mu * tk_block_sum(inv2, wsum);
    const double gcv = res2 / (trace * trace);
    if (tid == 0) w.gcv[blockIdx.x] = gcv;
    for (int i = tid; i < k; i += TK_THREADS) w.ysel[static_cast<int64_t>(blockIdx.x) * m + i] = y[i];
    __syncthreads();
    if (tid == 0) am_last = (ticket_acq_rel(w.counter, gridDim.x - 1) == gridDim.x - 1);
    __syncthreads();
    if (!am_last) return;
    __shared__ int best;
    if (tid == 0) {
      int bi = 0;
      double bv = __ldcg(w.gcv), bm = desc->mu_grid[0];
      for (unsigned u = 1; u < gridDim.x; ++u) {
        const double v = __ldcg(w.gcv + u), mm = desc->mu_grid[u];
        if (v < bv || (v == bv && mm > bm)) {
          bv = v;
          bm = mm;
          bi = static_cast<int>(u);
        }
      }
      best = bi;
      ctl->mu = bm;
      ctl->gcv_best = bv;
    }
    __syncthreads();
    for (int i = tid; i < k; i += TK_THREADS) w.y[i] = __ldcg(w.ysel + static_cast<int64_t>(best) * m + i);
    return;
  }
  for (int i = tid; i < k; i += TK_THREADS) w.y[i] = y[i];
  if (tid == 0) ctl->mu = mu;
}

// X = X0 + sum_{i<k} y_i V_i  (Eq. 10S); after a restart X holds the iterate
// the cycle started from and takes the place of X0 (elementwise in place)
template <typename T>
__global__ void k_assemble(Work w0, PtrRef X0r0, PtrRef Xr0, const int* gate) {
  const int64_t bo = bidx(w0.b).off;
  const Work w = w0.at(bo);
  const PtrRef X0r = X0r0.at(bo), Xr = Xr0.at(bo);
  gate = bsh(gate, bo);
  if (gate != nullptr && *gate) return;
  const int k = w.ctl->j;
  __shared__ T ys[kMaxK];
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = static_cast<T>(w.y[i]);
  __syncthreads();
  T* X = Xr.get<T>();
  const T* X0 = w.ctl->cycle > 0 ? X : X0r.get<const T>();
  const T* V = static_cast<const T*>(w.V);
  const int64_t n = w.n;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n;
       o += (int64_t)gridDim.x * blockDim.x) {
    T v = (X0 != nullptr) ? X0[o] : static_cast<T>(0);
    for (int i = 0; i < k; ++i) v += ys[i] * V[static_cast<int64_t>(i) * n + o];
    X[o] = v;
  }
}

__global__ void k_finalize(Work w0, InfoDev* info0) {
  const int64_t bo = bidx(w0.b).off;
  const Work w = w0.at(bo);
  InfoDev* info = bsh(info0, bo);
  const Ctl* c = w.ctl;
  const int t = threadIdx.x;
  if (t == 0) {
    info->iters = c->iters_total;
    info->restarts = c->cycle;
    info->breakdown = c->breakdown;
    info->converged = c->converged;
    info->status = c->status;
    info->k = c->j;
    info->beta = c->beta0;
    info->mu = c->mu;
    info->rho_final = c->rho;
    info->true_rel_resid = c->true_rr;
    info->true_rel_resid_theta = c->true_th;
  }
  for (int i = t; i < c->iters_total && i < kMaxK; i += blockDim.x) info->rho_hist[i] = w.rho_hist[i];
  for (int i = t; i < kMaxMu; i += blockDim.x) info->gcv[i] = w.gcv[i];
}

// Holds the stream until the host has queued a whole kernel group (phase
// timing): one thread polls a flag in mapped host memory.  The wait is
// bounded (limit_ns of globaltimer; phase timing gives 10 s, room for the
// lazy loading of modules on a first launch); on expiry the kernel records
// RTG_ERR_TIMEOUT in *status and returns, so the stream never stalls.
__global__ void k_gate(const volatile unsigned* flag, unsigned want, volatile unsigned* status,
                       unsigned long long limit_ns) {
  unsigned long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (*flag < want) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > limit_ns) {
      *status = RTG_ERR_TIMEOUT;
      return;
    }
    __nanosleep(500);
  }
}

cudaError_t launch_gate(const unsigned* flag, unsigned want, unsigned* status, cudaStream_t s,
                        unsigned long long limit_ns) {
  k_gate<<<1, 1, 0, s>>>(flag, want, status, limit_ns);
  return cudaGetLastError();
}

static unsigned ew_grid(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return static_cast<unsigned>(b < 1 ? 1 : b);
}

cudaError_t launch_tikhonov(const Work& w, const FinishOpts& f, cudaStream_t s, const int* gate) {
  const unsigned blocks = (f.mode == 2) ? static_cast<unsigned>(f.n_mu) : 1u;
  const size_t sm = static_cast<size_t>(tk_scratch_doubles(w.m)) * sizeof(double);
  const int in_smem = sm <= size_t(200) * 1024 ? 1 : 0;
  if (in_smem) {
    cudaError_t e = set_smem(k_tikhonov, sm);
    if (e != cudaSuccess) return e;
  }
  k_tikhonov<<<dim3(blocks, 1, w.b.n), TK_THREADS, in_smem ? sm : 0, s>>>(w, f.desc, f.mode,
                                                                         w.ysel + kMaxMu * w.m, in_smem, gate);
  return cudaGetLastError();
}

// X = X0 + sum_{i<k} y_i V_i with V in BF16 (FP32 arithmetic, 8 values per load);
// X0 after a restart as in k_assemble
__global__ void k_assemble_bf16(Work w0, PtrRef X0r0, PtrRef Xr0, const int* gate) {
  const int64_t bo = bidx(w0.b).off;
  const Work w = w0.at(bo);
  const PtrRef X0r = X0r0.at(bo), Xr = Xr0.at(bo);
  gate = bsh(gate, bo);
  if (gate != nullptr && *gate) return;
  const int k = w.ctl->j;
  __shared__ float ys[kMaxK];
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = static_cast<float>(w.y[i]);
  __syncthreads();
  float* X = Xr.get<float>();
  const float* X0 = w.ctl->cycle > 0 ? X : X0r.get<const float>();
  const uint4* V8 = static_cast<const uint4*>(w.V);
  const int64_t n8 = w.n / 8;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n8;
       o += (int64_t)gridDim.x * blockDim.x) {
    float acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = (X0 != nullptr) ? X0[8 * o + q] : 0.f;
    for (int i = 0; i < k; ++i) {
      const uint4 v = V8[static_cast<int64_t>(i) * n8 + o];
      const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[2 * q] = fmaf(ys[i], __uint_as_float(w4[q] << 16), acc[2 * q]);
        acc[2 * q + 1] = fmaf(ys[i], __uint_as_float(w4[q] & 0xffff0000u), acc[2 * q + 1]);
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) X[8 * o + q] = acc[q];
  }
}

cudaError_t launch_assemble(const Work& w, PtrRef X0, PtrRef X, cudaStream_t s, const int* gate) {
  if (w.vdtype == RTG_BF16) {
    k_assemble_bf16<<<dim3(ew_grid(w.n / 8 + 1), 1, w.b.n), 256, 0, s>>>(w, X0, X, gate);
    return cudaGetLastError();
  }
  if (w.dtype == RTG_F64) k_assemble<double><<<dim3(ew_grid(w.n), 1, w.b.n), 256, 0, s>>>(w, X0, X, gate);
  else k_assemble<float><<<dim3(ew_grid(w.n), 1, w.b.n), 256, 0, s>>>(w, X0, X, gate);
  return cudaGetLastError();
}

// Final residual of the Block GMRES algorithm (Section 4.4, its last steps:
// R_m = C - A *_N X_m and its Theta-norm).  R (in the V_0 slot) and S(R) (in
// Spart) come from the apply and sketch launched before this kernel.  Each
// block sums R.R, C.C (grid-stride over n) and S(R).S(R) (over d) in
// float-float (FP32) or FP64, writes one row of three partial sums, and the
// last block adds the rows in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) k_true_resid(Work w0, PtrRef Cr0) {
  const int64_t bo = bidx(w0.b).off;
  const Work w = w0.at(bo);
  const T* C = Cr0.at(bo).get<const T>();
  const T* R = static_cast<const T*>(w.V);
  const T* SR = static_cast<const T*>(w.Spart);
  __shared__ double red[8][3];
  __shared__ int am_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  DotAcc<T> rr, cc, ss;
  for (int64_t o = t0; o < w.n; o += stride) {
    const T r = R[o], c = C[o];
    rr.add(r, r);
    cc.add(c, c);
  }
  for (int64_t o = t0; o < w.d; o += stride) {
    const T v = SR[o];
    ss.add(v, v);
  }
  const double a = rr.warp_total(), b = cc.warp_total(), c = ss.warp_total();
  if (lane == 0) {
    red[warp][0] = a;
    red[warp][1] = b;
    red[warp][2] = c;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double v = 0.0;
    for (int u = 0; u < 8; ++u) v += red[u][threadIdx.x];
    w.part[static_cast<int64_t>(blockIdx.x) * 3 + threadIdx.x] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) am_last = (ticket_acq_rel(w.counter + 1, gridDim.x - 1) == gridDim.x - 1);
  __syncthreads();
  if (!am_last) return;
  if (warp == 0) {   // lane l sums rows l, l + 32, ...; then a fixed warp tree
    double s3[3] = {0.0, 0.0, 0.0};
    for (unsigned r = lane; r < gridDim.x; r += 32)
      for (int q = 0; q < 3; ++q) s3[q] += __ldcg(w.part + static_cast<int64_t>(r) * 3 + q);
    for (int q = 0; q < 3; ++q) s3[q] = warp_sum(s3[q]);
    if (lane == 0) {
      Ctl* ctl = w.ctl;
      ctl->true_rr = s3[1] > 0.0 ? sqrt(s3[0] / s3[1]) : (s3[0] > 0.0 ? INFINITY : 0.0);
      ctl->true_th = ctl->beta0 > 0.0 ? sqrt(s3[2]) / ctl->beta0 : (s3[2] > 0.0 ? INFINITY : 0.0);
    }
  }
}

cudaError_t launch_true_resid(const Work& w, PtrRef C, cudaStream_t s) {
  // rows of three partial sums must fit the partial-sum buffer
  int64_t blocks = ew_grid(w.n / 4 + 1);
  const int64_t cap = static_cast<int64_t>(w.part_rows) * (2 * w.m + 4) / 3;
  if (blocks > cap) blocks = cap;
  if (blocks > 304) blocks = 304;
  if (blocks < 1) blocks = 1;
  const dim3 g(static_cast<unsigned>(blocks), 1, static_cast<unsigned>(w.b.n));
  if (w.dtype == RTG_F64) k_true_resid<double><<<g, 256, 0, s>>>(w, C);
  else k_true_resid<float><<<g, 256, 0, s>>>(w, C);
  return cudaGetLastError();
}

// Learned warm start: ||S(R_0)|| and ||S(C)|| (float-float sums over the d
// sketch entries, one block), then the decision: fall back to X_0 = 0 with
// GCV when the prediction's sketched residual is not below the cold start's,
// else keep X_0, take lambda = exp(predicted log lambda) and rescale the stop
// level so that both stop at ||S(C - Phi X)|| <= tol ||S(C)||.
__global__ void __launch_bounds__(1024) k_ws_decide(const float* SR, const float* SC, int64_t d,
                                                    const float* loglam, double tol, WsDecision* dec) {
  __shared__ double red[32][2];
  DotAcc<float> r, c;
  for (int64_t i = threadIdx.x; i < d; i += blockDim.x) {
    const float a = SR[i], b = SC[i];
    r.add(a, a);
    c.add(b, b);
  }
  const double rr = r.warp_total(), cc = c.warp_total();
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5][0] = rr;
    red[threadIdx.x >> 5][1] = cc;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double sr = 0.0, sc = 0.0;
  for (int u = 0; u < (int)(blockDim.x >> 5); ++u) {
    sr += red[u][0];
    sc += red[u][1];
  }
  sr = sqrt(sr);
  sc = sqrt(sc);
  const bool warm = isfinite(sr) && sr < sc;
  dec->fell_back = warm ? 0 : 1;
  dec->sC = sc;
  dec->sR = sr;
  if (warm) {
    const double ll = static_cast<double>(*loglam);
    dec->lambda = isfinite(ll) ? exp(fmin(fmax(ll, -40.0), 20.0)) : 1e-3;
    dec->tol = sr > 0.0 ? tol * sc / sr : tol;
  } else {
    dec->lambda = -1.0;
    dec->tol = tol;
  }
}

__global__ void k_ws_zero_if(const WsDecision* dec, float* X, int64_t n) {
  if (!dec->fell_back) return;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x)
    X[o] = 0.f;
}

__global__ void k_ws_write_desc(const WsDecision* dec, SolveDesc* desc) {
  desc->tol = dec->tol;
  desc->lambda = dec->lambda;
}

cudaError_t launch_ws_decide(const float* SR, const float* SC, int64_t d, const float* loglam, double tol,
                             WsDecision* dec, cudaStream_t s) {
  k_ws_decide<<<1, 1024, 0, s>>>(SR, SC, d, loglam, tol, dec);
  return cudaGetLastError();
}

cudaError_t launch_ws_zero_if(const WsDecision* dec, float* X, int64_t n, cudaStream_t s) {
  k_ws_zero_if<<<ew_grid(n), 256, 0, s>>>(dec, X, n);
  return cudaGetLastError();
}

cudaError_t launch_ws_write_desc(const WsDecision* dec, SolveDesc* desc, cudaStream_t s) {
  k_ws_write_desc<<<1, 1, 0, s>>>(dec, desc);
  return cudaGetLastError();
}

// Work queue of a batched solve: a graph branch takes the next problem of
// its class with one atomic increment of the class's counter and copies that
// problem's descriptor into its own, which its kernels read.  With `done`
// set, the branch first returns the info record of the problem it has just
// solved to that problem's place.  The branch's loop condition is 1 while
// the class has problems left, else 0 (the branch then ends).  A nested loop
// condition keeps its value from one pass of the outer loop's body to the
// next, so the solve's own loop condition is set to 1 for the new problem
// (the first problem of a launch starts from the condition's default, 1).
__global__ void k_queue_next(QueueArgs q, int done) {
  __shared__ int next;
  const int cur = *q.cur;
  if (done && cur >= 0) {
    const uint64_t* src = reinterpret_cast<const uint64_t*>(q.my_info);
    uint64_t* dst = reinterpret_cast<uint64_t*>(q.info + cur);
    for (int i = threadIdx.x; i < int(sizeof(InfoDev) / 8); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();   // every thread has read *q.cur
  if (threadIdx.x == 0) {
    const unsigned k = atomicAdd(q.counter, 1u);
    next = k < static_cast<unsigned>(q.n) ? static_cast<int>(k) : -1;
    *q.cur = next;
    cudaGraphSetConditional(static_cast<cudaGraphConditionalHandle>(q.cond), next >= 0 ? 1u : 0u);
    if (next >= 0 && q.use_inner) cudaGraphSetConditional(static_cast<cudaGraphConditionalHandle>(q.inner), 1u);
  }
  __syncthreads();
  if (next >= 0) {
    const uint64_t* src = reinterpret_cast<const uint64_t*>(q.desc + next);
    uint64_t* dst = reinterpret_cast<uint64_t*>(q.my_desc);
    for (int i = threadIdx.x; i < int(sizeof(SolveDesc) / 8); i += blockDim.x) dst[i] = src[i];
  }
}
static_assert(sizeof(SolveDesc) % 8 == 0 && sizeof(InfoDev) % 8 == 0, "records are copied as 8-byte words");

cudaError_t launch_queue_next(const QueueArgs& q, int done, cudaStream_t s) {
  k_queue_next<<<1, 128, 0, s>>>(q, done);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const Work& w, InfoDev* info, cudaStream_t s) {
  k_finalize<<<dim3(1, 1, w.b.n), 256, 0, s>>>(w, info);
  return cudaGetLastError();
}

}  // namespace rtg
