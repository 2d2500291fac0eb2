// Sketched Golub-Kahan bidiagonalisation (Algorithm 4, "Block Golub-Kahan via
// Sketched Einstein Product"): the Theta-norms of its short recurrences and
// the recurrences themselves.  Only norms are sketched, and S is linear, so
//   S(Phi V_j - alpha_j U_j) = S(Phi V_j) - alpha_j S(U_j)
// with S(U_j) kept from the previous step: each norm is one reduction over
// the d sketch entries of the product's sketch.  The lower-bidiagonal
// matrix goes into the Hessenberg storage (alpha_j at (j, j), beta_{j+1}
// at (j+1, j)), so the Givens update, the projected Tikhonov / GCV solve
// and the assembly are the RTG-GMRES kernels.
#include "gs_common.cuh"

namespace rtg {

constexpr int GK_THREADS = 256;
constexpr int GK_ITEMS = 4;

// Blocks of the norm reduction: about 1024 sketch entries each.
static int gk_grid(int64_t d) {
  int64_t g = (d + GK_THREADS * GK_ITEMS - 1) / (GK_THREADS * GK_ITEMS);
  if (g > 1024) g = 1024;
  return static_cast<int>(g < 1 ? 1 : g);
}

// The coefficient of the subtracted vector and its sketch for a phase.
__device__ __forceinline__ double gk_coef(const Work& w, int phase) {
  const Ctl* ctl = w.ctl;
  const int ld = w.m + 1;
  if (phase == 2) {   // alpha_j, j = ctl->j
    const int J = ctl->j;
    return w.H[J + static_cast<int64_t>(ld) * J];
  }
  if (phase == 3) {   // beta_{j+1}, j = ctl->j - 1
    const int J = ctl->j - 1;
    return w.H[J + 1 + static_cast<int64_t>(ld) * J];
  }
  return 0.0;
}

template <typename T>
__global__ void __launch_bounds__(GK_THREADS) k_gk_norm(Work w, int phase, StepOpts o) {
  Ctl* ctl = w.ctl;
  if (ctl->stop) return;
  __shared__ double red[GS_MAXW][kRedCols];
  __shared__ double tot[4];
  __shared__ int am_last;
  const T* S = static_cast<const T*>(w.S);
  const T* q = static_cast<const T*>(w.Q) + (phase == 3 ? w.d : 0);
  const T c = static_cast<T>(gk_coef(w, phase));
  const int64_t d = w.d;
  DotAcc<T> a, b;
  const int64_t chunk = (d + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = (lo + chunk < d) ? lo + chunk : d;
  for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    const T s = S[e];
    const T r = (phase >= 2) ? s - c * q[e] : s;
    a.add(r, r);
    b.add(s, s);
  }
  const double ta = a.warp_total(), tb = b.warp_total();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[warp][0] = ta;
    red[warp][1] = tb;
  }
  __syncthreads();
  const int rowlen = 2 * w.m + 4;
  if (threadIdx.x < 2)
    w.part[static_cast<int64_t>(blockIdx.x) * rowlen + threadIdx.x] =
        warps_total(red, blockDim.x >> 5, threadIdx.x);
  if (!last_block_combine<false>(w, 2, tot, &am_last, &red[0][0])) return;
  if (threadIdx.x != 0) return;
  const double nrm = sqrt(tot[0] > 0.0 ? tot[0] : 0.0);
  const double pre = sqrt(tot[1] > 0.0 ? tot[1] : 0.0);
  const double bd_tol = o.desc_bd_tol ? *o.desc_bd_tol : o.bd_tol;
  const int ld = w.m + 1;
  if (!isfinite(nrm)) {
    ctl->status = RTG_ERR_NONFINITE;
    ctl->stop = 1;
    set_cond(o, 0);
    return;
  }
  if (phase == 0) {            // beta_0 = ||R_0||_Theta
    if (nrm == 0.0) {
      ctl->converged = 1;
      ctl->stop = 1;
    } else {
      ctl->beta = ctl->beta0 = nrm;
      w.g[0] = nrm;
      ctl->rho = 1.0;
      ctl->gk_scale = nrm;
    }
    set_cond(o, !ctl->stop);
  } else if (phase == 1) {     // alpha_0
    if (nrm <= bd_tol * ctl->beta0) {   // Phi^T R_0 = 0: R_0 is orthogonal to the range
      ctl->breakdown = 1;
      ctl->converged = 1;
      ctl->stop = 1;
    } else {
      w.H[0] = nrm;
      ctl->gk_scale = nrm;
    }
    set_cond(o, !ctl->stop);
  } else if (phase == 2) {     // beta_{J+1}: column J of the bidiagonal is complete
    const int J = ctl->j;
    double* Hc = w.H + static_cast<int64_t>(ld) * J;
    for (int i = 0; i < J; ++i) Hc[i] = 0.0;
    for (int i = J + 2; i < ld; ++i) Hc[i] = 0.0;
    const bool breakdown = nrm <= bd_tol * pre;
    Hc[J + 1] = breakdown ? 0.0 : nrm;
    if (breakdown) ctl->breakdown = 1;
    ctl->pre2 = pre * pre;
    ctl->hnext = nrm;
    ctl->gk_scale = nrm;
    ctl->skip_update = breakdown ? 1 : 0;
    ctl->j = J + 1;
    ctl->givens = 1;
  } else {                     // alpha_{J+1}, J = j - 1
    const int J = ctl->j - 1;
    if (nrm <= bd_tol * pre) { // Phi^T U_{J+1} lies in span(V_J): the process ends here
      ctl->breakdown = 1;
      ctl->converged = 1;
      ctl->stop = 1;
      set_cond(o, 0);
    } else {
      if (J + 1 < w.m) w.H[(J + 1) + static_cast<int64_t>(ld) * (J + 1)] = nrm;
      ctl->gk_scale = nrm;
    }
  }
}

// out = (src - c * prev) / scale over n entries (FP32 data as float4),
// and the same recurrence for the sketched vector (FP64 arithmetic).
template <typename T>
__global__ void k_gk_update(Work w, int phase, PtrRef srcr, StepOpts o) {
  Ctl* ctl = w.ctl;
  if (phase == 2 && blockIdx.x == gridDim.x - 1) {   // Givens of column j - 1 beside the update
    givens_step(w, o);
    return;
  }
  if (ctl->stop || ctl->skip_update) return;
  const int nblk = (phase == 2) ? gridDim.x - 1 : gridDim.x;
  const int64_t n = w.n, d = w.d;
  T* V = static_cast<T*>(w.V);
  T* U = static_cast<T*>(w.U);
  T* Qs = static_cast<T*>(w.Q);
  const T* src = nullptr;
  const T* prev = nullptr;
  T* out = nullptr;
  T* q = Qs;   // S(U) in slot 0, S(V) in slot 1
  const int Jn = ctl->j;   // phases 2 and 3: index of the new vector
  if (phase == 0) {
    src = srcr.get<const T>();
    out = U;
  } else if (phase == 1) {
    src = static_cast<const T*>(w.W);
    out = V;
    q = Qs + d;
  } else if (phase == 2) {
    src = static_cast<const T*>(w.W);
    prev = U + static_cast<int64_t>((Jn - 1) % 2) * n;
    out = U + static_cast<int64_t>(Jn % 2) * n;
  } else {
    if (Jn > w.m) return;
    src = static_cast<const T*>(w.W);
    prev = V + static_cast<int64_t>(Jn - 1) * n;
    out = V + static_cast<int64_t>(Jn) * n;
    q = Qs + d;
  }
  // coefficient of prev: alpha_{j-1} (phase 2, stored at (j-1, j-1)) or
  // beta_j (phase 3, stored at (j, j-1)); divisor: the norm just computed
  const int ld = w.m + 1;
  double cprev = 0.0;
  if (phase == 2) cprev = w.H[(Jn - 1) + static_cast<int64_t>(ld) * (Jn - 1)];
  if (phase == 3) cprev = w.H[Jn + static_cast<int64_t>(ld) * (Jn - 1)];
  const double inv = 1.0 / ctl->gk_scale;
  const T ci = static_cast<T>(cprev), si = static_cast<T>(inv);
  const int64_t stride = static_cast<int64_t>(nblk) * blockDim.x;
  const int64_t t0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (sizeof(T) == 4 && (n % 4) == 0 && (reinterpret_cast<uintptr_t>(src) % 16) == 0) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    const float4* p4 = reinterpret_cast<const float4*>(prev);
    float4* o4 = reinterpret_cast<float4*>(out);
    const float cf = static_cast<float>(ci), sf = static_cast<float>(si);
    for (int64_t e = t0; e < n / 4; e += stride) {
      float4 v = s4[e];
      if (p4 != nullptr) {
        const float4 p = p4[e];
        v.x -= cf * p.x; v.y -= cf * p.y; v.z -= cf * p.z; v.w -= cf * p.w;
      }
      v.x *= sf; v.y *= sf; v.z *= sf; v.w *= sf;
      o4[e] = v;
    }
  } else {
    for (int64_t e = t0; e < n; e += stride) {
      T v = src[e];
      if (prev != nullptr) v -= ci * prev[e];
      out[e] = v * si;
    }
  }
  const T* S = static_cast<const T*>(w.S);
  for (int64_t e = t0; e < d; e += stride) {
    double v = static_cast<double>(S[e]);
    if (phase >= 2) v -= cprev * static_cast<double>(q[e]);
    q[e] = static_cast<T>(v * inv);
  }
}

static unsigned gk_ew_grid(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return static_cast<unsigned>(b < 1 ? 1 : b);
}

cudaError_t launch_gk_norm(const Work& w, int phase, const StepOpts& o, cudaStream_t s) {
  const int g = gk_grid(w.d);
  if (w.dtype == RTG_F64) k_gk_norm<double><<<g, GK_THREADS, 0, s>>>(w, phase, o);
  else k_gk_norm<float><<<g, GK_THREADS, 0, s>>>(w, phase, o);
  return cudaGetLastError();
}

cudaError_t launch_gk_update(const Work& w, int phase, PtrRef src, const StepOpts& o, cudaStream_t s) {
  const unsigned extra = (phase == 2) ? 1u : 0u;   // the Givens block
  if (w.dtype == RTG_F64)
    k_gk_update<double><<<gk_ew_grid(w.n) + extra, 256, 0, s>>>(w, phase, src, o);
  else
    k_gk_update<float><<<gk_ew_grid(w.n / 4 + 1) + extra, 256, 0, s>>>(w, phase, src, o);
  return cudaGetLastError();
}

}  // namespace rtg
