// Device helpers shared by the kernels that finish a sketched Gram-Schmidt
// reduction (the sketch kernel fuses the first pass; k_arnoldi.cu holds
// the others): block partial dot products with the stored sketched basis,
// the last-block combine, the Givens update of Eq. 11S and the scalar
// epilogue of each pass (Section 4.3; the Block GMRES algorithm's steps).
#pragma once

#include <type_traits>

#include "rtg_internal.cuh"

namespace rtg {

constexpr int GS_MAXW = 8;   // warps per block of the reducing kernels (256 threads)
constexpr int kRedCols = 2 * kMaxK + 4;   // columns of one reduction (see gs_ncols)
// Gram matrices of up to this many rows are staged in shared memory by the
// step finish (rows of gram_smem_ld(r) <= r + 2 doubles; it needs
// (kMaxK + 6) + r (r + 2) + GS_MAXW r + 4 doubles of scratch)
constexpr int kGramSmemRows = 56;
static_assert((kMaxK + 6) + kGramSmemRows * (kGramSmemRows + 2) + GS_MAXW * kGramSmemRows + 4 <=
                  GS_MAXW * kRedCols,
              "Gram staging must fit the reduction scratch");
// row stride of the staged n x n Gram matrix: even, so that 16-byte copies
// land on 16-byte boundaries
__device__ __forceinline__ int gram_smem_ld(int n) { return (n + 2) & ~1; }

template <typename A>
__device__ __forceinline__ A warp_sum(A v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Last-block ticket: an atomic increment (wrapping to zero after `last`)
// with acquire-release semantics at GPU scope.  The barrier before it makes
// the block's writes (its partial row) precede the release; the barrier
// after it orders the last block's reads after the acquire.  Cheaper than
// two full fences around a relaxed atomic.
__device__ __forceinline__ unsigned ticket_acq_rel(unsigned* counter, unsigned last) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.inc.u32 %0, [%1], %2;" : "=r"(old) : "l"(counter), "r"(last) : "memory");
  return old;
}

// Condition of the device-side loop.  A lock-step batch (o.group_left set)
// keeps looping while any of its problems runs: each problem's stop is
// counted once, and the count reaching zero ends the loop.
// (The count is kept on direct launches too: the host reads it per step.)
__device__ __forceinline__ void set_cond(const StepOpts& o, int keep_going, Ctl* ctl = nullptr) {
  const cudaGraphConditionalHandle h = static_cast<cudaGraphConditionalHandle>(o.cond);
  if (o.group_left == nullptr) {
    if (o.use_cond) cudaGraphSetConditional(h, keep_going ? 1u : 0u);
    return;
  }
  if (!keep_going && ctl != nullptr && atomicExch(&ctl->counted, 1) == 0 && atomicSub(o.group_left, 1u) == 1u &&
      o.use_cond)
    cudaGraphSetConditional(h, 0u);
}

// Double-float ("float-float") accumulation for FP32 data: the FP64 pipe
// of this GPU runs at 1/64 of the FP32 rate with a long dependent latency,
// so sums of products of FP32 values are kept as unevaluated pairs
// hi + lo of floats with error-free transformations (exact product by
// FMA, Knuth's two-sum), about 48 significant bits.  IEEE intrinsics keep
// the compiler from contracting or reassociating them.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ FF ff_add(FF x, FF y) {
  const FF s = ff_two_sum(x.hi, y.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return ff_two_sum(s.hi, e);
}
// Sum of two pairs inside a reduction: the two-sum of the high parts is
// exact and the low parts are added in FP32, without renormalising the
// result (the pair still stands for hi + lo; every reduction here ends in
// a conversion to double, which needs no normalised pair).  8 FP32
// operations instead of ff_add's 14.
__device__ __forceinline__ FF ff_add_lazy(FF x, FF y) {
  const FF s = ff_two_sum(x.hi, y.hi);
  return {s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo))};
}
__device__ __forceinline__ FF ff_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ FF ff_warp_sum(FF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    FF w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = ff_add_lazy(v, w);
  }
  return v;
}
__device__ __forceinline__ double ff_to_double(FF v) {
  return static_cast<double>(v.hi) + static_cast<double>(v.lo);
}

// Dot-product accumulator: float-float for FP32 data, FP64 for FP64 data.
template <typename T>
struct DotAcc;
template <>
struct DotAcc<float> {
  FF v{0.f, 0.f};
  __device__ __forceinline__ void add(float a, float b) { v = ff_add_lazy(v, ff_prod(a, b)); }
  __device__ __forceinline__ double warp_total() { return ff_to_double(ff_warp_sum(v)); }
};
template <>
struct DotAcc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double a, double b) { v = fma(a, b, v); }
  __device__ __forceinline__ double warp_total() { return warp_sum(v); }
};

// Columns of the per-block partial sums of one Gram-Schmidt reduction:
// [0, J] s . Q_i, [J+1] s . s, [J+2, 2J+2] Q_J . Q_i (the new row of the
// Gram matrix G = Q^T Q).  The start of a process (J = -1) has only s . s.
__device__ __forceinline__ int gs_ncols(int J) { return J < 0 ? 1 : 2 * J + 3; }

// Reduce-scatter of 32 float-float values across a warp: in five halving
// rounds each lane keeps one half of its values and hands the other half
// to its partner, adding what it receives; afterwards v[0] of lane l is the
// warp total of value l.  31 exchanges per lane instead of 32 x 5 for 32
// separate warp sums, and the adds of a round are independent.  The tree
// is fixed, so the sums are deterministic.
__device__ __forceinline__ void ff_reduce_scatter32(FF (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const int half = 16 >> r;          // also the partner's lane offset
    const bool up = (lane & half) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const FF give = up ? v[k] : v[k + half];
      const FF keep = up ? v[k + half] : v[k];
      FF got;
      got.hi = __shfl_xor_sync(0xffffffffu, give.hi, half);
      got.lo = __shfl_xor_sync(0xffffffffu, give.lo, half);
      v[k] = ff_add_lazy(keep, got);
    }
  }
}

// The same for NV = 2, 4, ..., 32 values: log2(NV) halving rounds inside
// aligned groups of NV lanes, then butterfly sums across the groups;
// afterwards v[0] of lane l is the warp total of value l % NV.
template <int NV>
__device__ __forceinline__ void ff_reduce_scatter(FF (&v)[NV]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int half = NV / 2; half >= 1; half >>= 1) {
    const bool up = (lane & half) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const FF give = up ? v[k] : v[k + half];
      const FF keep = up ? v[k + half] : v[k];
      FF got;
      got.hi = __shfl_xor_sync(0xffffffffu, give.hi, half);
      got.lo = __shfl_xor_sync(0xffffffffu, give.lo, half);
      v[k] = ff_add_lazy(keep, got);
    }
  }
#pragma unroll
  for (int o = NV; o < 32; o <<= 1) {
    FF got;
    got.hi = __shfl_xor_sync(0xffffffffu, v[0].hi, o);
    got.lo = __shfl_xor_sync(0xffffffffu, v[0].lo, o);
    v[0] = ff_add_lazy(v[0], got);
  }
}

// One group of W columns i0 .. i0 + W - 1 (those <= J) of the FP32 partial
// sums: s . Q_i and Q_J . Q_i over this thread's ITEMS entries, reduced
// across the warp by one reduce-scatter of 2 W float-float values; lane
// l < 2 W writes column i0 + l % W of its warp's row (s . Q_i for l < W).
template <int W, int ITEMS>
__device__ __forceinline__ void ff_dot_group(const float* Q, int64_t d, const float (&sv)[ITEMS],
                                             const float (&qJ)[ITEMS], const int64_t* idx, int cnt, int i0, int J,
                                             FF (*rf)[kRedCols], int warp, int lane) {
  float qv[W][ITEMS];
#pragma unroll
  for (int g = 0; g < W; ++g)
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const bool ok = k < cnt && idx[k] >= 0 && i0 + g <= J;
      qv[g][k] = ok ? Q[static_cast<int64_t>(i0 + g) * d + idx[k]] : 0.f;
    }
  FF v[2 * W];
#pragma unroll
  for (int g = 0; g < W; ++g) {
    // the first product starts the pair (an exact product is already a
    // normalised pair, so adding it to zero would change nothing)
    FF p = ff_prod(sv[0], qv[g][0]), q = ff_prod(qJ[0], qv[g][0]);
#pragma unroll
    for (int k = 1; k < ITEMS; ++k) {
      p = ff_add_lazy(p, ff_prod(sv[k], qv[g][k]));
      q = ff_add_lazy(q, ff_prod(qJ[k], qv[g][k]));
    }
    v[g] = p;
    v[W + g] = q;
  }
  ff_reduce_scatter<2 * W>(v);
  if (lane < 2 * W) {
    const int g = lane % W;
    if (i0 + g <= J) rf[warp][lane < W ? i0 + g : J + 2 + i0 + g] = v[0];
  }
}

// Sum of the per-warp values of one column in a fixed order.
__device__ __forceinline__ double warps_total(const double (*red)[kRedCols], int nw, int i) {
  if (nw == 8)
    return ((red[0][i] + red[1][i]) + (red[2][i] + red[3][i])) +
           ((red[4][i] + red[5][i]) + (red[6][i] + red[7][i]));
  double acc = 0.0;
  for (int u = 0; u < nw; ++u) acc += red[u][i];
  return acc;
}

// Sum of the per-warp float-float values of one column in a fixed order.
__device__ __forceinline__ FF ff_warps_total(const FF (*red)[kRedCols], int nw, int i) {
  if (nw == 8)
    return ff_add_lazy(ff_add_lazy(ff_add_lazy(red[0][i], red[1][i]), ff_add_lazy(red[2][i], red[3][i])),
                       ff_add_lazy(ff_add_lazy(red[4][i], red[5][i]), ff_add_lazy(red[6][i], red[7][i])));
  FF acc{0.f, 0.f};
  for (int u = 0; u < nw; ++u) acc = ff_add_lazy(acc, red[u][i]);
  return acc;
}

// Per-block partial sums of the columns above: products of the stored
// values accumulated in double-float (FP32 data) or FP64 (FP64 data).
// Each thread passes up to ITEMS entries (vals at sketch indices idx);
// entries past cnt or with a negative index are ignored.  Writes row
// (linear block id) of w.part: float-float pairs for FP32 data (summed by
// last_block_combine<true> on the FP32 pipe), doubles for FP64 data.
// red: shared [GS_MAXW][kRedCols] doubles (float-float pairs for FP32).
template <typename T, int ITEMS>
__device__ void block_partials(const Work& w, const T* vals, const int64_t* idx, int cnt, int J,
                               double (*red)[kRedCols]) {
  const T* Q = static_cast<const T*>(w.Q);
  const int64_t d = w.d;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int ncols = gs_ncols(J);
  T sv[ITEMS], qJ[ITEMS];
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const bool ok = k < cnt && idx[k] >= 0;
    sv[k] = ok ? vals[k] : static_cast<T>(0);
    qJ[k] = (ok && J >= 0) ? Q[static_cast<int64_t>(J) * d + idx[k]] : static_cast<T>(0);
  }
  FF (*rf)[kRedCols] = reinterpret_cast<FF (*)[kRedCols]>(red);
  {   // s . s
    DotAcc<T> a;
    if constexpr (sizeof(T) == 4) a.v = ff_prod(sv[0], sv[0]);
    else a.add(sv[0], sv[0]);
#pragma unroll
    for (int k = 1; k < ITEMS; ++k) a.add(sv[k], sv[k]);
    if constexpr (sizeof(T) == 4) {
      const FF t = ff_warp_sum(a.v);
      if (lane == 0) rf[warp][J + 1] = t;
    } else {
      const double t = a.warp_total();
      if (lane == 0) red[warp][J + 1] = t;
    }
  }
  if constexpr (sizeof(T) == 4) {
    // 16 columns of Q at a time (the last group only as wide as it needs,
    // rounded up to a power of two): s . Q_i and Q_J . Q_i for each
    for (int i0 = 0; i0 <= J; i0 += 16) {
      const int nv = J + 1 - i0;
      if (nv > 8) ff_dot_group<16, ITEMS>(Q, d, sv, qJ, idx, cnt, i0, J, rf, warp, lane);
      else if (nv > 4) ff_dot_group<8, ITEMS>(Q, d, sv, qJ, idx, cnt, i0, J, rf, warp, lane);
      else if (nv > 2) ff_dot_group<4, ITEMS>(Q, d, sv, qJ, idx, cnt, i0, J, rf, warp, lane);
      else if (nv > 1) ff_dot_group<2, ITEMS>(Q, d, sv, qJ, idx, cnt, i0, J, rf, warp, lane);
      else ff_dot_group<1, ITEMS>(Q, d, sv, qJ, idx, cnt, i0, J, rf, warp, lane);
    }
  } else {
    // columns of Q in groups of 8: all loads of a group go out before any use
    constexpr int GRP = 8;
    for (int i0 = 0; i0 <= J; i0 += GRP) {
      T qv[GRP][ITEMS];
#pragma unroll
      for (int g = 0; g < GRP; ++g)
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
          const bool ok = k < cnt && idx[k] >= 0 && i0 + g <= J;
          qv[g][k] = ok ? Q[static_cast<int64_t>(i0 + g) * d + idx[k]] : static_cast<T>(0);
        }
#pragma unroll
      for (int g = 0; g < GRP; ++g) {
        if (i0 + g > J) break;
        DotAcc<T> p, q;
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
          p.add(sv[k], qv[g][k]);
          q.add(qJ[k], qv[g][k]);
        }
        const double tp = p.warp_total(), tq = q.warp_total();
        if (lane == 0) {
          red[warp][i0 + g] = tp;
          red[warp][J + 2 + i0 + g] = tq;
        }
      }
    }
  }
  __syncthreads();
  const int rowlen = 2 * w.m + 4;
  const int64_t row = static_cast<int64_t>(blockIdx.x + gridDim.x * blockIdx.y) * rowlen;
  for (int i = threadIdx.x; i < ncols; i += blockDim.x) {
    if constexpr (sizeof(T) == 4) reinterpret_cast<FF*>(w.part)[row + i] = ff_warps_total(rf, nw, i);
    else w.part[row + i] = warps_total(red, nw, i);
  }
}

// Ticket: returns true in every thread of the last block to finish, after
// tot[0..ncols) holds the sum of all blocks' rows.  Thread t takes column
// t % nc and every G-th row starting at t / nc, sixteen rows per round of
// loads, then one thread per column adds the G group sums in a pairwise
// tree.  FFROWS: the rows hold float-float pairs, summed with float-float
// adds on the FP32 pipe (an FP64 add occupies its SM sub-partition's FP64
// unit for about 64 cycles on this GPU; the pairs already carry the
// partial sums' precision); else doubles.  The order is fixed, so the
// result is deterministic.  The counter wraps back to zero by itself.
// scratch: >= blockDim doubles.  pre (optional): called by every thread of
// the last block right after the ticket, before its loads, e.g. to start
// asynchronous copies that the caller needs after the combine.
template <bool FFROWS, typename Pre = void (*)()>
__device__ inline bool last_block_combine(const Work& w, int ncols, double* tot, int* am_last,
                                          double* scratch, Pre pre = nullptr) {
  using V = typename std::conditional<FFROWS, FF, double>::type;
  __syncthreads();
  const unsigned nblk = gridDim.x * gridDim.y;
  if (threadIdx.x == 0) *am_last = (ticket_acq_rel(w.counter, nblk - 1) == nblk - 1);
  __syncthreads();
  if (!*am_last) return false;
  if constexpr (!std::is_same<Pre, void (*)()>::value) pre();   // e.g. start the Gram staging copies
  auto add = [](V x, V y) -> V {
    if constexpr (FFROWS) return ff_add_lazy(x, y);
    else return x + y;
  };
  auto load = [](const V* q) -> V {
    if constexpr (FFROWS) {
      const float2 f = __ldcg(reinterpret_cast<const float2*>(q));
      return FF{f.x, f.y};
    } else {
      return __ldcg(q);
    }
  };
  const V zero{};
  V* sc = reinterpret_cast<V*>(scratch);
  const int rowlen = 2 * w.m + 4;
  const int nt = blockDim.x;
  for (int c0 = 0; c0 < ncols; c0 += nt) {
    const int nc = (ncols - c0 < nt) ? ncols - c0 : nt;
    int G = nt / nc;
    if (G > 32) G = 32;
    const int t = threadIdx.x;
    const int c = t % nc, g = t / nc;
    if (g < G) {
      // rows g, g + G, ...: sixteen loads in flight per round (one L2
      // round trip per sixteen rows), summed in a fixed tree
      constexpr int U = 16;
      V acc = zero;
      const V* p = reinterpret_cast<const V*>(w.part) + c0 + c;
      for (unsigned b = g; b < nblk; b += U * G) {
        V v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const unsigned bb = b + u * G;
          v[u] = bb < nblk ? load(p + static_cast<int64_t>(bb) * rowlen) : zero;
        }
#pragma unroll
        for (int h = U / 2; h > 0; h >>= 1)
#pragma unroll
          for (int u = 0; u < h; ++u) v[u] = add(v[u], v[u + h]);
        acc = add(acc, v[0]);
      }
      sc[g * nc + c] = acc;
    }
    __syncthreads();
    if (t < nc) {   // pairwise tree over the G group sums (levels that would add only zeros skipped)
      V v[32];
#pragma unroll
      for (int u = 0; u < 32; ++u) v[u] = u < G ? sc[u * nc + t] : zero;
#pragma unroll
      for (int h = 16; h > 0; h >>= 1)
        if (h < G) {
#pragma unroll
          for (int u = 0; u < h; ++u) v[u] = add(v[u], v[u + h]);
        }
      if constexpr (FFROWS) tot[c0 + t] = ff_to_double(v[0]);
      else tot[c0 + t] = v[0];
    }
    __syncthreads();
  }
  return true;
}

// Start of a process (one thread): beta = ||R_0||_Theta = sqrt(s . s).
__device__ inline void gs_finish_start(const Work& w, const StepOpts& o, const double* tot) {
  Ctl* ctl = w.ctl;
  const double tol = o.desc_tol ? *o.desc_tol : o.tol;
  const double beta = sqrt(tot[0]);
  if (ctl->status != 0) {
    ctl->stop = 1;
  } else if (!isfinite(beta)) {
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
    if (ctl->rho <= tol) {   // (a warm start or a restart may already meet the stop level)
      ctl->converged = 1;
      ctl->stop = 1;
    }
    if (w.m == 0) ctl->stop = 1;
  }
  set_cond(o, !ctl->stop, ctl);
}

// Starts the asynchronous copies of the stored Gram matrix rows and columns
// 0..J-1 into the finish's shared staging area, so that they travel while
// the last block combines the partial rows; the finish called with
// staged = true waits for them.  Only where the finish stages G
// (J + 1 <= kGramSmemRows).  G is symmetric, so column k of G (contiguous
// in global memory) is copied to row k of the staging area, in 16-byte
// copies that bypass L1 (cp.async.cg): G's addresses are rewritten with
// other values by every cycle and every solve of the plan, and only L2 is
// coherent across the SMs that run successive finishes.  When J is odd the
// last pair of a column also brings G(J, k), which the finish overwrites
// with the new row.  sh: the finish's scratch, whose staging area starts
// after kMaxK + 6 doubles (past the combine's scratch, 16-byte aligned).
__device__ inline void gs_stage_gram_async(const Work& w, int J, double* sh) {
  const int n = J + 1;
  if (J < 1 || n > kGramSmemRows) return;
  const int lg = gram_smem_ld(n), ldg = gram_ld(w.m), pairs = (J + 1) / 2;
  double* Gs = sh + (kMaxK + 2) + 4;
  for (int e = threadIdx.x; e < J * pairs; e += blockDim.x) {
    const int p = e % pairs, k = e / pairs;
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(&Gs[k * lg + 2 * p]));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa),
                 "l"(w.G + static_cast<int64_t>(ldg) * k + 2 * p)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Step finish from one reduction (every thread of the last block).
// Classical Gram-Schmidt with one re-orthogonalisation pass, written with
// the Gram matrix G = Q^T Q of the stored sketched basis so that a single
// pass over Q suffices: h1 = Q^T s, h2 = Q^T (s - Q h1) = h1 - G h1,
// h = h1 + h2 and h_{j+1,j}^2 = ||s - Q h||^2 = s.s - 2 h.h1 + h.(G h), all
// in FP64.  Writes the Hessenberg column, h_{j+1,j} (0 on breakdown), the
// breakdown and non-finite flags, and advances j.  The Givens update of
// Eq. 11S, rho_j and the stop rule follow in givens_step, off this
// kernel's critical path.  Up to kGramSmemRows rows the Gram matrix is
// staged in shared memory and every warp takes part in the two products
// with it; beyond, one warp per row reads it from global memory.  sh:
// shared scratch of GS_MAXW * kRedCols doubles, 256 threads.
__device__ inline void gs_finish_gram(const Work& w, const StepOpts& o, const double* tot, double* sh,
                                      bool staged = false) {
  Ctl* ctl = w.ctl;
  const int J = ctl->j;
  const int ld = w.m + 1, ldg = gram_ld(w.m);
  const double bd_tol = o.desc_bd_tol ? *o.desc_bd_tol : o.bd_tol;   // loaded early, used at the end
  const double* h1 = tot;
  const double s2 = tot[J + 1];
  const double* grow = tot + J + 2;
  double* col = sh;                    // h
  double* red = col + (kMaxK + 2);     // a = h.h1, b = h.(G h)
  double* G = w.G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n = J + 1;
  if (n <= kGramSmemRows) {
    // G staged in shared memory (even row stride); each product G x runs
    // on every warp: warp w takes a slice of the columns, lane the rows
    // lane and lane + 32, and the warps' partial rows are summed in order
    const int lg = gram_smem_ld(n);
    double* Gs = red + 4;              // n x n
    double* pr = Gs + n * lg;          // [nw][n] partial products
    double* ab = pr + nw * n;          // [2][2] the two warps' sums of a and b
    if (staged) {   // rows and columns < J arrived by gs_stage_gram_async; J from the new row
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        Gs[J * lg + i] = grow[i];
        Gs[i * lg + J] = grow[i];
      }
    } else
    for (int e0 = 0; e0 < n * n; e0 += 8 * static_cast<int>(blockDim.x)) {   // eight loads in flight
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * blockDim.x + threadIdx.x;
        const int i = e % n, k = e / n;
        v[u] = (e >= n * n) ? 0.0 : (i == J) ? grow[k] : (k == J ? grow[i] : __ldcg(G + i + static_cast<int64_t>(ldg) * k));
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * blockDim.x + threadIdx.x;
        if (e < n * n) Gs[(e % n) * lg + e / n] = v[u];
      }
    }
    for (int i = threadIdx.x; i <= J; i += blockDim.x) {   // new row/column, for later steps
      G[i + static_cast<int64_t>(ldg) * J] = grow[i];
      G[J + static_cast<int64_t>(ldg) * i] = grow[i];
    }
    __syncthreads();
    const int ks = (n + nw - 1) / nw;
    const int k0 = warp * ks, k1 = (k0 + ks < n) ? k0 + ks : n;
    auto gmul = [&](const double* x) {   // pr[w][i] = sum over the warp's columns of G(i, k) x_k
      for (int i = lane; i < n; i += 32) {
        double u = 0.0;
        for (int k = k0; k < k1; ++k) u = fma(Gs[i * lg + k], x[k], u);
        pr[warp * n + i] = u;
      }
    };
    gmul(h1);
    __syncthreads();
    // sums of the warps' partial rows as a fixed tree (FP64 adds have a
    // long dependent latency on this GPU)
    auto wsum = [&](int i) {
      if (nw == 8)
        return ((pr[i] + pr[n + i]) + (pr[2 * n + i] + pr[3 * n + i])) +
               ((pr[4 * n + i] + pr[5 * n + i]) + (pr[6 * n + i] + pr[7 * n + i]));
      double u = 0.0;
      for (int v = 0; v < nw; ++v) u += pr[v * n + i];
      return u;
    };
    for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = 2.0 * h1[i] - wsum(i);
    __syncthreads();
    gmul(col);
    __syncthreads();
    if (warp < 4) {   // a = h . h1 (warps 0, 1), b = h . (G h) (warps 2, 3) over the n <= 64 rows
      // the FP64 products are split exactly into float pairs and summed by a
      // float-float warp tree on the FP32 pipe (a tree of FP64 shuffles and
      // adds is several times slower on this GPU)
      const int i = threadIdx.x & 63, which = warp >> 1;
      double p = 0.0;
      if (i < n) p = which == 0 ? col[i] * h1[i] : col[i] * wsum(i);
      const float hi = __double2float_rn(p);
      FF v{hi, __double2float_rn(p - static_cast<double>(hi))};
      v = ff_warp_sum(v);
      if (lane == 0) ab[warp] = ff_to_double(v);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      red[0] = ab[0] + ab[1];
      red[1] = ab[2] + ab[3];
    }
  } else {
    for (int i = threadIdx.x; i <= J; i += blockDim.x) {
      G[i + static_cast<int64_t>(ldg) * J] = grow[i];
      G[J + static_cast<int64_t>(ldg) * i] = grow[i];
    }
    __syncthreads();
    // h = 2 h1 - G h1: one warp per row, lanes across the columns
    for (int i = warp; i <= J; i += nw) {
      double gh = 0.0;
      for (int k = lane; k <= J; k += 32) gh += __ldcg(G + i + static_cast<int64_t>(ldg) * k) * h1[k];
      gh = warp_sum(gh);
      if (lane == 0) col[i] = 2.0 * h1[i] - gh;
    }
    __syncthreads();
    double* hgh_row = red + 4;         // (G h)_i * h_i per row
    for (int i = warp; i <= J; i += nw) {
      double gh = 0.0;
      for (int k = lane; k <= J; k += 32) gh += __ldcg(G + i + static_cast<int64_t>(ldg) * k) * col[k];
      gh = warp_sum(gh);
      if (lane == 0) hgh_row[i] = gh * col[i];
    }
    __syncthreads();
    if (warp == 0) {
      double a = 0.0, b = 0.0;
      for (int i = lane; i <= J; i += 32) {
        a += col[i] * h1[i];
        b += hgh_row[i];
      }
      a = warp_sum(a);
      b = warp_sum(b);
      if (lane == 0) {
        red[0] = a;
        red[1] = b;
      }
    }
  }
  __syncthreads();
  double* Hc = w.H + static_cast<int64_t>(ld) * J;
  int bad = 0;
  for (int i = threadIdx.x; i <= J; i += blockDim.x) {
    Hc[i] = col[i];
    bad |= !isfinite(col[i]);
  }
  for (int i = J + 2 + threadIdx.x; i < ld; i += blockDim.x) Hc[i] = 0.0;
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    const double hh1 = red[0], hgh = red[1];
    const bool finite = isfinite(s2) && isfinite(hh1) && isfinite(hgh) && !bad;
    const double hn2 = s2 - 2.0 * hh1 + hgh;
    const double hn2p = hn2 > 0.0 ? hn2 : 0.0;
    const double hn = sqrt(hn2p);
    // h_{j+1,j} <= bd_tol ||S(Phi V_j)||, compared in squares (one square root fewer)
    const bool breakdown = finite && (hn2p <= bd_tol * bd_tol * s2);
    Hc[J + 1] = breakdown ? 0.0 : hn;
    ctl->pre2 = s2;
    ctl->hnext = hn;
    ctl->j = J + 1;
    if (!finite) ctl->status = RTG_ERR_NONFINITE;
    if (breakdown) ctl->breakdown = 1;
    ctl->skip_update = (!finite || breakdown) ? 1 : 0;
    ctl->givens = 1;
  }
}

// Givens update of Eq. 11S for the Hessenberg column the last finish wrote
// (column J = j - 1), rho_j = |g_{J+1}| / beta_0, the stop rule and the
// condition of the device-side loop, which never runs more than m + 1
// bodies.  Called by every thread of one block, which runs beside the basis
// update (it does not depend on it): the block stages the column and the
// stored rotations in shared memory with one round of loads, then one
// thread applies the rotations (a dependent FP64 chain).
__device__ inline void givens_step(const Work& w, const StepOpts& o) {
  __shared__ double gv_h[kMaxK + 2], gv_c[kMaxK], gv_s[kMaxK];
  __shared__ int gv_J, gv_do;
  Ctl* ctl = w.ctl;
  if (threadIdx.x == 0) {
    gv_do = ctl->givens;
    gv_J = ctl->j - 1;
  }
  __syncthreads();
  const int ld = w.m + 1;
  if (gv_do) {
    const int J = gv_J;
    const double* Hc = w.H + static_cast<int64_t>(ld) * J;
    for (int i = threadIdx.x; i <= J + 1; i += blockDim.x) gv_h[i] = Hc[i];
    for (int i = threadIdx.x; i < J; i += blockDim.x) {
      gv_c[i] = w.cs[i];
      gv_s[i] = w.sn[i];
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  if (gv_do) {
    ctl->givens = 0;
    const int J = gv_J;
    const double tol = o.desc_tol ? *o.desc_tol : o.tol;
    double* Rc = w.R + static_cast<int64_t>(ld) * J;
    // rotations 0..J-1 on the new column, then the new rotation
    double x = gv_h[0];
    for (int i = 0; i < J; ++i) {
      const double y = gv_h[i + 1], c = gv_c[i], sv = gv_s[i];
      Rc[i] = c * x + sv * y;
      x = -sv * x + c * y;
    }
    const double y = gv_h[J + 1];
    const double den = hypot(x, y);
    double c = 1.0, sv = 0.0;
    if (den != 0.0) {
      c = x / den;
      sv = y / den;
    }
    Rc[J] = den;
    Rc[J + 1] = 0.0;
    w.cs[J] = c;
    w.sn[J] = sv;
    const double gJ = w.g[J];
    w.g[J + 1] = -sv * gJ;
    w.g[J] = c * gJ;
    const double rho = fabs(sv * gJ) / ctl->beta0;
    ctl->rho = rho;
    w.rho_hist[ctl->iters_total] = rho;
    ctl->iters_total += 1;
    const bool finite = ctl->status != RTG_ERR_NONFINITE && isfinite(rho);
    if (!finite && ctl->status == 0) ctl->status = RTG_ERR_NONFINITE;
    const bool breakdown = ctl->breakdown != 0;
    const bool conv = finite && rho <= tol;
    if (conv || breakdown) ctl->converged = 1;
    // a nonzero status (a bounded wait that gave up upstream) ends the solve
    if (!finite || breakdown || conv || ctl->status != 0) {
      ctl->stop = 1;
    } else if (J + 1 >= w.m) {
      // end of a cycle: restart from the least-squares iterate while cycles
      // remain (the body's restart kernels run when rs_skip is 0), else stop
      if (ctl->cycle + 1 < w.cycles) {
        ctl->rs_skip = 0;
        if (o.use_rs_cond) cudaGraphSetConditional(static_cast<cudaGraphConditionalHandle>(o.rs_cond), 1u);
      } else {
        ctl->stop = 1;
      }
    }
  }
  // the body runs at most m times per cycle
  const int loops = ++ctl->loops;
  const int cap = w.m * w.cycles;
  if (loops > cap) {
    ctl->stop = 1;
    ctl->rs_skip = 1;
    if (o.use_cond && loops > cap + 1 && ctl->status == 0) ctl->status = RTG_ERR_TIMEOUT;
  }
  set_cond(o, !ctl->stop, ctl);
}

}  // namespace rtg
