// Sketched global Arnoldi step (Section 4.3; algorithm "Block GMRES via
// Sketched Einstein Product"): Gram-Schmidt in the sketch space against the
// stored sketched basis Q = [S(V_0) .. S(V_j)], the full-space basis update,
// and the Givens update of the Hessenberg least-squares residual (Eq. 11S).
//
// The paper orthogonalises with modified Gram-Schmidt, recomputing the
// sketch of W after every subtraction.  Because S is linear,
// S(W - h V_i) = S(W) - h S(V_i), so the whole process can run on the
// sketch s = S(Phi V_j): classical Gram-Schmidt with one
// re-orthogonalisation pass, equal to MGS in exact arithmetic.  The second
// pass is taken through the Gram matrix G = Q^T Q of the stored sketches
// (kept one row per step): h2 = Q^T (s - Q h1) = h1 - G h1, so one
// reduction over Q per step gives h = h1 + h2 and
// h_{j+1,j}^2 = ||s - Q h||^2 = s.s - 2 h.h1 + h.G h, all in FP64.  The
// update then applies h once:
//   V_{j+1} = (W - sum_i h_i V_i) / h_{j+1,j},  Q_{j+1} = (s - Q h) / h_{j+1,j}.
//
// Reductions: each CTA reduces its slice (data-type partials, warp
// shuffles, FP64 across warps) into a row of `part`; the last CTA to finish
// (atomic ticket) sums the rows in FP64 and runs the scalar epilogue.
// Nothing waits on another CTA.
#include <cuda_bf16.h>

#include "gs_common.cuh"
#include "tma_common.cuh"

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

// pass 0: start of the process, beta = ||S|| with S summed from the
// chain's partial sketches; pass 1: one Arnoldi step's Gram-Schmidt
// reduction on S (s . Q_i, s . s and the new Gram row) and its finish.
template <typename T>
__global__ void __launch_bounds__(GS_THREADS) k_gs_pass(Work w0, int pass, StepOpts o0, const int* gate) {
  const int64_t bo = bidx(w0.b).off;
  const Work w = w0.at(bo);
  const StepOpts o = o0.at(bo);
  Ctl* ctl = w.ctl;
  gate = bsh(gate, bo);
  if (gate != nullptr && *gate) return;
  if (ctl->stop) return;
  const int J = (pass == 0) ? -1 : ctl->j;
  const int d = w.d;
  T* S = static_cast<T*>(w.S);
  __shared__ double red[GS_MAXW][kRedCols];
  __shared__ double tot[kRedCols];
  __shared__ int am_last;
  const int64_t chunk = (d + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = (lo + chunk < d) ? lo + chunk : d;
  T sv[GS_ITEMS];
  int64_t ix[GS_ITEMS];
  int cnt = 0;
  const T* P = static_cast<const T*>(w.Spart);
#pragma unroll
  for (int k = 0; k < GS_ITEMS; ++k) {
    ix[k] = lo + threadIdx.x + static_cast<int64_t>(k) * GS_THREADS;
    sv[k] = 0;
    if (ix[k] < hi) {
      cnt = k + 1;
      T v = 0;
      for (int p = 0; p < w.nparts; ++p) v += P[static_cast<int64_t>(p) * d + ix[k]];
      S[ix[k]] = v;
      sv[k] = v;
    } else {
      ix[k] = -1;
    }
  }
  block_partials<T, GS_ITEMS>(w, sv, ix, cnt, J, red);
  if (!last_block_combine<sizeof(T) == 4>(w, gs_ncols(J), tot, &am_last, &red[0][0])) return;
  if (pass == 0) {
    if (threadIdx.x == 0) gs_finish_start(w, o, tot);
  } else {
    gs_finish_gram(w, o, tot, &red[0][0]);
  }
}

// V_0 = src / beta, Q_0 = S / beta
template <typename T>
__global__ void k_start_scale(Work w0, PtrRef srcr0, const int* gate) {
  const int64_t bo = bidx(w0.b).off;
  const Work w = w0.at(bo);
  const PtrRef srcr = srcr0.at(bo);
  const Ctl* ctl = w.ctl;
  gate = bsh(gate, bo);
  if (gate != nullptr && *gate) return;
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
// The last block of the grid runs givens_step (Eq. 11S, rho_j, the stop
// rule) beside the update; the others share the update.
template <typename T>
__global__ void k_update(Work w0, StepOpts o0) {
  const int64_t bo = bidx(w0.b).off;
  const Work w = w0.at(bo);
  const StepOpts o = o0.at(bo);
  Ctl* ctl = w.ctl;
  if (blockIdx.x == gridDim.x - 1) {
    givens_step(w, o);
    return;
  }
  if (ctl->skip_update || ctl->j == 0) return;
  // lock-step batch: a problem that stopped in an earlier body has nothing to update
  if (o.group_left != nullptr && ctl->stop && !ctl->givens) return;
  const int jj = ctl->j;
  if (jj > w.m) {   // V holds m+1 tensors: never write past V_m
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctl->status = RTG_ERR_INVALID_ARG;
      ctl->stop = 1;
    }
    return;
  }
  __shared__ T hs[kMaxK + 1];
  __shared__ double hd[kMaxK + 1];
  const int ld = w.m + 1;
  for (int i = threadIdx.x; i < jj; i += blockDim.x) {
    const double h = w.H[static_cast<int64_t>(ld) * (jj - 1) + i];
    hs[i] = static_cast<T>(h);
    hd[i] = h;
  }
  T* V = static_cast<T*>(w.V);
  T* Q = static_cast<T*>(w.Q);
  const T* W = static_cast<const T*>(w.W);
  const T* S = static_cast<const T*>(w.S);
  const int64_t n = w.n, d = w.d;
  const int64_t stride = (int64_t)(gridDim.x - 1) * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (sizeof(T) == 4 && (n % 4) == 0) {
    const int64_t n4 = n / 4;
    const float4* W4 = reinterpret_cast<const float4*>(W);
    const float4* V4 = reinterpret_cast<const float4*>(V);
    float4* out = reinterpret_cast<float4*>(V) + static_cast<int64_t>(jj) * n4;
    // the first element's data loads go out before the barrier that publishes h
    constexpr int PRE = 8;
    float4 pre[PRE];
    float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t0 < n4) {
      w0 = W4[t0];
#pragma unroll
      for (int i = 0; i < PRE; ++i)
        if (i < jj) pre[i] = V4[static_cast<int64_t>(i) * n4 + t0];
    }
    __syncthreads();
    const T inv = static_cast<T>(1.0 / ctl->hnext);
    const float fi = static_cast<float>(inv);
    for (int64_t e = t0; e < n4; e += stride) {
      float4 acc;
      int i = 0;
      if (e == t0) {
        acc = w0;
#pragma unroll
        for (int u = 0; u < PRE; ++u) {
          if (u >= jj) break;
          const float h0 = hs[u];
          acc.x -= h0 * pre[u].x; acc.y -= h0 * pre[u].y; acc.z -= h0 * pre[u].z; acc.w -= h0 * pre[u].w;
        }
        i = jj < PRE ? jj : PRE;
      } else {
        acc = W4[e];
      }
      // eight basis loads in flight per round (the kernel is bound by HBM latency)
      for (; i + 8 <= jj; i += 8) {
        float4 a8[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a8[u] = V4[static_cast<int64_t>(i + u) * n4 + e];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float h0 = hs[i + u];
          acc.x -= h0 * a8[u].x; acc.y -= h0 * a8[u].y; acc.z -= h0 * a8[u].z; acc.w -= h0 * a8[u].w;
        }
      }
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
      acc.x *= fi; acc.y *= fi; acc.z *= fi; acc.w *= fi;
      out[e] = acc;
    }
  } else {
    __syncthreads();
    const T inv = static_cast<T>(1.0 / ctl->hnext);
    for (int64_t e = t0; e < n; e += stride) {
      T v = W[e];
      for (int i = 0; i < jj; ++i) v -= hs[i] * V[static_cast<int64_t>(i) * n + e];
      V[static_cast<int64_t>(jj) * n + e] = v * inv;
    }
  }
  // Q_{j} = (s - Q h) / h_{j,j-1}, accumulated in FP64 and rounded once
  const double invd = 1.0 / ctl->hnext;
  for (int64_t e = t0; e < d; e += stride) {
    double v = static_cast<double>(S[e]);
    for (int i = 0; i < jj; ++i) v -= hd[i] * static_cast<double>(Q[static_cast<int64_t>(i) * d + e]);
    Q[static_cast<int64_t>(jj) * d + e] = static_cast<T>(v * invd);
  }
}

// new_cycle = 0: start of a solve; 1: start of a restarted cycle (gated by
// rs_skip inside the step body: it keeps the body count, the lock-step
// count of running problems and the restart flag, which the restart
// sequence clears last).
__global__ void k_reset(Work w0, int new_cycle, unsigned* group_left, const int* gate) {
  const BIdx bi = bidx(w0.b);
  Ctl* ctl = bsh(w0.ctl, bi.off);
  gate = bsh(gate, bi.off);
  if (gate != nullptr && *gate) return;
  unsigned* counter = bsh(w0.counter, bi.off);
  // last-block counters wrap to zero by themselves; clearing them here also
  // recovers from a solve that ended inside a kernel
  for (int i = 0; i < 8; ++i) counter[i] = 0u;
  ctl->j = 0;
  ctl->stop = 0;
  ctl->breakdown = 0;
  ctl->converged = 0;
  ctl->skip_update = 0;
  ctl->pre2 = 0.0;
  ctl->hnext = 0.0;
  ctl->givens = 0;
  if (new_cycle) {
    ctl->cycle += 1;
  } else {
    if (group_left != nullptr && bi.p == 0) *group_left = static_cast<unsigned>(w0.b.n);
    ctl->counted = 0;
    ctl->loops = 0;
    ctl->rs_skip = 1;
    ctl->status = 0;
    ctl->iters_total = 0;
    ctl->cycle = 0;
    ctl->beta0 = 0.0;
    ctl->beta = 0.0;
    ctl->rho = 1.0;
    ctl->mu = 0.0;
    ctl->true_rr = -1.0;
    ctl->true_th = -1.0;
  }
}

static unsigned ew_grid(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return static_cast<unsigned>(b < 1 ? 1 : b);
}

cudaError_t launch_reset(const Work& w, int new_cycle, cudaStream_t s, unsigned* group_left, const int* gate) {
  k_reset<<<dim3(1, 1, w.b.n), 1, 0, s>>>(w, new_cycle, group_left, gate);
  return cudaGetLastError();
}

__global__ void k_restart_done(Work w0, StepOpts o) {
  Ctl* ctl = bsh(w0.ctl, bidx(w0.b).off);
  ctl->rs_skip = 1;
  if (o.use_rs_cond) cudaGraphSetConditional(static_cast<cudaGraphConditionalHandle>(o.rs_cond), 0u);
}

cudaError_t launch_restart_done(const Work& w, const StepOpts& o, cudaStream_t s) {
  k_restart_done<<<dim3(1, 1, w.b.n), 1, 0, s>>>(w, o);
  return cudaGetLastError();
}

// BF16 basis: V_0 = src / beta with src in FP32 (C) or BF16 (the V_0 slot).
// Eight values per 16-byte load (n is a multiple of 8).
__device__ __forceinline__ void bf8_to_f(const uint4& q, float* f) {
  const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    f[2 * i] = __uint_as_float(w4[i] << 16);
    f[2 * i + 1] = __uint_as_float(w4[i] & 0xffff0000u);
  }
}
__device__ __forceinline__ uint4 f_to_bf8(const float* f) {
  uint32_t w4[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
    w4[i] = *reinterpret_cast<const uint32_t*>(&h);
  }
  return make_uint4(w4[0], w4[1], w4[2], w4[3]);
}

template <bool SRC_BF16>
__global__ void k_start_scale_bf16(Work w0, PtrRef srcr0, const int* gate) {
  const int64_t bo = bidx(w0.b).off;
  const Work w = w0.at(bo);
  const PtrRef srcr = srcr0.at(bo);
  const Ctl* ctl = w.ctl;
  gate = bsh(gate, bo);
  if (gate != nullptr && *gate) return;
  if (ctl->stop) return;
  const float fi = static_cast<float>(1.0 / ctl->beta);
  uint4* V8 = static_cast<uint4*>(w.V);
  const int64_t n8 = w.n / 8;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t o = t0; o < n8; o += stride) {
    float f[8];
    if (SRC_BF16) {
      bf8_to_f(srcr.get<const uint4>()[o], f);
    } else {
      const float4* s4 = srcr.get<const float4>();
      const float4 a = s4[2 * o], b = s4[2 * o + 1];
      f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w; f[4] = b.x; f[5] = b.y; f[6] = b.z; f[7] = b.w;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) f[i] *= fi;
    V8[o] = f_to_bf8(f);
  }
  float* Q = static_cast<float*>(w.Q);
  const float* S = static_cast<const float*>(w.S);
  const float inv = static_cast<float>(1.0 / ctl->beta);
  for (int64_t o = t0; o < w.d; o += stride) Q[o] = S[o] * inv;
}

// BF16 basis: V_{j+1} = (W - sum_i h_i V_i) / h_{j+1,j} with FP32 arithmetic;
// Q_{j+1} as in k_update.  The last block runs givens_step.
__global__ void k_update_bf16(Work w0, StepOpts o0) {
  const int64_t bo = bidx(w0.b).off;
  const Work w = w0.at(bo);
  const StepOpts o = o0.at(bo);
  Ctl* ctl = w.ctl;
  if (blockIdx.x == gridDim.x - 1) {
    givens_step(w, o);
    return;
  }
  if (ctl->skip_update || ctl->j == 0) return;
  if (o.group_left != nullptr && ctl->stop && !ctl->givens) return;
  const int jj = ctl->j;
  if (jj > w.m) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctl->status = RTG_ERR_INVALID_ARG;
      ctl->stop = 1;
    }
    return;
  }
  __shared__ float hs[kMaxK + 1];
  __shared__ double hd[kMaxK + 1];
  const int ld = w.m + 1;
  for (int i = threadIdx.x; i < jj; i += blockDim.x) {
    const double h = w.H[static_cast<int64_t>(ld) * (jj - 1) + i];
    hs[i] = static_cast<float>(h);
    hd[i] = h;
  }
  __syncthreads();
  const uint4* W8 = static_cast<const uint4*>(w.W);
  const uint4* V8 = static_cast<const uint4*>(w.V);
  const int64_t n8 = w.n / 8;
  uint4* out = static_cast<uint4*>(w.V) + static_cast<int64_t>(jj) * n8;
  const float fi = static_cast<float>(1.0 / ctl->hnext);
  const int64_t stride = (int64_t)(gridDim.x - 1) * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t e = t0; e < n8; e += stride) {
    float acc[8];
    bf8_to_f(W8[e], acc);
    int i = 0;
    for (; i + 8 <= jj; i += 8) {
      uint4 q8[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) q8[u] = V8[static_cast<int64_t>(i + u) * n8 + e];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        float f[8];
        bf8_to_f(q8[u], f);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = fmaf(-hs[i + u], f[k], acc[k]);
      }
    }
    for (; i + 4 <= jj; i += 4) {
      const uint4 q0 = V8[static_cast<int64_t>(i) * n8 + e];
      const uint4 q1 = V8[static_cast<int64_t>(i + 1) * n8 + e];
      const uint4 q2 = V8[static_cast<int64_t>(i + 2) * n8 + e];
      const uint4 q3 = V8[static_cast<int64_t>(i + 3) * n8 + e];
      float f[8];
      bf8_to_f(q0, f);
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] = fmaf(-hs[i], f[k], acc[k]);
      bf8_to_f(q1, f);
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] = fmaf(-hs[i + 1], f[k], acc[k]);
      bf8_to_f(q2, f);
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] = fmaf(-hs[i + 2], f[k], acc[k]);
      bf8_to_f(q3, f);
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] = fmaf(-hs[i + 3], f[k], acc[k]);
    }
    for (; i < jj; ++i) {
      float f[8];
      bf8_to_f(V8[static_cast<int64_t>(i) * n8 + e], f);
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] = fmaf(-hs[i], f[k], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] *= fi;
    out[e] = f_to_bf8(acc);
  }
  float* Q = static_cast<float*>(w.Q);
  const float* S = static_cast<const float*>(w.S);
  const double invd = 1.0 / ctl->hnext;
  for (int64_t e = t0; e < w.d; e += stride) {
    double v = static_cast<double>(S[e]);
    for (int i = 0; i < jj; ++i) v -= hd[i] * static_cast<double>(Q[static_cast<int64_t>(i) * w.d + e]);
    Q[static_cast<int64_t>(jj) * w.d + e] = static_cast<float>(v * invd);
  }
}

// Basis update streamed through shared memory (FP32 or BF16 storage, FP32
// arithmetic): V_{j+1} = (W - sum_i h_i V_i) / h_{j+1,j}.  The tensor is cut
// into chunks of 16 KB, one CTA each; a CTA streams W and V_0 .. V_{j-1} of
// its chunk through a ring of UP_STAGES slots filled by bulk asynchronous
// copies, so 64 KB per CTA are in flight and the kernel runs at HBM
// bandwidth however many basis tensors it reads.  Each thread keeps 16 (FP32)
// or 32 (BF16) elements in 16-byte groups; the subtraction order (W, then
// V_0, V_1, ...) equals the register kernel's, so the results are the same
// bit for bit.  The next CTAs form Q_{j+1} (as in k_update), the last one
// runs givens_step.  At 512 x 512 x 3 the grid is one wave (192 chunk CTAs,
// 192 column CTAs, three CTAs per SM).
constexpr int UP_THREADS = 256;

// Ring geometries the autotuner chooses from: bytes of one slot (the chunk a
// CTA streams) and slots in flight.  Every geometry gives the same results
// bit for bit (each element is updated in the same order).  Index 0 is the
// default when no tuning has run.
struct UpCfg {
  int slot, stages;
};
constexpr UpCfg kUpCfgs[] = {{16384, 4}, {8192, 4}, {8192, 8}, {16384, 2}, {32768, 2}};
constexpr int kUpCfgCount = sizeof(kUpCfgs) / sizeof(kUpCfgs[0]);
int update_configs() { return kUpCfgCount; }

template <typename TV, int UP_SLOT, int UP_STAGES>
__global__ void __launch_bounds__(UP_THREADS) k_update_ring(Work w0, StepOpts o0, int nchunks) {
  constexpr int CE = UP_SLOT / static_cast<int>(sizeof(TV));   // elements of a chunk
  constexpr int VEC = 16 / static_cast<int>(sizeof(TV));       // elements per 16-byte group
  constexpr int NV = CE / VEC / UP_THREADS;                     // groups per thread
  const int64_t bo = bidx(w0.b).off;
  const Work w = w0.at(bo);
  const StepOpts o = o0.at(bo);
  Ctl* ctl = w.ctl;
  if (blockIdx.x == gridDim.x - 1) {
    givens_step(w, o);
    return;
  }
  if (ctl->skip_update || ctl->j == 0) return;
  if (o.group_left != nullptr && ctl->stop && !ctl->givens) return;
  const int jj = ctl->j;
  if (jj > w.m) {   // V holds m+1 tensors: never write past V_m
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctl->status = RTG_ERR_INVALID_ARG;
      ctl->stop = 1;
    }
    return;
  }
  // h_{i,j} as FP32 (hs) and, for the sketched column, as float-float
  // hs + hl; 1/h_{j+1,j} likewise, computed once per CTA (an FP64 division
  // in every thread would load the slow FP64 pipe).
  __shared__ float hs[kMaxK + 1];
  __shared__ float hl[kMaxK + 1];
  __shared__ float rinv[2];
  __shared__ __align__(8) uint64_t full[UP_STAGES];
  const int ld = w.m + 1;
  const bool qcta = static_cast<int>(blockIdx.x) >= nchunks;
  for (int i = threadIdx.x; i < jj; i += blockDim.x) {
    const double h = w.H[static_cast<int64_t>(ld) * (jj - 1) + i];
    const float f = static_cast<float>(h);
    hs[i] = f;
    if (qcta) hl[i] = static_cast<float>(h - static_cast<double>(f));
  }
  if (threadIdx.x == blockDim.x - 1) {
    const double r = 1.0 / ctl->hnext;
    const float f = static_cast<float>(r);
    rinv[0] = f;
    rinv[1] = static_cast<float>(r - static_cast<double>(f));
  }
  if (qcta) {   // Q_{j+1} = (S - sum_i h_i Q_i) / h_{j+1,j}, accumulated in float-float
    __syncthreads();
    float* Q = static_cast<float*>(w.Q);
    const float* S = static_cast<const float*>(w.S);
    const int64_t e = static_cast<int64_t>(blockIdx.x - nchunks) * blockDim.x + threadIdx.x;
    if (e >= w.d) return;
    FF v{S[e], 0.f};
    auto sub = [&](int i, float q) {   // v -= (hs_i + hl_i) q
      const FF p = ff_prod(hs[i], q);
      v = ff_add(v, FF{-p.hi, -__fmaf_rn(hl[i], q, p.lo)});
    };
    int i = 0;
    for (; i + 8 <= jj; i += 8) {   // eight loads in flight, then the chain in order
      float q8[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) q8[u] = Q[static_cast<int64_t>(i + u) * w.d + e];
#pragma unroll
      for (int u = 0; u < 8; ++u) sub(i + u, q8[u]);
    }
    for (; i < jj; ++i) sub(i, Q[static_cast<int64_t>(i) * w.d + e]);
    // (v.hi + v.lo)(r0 + r1), rounded once to FP32
    const FF p = ff_prod(v.hi, rinv[0]);
    const float lo = __fmaf_rn(v.hi, rinv[1], __fmaf_rn(v.lo, rinv[0], p.lo));
    Q[static_cast<int64_t>(jj) * w.d + e] = __fadd_rn(p.hi, lo);
    return;
  }
  extern __shared__ __align__(128) unsigned char smem[];
  TV* ring = reinterpret_cast<TV*>(smem);   // [UP_STAGES][CE]
  const int64_t n = w.n;
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * CE;
  const int ce = static_cast<int>(n - c0 < CE ? n - c0 : CE);   // a multiple of 8
  const uint32_t bytes = static_cast<uint32_t>(ce) * sizeof(TV);
  const TV* W = static_cast<const TV*>(w.W) + c0;
  const TV* V = static_cast<const TV*>(w.V) + c0;
  const int nt = jj + 1;   // W, then V_0 .. V_{jj-1}
  auto src = [&](int t) { return t == 0 ? W : V + static_cast<int64_t>(t - 1) * n; };
  if (threadIdx.x == 0) {
    for (int k = 0; k < UP_STAGES; ++k) mbar_init(&full[k]);
    for (int t = 0; t < UP_STAGES && t < nt; ++t) {
      mbar_expect(&full[t], bytes);
      bulk_g2s(ring + static_cast<size_t>(t) * CE, src(t), bytes, &full[t]);
    }
  }
  __syncthreads();
  // group k of this thread: elements (threadIdx.x + k * UP_THREADS) * VEC ..
  float acc[NV][VEC];
  bool ok = true;
  int t = 0;
  for (; t < nt; ++t) {
    const int sl = t % UP_STAGES;
    if (tc_wait_failed(&full[sl], static_cast<uint32_t>((t / UP_STAGES) & 1), &ctl->status)) {
      ok = false;
      break;
    }
    const uint4* slot = reinterpret_cast<const uint4*>(ring + static_cast<size_t>(sl) * CE);
    const float h0 = t > 0 ? hs[t - 1] : 0.f;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const uint4 q = slot[threadIdx.x + k * UP_THREADS];
      float v[VEC];
      if constexpr (sizeof(TV) == 4) {
        v[0] = __uint_as_float(q.x); v[1] = __uint_as_float(q.y); v[2] = __uint_as_float(q.z); v[3] = __uint_as_float(q.w);
      } else {
        bf8_to_f(q, v);
      }
      if (t == 0) {
#pragma unroll
        for (int u = 0; u < VEC; ++u) acc[k][u] = v[u];
      } else {
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
          if constexpr (sizeof(TV) == 4) acc[k][u] -= h0 * v[u];
          else acc[k][u] = fmaf(-h0, v[u], acc[k][u]);
        }
      }
    }
    __syncthreads();   // every thread is done with slot sl
    if (threadIdx.x == 0 && t + UP_STAGES < nt) {
      mbar_expect(&full[sl], bytes);
      bulk_g2s(ring + static_cast<size_t>(sl) * CE, src(t + UP_STAGES), bytes, &full[sl]);
    }
  }
  if (!ok) {   // a copy timed out: wait (bounded) for the others in flight, write nothing
    if (threadIdx.x == 0)
      for (int u = t + 1; u < nt && u < t + UP_STAGES; ++u)
        mbar_wait(&full[u % UP_STAGES], static_cast<uint32_t>((u / UP_STAGES) & 1));
    return;
  }
  const float fi = rinv[0];
  TV* out = static_cast<TV*>(w.V) + static_cast<int64_t>(jj) * n + c0;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const int e0 = (threadIdx.x + k * UP_THREADS) * VEC;
    if (e0 >= ce) break;
#pragma unroll
    for (int u = 0; u < VEC; ++u) acc[k][u] *= fi;
    if constexpr (sizeof(TV) == 4) {
      *reinterpret_cast<float4*>(out + e0) = make_float4(acc[k][0], acc[k][1], acc[k][2], acc[k][3]);
    } else {
      *reinterpret_cast<uint4*>(out + e0) = f_to_bf8(acc[k]);
    }
  }
}

cudaError_t launch_start(const Work& w, PtrRef src, const StepOpts& o, bool fused, cudaStream_t s,
                         int sdtype, const int* gate) {
  const unsigned g = static_cast<unsigned>(gs_grid(w.d)), nb = static_cast<unsigned>(w.b.n);
  if (sdtype < 0) sdtype = w.dtype;
  if (w.vdtype == RTG_BF16) {
    if (!fused) k_gs_pass<float><<<dim3(g, 1, nb), GS_THREADS, 0, s>>>(w, 0, o, gate);
    if (sdtype == RTG_BF16) k_start_scale_bf16<true><<<dim3(ew_grid(w.n / 8 + 1), 1, nb), 256, 0, s>>>(w, src, gate);
    else k_start_scale_bf16<false><<<dim3(ew_grid(w.n / 8 + 1), 1, nb), 256, 0, s>>>(w, src, gate);
    return cudaGetLastError();
  }
  if (w.dtype == RTG_F64) {
    if (!fused) k_gs_pass<double><<<dim3(g, 1, nb), GS_THREADS, 0, s>>>(w, 0, o, gate);
    k_start_scale<double><<<dim3(ew_grid(w.n), 1, nb), 256, 0, s>>>(w, src, gate);
  } else {
    if (!fused) k_gs_pass<float><<<dim3(g, 1, nb), GS_THREADS, 0, s>>>(w, 0, o, gate);
    k_start_scale<float><<<dim3(ew_grid(w.n / 4 + 1), 1, nb), 256, 0, s>>>(w, src, gate);
  }
  return cudaGetLastError();
}

cudaError_t launch_pass1(const Work& w, const StepOpts& o, cudaStream_t s) {
  const dim3 g(static_cast<unsigned>(gs_grid(w.d)), 1, static_cast<unsigned>(w.b.n));
  if (w.dtype == RTG_F64) k_gs_pass<double><<<g, GS_THREADS, 0, s>>>(w, 1, o, nullptr);
  else k_gs_pass<float><<<g, GS_THREADS, 0, s>>>(w, 1, o, nullptr);
  return cudaGetLastError();
}



template <typename TV, int SLOT, int STAGES>
static cudaError_t launch_update_ring_cfg(const Work& w, const StepOpts& o, cudaStream_t s) {
  constexpr size_t sm = size_t(STAGES) * SLOT;
  cudaError_t e = set_smem(k_update_ring<TV, SLOT, STAGES>, sm);
  if (e != cudaSuccess) return e;
  constexpr int64_t CE = SLOT / sizeof(TV);
  const int nchunks = static_cast<int>((w.n + CE - 1) / CE);
  const int qblocks = static_cast<int>((w.d + UP_THREADS - 1) / UP_THREADS);
  const dim3 grid(static_cast<unsigned>(nchunks + qblocks + 1), 1, static_cast<unsigned>(w.b.n));
  k_update_ring<TV, SLOT, STAGES><<<grid, UP_THREADS, sm, s>>>(w, o, nchunks);
  return cudaGetLastError();
}

template <typename TV>
static cudaError_t launch_update_ring(const Work& w, const StepOpts& o, cudaStream_t s) {
  switch (w.upcfg) {
    case 1: return launch_update_ring_cfg<TV, kUpCfgs[1].slot, kUpCfgs[1].stages>(w, o, s);
    case 2: return launch_update_ring_cfg<TV, kUpCfgs[2].slot, kUpCfgs[2].stages>(w, o, s);
    case 3: return launch_update_ring_cfg<TV, kUpCfgs[3].slot, kUpCfgs[3].stages>(w, o, s);
    case 4: return launch_update_ring_cfg<TV, kUpCfgs[4].slot, kUpCfgs[4].stages>(w, o, s);
    default: return launch_update_ring_cfg<TV, kUpCfgs[0].slot, kUpCfgs[0].stages>(w, o, s);
  }
}

bool update_uses_ring(const Work& w) {
  return w.dtype == RTG_F32 && w.n % 8 == 0 && w.n / 4096 < (int64_t(1) << 30);
}

cudaError_t launch_update(const Work& w, const StepOpts& o, cudaStream_t s) {
  // FP32 solves with whole 8-element groups stream the basis through shared memory
  if (update_uses_ring(w))
    return w.vdtype == RTG_BF16 ? launch_update_ring<__nv_bfloat16>(w, o, s) : launch_update_ring<float>(w, o, s);
  // one block more than the update needs: it runs the Givens step
  const unsigned nb = static_cast<unsigned>(w.b.n);
  if (w.vdtype == RTG_BF16) k_update_bf16<<<dim3(ew_grid(w.n / 8 + 1) + 1, 1, nb), 256, 0, s>>>(w, o);
  else if (w.dtype == RTG_F64) k_update<double><<<dim3(ew_grid(w.n) + 1, 1, nb), 256, 0, s>>>(w, o);
  else k_update<float><<<dim3(ew_grid(w.n / 4 + 1) + 1, 1, nb), 256, 0, s>>>(w, o);
  return cudaGetLastError();
}

}  // namespace rtg
