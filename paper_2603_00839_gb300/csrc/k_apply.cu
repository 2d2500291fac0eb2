// Operator apply Y = alpha * Phi(X) + beta * Z for the separable Einstein
// product Phi(X) = A *_N X (*_M B) (Section 1; Eq. 56-57 with zero
// boundary conditions).  Phi is a list of mode products with banded
// Toeplitz or dense matrices.
//
// Fused path (one HBM pass): a CTA owns a 64 x 16 tile of modes 1-2 for
// up to four channels of mode 3.  Per channel it stages the halo tile in
// shared memory, filters along mode 1 into a second shared tile, then
// along mode 2 into registers; the mode-3 matrix mixes the channels in
// registers before the single store.  Unfused path: one kernel per mode
// product, ping-ponging through scratch tensors.
#include <cuda_bf16.h>

#include <cstring>

#include "tma_common.cuh"

namespace rtg {

constexpr int FTX = 64;
constexpr int FTY = 16;
constexpr int FTHREADS = 256;

struct FusedArgs {
  int64_t I1, I2;
  int64_t nslab;               // independent slabs of nc channels
  int r1, r2;
  int nc;
  double t1[kMaxTaps], t2[kMaxTaps];
  double M[kMaxMix * kMaxMix]; // M[p + nc*c]
  double alpha, beta;
  // the same, rounded to FP32 on the host: an FP64-to-FP32 conversion runs on
  // this GPU's FP64 pipe (two lanes per SM per cycle), and converting the
  // taps and the mix in every thread made the FP32 kernels FP64-bound
  float t1f[kMaxTaps], t2f[kMaxTaps];
  float Mf[kMaxMix * kMaxMix];
  float alphaf, betaf;
  // the taps zero-padded to the register kernel's compile-time radius RR
  // (tap t of the padded filter is tap t - (RR - r) of the real one): with
  // compile-time indices they stay in the constant bank as FMA operands
  // instead of taking two registers per tap
  double t1p[kMaxTaps], t2p[kMaxTaps];
  float t1pf[kMaxTaps], t2pf[kMaxTaps];
};
// An argument in the kernel's arithmetic type.
template <typename T>
__device__ __forceinline__ T argT(double d, float f) {
  if constexpr (sizeof(T) == 4) return f;
  else return d;
}

template <typename T, int NC>
__global__ void __launch_bounds__(FTHREADS)
k_apply_fused(PtrRef Xr, PtrRef Yr, PtrRef Zr, const int* stop, FusedArgs a, Batch bt) {
  const BIdx bi = bidx(bt);
  Xr = Xr.at(bi.off);
  Yr = Yr.at(bi.off);
  Zr = Zr.at(bi.off);
  stop = bsh(stop, bi.off);
  if (stop != nullptr && *stop) return;
  const T* X = Xr.get<const T>();
  T* __restrict__ Y = Yr.get<T>();
  const T* Z = Zr.get<const T>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T t1s[kMaxTaps], t2s[kMaxTaps];
  const int Wd = FTX + 2 * a.r1;
  const int Ht = FTY + 2 * a.r2;
  T* in_s = reinterpret_cast<T*>(smem_raw);
  T* tmp = in_s + Ht * Wd;
  for (int t = threadIdx.x; t <= 2 * a.r1; t += FTHREADS) t1s[t] = argT<T>(a.t1[t], a.t1f[t]);
  for (int t = threadIdx.x; t <= 2 * a.r2; t += FTHREADS) t2s[t] = argT<T>(a.t2[t], a.t2f[t]);

  const int64_t x0 = static_cast<int64_t>(blockIdx.x) * FTX;
  const int64_t y0 = static_cast<int64_t>(blockIdx.y) * FTY;
  const int64_t plane = a.I1 * a.I2;
  const int tx = threadIdx.x & (FTX - 1);
  const int ty = threadIdx.x / FTX;          // 0..3, rows ty + 4k
  T acc[NC][FTY / 4];

  for (int64_t slab = bi.z; slab < a.nslab; slab += bi.nz) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const T* Xc = X + (slab * NC + c) * plane;
      __syncthreads();
      for (int idx = threadIdx.x; idx < Ht * Wd; idx += FTHREADS) {
        const int yy = idx / Wd, xx = idx - yy * Wd;
        const int64_t gx = x0 - a.r1 + xx, gy = y0 - a.r2 + yy;
        T v = 0;
        if (gx >= 0 && gx < a.I1 && gy >= 0 && gy < a.I2) v = Xc[gy * a.I1 + gx];
        in_s[idx] = v;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < Ht * FTX; idx += FTHREADS) {    // mode-1 filter
        const int yy = idx / FTX, xx = idx - yy * FTX;
        const T* row = in_s + yy * Wd + xx;
        T s = 0;
        for (int t = 0; t <= 2 * a.r1; ++t) s += t1s[t] * row[t];
        tmp[idx] = s;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < FTY / 4; ++k) {                              // mode-2 filter
        const T* col = tmp + (ty + 4 * k) * FTX + tx;
        T s = 0;
        for (int t = 0; t <= 2 * a.r2; ++t) s += t2s[t] * col[t * FTX];
        acc[c][k] = s;
      }
    }
#pragma unroll
    for (int k = 0; k < FTY / 4; ++k) {                                // mode-3 mix + store
      const int64_t gx = x0 + tx, gy = y0 + ty + 4 * k;
      if (gx >= a.I1 || gy >= a.I2) continue;
#pragma unroll
      for (int p = 0; p < NC; ++p) {
        T v = 0;
#pragma unroll
        for (int c = 0; c < NC; ++c) v += argT<T>(a.M[p + NC * c], a.Mf[p + NC * c]) * acc[c][k];
        const int64_t o = (slab * NC + p) * plane + gy * a.I1 + gx;
        T out = argT<T>(a.alpha, a.alphaf) * v;
        if (Z != nullptr) out += argT<T>(a.beta, a.betaf) * Z[o];
        Y[o] = out;
      }
    }
  }
}

// Register-blocked variant for a compile-time radius RR (taps zero-padded
// to 2*RR+1) and NC jointly mixed channels.  Tile 64 x 16 of modes 1-2,
// 256 threads.  All NC halo tiles are staged in shared memory at once with
// cp.async (zero fill outside the tensor: the zero boundary of Eq. 57), so
// the CTA waits on global memory once.  Per channel the mode-2 filter runs
// first, over the 16 output rows and every staged column (a task: two
// adjacent columns x 4 rows, paired FP32 FMAs), then the mode-1 filter over
// the 16 x 64 outputs (a thread: 4 consecutive outputs of one row from a
// register window of 4+2RR values): filtering the halo rows along mode 2
// first costs 16 (64 + 2RR) + 16 x 64 products per tap instead of
// (16 + 2RR) 64 + 16 x 64, and the thread's 4 outputs leave in one 16-byte
// store after the channel mix.
constexpr int RTX = 64;
constexpr int RTY = 16;


template <int RR, typename T>
struct RegGeom {
  // FP32 rows start on a 16-byte boundary: the halo is widened to RA >= RR
  // columns (a multiple of 4) and the filter window starts OFF = RA - RR in.
  static constexpr int RA = (sizeof(T) == 4) ? ((RR + 3) / 4) * 4 : RR;
  static constexpr int OFF = RA - RR;
  static constexpr int Wd = RTX + 2 * RA;
  static constexpr int Ht = RTY + 2 * RR;
};

// Paired FP32 FMA (fma.rn.f32x2): two lanes of independent multiply-adds
// in one instruction.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mov.b64 rc, {%6, %7};\n"
      " fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}\n"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
template <typename T>
struct Pair {
  T x, y;
};
__device__ __forceinline__ Pair<float> pfma(float t, Pair<float> v, Pair<float> acc) {
  const float2 r = ffma2(make_float2(t, t), make_float2(v.x, v.y), make_float2(acc.x, acc.y));
  return {r.x, r.y};
}
__device__ __forceinline__ Pair<double> pfma(double t, Pair<double> v, Pair<double> acc) {
  return {fma(t, v.x, acc.x), fma(t, v.y, acc.y)};
}
// Two adjacent values (8-byte aligned for FP32: one 64-bit shared load).
__device__ __forceinline__ Pair<float> load_pair(const float* p) {
  const float2 q = *reinterpret_cast<const float2*>(p);
  return {q.x, q.y};
}
__device__ __forceinline__ Pair<double> load_pair(const double* p) { return {p[0], p[1]}; }

// the taps as kernel-parameter (constant-bank) operands, see FusedArgs
#define t1(t) argT<T>(a.t1p[t], a.t1pf[t])
#define t2(t) argT<T>(a.t2p[t], a.t2pf[t])

template <typename T, int NC, int RR>
__global__ void __launch_bounds__(FTHREADS, (RR <= 7 ? 4 : 1))
k_apply_reg(PtrRef Xr, PtrRef Yr, PtrRef Zr, const int* stop, FusedArgs a,
            const __grid_constant__ CUtensorMap xmap, int xtma, Batch bt) {
  const BIdx bi = bidx(bt);
  Xr = Xr.at(bi.off);
  Yr = Yr.at(bi.off);
  Zr = Zr.at(bi.off);
  stop = bsh(stop, bi.off);
  if (stop != nullptr && *stop) return;
  const T* X = Xr.get<const T>();
  T* __restrict__ Y = Yr.get<T>();
  const T* Z = Zr.get<const T>();
  using G = RegGeom<RR, T>;
  constexpr int NT = 2 * RR + 1;
  constexpr int Wd = G::Wd, Ht = G::Ht, RA = G::RA, OFF = G::OFF;
  constexpr int NPAIR = Wd / 2;                 // mode-2 pass: column pairs
  constexpr int V2 = 4;                          // mode-2 pass: output rows per task
  constexpr int M1 = 4;                          // mode-1 pass: outputs per thread
  static_assert(Wd % 2 == 0 && NPAIR * (RTY / V2) <= 2 * FTHREADS, "mode-2 tasks");
  static_assert(RTY * (RTX / M1) == FTHREADS, "mode-1 tasks: one per thread");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t xbar;
  // the tiled copy's destination must start on 128 bytes: the tile is placed
  // there explicitly (the launch adds 128 bytes of slack)
  const uint32_t raw = static_cast<uint32_t>(__cvta_generic_to_shared(smem_raw));
  T* in_s = reinterpret_cast<T*>(smem_raw + (((raw + 127u) & ~127u) - raw));   // NC x Ht x Wd
  T* tmp = in_s + NC * Ht * Wd;                  // RTY x Wd
  const int x0 = blockIdx.x * RTX;
  const int y0 = blockIdx.y * RTY;
  const int I1 = static_cast<int>(a.I1), I2 = static_cast<int>(a.I2);
  const int64_t plane = a.I1 * a.I2;
  const int oy = threadIdx.x / (RTX / M1);       // mode-1 pass: output row
  const int ox = (threadIdx.x % (RTX / M1)) * M1; // mode-1 pass: first of 4 outputs
  // with a tensor map of the input (FP32; the basis slot and the problem as
  // its outer coordinates), one tiled TMA copy stages the halo tile of all
  // NC channels, zero filled outside the tensor (the zero boundary of Eq. 57)
  const int slot = (xtma && Xr.jidx != nullptr) ? *Xr.jidx + Xr.joff : 0;
  // the copy engine's rules, checked: a 128-byte aligned destination and an
  // innermost start coordinate on 16 bytes; otherwise the threads stage the tile
  const bool tma = xtma && (static_cast<uint32_t>(__cvta_generic_to_shared(in_s)) & 127u) == 0 &&
                   ((static_cast<int64_t>(x0 - RA) * static_cast<int64_t>(sizeof(T))) & 15) == 0;
  if (tma && threadIdx.x == 0) mbar_init(&xbar);
  uint32_t xphase = 0;
  for (int64_t slab = bi.z; slab < a.nslab; slab += bi.nz) {
    __syncthreads();
    const T* Xs = X + slab * NC * plane;
    if (tma) {
      if (threadIdx.x == 0) {
        mbar_expect(&xbar, static_cast<uint32_t>(NC * Ht * Wd * sizeof(T)));
        tma_load_5d(in_s, &xmap, x0 - RA, y0 - RR, static_cast<int>(slab * NC), slot, bi.p, &xbar);
      }
      const bool landed = mbar_wait(&xbar, xphase);
      xphase ^= 1u;
      if (__syncthreads_or(!landed)) {
        // the copy did not land in time: wait once more (bounded) for it, then
        // poison the tile so that the solve stops with a non-finite status
        if (threadIdx.x == 0) mbar_wait(&xbar, xphase ^ 1u);
        __syncthreads();
        for (int idx = threadIdx.x; idx < NC * Ht * Wd; idx += FTHREADS) in_s[idx] = static_cast<T>(__int_as_float(0x7fc00000));
      }
    } else if (sizeof(T) == 4 && (reinterpret_cast<uintptr_t>(X) & 15) == 0) {
      // 16-byte copies; a float4 lies wholly inside or outside (I1 % 4 == 0)
      constexpr int W4 = Wd / 4;
      for (int idx = threadIdx.x; idx < NC * Ht * W4; idx += FTHREADS) {
        const int row = idx / W4, f4 = idx - row * W4;
        const int c = row / Ht, yy = row - c * Ht;
        const int gy = y0 - RR + yy, gx = x0 - RA + 4 * f4;
        const bool v = gy >= 0 && gy < I2 && gx >= 0 && gx < I1;
        const T* src = v ? Xs + c * plane + static_cast<int64_t>(gy) * I1 + gx : X;
        const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(&in_s[row * Wd + 4 * f4]));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src), "r"(v ? 16 : 0));
      }
    } else {
      for (int idx = threadIdx.x; idx < NC * Ht * Wd; idx += FTHREADS) {
        const int row = idx / Wd, xx = idx - row * Wd;
        const int c = row / Ht, yy = row - c * Ht;
        const int gy = y0 - RR + yy, gx = x0 - RA + xx;
        const bool v = gy >= 0 && gy < I2 && gx >= 0 && gx < I1;
        const T* src = v ? Xs + c * plane + static_cast<int64_t>(gy) * I1 + gx : X;
        // element loads through L2 (the basis slots are rewritten by every
        // cycle and solve; only L2 is coherent across SMs)
        in_s[idx] = v ? __ldcg(src) : static_cast<T>(0);
      }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    T acc[NC][M1];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const T* ins = in_s + c * Ht * Wd;
      // mode 2 first (along y, all Wd staged columns): task = (column pair,
      // 4 output rows), paired FMAs over the two columns
      for (int task = threadIdx.x; task < NPAIR * (RTY / V2); task += FTHREADS) {
        const int pr = task % NPAIR, g = task / NPAIR;
        Pair<T> win[V2 + 2 * RR];
#pragma unroll
        for (int u = 0; u < V2 + 2 * RR; ++u) {
          win[u] = load_pair(ins + (g * V2 + u) * Wd + 2 * pr);
        }
#pragma unroll
        for (int o = 0; o < V2; ++o) {
          Pair<T> s{static_cast<T>(0), static_cast<T>(0)};
#pragma unroll
          for (int t = 0; t < NT; ++t) s = pfma(t2(t), win[o + t], s);
          T* q = tmp + (g * V2 + o) * Wd + 2 * pr;
          if constexpr (sizeof(T) == 4) {
            *reinterpret_cast<float2*>(q) = make_float2(s.x, s.y);
          } else {
            q[0] = s.x;
            q[1] = s.y;
          }
        }
      }
      __syncthreads();
      // mode 1 (along x): 4 consecutive outputs of one row per thread
      {
        T win[M1 + 2 * RR];
        if (sizeof(T) == 4) {
          // aligned 16-byte loads covering the window, which starts OFF & 3 floats in
          constexpr int A0 = OFF & ~3, SH = OFF & 3;
          constexpr int NV = (SH + M1 + 2 * RR + 3) / 4;
          const float4* rp = reinterpret_cast<const float4*>(tmp + oy * Wd + ox + A0);
          float buf[NV * 4];
#pragma unroll
          for (int v4 = 0; v4 < NV; ++v4) {
            const float4 q = rp[v4];
            buf[4 * v4] = q.x;
            buf[4 * v4 + 1] = q.y;
            buf[4 * v4 + 2] = q.z;
            buf[4 * v4 + 3] = q.w;
          }
#pragma unroll
          for (int u = 0; u < M1 + 2 * RR; ++u) win[u] = static_cast<T>(buf[SH + u]);
        } else {
          const T* row = tmp + oy * Wd + ox + OFF;
#pragma unroll
          for (int u = 0; u < M1 + 2 * RR; ++u) win[u] = row[u];
        }
#pragma unroll
        for (int o = 0; o < M1; ++o) {
          T sacc = 0;
#pragma unroll
          for (int t = 0; t < NT; ++t) sacc += t1(t) * win[o + t];
          acc[c][o] = sacc;
        }
      }
      __syncthreads();
    }
    const int gy = y0 + oy;
    if (gy < I2) {
      T out[M1];
#pragma unroll
      for (int p = 0; p < NC; ++p) {
        const int64_t base = (slab * NC + p) * plane + static_cast<int64_t>(gy) * I1 + x0 + ox;
#pragma unroll
        for (int o = 0; o < M1; ++o) {
          T v = 0;
#pragma unroll
          for (int c = 0; c < NC; ++c) v += argT<T>(a.M[p + NC * c], a.Mf[p + NC * c]) * acc[c][o];
          out[o] = argT<T>(a.alpha, a.alphaf) * v;
        }
        if (sizeof(T) == 4 && x0 + ox + M1 <= I1 && ((reinterpret_cast<uintptr_t>(Y + base)) & 15) == 0 &&
            (Z == nullptr || ((reinterpret_cast<uintptr_t>(Z + base)) & 15) == 0)) {
          if (Z != nullptr) {
            const float4 z = __ldcg(reinterpret_cast<const float4*>(Z + base));
            const T bz = argT<T>(a.beta, a.betaf);
            out[0] += bz * static_cast<T>(z.x);
            out[1] += bz * static_cast<T>(z.y);
            out[2] += bz * static_cast<T>(z.z);
            out[3] += bz * static_cast<T>(z.w);
          }
          *reinterpret_cast<float4*>(Y + base) = make_float4(static_cast<float>(out[0]), static_cast<float>(out[1]),
                                                             static_cast<float>(out[2]), static_cast<float>(out[3]));
        } else {
#pragma unroll
          for (int o = 0; o < M1; ++o) {
            if (x0 + ox + o >= I1) break;
            T v = out[o];
            if (Z != nullptr) v += argT<T>(a.beta, a.betaf) * Z[base + o];
            Y[base + o] = v;
          }
        }
      }
    }
  }
}
#undef t1
#undef t2

// ---------------------------------------------------------------- spatio-temporal path
// One HBM pass for the video operator (order 4: blur on modes 1-2, channel
// mix on mode 3, banded temporal filter of radius <= 2 on mode 4) and for
// any image operator whose tensors are stored in BF16.  A CTA owns a
// 64 x 16 tile of modes 1-2, all NC channels of one channel group and a
// chunk of output frames.  It walks the input frames in order: each frame's
// halo tile is loaded into registers (16-byte loads, BF16 or FP32) while
// the previous frame is being filtered, converted to FP32 in shared memory,
// filtered along mode 2 and then mode 1 as in the image kernel, and added into a
// ring of five partial output frames held in registers; the oldest ring
// entry is complete after each input frame, is mixed across the channels
// and stored.  Arithmetic is FP32 in every storage format.
constexpr int STX = 64, STY = 16, ST_THREADS = 256, ST_RING = 5, ST_VSEG = 4;

struct StArgs {
  int64_t I1, I2, I3, nF;   // mode sizes; nF = 1 for order 3
  int F;                    // output frames per CTA
  int nchunk;               // frame chunks
  int rt;                   // temporal radius (0..2)
  float t1[kMaxTaps], t2[kMaxTaps];   // spatial taps zero-padded to the compiled radius
  float t4[ST_RING];                  // temporal taps zero-padded to radius 2: t4[2 + s]
  float M[kMaxMix * kMaxMix];         // channel mix M[p + nc * c]
  float alpha, beta;
};

template <typename TI>
struct StVec {   // elements of TI in one 16-byte load
  static constexpr int V = 16 / static_cast<int>(sizeof(TI));
};

template <int RR, typename TI>
struct StGeom {
  static constexpr int V = StVec<TI>::V;
  static constexpr int RA = ((RR + V - 1) / V) * V;   // halo widened to whole 16-byte loads
  static constexpr int OFF = RA - RR;
  static constexpr int Wd = STX + 2 * RA;
  static constexpr int Ht = STY + 2 * RR;
};

__device__ __forceinline__ void st_to_float(const uint4& q, float* dst, float) {
  dst[0] = __uint_as_float(q.x);
  dst[1] = __uint_as_float(q.y);
  dst[2] = __uint_as_float(q.z);
  dst[3] = __uint_as_float(q.w);
}
__device__ __forceinline__ void st_to_float(const uint4& q, float* dst, __nv_bfloat16) {
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    dst[2 * i] = __uint_as_float(w[i] << 16);
    dst[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}
__device__ __forceinline__ void st_store(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
// Four consecutive outputs (plus beta Z, if Z is given): one 16-byte (FP32)
// or 8-byte (BF16) store when all four lie inside the row (`room` entries
// left in it) and the address is aligned, else element by element.
template <typename TO>
__device__ __forceinline__ void st_store4(TO* p, const float* z, float beta, const float (&v)[4], int room) {
  float o[4] = {v[0], v[1], v[2], v[3]};
  const bool vec = room >= 4 && (reinterpret_cast<uintptr_t>(p) % (4 * sizeof(TO))) == 0 &&
                   (z == nullptr || (reinterpret_cast<uintptr_t>(z) % 16) == 0);
  if (vec) {
    if (z != nullptr) {
      const float4 q = __ldcg(reinterpret_cast<const float4*>(z));
      o[0] = fmaf(beta, q.x, o[0]);
      o[1] = fmaf(beta, q.y, o[1]);
      o[2] = fmaf(beta, q.z, o[2]);
      o[3] = fmaf(beta, q.w, o[3]);
    }
    if constexpr (sizeof(TO) == 4) {
      *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
      const __nv_bfloat162 lo = __floats2bfloat162_rn(o[0], o[1]), hi = __floats2bfloat162_rn(o[2], o[3]);
      uint2 w;
      w.x = *reinterpret_cast<const uint32_t*>(&lo);
      w.y = *reinterpret_cast<const uint32_t*>(&hi);
      *reinterpret_cast<uint2*>(p) = w;
    }
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (e >= room) break;
      float x = o[e];
      if (z != nullptr) x = fmaf(beta, z[e], x);
      st_store(p + e, x);
    }
  }
}

template <typename TI, typename TO, int NC, int RR>
__global__ void __launch_bounds__(ST_THREADS, 2)
k_apply_st(PtrRef Xr, PtrRef Yr, PtrRef Zr, const int* stop, StArgs a, Batch bt) {
  const BIdx bi = bidx(bt);
  Xr = Xr.at(bi.off);
  Yr = Yr.at(bi.off);
  Zr = Zr.at(bi.off);
  stop = bsh(stop, bi.off);
  if (stop != nullptr && *stop) return;
  const TI* X = Xr.get<const TI>();
  TO* __restrict__ Y = Yr.get<TO>();
  const float* Z = Zr.get<const float>();
  using G = StGeom<RR, TI>;
  constexpr int V = G::V, Wd = G::Wd, Ht = G::Ht, RA = G::RA, OFF = G::OFF;
  constexpr int NT = 2 * RR + 1;
  constexpr int NCH = NC * Ht * (Wd / V);                    // 16-byte loads per frame
  constexpr int NPT = (NCH + ST_THREADS - 1) / ST_THREADS;   // per thread
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* in_s = reinterpret_cast<float*>(smem_raw);   // NC x Ht x Wd
  float* tmp = in_s + NC * Ht * Wd;                   // STY x Wd
  const int x0 = blockIdx.x * STX, y0 = blockIdx.y * STY;
  const int I1 = static_cast<int>(a.I1), I2 = static_cast<int>(a.I2);
  const int64_t plane = a.I1 * a.I2;
  const int group = static_cast<int>(bi.z / a.nchunk);
  const int chunk = static_cast<int>(bi.z % a.nchunk);
  const int64_t f0 = static_cast<int64_t>(chunk) * a.F;
  const int64_t f1 = (f0 + a.F < a.nF) ? f0 + a.F : a.nF;
  const int rt = a.rt;
  // mode-1 pass and output: row oy, columns ox .. ox + 3 of the tile
  static_assert(STY * (STX / ST_VSEG) == ST_THREADS, "one output quad per thread");
  const int oy = threadIdx.x / (STX / ST_VSEG);
  const int ox = (threadIdx.x % (STX / ST_VSEG)) * ST_VSEG;
  constexpr int NPAIR = Wd / 2;                       // mode-2 pass: column pairs x 4 output rows
  uint4 pre[NPT];
  auto load_frame = [&](int64_t u) {
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
      pre[q] = make_uint4(0u, 0u, 0u, 0u);
      const int idx = threadIdx.x + q * ST_THREADS;
      if (idx >= NCH) continue;
      const int row = idx / (Wd / V), f = idx - row * (Wd / V);
      const int c = row / Ht, yy = row - c * Ht;
      const int gy = y0 - RR + yy, gx = x0 - RA + V * f;
      if (gy < 0 || gy >= I2 || gx < 0 || gx >= I1) continue;
      const int64_t pl = (static_cast<int64_t>(group) * NC + c) + a.I3 * u;
      pre[q] = __ldcg(reinterpret_cast<const uint4*>(X + pl * plane + static_cast<int64_t>(gy) * I1 + gx));
    }
  };
  auto store_frame = [&]() {
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
      const int idx = threadIdx.x + q * ST_THREADS;
      if (idx >= NCH) continue;
      const int row = idx / (Wd / V), f = idx - row * (Wd / V);
      float v[V];
      st_to_float(pre[q], v, TI());
      float4* d = reinterpret_cast<float4*>(in_s + row * Wd + V * f);
#pragma unroll
      for (int h = 0; h < V / 4; ++h) d[h] = make_float4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
    }
  };
  float ring[ST_RING][NC][ST_VSEG];
#pragma unroll
  for (int k = 0; k < ST_RING; ++k)
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int o = 0; o < ST_VSEG; ++o) ring[k][c][o] = 0.f;
  const int64_t u0 = f0 - rt, u1 = f1 + rt;
  {   // the first frame inside the tensor; each frame then prefetches the next
    const int64_t uf = u0 > 0 ? u0 : 0;
    if (uf < u1 && uf < a.nF) load_frame(uf);
  }
  for (int64_t u = u0; u < u1; ++u) {
    const bool have = u >= 0 && u < a.nF;
    float P[NC][ST_VSEG];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int o = 0; o < ST_VSEG; ++o) P[c][o] = 0.f;
    if (have) {
      __syncthreads();              // the previous frame's filters are done with in_s
      store_frame();
      __syncthreads();
      if (u + 1 < u1 && u + 1 < a.nF) load_frame(u + 1);   // in flight during the filters
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float* ins = in_s + c * Ht * Wd;
        // mode 2 first over every staged column: task = (column pair, 4 output rows)
        for (int task = threadIdx.x; task < NPAIR * (STY / ST_VSEG); task += ST_THREADS) {
          const int pr = task % NPAIR, g = task / NPAIR;
          float2 win[ST_VSEG + 2 * RR];
#pragma unroll
          for (int u2 = 0; u2 < ST_VSEG + 2 * RR; ++u2)
            win[u2] = *reinterpret_cast<const float2*>(ins + (g * ST_VSEG + u2) * Wd + 2 * pr);
#pragma unroll
          for (int o = 0; o < ST_VSEG; ++o) {
            float2 sacc = make_float2(0.f, 0.f);
#pragma unroll
            for (int t = 0; t < NT; ++t) sacc = ffma2(make_float2(a.t2[t], a.t2[t]), win[o + t], sacc);
            *reinterpret_cast<float2*>(tmp + (g * ST_VSEG + o) * Wd + 2 * pr) = sacc;
          }
        }
        __syncthreads();
        // mode 1: 4 consecutive outputs of row oy
        {
          constexpr int A0 = OFF & ~3, SH = OFF & 3;
          constexpr int NV = (SH + ST_VSEG + 2 * RR + 3) / 4;
          const float4* rp = reinterpret_cast<const float4*>(tmp + oy * Wd + ox + A0);
          float buf[NV * 4];
#pragma unroll
          for (int v4 = 0; v4 < NV; ++v4) {
            const float4 q = rp[v4];
            buf[4 * v4] = q.x;
            buf[4 * v4 + 1] = q.y;
            buf[4 * v4 + 2] = q.z;
            buf[4 * v4 + 3] = q.w;
          }
#pragma unroll
          for (int o = 0; o < ST_VSEG; ++o) {
            float sacc = 0.f;
#pragma unroll
            for (int t = 0; t < NT; ++t) sacc = fmaf(a.t1[t], buf[SH + o + t], sacc);
            P[c][o] = sacc;
          }
        }
        if (c + 1 < NC) __syncthreads();   // the next channel's mode-2 pass rewrites tmp
      }
    }
    // ring[k] is output frame u - rt + k; frame u enters with tap t4[2 + rt - k]
#pragma unroll
    for (int k = 0; k < ST_RING; ++k) {
      if (k > 2 * rt) break;
      const float tk = a.t4[2 + rt - k];
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int o = 0; o < ST_VSEG; ++o) ring[k][c][o] = fmaf(tk, P[c][o], ring[k][c][o]);
    }
    const int64_t t = u - rt;
    const int gy = y0 + oy;
    if (t >= f0 && t < f1 && gy < I2) {
#pragma unroll
      for (int p = 0; p < NC; ++p) {
        const int64_t base = ((static_cast<int64_t>(group) * NC + p) + a.I3 * t) * plane +
                             static_cast<int64_t>(gy) * I1 + x0 + ox;
        float out[ST_VSEG];
#pragma unroll
        for (int o = 0; o < ST_VSEG; ++o) {
          float v = 0.f;
#pragma unroll
          for (int c = 0; c < NC; ++c) v = fmaf(a.M[p + NC * c], ring[0][c][o], v);
          out[o] = a.alpha * v;
        }
        st_store4(Y + base, Z != nullptr ? Z + base : nullptr, a.beta, out, I1 - (x0 + ox));
      }
    }
#pragma unroll
    for (int k = 0; k + 1 < ST_RING; ++k)
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int o = 0; o < ST_VSEG; ++o) ring[k][c][o] = ring[k + 1][c][o];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int o = 0; o < ST_VSEG; ++o) ring[ST_RING - 1][c][o] = 0.f;
  }
}

// Spatial radius bucket of the spatio-temporal kernel (0 when none holds r).
int st_bucket(int r) {
  const int b[] = {3, 5, 7, 9};
  for (int v : b)
    if (r <= v) return v;
  return 0;
}

// Smallest compiled radius bucket that holds r (0 when none does).
static int reg_bucket(int r) {
  const int b[] = {3, 5, 7, 9, 12, 16};
  for (int v : b)
    if (r <= v) return v;
  return 0;
}

struct TapArgs {
  double t[kMaxTaps];
  float tf[kMaxTaps];   // rounded to FP32 on the host (see FusedArgs)
};

// out(l, i, r) = sum_t taps[r+t] X(l, i+t, r), zero outside [0, I)
template <typename T>
__global__ void k_pass_band(PtrRef Xr, PtrRef Yr, int64_t L, int64_t I, int64_t R, int rad,
                            TapArgs taps, const int* stop, Batch bt) {
  const int64_t bo = bidx(bt).off;
  Xr = Xr.at(bo);
  Yr = Yr.at(bo);
  stop = bsh(stop, bo);
  if (stop != nullptr && *stop) return;
  const T* X = Xr.get<const T>();
  T* __restrict__ Y = Yr.get<T>();
  const int64_t total = L * I * R;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total;
       o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = o % L;
    const int64_t i = (o / L) % I;
    const int64_t r = o / (L * I);
    T s = 0;
    for (int t = -rad; t <= rad; ++t) {
      const int64_t ii = i + t;
      if (ii >= 0 && ii < I) s += argT<T>(taps.t[rad + t], taps.tf[rad + t]) * X[l + L * (ii + I * r)];
    }
    Y[o] = s;
  }
}

// out(l, p, r) = sum_i M(p, i) X(l, i, r), M column-major on the device
template <typename T>
__global__ void k_pass_dense(PtrRef Xr, PtrRef Yr, int64_t L, int64_t I, int64_t R,
                             const double* M, const int* stop, Batch bt) {
  const int64_t bo = bidx(bt).off;
  Xr = Xr.at(bo);
  Yr = Yr.at(bo);
  stop = bsh(stop, bo);
  if (stop != nullptr && *stop) return;
  const T* X = Xr.get<const T>();
  T* __restrict__ Y = Yr.get<T>();
  const int64_t total = L * I * R;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total;
       o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = o % L;
    const int64_t p = (o / L) % I;
    const int64_t r = o / (L * I);
    T s = 0;
    for (int64_t i = 0; i < I; ++i) s += static_cast<T>(M[p + I * i]) * X[l + L * (i + I * r)];
    Y[o] = s;
  }
}

// Y = alpha * A + beta * Z (Y may alias A)
template <typename T>
__global__ void k_axpby(PtrRef Ar, PtrRef Yr, PtrRef Zr, double alpha, double beta, int64_t n,
                        const int* stop, Batch bt) {
  const int64_t bo = bidx(bt).off;
  Ar = Ar.at(bo);
  Yr = Yr.at(bo);
  Zr = Zr.at(bo);
  stop = bsh(stop, bo);
  if (stop != nullptr && *stop) return;
  const T* A = Ar.get<const T>();
  T* Y = Yr.get<T>();
  const T* Z = Zr.get<const T>();
  const T al = static_cast<T>(alpha), be = static_cast<T>(beta);   // once per thread
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n;
       o += (int64_t)gridDim.x * blockDim.x) {
    T v = al * A[o];
    if (Z != nullptr) v += be * Z[o];
    Y[o] = v;
  }
}

static unsigned grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 64) b = 152 * 64;
  if (b < 1) b = 1;
  return static_cast<unsigned>(b);
}

static size_t fused_smem(const OpPlan& op, size_t elem) {
  const size_t Wd = FTX + 2 * op.r1, Ht = FTY + 2 * op.r2;
  return (Ht * Wd + Ht * FTX) * elem;
}

int64_t apply_scratch_elems(const OpPlan& op) {
  if (op.fused || op.npass <= 1) return 0;
  int64_t n = 1;
  for (int k = 0; k < op.order; ++k) n *= op.dims[k];
  return n;
}

bool apply_uses_st(const OpPlan& op, int dtype, int tin, int tout) {
  if (tin < 0) tin = dtype;
  if (tout < 0) tout = dtype;
  const bool want = tin == RTG_BF16 || tout == RTG_BF16 || (dtype == RTG_F32 && op.st && op.r4 > 0);
  return want && st_supported(op, tin);
}

int apply_launches(const OpPlan& op, bool combine, int dtype, int tin, int tout) {
  if (op.fused || op.npass == 0 || apply_uses_st(op, dtype, tin, tout)) return 1;
  return op.npass + (combine ? 1 : 0);
}

static bool has_ptr(const PtrRef& r) { return r.base != nullptr || r.ind != nullptr; }

// Tensor map of an FP32 input of the register kernel: dims (I1, I2, planes,
// slots, problems) where `planes` counts the tensor's I1 x I2 planes, slots
// the basis slots of a slot-indexed buffer (1 for a direct pointer) and
// problems the lock-step batch; boxes of the CTA's halo tile (Wd x Ht x NC),
// zero filled outside.  False for inputs read through a pointer slot or a
// ring, or that break the copy engine's 16-byte rules.
static bool make_apply_map(CUtensorMap* m, const PtrRef& X, int64_t I1, int64_t I2, int64_t planes, int Wd, int Ht,
                           int NC, const Batch& b) {
  const PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
  if (fn == nullptr || X.base == nullptr || X.ind != nullptr || X.mod != 0) return false;
  const bool slotted = X.jidx != nullptr;
  if (slotted && X.nslot <= 0) return false;
  const uint64_t pitch = static_cast<uint64_t>(I1) * 4, plane = pitch * static_cast<uint64_t>(I2);
  const uint64_t tens = plane * static_cast<uint64_t>(planes);
  const uint64_t sstride = slotted ? static_cast<uint64_t>(X.stride) * 4 : ((tens + 15) & ~uint64_t(15));
  const uint64_t nslot = slotted ? static_cast<uint64_t>(X.nslot) : 1;
  const uint64_t pstride = b.n > 1 ? static_cast<uint64_t>(b.stride) : ((sstride * nslot + 15) & ~uint64_t(15));
  const uint64_t lim = uint64_t(1) << 40;
  if (reinterpret_cast<uintptr_t>(X.base) % 16 || pitch % 16 || plane % 16 || sstride % 16 || pstride % 16 ||
      sstride < tens || pstride < sstride * nslot || pstride >= lim || I1 > 0x7fffffffll || I2 > 0x7fffffffll ||
      planes > 0x7fffffffll)
    return false;
  const cuuint64_t dims[5] = {static_cast<cuuint64_t>(I1), static_cast<cuuint64_t>(I2),
                              static_cast<cuuint64_t>(planes), nslot, static_cast<cuuint64_t>(b.n)};
  const cuuint64_t strides[4] = {pitch, plane, sstride, pstride};
  const cuuint32_t box[5] = {static_cast<cuuint32_t>(Wd), static_cast<cuuint32_t>(Ht), static_cast<cuuint32_t>(NC), 1u, 1u};
  const cuuint32_t estr[5] = {1u, 1u, 1u, 1u, 1u};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void*>(X.base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T>
static cudaError_t apply_t(const OpPlan& op, PtrRef X, PtrRef Y, double alpha, double beta,
                           PtrRef Z, T* tmp, T* tmp2, const int* stop, cudaStream_t s, Batch b) {
  int64_t n = 1;
  for (int k = 0; k < op.order; ++k) n *= op.dims[k];
  if (n == 0) return cudaSuccess;
  if (op.fused) {
    FusedArgs a{};
    a.I1 = op.dims[0];
    a.I2 = op.order > 1 ? op.dims[1] : 1;
    const int64_t I3 = op.order > 2 ? op.dims[2] : 1;
    int64_t rest = 1;
    for (int k = 3; k < op.order; ++k) rest *= op.dims[k];
    a.r1 = op.r1;
    a.r2 = op.r2;
    for (int t = 0; t <= 2 * op.r1; ++t) a.t1[t] = op.t1[t];
    for (int t = 0; t <= 2 * op.r2; ++t) a.t2[t] = op.t2[t];
    a.alpha = alpha;
    a.beta = has_ptr(Z) ? beta : 0.0;
    for (int t = 0; t < kMaxTaps; ++t) {
      a.t1f[t] = static_cast<float>(a.t1[t]);
      a.t2f[t] = static_cast<float>(a.t2[t]);
    }
    a.alphaf = static_cast<float>(a.alpha);
    a.betaf = static_cast<float>(a.beta);
    if (op.mix > 0) {
      a.nc = op.mix;
      a.nslab = rest;
      for (int i = 0; i < op.mix * op.mix; ++i) a.M[i] = op.M3[i];
    } else {
      a.nc = 1;
      a.nslab = I3 * rest;
      a.M[0] = 1.0;
    }
    for (int i = 0; i < kMaxMix * kMaxMix; ++i) a.Mf[i] = static_cast<float>(a.M[i]);
    const int rr = reg_bucket(op.r1 > op.r2 ? op.r1 : op.r2);
    const bool fits = a.I1 < (int64_t(1) << 30) && a.I2 < (int64_t(1) << 30) &&
                      (sizeof(T) == 8 || (a.I1 % 4) == 0);
    if (rr > 0 && fits && (a.nc == 1 || a.nc == 3)) {
      for (int t = 0; t <= 2 * rr; ++t) {
        const int u1 = t - (rr - op.r1), u2 = t - (rr - op.r2);
        a.t1p[t] = (u1 >= 0 && u1 <= 2 * op.r1) ? a.t1[u1] : 0.0;
        a.t2p[t] = (u2 >= 0 && u2 <= 2 * op.r2) ? a.t2[u2] : 0.0;
        a.t1pf[t] = static_cast<float>(a.t1p[t]);
        a.t2pf[t] = static_cast<float>(a.t2p[t]);
      }
      dim3 grid(static_cast<unsigned>((a.I1 + RTX - 1) / RTX), static_cast<unsigned>((a.I2 + RTY - 1) / RTY),
                batch_z(a.nslab, b));
      cudaError_t e = cudaSuccess;
#define RTG_REG_CASE(NC, RR)                                                                          \
  if (a.nc == NC && rr == RR) {                                                                       \
    using Gm = RegGeom<RR, T>;                                                                        \
    const size_t smem = static_cast<size_t>(NC * Gm::Ht * Gm::Wd + RTY * Gm::Wd) * sizeof(T) + 128;   \
    e = set_smem(k_apply_reg<T, NC, RR>, smem);                                                       \
    if (e != cudaSuccess) return e;                                                                   \
    CUtensorMap xm;                                                                                   \
    std::memset(&xm, 0, sizeof xm);                                                                   \
    const int xtma = (sizeof(T) == 4 && make_apply_map(&xm, X, a.I1, a.I2, a.nslab * NC, Gm::Wd, Gm::Ht, NC, b)) \
                         ? 1 : 0;                                                                     \
    k_apply_reg<T, NC, RR><<<grid, FTHREADS, smem, s>>>(X, Y, Z, stop, a, xm, xtma, b);                  \
    return cudaGetLastError();                                                                        \
  }
      RTG_REG_CASE(1, 3) RTG_REG_CASE(1, 5) RTG_REG_CASE(1, 7) RTG_REG_CASE(1, 9) RTG_REG_CASE(1, 12) RTG_REG_CASE(1, 16)
      RTG_REG_CASE(3, 3) RTG_REG_CASE(3, 5) RTG_REG_CASE(3, 7) RTG_REG_CASE(3, 9) RTG_REG_CASE(3, 12) RTG_REG_CASE(3, 16)
#undef RTG_REG_CASE
    }
    const size_t smem = fused_smem(op, sizeof(T));
    dim3 grid(static_cast<unsigned>((a.I1 + FTX - 1) / FTX),
              static_cast<unsigned>((a.I2 + FTY - 1) / FTY),
              batch_z(a.nslab, b));
    cudaError_t e = cudaSuccess;
    switch (a.nc) {
#define RTG_FUSED_CASE(NC)                                                                        \
  case NC:                                                                                        \
    e = set_smem(k_apply_fused<T, NC>, smem);                                                     \
    if (e != cudaSuccess) return e;                                                               \
    k_apply_fused<T, NC><<<grid, FTHREADS, smem, s>>>(X, Y, Z, stop, a, b);                          \
    break;
      RTG_FUSED_CASE(1)
      RTG_FUSED_CASE(2)
      RTG_FUSED_CASE(3)
      RTG_FUSED_CASE(4)
#undef RTG_FUSED_CASE
      default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  // unfused: one kernel per mode product
  if (op.npass == 0) {
    k_axpby<T><<<dim3(grid_for(n, 256), 1, b.n), 256, 0, s>>>(X, Y, Z, alpha, has_ptr(Z) ? beta : 0.0, n, stop, b);
    return cudaGetLastError();
  }
  PtrRef src = X;
  for (int p = 0; p < op.npass; ++p) {
    const Pass& ps = op.pass[p];
    PtrRef dst = (p == op.npass - 1) ? Y : ref((p % 2 == 0) ? tmp : tmp2);
    int64_t L = 1, R = 1;
    for (int k = 0; k < ps.mode; ++k) L *= op.dims[k];
    for (int k = ps.mode + 1; k < op.order; ++k) R *= op.dims[k];
    const int64_t I = op.dims[ps.mode];
    if (ps.kind == PK_BAND) {
      TapArgs ta{};
      for (int t = 0; t <= 2 * ps.radius; ++t) {
        ta.t[t] = ps.taps[t];
        ta.tf[t] = static_cast<float>(ps.taps[t]);
      }
      k_pass_band<T><<<dim3(grid_for(n, 256), 1, b.n), 256, 0, s>>>(src, dst, L, I, R, ps.radius, ta, stop, b);
    } else {
      k_pass_dense<T><<<dim3(grid_for(n, 256), 1, b.n), 256, 0, s>>>(src, dst, L, I, R, ps.dense, stop, b);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    src = dst;
  }
  if (alpha != 1.0 || has_ptr(Z)) {
    k_axpby<T><<<dim3(grid_for(n, 256), 1, b.n), 256, 0, s>>>(Y, Y, Z, alpha, has_ptr(Z) ? beta : 0.0, n, stop, b);
  }
  return cudaGetLastError();
}

// Frame chunking of the spatio-temporal kernel: about two CTAs per SM.
static void st_chunks(int64_t tiles, int64_t nF, int* F, int* nchunk) {
  int64_t want = (304 + tiles - 1) / tiles;
  if (want < 1) want = 1;
  if (want > nF) want = nF;
  int64_t f = (nF + want - 1) / want;
  *F = static_cast<int>(f);
  *nchunk = static_cast<int>((nF + f - 1) / f);
}

bool st_supported(const OpPlan& op, int tin) {
  if (!op.st) return false;
  const int64_t V = (tin == RTG_BF16) ? 8 : 4;
  return op.dims[0] % V == 0 && st_bucket(op.r1 > op.r2 ? op.r1 : op.r2) > 0;
}

template <typename TI, typename TO>
static cudaError_t apply_st_t(const OpPlan& op, PtrRef X, PtrRef Y, double alpha, double beta,
                              PtrRef Z, const int* stop, cudaStream_t s, Batch b) {
  StArgs a{};
  a.I1 = op.dims[0];
  a.I2 = op.order > 1 ? op.dims[1] : 1;
  a.I3 = op.order > 2 ? op.dims[2] : 1;
  a.nF = op.order > 3 ? op.dims[3] : 1;
  const int nc = op.st_nc;
  const int rr = st_bucket(op.r1 > op.r2 ? op.r1 : op.r2);
  for (int t = 0; t <= 2 * rr; ++t) {
    const int u1 = t - (rr - op.r1), u2 = t - (rr - op.r2);
    a.t1[t] = (u1 >= 0 && u1 <= 2 * op.r1) ? static_cast<float>(op.t1[u1]) : 0.f;
    a.t2[t] = (u2 >= 0 && u2 <= 2 * op.r2) ? static_cast<float>(op.t2[u2]) : 0.f;
  }
  a.rt = op.r4;
  for (int k = 0; k < ST_RING; ++k) {
    const int sft = k - 2;
    a.t4[k] = (sft >= -op.r4 && sft <= op.r4) ? static_cast<float>(op.t4[sft + op.r4]) : 0.f;
  }
  for (int i = 0; i < nc * nc; ++i) a.M[i] = static_cast<float>(op.st_M[i]);
  a.alpha = static_cast<float>(alpha);
  a.beta = has_ptr(Z) ? static_cast<float>(beta) : 0.f;
  const int64_t gx = (a.I1 + STX - 1) / STX, gy = (a.I2 + STY - 1) / STY, groups = a.I3 / nc;
  st_chunks(gx * gy * groups, a.nF, &a.F, &a.nchunk);
  if (groups * a.nchunk * b.n > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy), static_cast<unsigned>(groups * a.nchunk * b.n));
#define RTG_ST_CASE(NC, RR)                                                                         \
  if (nc == NC && rr == RR) {                                                                       \
    using Gm = StGeom<RR, TI>;                                                                      \
    const size_t smem = static_cast<size_t>(NC * Gm::Ht * Gm::Wd + STY * Gm::Wd) * sizeof(float);   \
    cudaError_t e = set_smem(k_apply_st<TI, TO, NC, RR>, smem);                                     \
    if (e != cudaSuccess) return e;                                                                 \
    k_apply_st<TI, TO, NC, RR><<<grid, ST_THREADS, smem, s>>>(X, Y, Z, stop, a, b);                    \
    return cudaGetLastError();                                                                      \
  }
  RTG_ST_CASE(1, 3) RTG_ST_CASE(1, 5) RTG_ST_CASE(1, 7) RTG_ST_CASE(1, 9)
  RTG_ST_CASE(3, 3) RTG_ST_CASE(3, 5) RTG_ST_CASE(3, 7) RTG_ST_CASE(3, 9)
#undef RTG_ST_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_apply(const OpPlan& op, int dtype, PtrRef X, PtrRef Y, double alpha,
                         double beta, PtrRef Z, void* tmp, void* tmp2, const int* stop,
                         cudaStream_t s, int tin, int tout, Batch b) {
  if (tin < 0) tin = dtype;
  if (tout < 0) tout = dtype;
  if (tin == RTG_BF16 || tout == RTG_BF16 || (dtype == RTG_F32 && op.st && op.r4 > 0)) {
    if (!apply_uses_st(op, dtype, tin, tout)) {
      if (tin == RTG_BF16 || tout == RTG_BF16) return cudaErrorInvalidValue;
    } else if (tin == RTG_BF16 && tout == RTG_BF16) {
      return apply_st_t<__nv_bfloat16, __nv_bfloat16>(op, X, Y, alpha, beta, Z, stop, s, b);
    } else if (tin == RTG_F32 && tout == RTG_BF16) {
      return apply_st_t<float, __nv_bfloat16>(op, X, Y, alpha, beta, Z, stop, s, b);
    } else if (tin == RTG_F32 && tout == RTG_F32) {
      return apply_st_t<float, float>(op, X, Y, alpha, beta, Z, stop, s, b);
    } else {
      return cudaErrorInvalidValue;
    }
  }
  if (dtype == RTG_F64)
    return apply_t<double>(op, X, Y, alpha, beta, Z, static_cast<double*>(tmp),
                           static_cast<double*>(tmp2), stop, s, b);
  return apply_t<float>(op, X, Y, alpha, beta, Z, static_cast<float*>(tmp),
                        static_cast<float*>(tmp2), stop, s, b);
}

}  // namespace rtg
