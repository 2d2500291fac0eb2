// Mode-wise Rademacher sketch S(X) = X x_1 Theta_1 x_2 ... x_d Theta_d
// (Section 3, the global tensor sketching operator; Section 3.1).
//
// Each sketched mode k is one contraction of the current tensor, viewed as
// (L, I_k, R) column-major: Y(l, q, r) = sum_i Theta_k(q, i) X(l, i, r).
// The scale prod_k 1/sqrt(s_k) is applied once, by the last contraction.
//
// FP32 data: every contraction is a GEMM on the tensor cores
// (mma.sync m16n8k16, BF16 in, FP32 accumulate).  Theta_k has entries
// exactly +-1 in BF16; each FP32 value x is split into three BF16 limbs
// h + m + l by truncation (h the top 8 significant bits of x, m the top 8
// of x - h, l the rest; both differences exact in FP32), so the three
// products per pair carry the full 24-bit significand and the sum is
// accumulated in FP32.  The first
// contraction on mode 1 (L = 1) is Theta (A operand, rows q) times the
// columns of X (B operand); later ones multiply X (A operand, rows l) by
// Theta^T (B operand).  Theta is expanded once per sketch into fragment
// order.  A CTA stages its operands (fragments and the data block) in
// shared memory with cp.async in one round trip, its 8 warps split K, and
// their partial tiles are summed through shared memory, so every stage
// writes final values.  The last contraction of a solve step also takes
// the first Gram-Schmidt pass: each CTA holds a final tile of the sketch
// and adds its dot products with every stored sketched basis vector.
//
// FP64 data: the same chain on CUDA cores with exact sign flips.
#include <cuda_bf16.h>

#include "gs_common.cuh"
#include "tma_common.cuh"

namespace rtg {

constexpr int TC_THREADS = 256;   // 8 warps split K
constexpr int F_COLS = 16;        // first stage: columns of X per CTA
constexpr int F_MT = 4;           // first stage: m16 tiles (64 Theta rows) per CTA
constexpr int N_NT = 2;           // later stages: n8 tiles (16 Theta rows) per CTA
constexpr int XA = 20;            // blocked row: 16 values of l + 4 pad (conflict-free A loads)

// ------------------------------------------------------------------ plan

const char* make_sketch_plan(int order, const int64_t* dims, const int64_t* sdims_in,
                             uint64_t seed, uint64_t pid, int dtype, SketchPlan& sp) {
  sp = SketchPlan{};
  if (sdims_in == nullptr) return "sketch_dims is NULL";
  sp.order = order;
  sp.seed = seed;
  sp.pid = pid;
  sp.dtype = dtype;
  int64_t bit = 0, word = 0, d = 1;
  double scale = 1.0;
  for (int k = 0; k < order; ++k) {
    if (sdims_in[k] < 1) return "sketch_dims must be >= 1";
    sp.dims[k] = dims[k];
    if (sdims_in[k] < dims[k]) {
      sp.sketched[k] = 1;
      sp.sdims[k] = sdims_in[k];
      sp.bit_off[k] = bit;
      sp.word_off[k] = word;
      sp.wpr[k] = static_cast<int>((dims[k] + 31) / 32);
      bit += sdims_in[k] * dims[k];
      word += sdims_in[k] * sp.wpr[k];
      scale /= sqrt(static_cast<double>(sdims_in[k]));
    } else {
      sp.sketched[k] = 0;
      sp.sdims[k] = dims[k];
    }
    d *= sp.sdims[k];
  }
  if (d > (int64_t(1) << 31) - 1) return "sketch size too large";
  sp.total_words = word;
  sp.d = d;
  sp.scale = scale;
  // contraction chain in increasing mode order
  int64_t cur[kMaxOrder];
  for (int k = 0; k < order; ++k) cur[k] = dims[k];
  sp.nstage = 0;
  int64_t frag = 0;
  for (int k = 0; k < order; ++k) {
    if (!sp.sketched[k]) continue;
    const int t = sp.nstage++;
    int64_t L = 1, R = 1;
    for (int u = 0; u < k; ++u) L *= cur[u];
    for (int u = k + 1; u < order; ++u) R *= cur[u];
    const int64_t I = cur[k], s = sp.sdims[k];
    sp.stage_mode[t] = k;
    sp.stage_L[t] = L;
    sp.stage_I[t] = I;
    sp.stage_R[t] = R;
    sp.stage_s[t] = s;
    sp.stage_first[t] = (L == 1) ? 1 : 0;
    sp.stage_kt[t] = static_cast<int>((I + 15) / 16);
    sp.stage_out[t] = L * s * R;
    sp.stage_split[t] = 1;
    if (dtype == RTG_F32) {
      sp.frag_off[t] = frag;
      if (sp.stage_first[t]) {
        sp.stage_ntile[t] = static_cast<int>((s + 15) / 16);            // m16 tiles of Theta rows
        const int64_t blocks = (sp.stage_ntile[t] + F_MT - 1) / F_MT;   // F_MT tiles per CTA
        frag += blocks * sp.stage_kt[t] * F_MT * 32 * 4;                // uint4 per lane
      } else {
        sp.stage_ntile[t] = static_cast<int>((s + 7) / 8);             // n8 tiles of Theta rows
        const int64_t blocks = (sp.stage_ntile[t] + N_NT - 1) / N_NT;   // N_NT tiles per CTA
        frag += blocks * sp.stage_kt[t] * N_NT * 32 * 2;                // uint2 per lane
      }
    }
    cur[k] = s;
  }
  sp.frag_words = frag;
  // layouts between stages (FP32 chain)
  int64_t part = 1;
  for (int t = 0; t < sp.nstage; ++t)
    sp.stage_in_blocked[t] = (dtype == RTG_F32 && t > 0 && !sp.stage_first[t]) ? 1 : 0;
  for (int t = 0; t < sp.nstage; ++t) {
    if (t + 1 < sp.nstage) {
      const int k = sp.stage_mode[t], k2 = sp.stage_mode[t + 1];
      int64_t M = 1;
      for (int u = k + 1; u < k2; ++u) M *= dims[u];
      sp.next_M[t] = M;
      sp.next_L[t] = sp.stage_L[t + 1];
      sp.next_I[t] = sp.stage_I[t + 1];
      sp.next_LT[t] = (sp.stage_L[t + 1] + 15) / 16;
      sp.stage_out_alloc[t] = sp.stage_in_blocked[t + 1]
                                  ? sp.stage_R[t + 1] * sp.next_LT[t] * sp.stage_I[t + 1] * 20
                                  : sp.stage_out[t];
      if (sp.stage_out_alloc[t] > part) part = sp.stage_out_alloc[t];
    } else {
      sp.stage_out_alloc[t] = sp.stage_out[t];
    }
  }
  sp.part_elems = part;
  sp.last_split = 1;
  sp.tmp_elems = part;
  sp.fused_dots = (dtype == RTG_F32 && sp.nstage > 0 && !sp.stage_first[sp.nstage - 1]) ? 1 : 0;
  sp.dots_blocks = 0;
  if (sp.fused_dots) {
    const int t = sp.nstage - 1;
    sp.dots_blocks = ((sp.stage_L[t] + 15) / 16) * sp.stage_R[t] * ((sp.stage_ntile[t] + N_NT - 1) / N_NT);
  }
  return nullptr;
}

static size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

size_t sketch_scratch_bytes(const SketchPlan& sp) {
  const size_t elt = sp.dtype == RTG_F64 ? 8 : 4;
  return al256((sp.total_words + 1) * 4) + al256((sp.frag_words + 1) * 4) +
         2 * al256(size_t(sp.part_elems) * elt) + 256 + 256;
}

SketchScratch carve_sketch_scratch(const SketchPlan& sp, void* base) {
  const size_t elt = sp.dtype == RTG_F64 ? 8 : 4;
  char* p = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(base) + 255) & ~uintptr_t(255));
  SketchScratch sc;
  sc.bits = reinterpret_cast<uint32_t*>(p);
  p += al256((sp.total_words + 1) * 4);
  sc.frags = reinterpret_cast<uint32_t*>(p);
  p += al256((sp.frag_words + 1) * 4);
  sc.tmp0 = p;
  p += al256(size_t(sp.part_elems) * elt);
  sc.tmp1 = p;
  return sc;
}

// ------------------------------------------------------------------ Theta fragments

__device__ __forceinline__ uint32_t pm1_pair(uint32_t b0, uint32_t b1, bool v0, bool v1) {
  // packed bf16x2: +1 = 0x3F80, -1 = 0xBF80, padding = 0
  const uint32_t lo = v0 ? (0x3F80u | (b0 << 15)) : 0u;
  const uint32_t hi = v1 ? (0x3F80u | (b1 << 15)) : 0u;
  return lo | (hi << 16);
}

__device__ __forceinline__ uint32_t theta_bit(const uint32_t* rowbits, int64_t i) {
  return (rowbits[i >> 5] >> (i & 31)) & 1u;
}

struct FragArgs {
  int nstage;
  int first[kMaxOrder];
  int64_t s[kMaxOrder], I[kMaxOrder], word_off[kMaxOrder], frag_off[kMaxOrder];
  int wpr[kMaxOrder], kt[kMaxOrder], ntile[kMaxOrder];
  int64_t total_lanes;
  int64_t lane_off[kMaxOrder + 1];
};

// One thread per (tile, k-tile, lane) of every stage: the fragment
// registers of mma.m16n8k16 for Theta (A operand, first stage) or
// Theta^T (B operand, later stages).
__global__ void k_theta_frags(FragArgs a, const uint32_t* bits0, uint32_t* frags0, Batch bt) {
  const int64_t bo = bidx(bt).off;
  const uint32_t* bits = bsh(bits0, bo);
  uint32_t* frags = bsh(frags0, bo);
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= a.total_lanes) return;
  int t = 0;
  while (t + 1 < a.nstage && g >= a.lane_off[t + 1]) ++t;
  const int64_t local = g - a.lane_off[t];
  const int lane = static_cast<int>(local & 31);
  // blocked layout: ((block * kt + kk) * per + tile_in_block) * 32 + lane, per = F_MT or N_NT
  const int per = a.first[t] ? F_MT : N_NT;
  const int64_t idx = local >> 5;
  const int tin = static_cast<int>(idx % per);
  const int kk = static_cast<int>((idx / per) % a.kt[t]);
  const int64_t blk = idx / (static_cast<int64_t>(per) * a.kt[t]);
  const int64_t tile = blk * per + tin;
  const int64_t tile_k = idx;
  const int gid = lane >> 2, tig = lane & 3;
  const uint32_t* rows = bits + a.word_off[t];
  const int64_t k0 = static_cast<int64_t>(kk) * 16 + tig * 2;
  if (a.first[t]) {
    // A (16 x 16, row-major): reg0 (r, k0..k0+1), reg1 (r+8, ..), reg2 (r, k0+8..), reg3 (r+8, k0+8..)
    uint32_t reg[4];
    for (int h = 0; h < 4; ++h) {
      const int64_t q = tile * 16 + gid + ((h & 1) ? 8 : 0);
      const int64_t i = k0 + ((h & 2) ? 8 : 0);
      const bool rv = q < a.s[t];
      const uint32_t* rb = rows + (rv ? q : 0) * a.wpr[t];
      const bool v0 = rv && i < a.I[t], v1 = rv && (i + 1) < a.I[t];
      reg[h] = pm1_pair(v0 ? theta_bit(rb, i) : 0u, v1 ? theta_bit(rb, i + 1) : 0u, v0, v1);
    }
    uint4* out = reinterpret_cast<uint4*>(frags + a.frag_off[t]);
    out[tile_k * 32 + lane] = make_uint4(reg[0], reg[1], reg[2], reg[3]);
  } else {
    // B (16 x 8, "col"): reg0 (k0..k0+1, n), reg1 (k0+8.., n); B(k = i, n = q) = Theta(q, i)
    const int64_t q = tile * 8 + gid;
    const bool rv = q < a.s[t];
    const uint32_t* rb = rows + (rv ? q : 0) * a.wpr[t];
    uint32_t reg[2];
    for (int h = 0; h < 2; ++h) {
      const int64_t i = k0 + (h ? 8 : 0);
      const bool v0 = rv && i < a.I[t], v1 = rv && (i + 1) < a.I[t];
      reg[h] = pm1_pair(v0 ? theta_bit(rb, i) : 0u, v1 ? theta_bit(rb, i + 1) : 0u, v0, v1);
    }
    uint2* out = reinterpret_cast<uint2*>(frags + a.frag_off[t]);
    out[tile_k * 32 + lane] = make_uint2(reg[0], reg[1]);
  }
}

cudaError_t launch_theta(const SketchPlan& sp, uint32_t* bits, uint32_t* frags, cudaStream_t s,
                         const uint64_t* key_dev, Batch b) {
  cudaError_t e = launch_theta_bits(sp, bits, s, key_dev, b);
  if (e != cudaSuccess || sp.dtype != RTG_F32 || sp.nstage == 0) return e;
  FragArgs a{};
  a.nstage = sp.nstage;
  int64_t lanes = 0;
  for (int t = 0; t < sp.nstage; ++t) {
    const int k = sp.stage_mode[t];
    a.first[t] = sp.stage_first[t];
    a.s[t] = sp.stage_s[t];
    a.I[t] = sp.stage_I[t];
    a.word_off[t] = sp.word_off[k];
    a.frag_off[t] = sp.frag_off[t];
    a.wpr[t] = sp.wpr[k];
    a.kt[t] = sp.stage_kt[t];
    a.ntile[t] = sp.stage_ntile[t];
    a.lane_off[t] = lanes;
    const int per = sp.stage_first[t] ? F_MT : N_NT;
    lanes += ((sp.stage_ntile[t] + per - 1) / per) * per * int64_t(sp.stage_kt[t]) * 32;
  }
  a.lane_off[sp.nstage] = lanes;
  a.total_lanes = lanes;
  k_theta_frags<<<dim3(static_cast<unsigned>((lanes + 255) / 256), 1, b.n), 256, 0, s>>>(a, bits, frags, b);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ tensor-core contractions

// Exact three-limb split of a pair of FP32 values into BF16 limbs by
// truncation: h keeps the top 8 significant bits of x (the low 16 bits of
// its encoding cleared), m the top 8 of the exact remainder x - h, and
// l = x - h - m has at most 8 significant bits, so it is a BF16 value too;
// x = h + m + l exactly (normal x).  Each limb is the high half of an FP32
// encoding, so the pairs are packed with one byte permute: out[0] holds
// (h0, h1), out[1] (m0, m1), out[2] (l0, l1), element 0 in the low half.
__device__ __forceinline__ void split_pair(float x0, float x1, uint32_t out[3]) {
  const uint32_t u0 = __float_as_uint(x0), u1 = __float_as_uint(x1);
  const float r0 = x0 - __uint_as_float(u0 & 0xffff0000u);
  const float r1 = x1 - __uint_as_float(u1 & 0xffff0000u);
  const uint32_t v0 = __float_as_uint(r0), v1 = __float_as_uint(r1);
  const float l0 = r0 - __uint_as_float(v0 & 0xffff0000u);
  const float l1 = r1 - __uint_as_float(v1 & 0xffff0000u);
  out[0] = __byte_perm(u0, u1, 0x7632);
  out[1] = __byte_perm(v0, v1, 0x7632);
  out[2] = __byte_perm(__float_as_uint(l0), __float_as_uint(l1), 0x7632);
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

constexpr int F_NT = F_COLS / 8;  // first stage: n8 tiles per CTA
constexpr int F_RED = F_COLS + 1; // padded row of the first stage's cross-warp reduction

template <int CH>
constexpr size_t first_smem() {
  return size_t(CH) * F_MT * 32 * 16 + size_t(F_COLS) * (CH * 16 + 8) * 4 >
                 size_t(8) * F_MT * 16 * F_RED * 4
             ? size_t(CH) * F_MT * 32 * 16 + size_t(F_COLS) * (CH * 16 + 8) * 4
             : size_t(8) * F_MT * 16 * F_RED * 4;
}

// Output placement of a stage: natural column-major (last stage) or blocked
// for the next stage (see SketchPlan).  e_r is the r-part of the natural
// index, already split by the caller into (l-offset, i', r').
struct OutMap {
  int blocked;
  int small;              // every index part below 2^31: 32-bit divisions
  int64_t L, s;           // this stage
  int64_t M, I2, LT2;     // next stage
};
__device__ __forceinline__ int64_t out_pos(const OutMap& om, int64_t l, int64_t q, int64_t r) {
  if (!om.blocked) return l + om.L * (q + om.s * r);
  if (om.small) {
    const uint32_t M = static_cast<uint32_t>(om.M), I2 = static_cast<uint32_t>(om.I2);
    const uint32_t rr = static_cast<uint32_t>(r), rm = rr % M, rq = rr / M;
    const uint32_t L = static_cast<uint32_t>(om.L);
    const uint32_t l2 = static_cast<uint32_t>(l) + L * static_cast<uint32_t>(q) + L * static_cast<uint32_t>(om.s) * rm;
    const uint32_t i2 = rq % I2, r2 = rq / I2;
    return (static_cast<int64_t>(r2) * om.LT2 + l2 / 16) * om.I2 * XA + static_cast<int64_t>(i2) * XA + (l2 % 16);
  }
  const int64_t rm = r % om.M, rq = r / om.M;
  const int64_t l2 = l + om.L * q + om.L * om.s * rm;
  const int64_t i2 = rq % om.I2, r2 = rq / om.I2;
  return ((r2 * om.LT2 + l2 / 16) * om.I2 + i2) * XA + (l2 % 16);
}

// First contraction (mode 1, L = 1): out(q, r) = scale * sum_i Theta(q, i) X(i, r).
// CTA: 64 rows of Theta x 16 columns of X.  Each K chunk (CH tiles) arrives
// by TMA bulk copies: one for the Theta fragments, one per column of X.
// Warp w takes the K tiles w, w+8, ...; the 8 partial tiles are summed in
// shared memory.
template <int CH, typename TI>
__global__ void __launch_bounds__(TC_THREADS)
k_sk_first_tc(PtrRef Xr, float* __restrict__ out, int64_t I, int64_t R, int64_t s, int kt_total,
              const uint4* fragA, int mt_total, float scale, OutMap om,
              int* status, int poison, const int* stop, Batch bt) {
  {
    const int64_t bo = bidx(bt).off;
    Xr = Xr.at(bo);
    out = bsh(out, bo);
    fragA = bsh(fragA, bo);
    status = bsh(status, bo);
    stop = bsh(stop, bo);
  }
  if (stop != nullptr && *stop) return;
  // BF16 data are exact in one limb; FP32 data take three (see split_pair)
  constexpr int LIMBS = sizeof(TI) == 4 ? 3 : 1;
  constexpr int EV = 16 / static_cast<int>(sizeof(TI));   // elements per 16 bytes
  const TI* X = Xr.get<const TI>();
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  constexpr int XS = CH * 16 + 8;
  uint4* fA = reinterpret_cast<uint4*>(smem);                                   // [CH][F_MT][32]
  TI* xs = reinterpret_cast<TI*>(smem + size_t(CH) * F_MT * 32 * 16);             // [F_COLS][XS]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, gid = lane >> 2, tig = lane & 3;
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * F_COLS;
  const int mb = blockIdx.y;
  const int nmt = min(F_MT, mt_total - mb * F_MT);
  const bool bulk = (I % EV == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0);
  if (tid == 0) mbar_init(&bar);
  __syncthreads();
  float acc[F_MT][F_NT][4];
#pragma unroll
  for (int a = 0; a < F_MT; ++a)
#pragma unroll
    for (int b = 0; b < F_NT; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  bool ok = true;
  uint32_t phase = 0;
  for (int kc0 = 0; kc0 < kt_total; kc0 += CH) {
    const int nk = min(CH, kt_total - kc0);
    const int64_t i0 = static_cast<int64_t>(kc0) * 16;
    const int rows = static_cast<int>((static_cast<int64_t>(nk) * 16 < I - i0) ? static_cast<int64_t>(nk) * 16 : I - i0);   // valid rows of X
    const int ncol = static_cast<int>((static_cast<int64_t>(F_COLS) < R - c0) ? static_cast<int64_t>(F_COLS) : R - c0);
    if (warp == 0) {   // lane 0 announces the bytes; the lanes issue one copy each
      const uint32_t fbytes = static_cast<uint32_t>(nk) * F_MT * 32 * 16;
      const uint32_t xbytes = bulk ? static_cast<uint32_t>(ncol) * rows * sizeof(TI) : 0u;
      if (lane == 0) mbar_expect(&bar, fbytes + xbytes);
      __syncwarp();
      if (lane == 0) bulk_g2s(fA, fragA + (static_cast<int64_t>(mb) * kt_total + kc0) * F_MT * 32, fbytes, &bar);
      if (bulk && lane < ncol)
        bulk_g2s(&xs[lane * XS], X + (c0 + lane) * I + i0, static_cast<uint32_t>(rows * sizeof(TI)), &bar);
    }
    // zero the rows and columns the copies do not cover; without bulk, plain loads
    if (!bulk || ncol < F_COLS || rows < nk * 16) {
      for (int idx = tid; idx < F_COLS * nk * 16; idx += TC_THREADS) {
        const int col = idx / (nk * 16), k = idx - col * (nk * 16);
        if (bulk && col < ncol && k < rows) continue;
        xs[col * XS + k] = (col < ncol && k < rows) ? X[(c0 + col) * I + i0 + k] : static_cast<TI>(0.f);
      }
    }
    if (tc_wait_failed(&bar, phase, status)) {
      ok = false;
      break;
    }
    phase ^= 1u;
    {
      for (int kk = warp; kk < nk; kk += 8) {
        uint32_t B[F_NT][2][3];
#pragma unroll
        for (int nt = 0; nt < F_NT; ++nt)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const TI* xp = &xs[(nt * 8 + gid) * XS + kk * 16 + tig * 2 + h * 8];
            if constexpr (sizeof(TI) == 4) {
              const float2 v = *reinterpret_cast<const float2*>(xp);
              split_pair(v.x, v.y, B[nt][h]);
            } else {
              B[nt][h][0] = *reinterpret_cast<const uint32_t*>(xp);   // two BF16 values, k and k+1
            }
          }
        uint32_t A[F_MT][4];
#pragma unroll
        for (int mt = 0; mt < F_MT; ++mt) {
          const uint4 av = fA[(kk * F_MT + mt) * 32 + lane];
          A[mt][0] = av.x;
          A[mt][1] = av.y;
          A[mt][2] = av.z;
          A[mt][3] = av.w;
        }
        // limb-outer order: consecutive MMAs update independent accumulators
#pragma unroll
        for (int l = 0; l < LIMBS; ++l)
#pragma unroll
          for (int mt = 0; mt < F_MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < F_NT; ++nt) mma_bf16(acc[mt][nt], A[mt], B[nt][0][l], B[nt][1][l]);
      }
    }
    __syncthreads();
  }
  if (!ok) {   // timed out: zeros where the solve records the timeout, else NaN (never a silent partial sum)
    const float fill = poison ? __int_as_float(0x7fc00000) : 0.f;
#pragma unroll
    for (int a = 0; a < F_MT; ++a)
#pragma unroll
      for (int b = 0; b < F_NT; ++b)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][b][c] = fill;
  }
  __syncthreads();
  constexpr int ROWS = F_MT * 16;
  float* red = reinterpret_cast<float*>(smem);                // [8][ROWS][F_RED]
#pragma unroll
  for (int mt = 0; mt < F_MT; ++mt)
#pragma unroll
    for (int nt = 0; nt < F_NT; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = mt * 16 + gid + h * 8, col = nt * 8 + tig * 2;
        red[(warp * ROWS + row) * F_RED + col] = acc[mt][nt][2 * h];
        red[(warp * ROWS + row) * F_RED + col + 1] = acc[mt][nt][2 * h + 1];
      }
  __syncthreads();
  for (int idx = tid; idx < ROWS * F_COLS; idx += TC_THREADS) {
    const int row = idx % ROWS, col = idx / ROWS;
    const int64_t q = static_cast<int64_t>(mb) * ROWS + row, c = c0 + col;
    if (q >= s || c >= R || row >= nmt * 16) continue;
    float v = 0.f;
#pragma unroll
    for (int wv = 0; wv < 8; ++wv) v += red[(wv * ROWS + row) * F_RED + col];
    out[out_pos(om, 0, q, c)] = v * scale;
  }
}

// Dynamic shared memory of the later stage: the K chunk (fragments and
// blocked input) during the contraction, then the reduction scratch of the
// fused Gram-Schmidt pass (GS_MAXW rows of partial sums and the totals).
template <int CH>
constexpr size_t inner_smem() {
  constexpr size_t mma = size_t(CH) * N_NT * 32 * 8 + size_t(CH) * 16 * XA * 4;
  constexpr size_t red = size_t(GS_MAXW + 1) * kRedCols * 8;
  return mma > red ? mma : red;
}

// Later contraction (L > 1): out(l, q, r) = scale * sum_i X(l, i, r) Theta(q, i).
// CTA: 16 values of l x 8 N_NT values of q for one r.  Input blocked for this
// stage (one bulk copy of I rows x 20 floats per K chunk) or natural
// (plain loads).  Warp w takes the K tiles w, w+8, ...  With dots_pass >= 0
// the CTA then runs that Gram-Schmidt pass on its final tile.
template <int CH>
__global__ void __launch_bounds__(TC_THREADS, 3)
k_sk_inner_tc(PtrRef Xr, int in_blocked, float* __restrict__ out, int64_t L, int64_t I, int64_t R,
              int64_t s, int kt_total, const uint2* fragB, int nt_total, float scale,
              OutMap om, int dots_pass, Work w, StepOpts o, int* status, int poison, const int* stop,
              Batch bt) {
  {
    const int64_t bo = bidx(bt).off;
    Xr = Xr.at(bo);
    out = bsh(out, bo);
    fragB = bsh(fragB, bo);
    w = w.at(bo);
    o = o.at(bo);
    status = bsh(status, bo);
    stop = bsh(stop, bo);
  }
  if (stop != nullptr && *stop) return;
  const float* X = Xr.get<const float>();
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  uint2* fB = reinterpret_cast<uint2*>(smem);                                    // [CH][N_NT][32]
  float* xa = reinterpret_cast<float*>(smem + size_t(CH) * N_NT * 32 * 8);        // [CH*16][XA]
  __shared__ int am_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, gid = lane >> 2, tig = lane & 3;
  const int64_t ltiles = (L + 15) / 16;
  const int64_t lt = blockIdx.x % ltiles, r = blockIdx.x / ltiles;
  const int64_t l0 = lt * 16;
  const int nb = blockIdx.y;
  const int nt0 = nb * N_NT;
  const bool bulk_in = in_blocked && (reinterpret_cast<uintptr_t>(X) % 16 == 0);
  if (tid == 0) mbar_init(&bar);
  __syncthreads();
  float acc[N_NT][4];
#pragma unroll
  for (int a = 0; a < N_NT; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;
  bool ok = true;
  uint32_t phase = 0;
  for (int kc0 = 0; kc0 < kt_total; kc0 += CH) {
    const int nk = min(CH, kt_total - kc0);
    const int64_t i0 = static_cast<int64_t>(kc0) * 16;
    const int rows = static_cast<int>((static_cast<int64_t>(nk) * 16 < I - i0) ? static_cast<int64_t>(nk) * 16 : I - i0);
    if (tid == 0) {
      const uint32_t fbytes = static_cast<uint32_t>(nk) * N_NT * 32 * 8;
      const uint32_t xbytes = bulk_in ? static_cast<uint32_t>(rows) * XA * 4 : 0u;
      mbar_expect(&bar, fbytes + xbytes);
      bulk_g2s(fB, fragB + (static_cast<int64_t>(nb) * kt_total + kc0) * N_NT * 32, fbytes, &bar);
      if (bulk_in) bulk_g2s(xa, X + ((r * ltiles + lt) * I + i0) * XA, static_cast<uint32_t>(rows) * XA * 4, &bar);
    }
    // rows past I are zero; without bulk input, load the natural layout
    if (!bulk_in || rows < nk * 16)
    for (int idx = tid; idx < nk * 16 * 16; idx += TC_THREADS) {
      const int k = idx >> 4, ll = idx & 15;
      if (k < rows && bulk_in) continue;
      float v = 0.f;
      if (k < rows) {
        if (in_blocked) v = __ldcg(&X[((r * ltiles + lt) * I + i0 + k) * XA + ll]);
        else if (l0 + ll < L) v = __ldcg(&X[l0 + ll + L * (i0 + k) + L * I * r]);
      }
      xa[k * XA + ll] = v;
    }
    if (tc_wait_failed(&bar, phase, status)) {
      ok = false;
      break;
    }
    phase ^= 1u;
    {
      for (int kk = warp; kk < nk; kk += 8) {
        uint32_t A[3][4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const int l = gid + ((h & 1) ? 8 : 0);
          const int k = kk * 16 + tig * 2 + ((h & 2) ? 8 : 0);
          uint32_t lim[3];
          split_pair(xa[k * XA + l], xa[(k + 1) * XA + l], lim);
          A[0][h] = lim[0];
          A[1][h] = lim[1];
          A[2][h] = lim[2];
        }
        uint2 Bv[N_NT];
#pragma unroll
        for (int nt = 0; nt < N_NT; ++nt) Bv[nt] = fB[(kk * N_NT + nt) * 32 + lane];
#pragma unroll
        for (int l = 0; l < 3; ++l)
#pragma unroll
          for (int nt = 0; nt < N_NT; ++nt) mma_bf16(acc[nt], A[l], Bv[nt].x, Bv[nt].y);
      }
    }
    __syncthreads();
  }
  if (!ok) {   // timed out: zeros where the solve records the timeout (the CTA still takes
               // part in the dots), else NaN (never a silent partial sum)
    const float fill = poison ? __int_as_float(0x7fc00000) : 0.f;
#pragma unroll
    for (int nt = 0; nt < N_NT; ++nt)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[nt][c] = fill;
  }
  __syncthreads();
  float* red = reinterpret_cast<float*>(smem);               // [8][16][N_NT*8]
  constexpr int TW = N_NT * 8;
#pragma unroll
  for (int nt = 0; nt < N_NT; ++nt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int l = gid + h * 8, q = nt * 8 + tig * 2;
      red[(warp * 16 + l) * TW + q] = acc[nt][2 * h];
      red[(warp * 16 + l) * TW + q + 1] = acc[nt][2 * h + 1];
    }
  __syncthreads();
  constexpr int ITEMS = (16 * TW + TC_THREADS - 1) / TC_THREADS;
  float vals[ITEMS];
  int64_t ix[ITEMS];
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    vals[k] = 0.f;   // entries outside the tensor are marked invalid (index -1)
    ix[k] = -1;
    const int e = tid + k * TC_THREADS;
    if (e >= 16 * TW) continue;
    const int l = e & 15, q = e >> 4;
    const int64_t gl = l0 + l, gq = static_cast<int64_t>(nt0) * 8 + q;
    if (gl >= L || gq >= s) continue;
    float v = 0.f;
#pragma unroll
    for (int wv = 0; wv < 8; ++wv) v += red[(wv * 16 + l) * TW + q];
    v *= scale;
    const int64_t g = out_pos(om, gl, gq, r);
    out[g] = v;
    vals[k] = v;
    ix[k] = g;
  }
  if (dots_pass < 0) return;
  const int J = (dots_pass == 0) ? -1 : w.ctl->j;
  // the reduction scratch reuses the dynamic shared memory
  __syncthreads();
  double(*red2)[kRedCols] = reinterpret_cast<double(*)[kRedCols]>(smem);
  double* tot = reinterpret_cast<double*>(smem) + GS_MAXW * kRedCols;
  block_partials<float, ITEMS>(w, vals, ix, ITEMS, J, red2);
  double* fin_sh = &red2[0][0];
  auto stage = [&]() { if (dots_pass > 0) gs_stage_gram_async(w, J, fin_sh); };
  if (!last_block_combine<true>(w, gs_ncols(J), tot, &am_last, &red2[0][0], stage)) return;
  if (dots_pass == 0) {
    if (tid == 0) gs_finish_start(w, o, tot);
  } else {
    gs_finish_gram(w, o, tot, &red2[0][0], true);
  }
}

// ------------------------------------------------------------------ CUDA-core chain (FP64)

// Y(l, q, r) = scale * sum_i (-1)^bit(q, i) X(l, i, r)
template <typename T>
__global__ void k_sketch_mode(PtrRef Xr, T* __restrict__ Y, int64_t L, int64_t I, int64_t R,
                              int64_t s, const uint32_t* bits, int wpr, T scale,
                              const int* stop, Batch bt) {
  {
    const int64_t bo = bidx(bt).off;
    Xr = Xr.at(bo);
    Y = bsh(Y, bo);
    bits = bsh(bits, bo);
    stop = bsh(stop, bo);
  }
  if (stop != nullptr && *stop) return;
  const T* X = Xr.get<const T>();
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
      const uint32_t b = __ldcg(brow + w);
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
__global__ void k_copy(PtrRef Xr, T* __restrict__ Y, int64_t n, const int* stop, Batch bt) {
  {
    const int64_t bo = bidx(bt).off;
    Xr = Xr.at(bo);
    Y = bsh(Y, bo);
    stop = bsh(stop, bo);
  }
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

int sketch_launches(const SketchPlan& sp) { return sp.nstage == 0 ? 1 : sp.nstage; }

static cudaError_t sketch_f64(const SketchPlan& sp, const SketchScratch& sc, PtrRef X, double* out,
                              const int* stop, cudaStream_t s, Batch b) {
  PtrRef src = X;
  for (int t = 0; t < sp.nstage; ++t) {
    const int k = sp.stage_mode[t];
    const bool last = (t == sp.nstage - 1);
    double* dst = last ? out : static_cast<double*>((t % 2 == 0) ? sc.tmp0 : sc.tmp1);
    const double scale = last ? sp.scale : 1.0;
    k_sketch_mode<double><<<dim3(grid_for(sp.stage_out[t]), 1, b.n), 256, 0, s>>>(
        src, dst, sp.stage_L[t], sp.stage_I[t], sp.stage_R[t], sp.stage_s[t],
        sc.bits + sp.word_off[k], sp.wpr[k], scale, stop, b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    src = ref(dst);
  }
  return cudaSuccess;
}

static OutMap stage_out_map(const SketchPlan& sp, int t) {
  OutMap om{};
  om.L = sp.stage_L[t];
  om.s = sp.stage_s[t];
  om.blocked = (t + 1 < sp.nstage) ? sp.stage_in_blocked[t + 1] : 0;
  om.M = om.blocked ? sp.next_M[t] : 1;
  om.I2 = om.blocked ? sp.next_I[t] : 1;
  om.LT2 = om.blocked ? sp.next_LT[t] : 1;
  // l2 < L s M and r < R (the stage's columns) stay below 2^31
  om.small = (om.L * om.s * om.M < (int64_t(1) << 31)) && (sp.stage_R[t] < (int64_t(1) << 31)) ? 1 : 0;
  return om;
}

template <int CH, typename TI>
static cudaError_t launch_first(dim3 grid, PtrRef src, float* dst, const SketchPlan& sp, int t, int kt,
                                const uint32_t* fr, float scale, OutMap om, int* status, int poison,
                                const int* stop, cudaStream_t s, Batch b) {
  constexpr size_t sm = first_smem<CH>();
  cudaError_t e = set_smem(k_sk_first_tc<CH, TI>, sm);
  if (e != cudaSuccess) return e;
  k_sk_first_tc<CH, TI><<<grid, TC_THREADS, sm, s>>>(src, dst, sp.stage_I[t], sp.stage_R[t], sp.stage_s[t], kt,
                                                     reinterpret_cast<const uint4*>(fr), sp.stage_ntile[t],
                                                     scale, om, status, poison, stop, b);
  return cudaGetLastError();
}

static cudaError_t sketch_f32(const SketchPlan& sp, const SketchScratch& sc, PtrRef X, float* out,
                              const SketchDots* dots, const int* stop, cudaStream_t s, int xdtype, Batch b) {
  PtrRef src = X;
  for (int t = 0; t < sp.nstage; ++t) {
    const bool last = (t == sp.nstage - 1);
    float* dst = last ? out : static_cast<float*>((t % 2 == 0) ? sc.tmp0 : sc.tmp1);
    const float scale = last ? static_cast<float>(sp.scale) : 1.f;
    const int kt = sp.stage_kt[t];
    const uint32_t* fr = sc.frags + sp.frag_off[t];
    const OutMap om = stage_out_map(sp, t);
    // a bounded wait that gives up is recorded in the solve's status when the
    // chain belongs to a solve with fused dots; elsewhere nothing would read a
    // status word, so the affected outputs become NaN instead
    int* status = (dots != nullptr) ? &dots->w->ctl->status : nullptr;
    const int poison = (dots != nullptr) ? 0 : 1;
    cudaError_t e = cudaSuccess;
    if (sp.stage_first[t]) {
      dim3 grid(static_cast<unsigned>((sp.stage_R[t] + F_COLS - 1) / F_COLS),
                static_cast<unsigned>((sp.stage_ntile[t] + F_MT - 1) / F_MT), static_cast<unsigned>(b.n));
      const bool bf = (t == 0 && xdtype == RTG_BF16);
      // K chunks of 16 tiles up to I = 512 (about 50 KB of shared memory, four
      // CTAs per SM: in throughput the occupancy outweighs the second chunk's load)
      if (kt > 32)
        e = bf ? launch_first<32, __nv_bfloat16>(grid, src, dst, sp, t, kt, fr, scale, om, status, poison, stop, s, b)
               : launch_first<32, float>(grid, src, dst, sp, t, kt, fr, scale, om, status, poison, stop, s, b);
      else
        e = bf ? launch_first<16, __nv_bfloat16>(grid, src, dst, sp, t, kt, fr, scale, om, status, poison, stop, s, b)
               : launch_first<16, float>(grid, src, dst, sp, t, kt, fr, scale, om, status, poison, stop, s, b);
    } else {
      const int64_t ltiles = (sp.stage_L[t] + 15) / 16;
      dim3 grid(static_cast<unsigned>(ltiles * sp.stage_R[t]),
                static_cast<unsigned>((sp.stage_ntile[t] + N_NT - 1) / N_NT), static_cast<unsigned>(b.n));
      const int dpass = (last && dots != nullptr) ? dots->pass : -1;
      const Work wk = (dots != nullptr) ? *dots->w : Work{};
      const StepOpts so = (dots != nullptr) ? dots->o : StepOpts{};
      const int inb = sp.stage_in_blocked[t];
      if (kt > 16) {
        constexpr size_t sm = inner_smem<32>();
        e = set_smem(k_sk_inner_tc<32>, sm);
        if (e != cudaSuccess) return e;
        k_sk_inner_tc<32><<<grid, TC_THREADS, sm, s>>>(src, inb, dst, sp.stage_L[t], sp.stage_I[t],
                                                       sp.stage_R[t], sp.stage_s[t], kt,
                                                       reinterpret_cast<const uint2*>(fr), sp.stage_ntile[t],
                                                       scale, om, dpass, wk, so, status, poison, stop, b);
      } else {
        constexpr size_t sm = inner_smem<16>();
        e = set_smem(k_sk_inner_tc<16>, sm);
        if (e != cudaSuccess) return e;
        k_sk_inner_tc<16><<<grid, TC_THREADS, sm, s>>>(src, inb, dst, sp.stage_L[t], sp.stage_I[t],
                                                       sp.stage_R[t], sp.stage_s[t], kt,
                                                       reinterpret_cast<const uint2*>(fr), sp.stage_ntile[t],
                                                       scale, om, dpass, wk, so, status, poison, stop, b);
      }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    src = ref(dst);
  }
  return cudaSuccess;
}

cudaError_t launch_sketch(const SketchPlan& sp, const SketchScratch& sc, PtrRef X, void* out,
                          const SketchDots* dots, const int* stop, cudaStream_t s, int xdtype, Batch b) {
  if (xdtype < 0) xdtype = sp.dtype;
  // BF16 input is read only by a first stage on mode 1 (FP32 plans)
  if (xdtype == RTG_BF16 && (sp.dtype != RTG_F32 || sp.nstage == 0 || !sp.stage_first[0]))
    return cudaErrorInvalidValue;
  int64_t n = 1;
  for (int k = 0; k < sp.order; ++k) n *= sp.dims[k];
  if (sp.nstage == 0) {     // no sketched mode: S = identity
    const dim3 g(grid_for(n), 1, static_cast<unsigned>(b.n));
    if (sp.dtype == RTG_F64) k_copy<double><<<g, 256, 0, s>>>(X, static_cast<double*>(out), n, stop, b);
    else k_copy<float><<<g, 256, 0, s>>>(X, static_cast<float*>(out), n, stop, b);
    return cudaGetLastError();
  }
  if (sp.dtype == RTG_F64) return sketch_f64(sp, sc, X, static_cast<double*>(out), stop, s, b);
  return sketch_f32(sp, sc, X, static_cast<float*>(out), sp.fused_dots ? dots : nullptr, stop, s, xdtype, b);
}

}  // namespace rtg
