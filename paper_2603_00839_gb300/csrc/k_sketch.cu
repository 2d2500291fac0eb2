// Mode-wise Rademacher sketch S(X) = X x_1 Theta_1 x_2 ... x_d Theta_d
// (Section 3, the global tensor sketching operator; Section 3.1).
//
// Each sketched mode k is one contraction of the current tensor, viewed as
// (L, I_k, R) column-major: Y(l, q, r) = sum_i Theta_k(q, i) X(l, i, r).
// The scale prod_k 1/sqrt(s_k) is applied once, by the last contraction.
//
// FP32 data: every contraction is a GEMM on the tensor cores (BF16 in,
// FP32 accumulate).  Theta_k has entries exactly +-1 in BF16; each FP32
// value x is split into three BF16 limbs h + m + l by truncation (h the top
// 8 significant bits of x, m the top 8 of x - h, l the rest; both
// differences exact in FP32), so the three products per pair carry the full
// 24-bit significand and the sum is accumulated in FP32.  A contraction with
// L = 1 (the first, on mode 1) runs on the fifth-generation tensor cores
// (tcgen05.mma, accumulator in tensor memory): Theta (A operand, 128 rows q
// per CTA) times the columns of X (B operand), Theta expanded once per
// sketch into swizzled shared-memory images.  Later contractions multiply X
// (A operand, rows l) by Theta^T (B operand) with mma.sync m16n8k16, Theta
// expanded into fragment order; a CTA stages its operands in shared memory
// with bulk copies, its 8 warps split K and their partial tiles are summed
// through shared memory, so every stage writes final values.  The last
// contraction of a solve step also takes the first Gram-Schmidt pass: each
// CTA holds a final tile of the sketch and adds its dot products with every
// stored sketched basis vector.
//
// FP64 data: the same chain on CUDA cores with exact sign flips.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <cuda_bf16.h>

#include "gs_common.cuh"
#include "tma_common.cuh"
#include "umma_common.cuh"

namespace rtg {

constexpr int TC_THREADS = 256;   // 8 warps split K
constexpr int N_NT = 4;           // later stages: n8 tiles (32 Theta rows) per CTA
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
        // tcgen05: Theta as 16 KB swizzled images of 128 rows x 64 values of K
        // (every stage with L == 1: after sketch sizes of 1 a later stage is one too)
        sp.stage_umma[t] = 1;
        sp.stage_ntile[t] = static_cast<int>((s + 127) / 128);
        sp.stage_kb[t] = static_cast<int>((I + 63) / 64);
        frag += int64_t(sp.stage_ntile[t]) * sp.stage_kb[t] * 4096;
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
  int64_t s[kMaxOrder], I[kMaxOrder], word_off[kMaxOrder], frag_off[kMaxOrder];
  int wpr[kMaxOrder], kt[kMaxOrder], ntile[kMaxOrder];
  int64_t total_lanes;
  int64_t lane_off[kMaxOrder + 1];
};

// One thread per (tile, k-tile, lane) of every later stage (L > 1): the
// fragment registers of mma.m16n8k16 for Theta^T (the B operand).
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
  // blocked layout: ((block * kt + kk) * N_NT + tile_in_block) * 32 + lane
  constexpr int per = N_NT;
  const int64_t idx = local >> 5;
  const int tin = static_cast<int>(idx % per);
  const int kk = static_cast<int>((idx / per) % a.kt[t]);
  const int64_t blk = idx / (static_cast<int64_t>(per) * a.kt[t]);
  const int64_t tile = blk * per + tin;
  const int64_t tile_k = idx;
  const int gid = lane >> 2, tig = lane & 3;
  const uint32_t* rows = bits + a.word_off[t];
  const int64_t k0 = static_cast<int64_t>(kk) * 16 + tig * 2;
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

// One thread per 16-byte chunk of the first stage's tcgen05 operand: Theta
// rows q of M tile mt and K block kb as a 128-row x 64-value BF16 tile in
// the 128-byte swizzled K-major layout (umma_common.cuh), one 16 KB image
// per (mt, kb), rows q >= s and values i >= I zero.
__global__ void k_theta_image(const uint32_t* bits0, uint32_t* frags0, int64_t word_off, int wpr, int64_t s,
                              int64_t I, int kblocks, int64_t frag_off, int64_t nchunks, Batch bt) {
  const int64_t bo = bidx(bt).off;
  const uint32_t* bits = bsh(bits0, bo);
  uint32_t* frags = bsh(frags0, bo);
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= nchunks) return;
  const uint32_t j = static_cast<uint32_t>(g & 7);
  const uint32_t r = static_cast<uint32_t>((g >> 3) & 127);
  const int64_t tile = g >> 10;                       // mt * kblocks + kb
  const int64_t kb = tile % kblocks, mt = tile / kblocks;
  const int64_t q = mt * 128 + r, i0 = kb * 64 + 8 * j;
  const bool rv = q < s;
  const uint32_t* rb = bits + word_off + (rv ? q : 0) * wpr;
  uint32_t w[4];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const int64_t i = i0 + 2 * h;
    const bool v0 = rv && i < I, v1 = rv && (i + 1) < I;
    w[h] = pm1_pair(v0 ? theta_bit(rb, i) : 0u, v1 ? theta_bit(rb, i + 1) : 0u, v0, v1);
  }
  unsigned char* img = reinterpret_cast<unsigned char*>(frags + frag_off) + tile * 16384;
  *reinterpret_cast<uint4*>(img + sw128_off(r, j)) = make_uint4(w[0], w[1], w[2], w[3]);
}

cudaError_t launch_theta(const SketchPlan& sp, uint32_t* bits, uint32_t* frags, cudaStream_t s,
                         const uint64_t* key_dev, Batch b) {
  cudaError_t e = launch_theta_bits(sp, bits, s, key_dev, b);
  if (e != cudaSuccess || sp.dtype != RTG_F32 || sp.nstage == 0) return e;
  bool frag_stages = false;
  for (int t = 0; t < sp.nstage; ++t) {
    if (!sp.stage_umma[t]) {
      frag_stages = true;
      continue;
    }
    const int k = sp.stage_mode[t];
    const int64_t nchunks = int64_t(sp.stage_ntile[t]) * sp.stage_kb[t] * 1024;
    k_theta_image<<<dim3(static_cast<unsigned>((nchunks + 255) / 256), 1, b.n), 256, 0, s>>>(
        bits, frags, sp.word_off[k], sp.wpr[k], sp.stage_s[t], sp.stage_I[t], sp.stage_kb[t], sp.frag_off[t],
        nchunks, b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (!frag_stages) return cudaSuccess;
  FragArgs a{};
  a.nstage = sp.nstage;
  int64_t lanes = 0;
  for (int t = 0; t < sp.nstage; ++t) {
    if (sp.stage_umma[t]) {   // no fragments for this stage: zero lanes
      a.lane_off[t] = lanes;
      a.kt[t] = 1;
      continue;
    }
    const int k = sp.stage_mode[t];
    a.s[t] = sp.stage_s[t];
    a.I[t] = sp.stage_I[t];
    a.word_off[t] = sp.word_off[k];
    a.frag_off[t] = sp.frag_off[t];
    a.wpr[t] = sp.wpr[k];
    a.kt[t] = sp.stage_kt[t];
    a.ntile[t] = sp.stage_ntile[t];
    a.lane_off[t] = lanes;
    lanes += ((sp.stage_ntile[t] + N_NT - 1) / N_NT) * N_NT * int64_t(sp.stage_kt[t]) * 32;
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

// First contraction on the fifth-generation tensor cores (mode 1, L = 1):
// out(q, c) = scale * sum_i Theta(q, i) X(i, c) as D = A B^T with
// A = Theta (M = 128 rows q per CTA, K = i) and B = the columns of X
// (N = U_BN columns c, K = i), both K-major in shared memory with the
// 128-byte swizzle, D in tensor memory (128 lanes = q, U_BN FP32 columns).
// K runs in blocks of 64, and the CTA's warps take three roles:
//  - warps 0-7 copy their pieces of each block of X into a ring of
//    U_XSTAGES stages (16-byte cp.async, zero fill past the tensor, issued
//    U_XSTAGES blocks ahead), split the staged FP32 values into their three
//    BF16 limbs (split_pair), store them into the swizzled limb tiles (a
//    ring of U_LBUF buffers) and arrive on the buffer's "ready" mbarrier;
//  - warp 8 allocates the tensor memory, waits for ready limbs and the
//    block's Theta image, and one elected lane issues 4 k-slices x LIMBS
//    MMAs accumulating into D and commits them to the mbarriers that free
//    the Theta stage and the limb buffer;
//  - warp 9 fills the Theta ring (16 KB bulk copy per block, the first
//    U_TSTAGES blocks at the start) and refills a stage as soon as its MMAs
//    have completed;
//  - with a tensor map of X (a direct input whose column blocks start on 16
//    bytes), warp 10 fills the X ring instead of the split warps: one tiled
//    TMA copy (cp.async.bulk.tensor) of the 64 x U_BN block per stage, zero
//    filled past the tensor, issued as soon as the split warps have
//    released the stage.
// The copies start before the tensor memory is allocated.  The rings are
// sized for two CTAs per SM (105 KB of shared memory each): with one limb
// buffer the split of block kb + 1 waits for the MMAs of block kb, and the
// other CTA on the SM splits or issues meanwhile (more stages and limb
// buffers at one CTA per SM overlapped the two inside the CTA, which was
// faster for one solve alone and slower for many problems at once).  The
// epilogue (warps 0-7) reads D back (tcgen05.ld, warp w: lanes 32 (w % 4),
// columns U_BN / 2 (w / 4) ..) and stores through the stage's output map,
// advancing the output position without divisions.  X not aligned to 16
// bytes per column block is read with plain loads by the split instead.
constexpr int U_BN = 64;        // columns of X per CTA (MMA N)
constexpr int U_TSTAGES = 3;    // Theta ring
constexpr int U_XSTAGES = 2;    // X ring
constexpr int U_LBUF = 1;       // limb buffers (105 KB in all: two CTAs per SM)
constexpr uint32_t kTileBlk = 5184;   // epilogue staging pitch per 16-row block (U_BN * 20 floats + 16 floats)
constexpr int U_SPLIT = 256;    // threads of the split warps
constexpr int U_THREADS = U_SPLIT + 96;
template <typename TI>
__host__ __device__ constexpr int u_limbs() { return sizeof(TI) == 4 ? 3 : 1; }
template <typename TI>
__host__ __device__ constexpr uint32_t u_xstage_bytes() { return uint32_t(U_BN) * 64u * uint32_t(sizeof(TI)); }
template <typename TI>
__host__ __device__ constexpr uint32_t u_limb_bytes() { return uint32_t(u_limbs<TI>()) * U_BN * 128u; }
template <typename TI>
constexpr size_t u_smem() {   // Theta ring, X ring, limb buffers, alignment slack
  return size_t(U_TSTAGES) * 16384u + size_t(U_XSTAGES) * u_xstage_bytes<TI>() + U_LBUF * size_t(u_limb_bytes<TI>()) +
         1024;
}

template <typename TI>
__global__ void __launch_bounds__(U_THREADS, 1)
k_sk_first_umma(PtrRef Xr, float* __restrict__ out, int64_t I, int64_t R, int64_t s, int kblocks,
                const unsigned char* img, float scale, OutMap om, int* status, int poison, const int* stop,
                const __grid_constant__ CUtensorMap xmap, int xtma, Batch bt) {
  const int prob = bidx(bt).p;   // the problem: the tensor map's third coordinate
  {
    const int64_t bo = bidx(bt).off;
    Xr = Xr.at(bo);
    out = bsh(out, bo);
    img = bsh(img, bo);
    status = bsh(status, bo);
    stop = bsh(stop, bo);
  }
  if (stop != nullptr && *stop) return;
  constexpr int LIMBS = u_limbs<TI>();
  constexpr uint32_t XST = u_xstage_bytes<TI>(), LB = u_limb_bytes<TI>();
  constexpr uint32_t XOFF = U_TSTAGES * 16384u;           // X ring
  constexpr uint32_t LOFF = XOFF + U_XSTAGES * XST;       // limb buffers
  constexpr uint32_t IDESC = umma_idesc_bf16_f32(128, U_BN);
  constexpr int EV = 16 / static_cast<int>(sizeof(TI));   // elements per 16 bytes
  constexpr int UPC = 64 / EV;                            // 16-byte units per column block
  constexpr int UNITS = U_BN * UPC / U_SPLIT;             // units per split thread per block
  static_assert(UNITS * U_SPLIT == U_BN * UPC, "units must divide evenly");
  extern __shared__ __align__(128) unsigned char smem_raw[];   // tiles aligned to 1024 below
  __shared__ __align__(8) uint64_t full[U_TSTAGES], empty[U_TSTAGES], lready[U_LBUF], lfree[U_LBUF];
  __shared__ __align__(8) uint64_t x_full[U_XSTAGES], x_empty[U_XSTAGES];
  __shared__ uint32_t tmem_holder;
  __shared__ int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;               // 1024-byte aligned tiles
  unsigned char* smem = smem_raw + (sbase - raw);
  const TI* X = Xr.get<const TI>();
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * U_BN;
  const int mt = blockIdx.y;
  const int ncol = static_cast<int>((R - c0 < U_BN) ? R - c0 : U_BN);
  // asynchronous column copies need every column block to start on 16 bytes;
  // with the tensor map, warp 10 stages X instead
  const bool acp = !xtma && (I % EV == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0);
  const bool staged = xtma || acp;
  if (tid == 0) {
#pragma unroll
    for (int st = 0; st < U_TSTAGES; ++st) {
      mbar_init(&full[st]);
      mbar_init(&empty[st]);
    }
    for (int b = 0; b < U_LBUF; ++b) {
      mbar_init_n(&lready[b], U_SPLIT);
      mbar_init(&lfree[b]);
    }
    for (int st = 0; st < U_XSTAGES; ++st) {
      mbar_init(&x_full[st]);
      mbar_init_n(&x_empty[st], U_SPLIT);
    }
    s_bad = 0;
  }
  __syncthreads();
  auto rows_of = [&](int kb) {
    const int64_t i0 = static_cast<int64_t>(kb) * 64;
    return static_cast<int>((I - i0 < 64) ? I - i0 : 64);
  };
  auto fail = [&]() { atomicExch(&s_bad, 1); };
  auto failed = [&]() { return *reinterpret_cast<volatile int*>(&s_bad) != 0; };
  bool bad = false;
  if (warp < U_SPLIT / 32) {
    // ---------------------------------------------------------------- split warps
    auto fill_x = [&](int kb) {   // this thread's units of block kb, one cp.async group
      if (acp && kb < kblocks) {
        const int st = kb % U_XSTAGES;
        const int rows = rows_of(kb);
#pragma unroll
        for (int k = 0; k < UNITS; ++k) {
          const int u = tid + k * U_SPLIT;
          const int n = u / UPC, e0 = (u % UPC) * EV;
          const bool v = n < ncol && e0 < rows;
          const TI* src = v ? X + (c0 + n) * I + static_cast<int64_t>(kb) * 64 + e0 : X;
          const unsigned dst = sbase + XOFF + st * XST + static_cast<uint32_t>((n * 64 + e0) * sizeof(TI));
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(v ? 16 : 0)
                       : "memory");
        }
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    for (int kb = 0; kb < U_XSTAGES; ++kb) fill_x(kb);
    for (int kb = 0; kb < kblocks; ++kb) {
      const int st = kb % U_XSTAGES, lb = kb % U_LBUF;
      const int rows = rows_of(kb);
      unsigned char* Ls = smem + LOFF + lb * LB;
      asm volatile("cp.async.wait_group %0;\n" ::"n"(U_XSTAGES - 1) : "memory");   // this thread's units of block kb
      if (xtma && !mbar_wait(&x_full[st], static_cast<uint32_t>((kb / U_XSTAGES) & 1))) fail();   // the TMA block
      if (kb >= U_LBUF && !mbar_wait(&lfree[lb], static_cast<uint32_t>(((kb - U_LBUF) / U_LBUF) & 1))) fail();
      if (failed()) {
        bad = true;
        break;
      }
      const unsigned char* Xs = smem + XOFF + st * XST;
#pragma unroll
      for (int k = 0; k < UNITS; ++k) {
        const int u = tid + k * U_SPLIT;
        const int n = u / UPC, e0 = (u % UPC) * EV;
        if constexpr (sizeof(TI) == 4) {
          float v[4] = {0.f, 0.f, 0.f, 0.f};
          if (staged) {
            const float4 q4 = *reinterpret_cast<const float4*>(Xs + (n * 64 + e0) * 4);
            v[0] = q4.x;
            v[1] = q4.y;
            v[2] = q4.z;
            v[3] = q4.w;
          } else if (n < ncol) {
            const float* src = reinterpret_cast<const float*>(X) + (c0 + n) * I + static_cast<int64_t>(kb) * 64 + e0;
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if (e0 + e < rows) v[e] = __ldcg(src + e);
          }
          uint32_t lo[3], hi[3];
          split_pair(v[0], v[1], lo);
          split_pair(v[2], v[3], hi);
          const uint32_t off = sw128_off(static_cast<uint32_t>(n), static_cast<uint32_t>(e0 >> 3)) + (e0 & 4) * 2u;
#pragma unroll
          for (int l = 0; l < 3; ++l) *reinterpret_cast<uint2*>(Ls + l * (U_BN * 128) + off) = make_uint2(lo[l], hi[l]);
        } else {
          uint4 v = make_uint4(0u, 0u, 0u, 0u);
          if (staged) {
            v = *reinterpret_cast<const uint4*>(Xs + (n * 64 + e0) * 2);
          } else if (n < ncol) {
            const unsigned short* src =
                reinterpret_cast<const unsigned short*>(X) + (c0 + n) * I + static_cast<int64_t>(kb) * 64 + e0;
            uint32_t e16[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) e16[e] = (e0 + e < rows) ? __ldcg(src + e) : 0u;
            v = make_uint4(e16[0] | (e16[1] << 16), e16[2] | (e16[3] << 16), e16[4] | (e16[5] << 16),
                           e16[6] | (e16[7] << 16));
          }
          *reinterpret_cast<uint4*>(Ls + sw128_off(static_cast<uint32_t>(n), static_cast<uint32_t>(e0 >> 3))) = v;
        }
      }
      if (xtma) mbar_arrive(&x_empty[st]);   // this thread is done with the block's X stage
      else fill_x(kb + U_XSTAGES);          // this thread's X stage is free again
      // the limb tiles were written through the generic proxy; the tensor core reads them through the async proxy
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_arrive(&lready[lb]);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
  } else if (warp == U_SPLIT / 32) {
    // ---------------------------------------------------------------- MMA issue
    // the whole warp runs the loop (its operands stay warp-uniform) and one
    // elected lane issues
    tmem_alloc(&tmem_holder, U_BN);
    tc_fence_before();
    __syncwarp();
    tc_fence_after();
    const uint32_t tmem = tmem_holder;
    int last = -1;
    for (int kb = 0; kb < kblocks; ++kb) {
      const int st = kb % U_TSTAGES, lb = kb % U_LBUF;
      const bool ok = mbar_wait(&lready[lb], static_cast<uint32_t>((kb / U_LBUF) & 1)) &&
                      mbar_wait(&full[st], static_cast<uint32_t>((kb / U_TSTAGES) & 1)) && !failed();
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) fail();
        break;
      }
      tc_fence_after();
      const uint32_t a0 = sbase + st * 16384u, b0 = sbase + LOFF + lb * LB;
      if (elect_one()) {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
          for (int l = 0; l < LIMBS; ++l)
            umma_bf16(tmem, umma_desc_sw128(a0 + kk * 32u), umma_desc_sw128(b0 + l * (U_BN * 128u) + kk * 32u),
                      IDESC, (kb | kk | l) != 0 ? 1u : 0u);
        umma_commit(&empty[st]);
        umma_commit(&lfree[lb]);
      }
      __syncwarp();
      last = kb;
    }
    // a failure leaves MMAs in flight: wait (bounded) for the last commit
    if (failed() && last >= 0) mbar_wait(&lfree[last % U_LBUF], static_cast<uint32_t>((last / U_LBUF) & 1));
  } else if (warp == U_SPLIT / 32 + 1) {
    // ---------------------------------------------------------------- Theta ring
    int issued = 0;
    for (int kb = 0; kb < kblocks; ++kb) {
      const int st = kb % U_TSTAGES;
      const bool ok = kb < U_TSTAGES ||
                      (mbar_wait(&empty[st], static_cast<uint32_t>(((kb - U_TSTAGES) / U_TSTAGES) & 1)) && !failed());
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) fail();
        break;
      }
      if (elect_one()) {
        mbar_expect(&full[st], 16384u);
        bulk_g2s(smem + st * 16384u, img + (static_cast<int64_t>(mt) * kblocks + kb) * 16384, 16384u, &full[st]);
      }
      __syncwarp();
      issued = kb + 1;
    }
    // a failure can leave copies in flight: wait (bounded) for the last one of each stage
    if (failed())
      for (int kb = issued - U_TSTAGES > 0 ? issued - U_TSTAGES : 0; kb < issued; ++kb)
        mbar_wait(&full[kb % U_TSTAGES], static_cast<uint32_t>((kb / U_TSTAGES) & 1));
  } else if (xtma) {
    // ---------------------------------------------------------------- X ring (tensor map)
    int issued = 0;
    for (int kb = 0; kb < kblocks; ++kb) {
      const int st = kb % U_XSTAGES;
      const bool ok = kb < U_XSTAGES ||
                      (mbar_wait(&x_empty[st], static_cast<uint32_t>(((kb - U_XSTAGES) / U_XSTAGES) & 1)) && !failed());
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) fail();
        break;
      }
      if (elect_one()) {
        mbar_expect(&x_full[st], XST);
        tma_load_3d(smem + XOFF + st * XST, &xmap, kb * 64, static_cast<int>(c0), prob, &x_full[st]);
      }
      __syncwarp();
      issued = kb + 1;
    }
    if (failed())
      for (int kb = issued - U_XSTAGES > 0 ? issued - U_XSTAGES : 0; kb < issued; ++kb)
        mbar_wait(&x_full[kb % U_XSTAGES], static_cast<uint32_t>((kb / U_XSTAGES) & 1));
  }
  // every MMA has completed once the last commit has arrived
  if (!bad && warp < U_SPLIT / 32 && kblocks > 0 &&
      !mbar_wait(&lfree[(kblocks - 1) % U_LBUF], static_cast<uint32_t>(((kblocks - 1) / U_LBUF) & 1)))
    fail();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_holder;
  bad = failed();
  // whole-tile output: the blocked layout of the next stage with M = 1, the
  // CTA's U_BN columns inside one r2 and inside the tensor, 16-byte aligned
  const bool tile_out = om.blocked && om.M == 1 && om.L == 1 && om.I2 % U_BN == 0 && c0 + U_BN <= R &&
                        (reinterpret_cast<uintptr_t>(out) % 16) == 0;
  if (bad && tid == 0 && status != nullptr) atomicExch(status, RTG_ERR_TIMEOUT);
  tc_fence_after();
  if (warp < U_SPLIT / 32) {
    // warp w: lanes 32 (w % 4) .. (rows q), columns (w / 4) U_BN / 2 .. in chunks of 16
    constexpr int HALF = U_BN / 2;
    const int quarter = warp & 3, half = warp >> 2;
    const int64_t q = static_cast<int64_t>(mt) * 128 + quarter * 32 + lane;
    const float sc = bad ? 1.f : scale;
    const float fill_v = poison ? __int_as_float(0x7fc00000) : 0.f;   // timed out: zeros where the solve records it, else NaN
    // output position of (q, c), advanced column by column without divisions:
    // natural layout pos += L s; blocked layout with M = 1 (the usual case:
    // no unsketched mode between this stage's mode and the next) l2 = L q
    // is fixed and pos += XA until i2 wraps to the next r2
    int64_t c = c0 + half * HALF;
    int64_t pos = 0, rm = 0, i2 = 0, r2 = 0;
    const int64_t Lq = om.L * q, Ls = om.L * om.s;
    if (!om.blocked) {
      pos = om.L * (q + om.s * c);
    } else {
      if (om.small) {
        const uint32_t c32 = static_cast<uint32_t>(c), M32 = static_cast<uint32_t>(om.M);
        const uint32_t rq32 = c32 / M32;
        rm = c32 - rq32 * M32;
        i2 = rq32 % static_cast<uint32_t>(om.I2);
        r2 = rq32 / static_cast<uint32_t>(om.I2);
      } else {
        const int64_t rq = c / om.M;
        rm = c % om.M;
        i2 = rq % om.I2;
        r2 = rq / om.I2;
      }
      const int64_t l2 = Lq + Ls * rm;
      pos = ((r2 * om.LT2 + (l2 >> 4)) * om.I2 + i2) * XA + (l2 & 15);
    }
    static_assert(HALF == 32, "one 32-column tensor-memory load per thread");
    float v[32];
    if (!bad) {
      tmem_ld32(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + static_cast<uint32_t>(half * HALF), v);
    } else {
#pragma unroll
      for (int n = 0; n < 32; ++n) v[n] = fill_v;
    }
    if (tile_out) {
      // the tile in the next stage's blocked layout: per 16-row block of q,
      // U_BN rows of XA floats (16 values of q, 4 pad) at a pitch of 5184
      // bytes (16 banks apart: the two half-warps do not collide)
      float* stg = reinterpret_cast<float*>(smem) + (quarter * 2 + (lane >> 4)) * (kTileBlk / 4);
#pragma unroll
      for (int n = 0; n < 32; ++n) stg[(half * HALF + n) * XA + (lane & 15)] = v[n] * sc;
    } else if (q < s) {
      if (!om.blocked) {
#pragma unroll
        for (int n = 0; n < 32; ++n, ++c, pos += Ls)
          if (c < R) out[pos] = v[n] * sc;
      } else if (om.M == 1) {
        const int64_t wrap = (om.LT2 - 1) * om.I2 * XA;   // from (r2, I2 - 1) to (r2 + 1, 0): XA + wrap
#pragma unroll
        for (int n = 0; n < 32; ++n, ++c) {
          if (c < R) out[pos] = v[n] * sc;
          pos += XA;
          if (++i2 == om.I2) {
            i2 = 0;
            pos += wrap;
          }
        }
      } else {
#pragma unroll
        for (int n = 0; n < 32; ++n, ++c) {
          if (c < R) out[pos] = v[n] * sc;
          if (++rm == om.M) {
            rm = 0;
            if (++i2 == om.I2) {
              i2 = 0;
              ++r2;
            }
          }
          const int64_t l2 = Lq + Ls * rm;
          pos = ((r2 * om.LT2 + (l2 >> 4)) * om.I2 + i2) * XA + (l2 & 15);
        }
      }
    }
  }
  if (tile_out) {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      // one bulk store of U_BN x XA floats per 16-row block of q inside the output
      const int64_t r2 = c0 / om.I2, i20 = c0 % om.I2;
      const int nblk = static_cast<int>((s - static_cast<int64_t>(mt) * 128 + 15) / 16);
      for (int b = 0; b < 8 && b < nblk; ++b) {
        const int64_t l2b = static_cast<int64_t>(mt) * 8 + b;   // q / 16
        bulk_s2g(out + ((r2 * om.LT2 + l2b) * om.I2 + i20) * XA, smem + b * kTileBlk, U_BN * XA * 4u);
      }
      bulk_s2g_commit_and_wait_read();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == U_SPLIT / 32) tmem_dealloc(tmem, U_BN);
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

// Tensor map of a first-stage input X (I x R elements of `elt` bytes per
// problem, problems `b.stride` bytes apart): dims (I, R, problems), boxes of
// 64 x U_BN x 1, zero fill outside.  False when the encoder refuses it or X
// does not meet the copy engine's alignment rules (base, row pitch and
// problem stride multiples of 16 bytes).
static bool make_xmap(CUtensorMap* m, const void* base, size_t elt, int64_t I, int64_t R, const Batch& b) {
  const PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
  if (fn == nullptr || base == nullptr) return false;
  const uint64_t pitch = static_cast<uint64_t>(I) * elt, plane = pitch * static_cast<uint64_t>(R);
  const uint64_t pstride = b.n > 1 ? static_cast<uint64_t>(b.stride) : ((plane + 15) & ~uint64_t(15));
  if (reinterpret_cast<uintptr_t>(base) % 16 || pitch % 16 || pstride % 16 || pstride < plane ||
      pstride >= (uint64_t(1) << 40) || I > 0xffffffffll || R > 0x7fffffffll)
    return false;
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(I), static_cast<cuuint64_t>(R), static_cast<cuuint64_t>(b.n)};
  const cuuint64_t strides[2] = {pitch, pstride};
  const cuuint32_t box[3] = {64u, static_cast<cuuint32_t>(U_BN), 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUresult r = fn(m, elt == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                        const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <typename TI>
static cudaError_t launch_first_umma(PtrRef src, float* dst, const SketchPlan& sp, int t, const uint32_t* fr,
                                     float scale, OutMap om, int* status, int poison, const int* stop,
                                     cudaStream_t s, Batch b) {
  constexpr size_t sm = u_smem<TI>();
  cudaError_t e = set_smem(k_sk_first_umma<TI>, sm);
  if (e != cudaSuccess) return e;
  // a direct input gets a tensor map (the copy engine stages X); an input
  // read through a pointer slot is staged by the split warps
  CUtensorMap xm;
  std::memset(&xm, 0, sizeof xm);
  const int xtma = (src.ind == nullptr && src.jidx == nullptr &&
                    make_xmap(&xm, src.base, sizeof(TI), sp.stage_I[t], sp.stage_R[t], b)) ? 1 : 0;
  const dim3 grid(static_cast<unsigned>((sp.stage_R[t] + U_BN - 1) / U_BN), static_cast<unsigned>(sp.stage_ntile[t]),
                  static_cast<unsigned>(b.n));
  k_sk_first_umma<TI><<<grid, U_THREADS, sm, s>>>(src, dst, sp.stage_I[t], sp.stage_R[t], sp.stage_s[t],
                                                  sp.stage_kb[t], reinterpret_cast<const unsigned char*>(fr), scale,
                                                  om, status, poison, stop, xm, xtma, b);
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
    if (sp.stage_umma[t]) {
      e = (t == 0 && xdtype == RTG_BF16)
              ? launch_first_umma<__nv_bfloat16>(src, dst, sp, t, fr, scale, om, status, poison, stop, s, b)
              : launch_first_umma<float>(src, dst, sp, t, fr, scale, om, status, poison, stop, s, b);
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
