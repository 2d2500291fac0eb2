// Philox4x64-10 and the Rademacher sketch signs (the random projections
// Theta_k of Section 3).
//
// Philox4x64-10 is written from its published definition (Salmon, Moraes,
// Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): the
// round maps (x0,x1,x2,x3) with key (k0,k1) to
// (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1, lo(M0 x0)); after
// each round the key is bumped by the Weyl constants.  Stream word w is
// lane w%4 of the block with counter (w/4 + 1, 0, 0, 0) and key
// (seed, problem_id); sign e is bit e%64 of word e/64, a set bit meaning -1.
#include "rtg_internal.cuh"
#include "philox.cuh"

namespace rtg {

__global__ void k_philox_words(uint64_t seed, uint64_t pid, int64_t n_words, uint64_t* out) {
  int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // one Philox block per thread
  if (4 * b >= n_words) return;
  uint64_t r[4];
  philox4x64_10(static_cast<uint64_t>(b) + 1, 0, 0, 0, seed, pid, r);
  for (int l = 0; l < 4; ++l)
    if (4 * b + l < n_words) out[4 * b + l] = r[l];
}

cudaError_t launch_philox_words(uint64_t seed, uint64_t pid, int64_t n_words, uint64_t* out,
                                cudaStream_t s) {
  if (n_words <= 0) return cudaSuccess;
  int64_t blocks = (n_words + 3) / 4;
  k_philox_words<<<(unsigned)((blocks + 127) / 128), 128, 0, s>>>(seed, pid, n_words, out);
  return cudaGetLastError();
}

struct ThetaArgs {
  int nmodes;                   // sketched modes
  int64_t s[kMaxOrder], I[kMaxOrder], bit_off[kMaxOrder], word_off[kMaxOrder];
  int wpr[kMaxOrder];
  int64_t total_words;
  uint64_t seed, pid;
  const uint64_t* key;          // if set: (seed, pid) read from device memory at run time
};

// One thread per packed 32-bit word: bit b of word (q, w) of mode k holds
// the sign of Theta_k(q, 32 w + b); padding bits past I_k are 0 (+1).
__global__ void k_theta_bits(ThetaArgs a, uint32_t* bits0, Batch bt) {
  const int64_t bo = bidx(bt).off;
  uint32_t* bits = bsh(bits0, bo);
  a.key = bsh(a.key, bo);
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.total_words) return;
  int k = 0;
  while (k + 1 < a.nmodes && t >= a.word_off[k + 1]) ++k;
  int64_t local = t - a.word_off[k];
  int64_t q = local / a.wpr[k];
  int64_t wi = local % a.wpr[k];
  int64_t i0 = wi * 32;
  int64_t e0 = a.bit_off[k] + q * a.I[k] + i0;
  const uint64_t seed = a.key ? a.key[0] : a.seed, pid = a.key ? a.key[1] : a.pid;
  // the 32 signs span at most two 64-bit stream words
  int64_t w0 = e0 / 64;
  uint64_t r[4];
  philox4x64_10(static_cast<uint64_t>(w0 / 4) + 1, 0, 0, 0, seed, pid, r);
  uint64_t word0 = r[w0 % 4];
  uint64_t word1 = word0;
  int64_t w1 = (e0 + 31) / 64;
  if (w1 != w0) {
    if (w1 / 4 != w0 / 4) philox4x64_10(static_cast<uint64_t>(w1 / 4) + 1, 0, 0, 0, seed, pid, r);
    word1 = r[w1 % 4];
  }
  uint32_t out = 0;
  for (int b = 0; b < 32; ++b) {
    if (i0 + b >= a.I[k]) break;
    int64_t e = e0 + b;
    uint64_t wd = (e / 64 == w0) ? word0 : word1;
    out |= static_cast<uint32_t>((wd >> (e % 64)) & 1ull) << b;
  }
  bits[t] = out;
}

cudaError_t launch_theta_bits(const SketchPlan& sp, uint32_t* bits, cudaStream_t s,
                              const uint64_t* key_dev, Batch b) {
  ThetaArgs a{};
  a.key = key_dev;
  int k = 0;
  for (int m = 0; m < sp.order; ++m) {
    if (!sp.sketched[m]) continue;
    a.s[k] = sp.sdims[m];
    a.I[k] = sp.dims[m];
    a.bit_off[k] = sp.bit_off[m];
    a.word_off[k] = sp.word_off[m];
    a.wpr[k] = sp.wpr[m];
    ++k;
  }
  a.nmodes = k;
  a.total_words = sp.total_words;
  a.seed = sp.seed;
  a.pid = sp.pid;
  if (k == 0 || sp.total_words == 0) return cudaSuccess;
  k_theta_bits<<<dim3((unsigned)((sp.total_words + 255) / 256), 1, b.n), 256, 0, s>>>(a, bits, b);
  return cudaGetLastError();
}

}  // namespace rtg
