// rtg_sketch_noalloc: the sketch S(X) for callers that cannot allocate
// device memory.
//
// rtg_sketch keeps its scratch (the packed Rademacher signs and the
// intermediates of the mode-wise contraction chain) in buffers that its
// handle allocates with cudaMalloc.  Some callers cannot do that: code
// running next to a framework that has already reserved the device memory
// for its own pool, or latency-critical code that cannot afford the
// implicit device synchronisation of cudaMalloc/cudaFree.  This entry point
// instead uses one fixed array in the library's static device memory, so
// it allocates nothing.  That array (kNoAllocBytes) is held by every GPU
// that loads the library, until the process exits.
#include <cstdio>
#include <mutex>

#include "rtg_internal.cuh"

namespace {

constexpr size_t kNoAllocBytes = size_t(4) << 20;   // 4 MiB of static device scratch

// Shared by every call on a device; keeps the contents of the last call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};


// In host code the symbol is only a host-side stand-in: the device address
// comes from cudaGetSymbolAddress, once per device, with that device current.
cudaError_t scratch_address(int device, void** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_addr[device] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

// The message is what rtg_last_error() returns afterwards.
rtg_status noalloc_fail(rtg_status st, const char* msg) {
  rtg::record_error(msg);
  return st;
}

bool on_device(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" rtg_status rtg_sketch_noalloc(rtg_shape shape, rtg_dtype dtype,
                                         const int64_t* sketch_dims, uint64_t seed,
                                         uint64_t problem_id, const void* X, void* SX,
                                         rtg_stream stream) {
  using namespace rtg;
  if (dtype != RTG_F64 && dtype != RTG_F32) return noalloc_fail(RTG_ERR_UNSUPPORTED, "dtype must be RTG_F64 or RTG_F32");
  if (shape.order < 1 || shape.order > kMaxOrder) return noalloc_fail(RTG_ERR_INVALID_ARG, "shape.order must be 1..4");
  if (sketch_dims == nullptr || X == nullptr || SX == nullptr || X == SX)
    return noalloc_fail(RTG_ERR_INVALID_ARG, "sketch_dims, X and SX must be non-NULL and SX must not alias X");
  if (!on_device(X) || !on_device(SX)) return noalloc_fail(RTG_ERR_INVALID_ARG, "X and SX must be device pointers");
  SketchPlan sp{};
  sp.order = shape.order;
  sp.seed = seed;
  sp.pid = problem_id;
  int64_t bit = 0, word = 0, d = 1;
  double scale = 1.0;
  for (int k = 0; k < shape.order; ++k) {
    if (shape.dims[k] < 1 || shape.dims[k] > (int64_t(1) << 31)) return noalloc_fail(RTG_ERR_INVALID_ARG, "shape.dims must be in 1..2^31");
    if (sketch_dims[k] < 1) return noalloc_fail(RTG_ERR_INVALID_ARG, "sketch_dims must be >= 1");
    sp.dims[k] = shape.dims[k];
    if (sketch_dims[k] < shape.dims[k]) {
      sp.sketched[k] = 1;
      sp.sdims[k] = sketch_dims[k];
      sp.bit_off[k] = bit;
      sp.word_off[k] = word;
      sp.wpr[k] = static_cast<int>((shape.dims[k] + 31) / 32);
      bit += sketch_dims[k] * shape.dims[k];
      word += sketch_dims[k] * sp.wpr[k];
      scale /= sqrt(static_cast<double>(sketch_dims[k]));
    } else {
      sp.sdims[k] = shape.dims[k];
    }
    d *= sp.sdims[k];
  }
  sp.total_words = word;
  sp.d = d;
  sp.scale = scale;
  int64_t cur[kMaxOrder], tmx = 1;
  int last = -1;
  for (int k = 0; k < shape.order; ++k) {
    cur[k] = shape.dims[k];
    if (sp.sketched[k]) last = k;
  }
  for (int k = 0; k < shape.order; ++k) {
    if (!sp.sketched[k]) continue;
    cur[k] = sp.sdims[k];
    if (k == last) break;
    int64_t sz = 1;
    for (int u = 0; u < shape.order; ++u) sz *= cur[u];
    if (sz > tmx) tmx = sz;
  }
  sp.tmp_elems = tmx;
  // scratch layout: [sign bits | intermediate 0 | intermediate 1], 256-byte aligned
  const size_t elt = dtype == RTG_F64 ? 8 : 4;
  const size_t bits_bytes = ((size_t(word) + 1) * 4 + 255) & ~size_t(255);
  const size_t tmp_bytes = (size_t(tmx) * elt + 255) & ~size_t(255);
  const size_t need = bits_bytes + 2 * tmp_bytes;
  if (need > kNoAllocBytes) {
    char msg[256];
    snprintf(msg, sizeof msg, "sketch needs %zu bytes of scratch; the static scratch holds %zu bytes",
             need, kNoAllocBytes);
    return noalloc_fail(RTG_ERR_INVALID_ARG, msg);
  }
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices)
    return noalloc_fail(RTG_ERR_CUDA, "cudaGetDevice failed");
  void* base = nullptr;
  cudaError_t e = scratch_address(device, &base);
  if (e != cudaSuccess) return noalloc_fail(RTG_ERR_CUDA, cudaGetErrorString(e));
  uint32_t* bits = static_cast<uint32_t*>(base);
  char* t0 = static_cast<char*>(base) + bits_bytes;
  char* t1 = t0 + tmp_bytes;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // every byte the chain reads is written first in this call: the signs by
  // launch_theta_bits, the intermediates by the contraction that produces
  // them, so nothing in the shared scratch needs clearing
  e = launch_theta_bits(sp, bits, s);
  if (e == cudaSuccess) e = launch_sketch(sp, dtype, bits, ref(X), SX, t0, t1, nullptr, s);
  if (e != cudaSuccess) return noalloc_fail(RTG_ERR_CUDA, cudaGetErrorString(e));
  return RTG_OK;
}
