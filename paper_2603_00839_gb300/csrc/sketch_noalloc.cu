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

constexpr size_t kNoAllocBytes = size_t(16) << 20;  // 16 MiB of static device scratch

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
  if (sketch_dims == nullptr || X == nullptr || SX == nullptr)
    return noalloc_fail(RTG_ERR_INVALID_ARG, "sketch_dims, X and SX must be non-NULL");
  if (!on_device(X) || !on_device(SX)) return noalloc_fail(RTG_ERR_INVALID_ARG, "X and SX must be device pointers");
  // the same size bound as rtg_sketch: at most 2^40 elements, checked before
  // each product so that no int64 product of the plan can wrap
  int64_t n = 1;
  for (int k = 0; k < shape.order; ++k) {
    if (shape.dims[k] < 1) return noalloc_fail(RTG_ERR_INVALID_ARG, "shape.dims must be >= 1");
    if (n > (int64_t(1) << 40) / shape.dims[k]) return noalloc_fail(RTG_ERR_INVALID_ARG, "tensor too large");
    n *= shape.dims[k];
  }
  SketchPlan sp;
  const char* perr = make_sketch_plan(shape.order, shape.dims, sketch_dims, seed, problem_id, dtype, sp);
  if (perr != nullptr) return noalloc_fail(RTG_ERR_INVALID_ARG, perr);
  {   // SX may not overlap the part of X the chain reads while it writes SX
    const size_t elt = dtype == RTG_F64 ? 8 : 4;
    const size_t span = size_t(n < sp.d ? n : sp.d) * elt;
    const char* x = static_cast<const char*>(X);
    const char* y = static_cast<const char*>(SX);
    if (x < y + span && y < x + span) return noalloc_fail(RTG_ERR_INVALID_ARG, "SX must not overlap X");
  }
  // scratch: packed signs, Theta operand images and two contraction intermediates
  const size_t need = sketch_scratch_bytes(sp);
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
  const SketchScratch sc = carve_sketch_scratch(sp, base);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // every byte the chain reads is written first in this call: the signs and
  // images by launch_theta, the intermediates by the contraction that
  // produces them, so nothing in the shared scratch needs clearing
  e = launch_theta(sp, sc.bits, sc.frags, s);
  if (e == cudaSuccess) e = launch_sketch(sp, sc, ref(X), SX, nullptr, nullptr, s);
  if (e != cudaSuccess) return noalloc_fail(RTG_ERR_CUDA, cudaGetErrorString(e));
  return RTG_OK;
}
