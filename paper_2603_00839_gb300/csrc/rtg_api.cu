// C ABI of librtg (declared in include/rtg.h): handles, argument
// validation, operator and sketch plans, the Krylov state, and the solve,
// which runs as one CUDA graph per configuration: prologue (sketch signs,
// R_0, beta), a device-controlled WHILE node whose body is one sketched
// Arnoldi step, and the epilogue (Tikhonov/GCV, assembly, summary).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "queue.cuh"
#include "rtg_internal.cuh"

using namespace rtg;


namespace {

thread_local std::string g_err = "no error";

rtg_status fail(rtg_status st, const char* fmt, ...) {
  char buf[768];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

rtg_status cuda_fail(cudaError_t e, const char* what) {
  return fail(RTG_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define CK(call)                                          \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
  } while (0)

#define RK(call)                        \
  do {                                  \
    rtg_status s_ = (call);             \
    if (s_ != RTG_OK) return s_;        \
  } while (0)

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  rtg_status ensure(size_t b) {
    if (b <= bytes && p) return RTG_OK;
    if (p) {
      cudaDeviceSynchronize();
      release();
    }
    if (b == 0) return RTG_OK;
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return fail(RTG_ERR_ALLOC, "cudaMalloc(%zu bytes) failed: %s", b, cudaGetErrorString(e));
    }
    bytes = b;
    return RTG_OK;
  }
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int d) {
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

size_t elt_size(int dtype) { return dtype == RTG_F64 ? 8 : (dtype == RTG_BF16 ? 2 : 4); }

// ------------------------------------------------------------------ operator plans

struct OpHolder {
  OpPlan op{};
  std::vector<std::unique_ptr<DevBuf>> dense;
};

rtg_status check_shape(const rtg_shape& sh, int64_t* n_out) {
  if (sh.order < 1 || sh.order > kMaxOrder) return fail(RTG_ERR_INVALID_ARG, "shape.order=%d not in 1..%d", sh.order, kMaxOrder);
  int64_t n = 1;
  for (int k = 0; k < sh.order; ++k) {
    if (sh.dims[k] < 1) return fail(RTG_ERR_INVALID_ARG, "shape.dims[%d]=%lld must be >= 1", k, (long long)sh.dims[k]);
    if (n > (int64_t(1) << 40) / sh.dims[k]) return fail(RTG_ERR_INVALID_ARG, "tensor too large");
    n *= sh.dims[k];
  }
  *n_out = n;
  return RTG_OK;
}

rtg_status check_dtype(rtg_dtype dt, bool bf16_ok = false) {
  if (dt == RTG_F64 || dt == RTG_F32) return RTG_OK;
  if (dt == RTG_BF16) {
    if (bf16_ok) return RTG_OK;
    return fail(RTG_ERR_UNSUPPORTED, "dtype RTG_BF16 is not supported by this call");
  }
  return fail(RTG_ERR_INVALID_ARG, "unknown dtype %d", (int)dt);
}

rtg_status check_factors(const rtg_factor* f, int nf, const rtg_shape& sh, const char* which) {
  if (nf < 0) return fail(RTG_ERR_INVALID_ARG, "%s count %d < 0", which, nf);
  if (nf > 0 && f == nullptr) return fail(RTG_ERR_INVALID_ARG, "%s is NULL with count %d", which, nf);
  for (int i = 0; i < nf; ++i) {
    const rtg_factor& x = f[i];
    if (x.mode < 1 || x.mode > sh.order) return fail(RTG_ERR_INVALID_ARG, "%s[%d].mode=%d outside 1..%d", which, i, x.mode, sh.order);
    if (x.n != sh.dims[x.mode - 1]) return fail(RTG_ERR_INVALID_ARG, "%s[%d].n=%d but dims[%d]=%lld", which, i, x.n, x.mode - 1, (long long)sh.dims[x.mode - 1]);
    if (x.kind == RTG_FACTOR_IDENTITY) continue;
    if (x.kind == RTG_FACTOR_BANDED_TOEPLITZ) {
      if (x.radius < 0 || x.radius > kMaxRadius) return fail(RTG_ERR_INVALID_ARG, "%s[%d].radius=%d outside 0..%d", which, i, x.radius, kMaxRadius);
      if (x.taps == nullptr) return fail(RTG_ERR_INVALID_ARG, "%s[%d].taps is NULL", which, i);
      for (int t = 0; t <= 2 * x.radius; ++t)
        if (!std::isfinite(x.taps[t])) return fail(RTG_ERR_INVALID_ARG, "%s[%d].taps[%d] is not finite", which, i, t);
      continue;
    }
    if (x.kind == RTG_FACTOR_DENSE) {
      if (x.dense == nullptr) return fail(RTG_ERR_INVALID_ARG, "%s[%d].dense is NULL", which, i);
      if (x.n > 4096) return fail(RTG_ERR_UNSUPPORTED, "%s[%d]: dense factor of size %d > 4096", which, i, x.n);
      for (int64_t t = 0; t < int64_t(x.n) * x.n; ++t)
        if (!std::isfinite(x.dense[t])) return fail(RTG_ERR_INVALID_ARG, "%s[%d].dense has a non-finite entry", which, i);
      continue;
    }
    return fail(RTG_ERR_INVALID_ARG, "%s[%d].kind=%d unknown", which, i, x.kind);
  }
  return RTG_OK;
}

void append_bytes(std::string& k, const void* p, size_t n) { k.append(static_cast<const char*>(p), n); }

std::string op_key(const rtg_factor* A, int nA, const rtg_factor* B, int nB, const rtg_shape& sh) {
  std::string k;
  append_bytes(k, &sh.order, sizeof sh.order);
  append_bytes(k, sh.dims, sizeof(int64_t) * sh.order);
  for (int side = 0; side < 2; ++side) {
    const rtg_factor* f = side ? B : A;
    const int nf = side ? nB : nA;
    k.push_back(side ? 'B' : 'A');
    for (int i = 0; i < nf; ++i) {
      append_bytes(k, &f[i].mode, sizeof(int32_t));
      append_bytes(k, &f[i].kind, sizeof(int32_t));
      append_bytes(k, &f[i].n, sizeof(int32_t));
      if (f[i].kind == RTG_FACTOR_BANDED_TOEPLITZ) {
        append_bytes(k, &f[i].radius, sizeof(int32_t));
        append_bytes(k, f[i].taps, sizeof(double) * (2 * f[i].radius + 1));
      } else if (f[i].kind == RTG_FACTOR_DENSE) {
        append_bytes(k, f[i].dense, sizeof(double) * size_t(f[i].n) * f[i].n);
      }
    }
  }
  return k;
}

// Mode products in application order: left factors, then right factors
// (a right factor B acts as the mode matrix B^T; for banded B the taps reverse).
rtg_status build_op(const rtg_factor* A, int nA, const rtg_factor* B, int nB, const rtg_shape& sh,
                    OpHolder& H) {
  OpPlan& op = H.op;
  op = OpPlan{};
  op.order = sh.order;
  for (int k = 0; k < sh.order; ++k) op.dims[k] = sh.dims[k];
  for (int side = 0; side < 2; ++side) {
    const rtg_factor* f = side ? B : A;
    const int nf = side ? nB : nA;
    for (int i = 0; i < nf; ++i) {
      const rtg_factor& x = f[i];
      if (x.kind == RTG_FACTOR_IDENTITY) continue;
      if (op.npass >= kMaxPasses) return fail(RTG_ERR_UNSUPPORTED, "more than %d non-identity factors", kMaxPasses);
      Pass& p = op.pass[op.npass++];
      p = Pass{};
      p.mode = x.mode - 1;
      p.n = x.n;
      if (x.kind == RTG_FACTOR_BANDED_TOEPLITZ) {
        p.kind = PK_BAND;
        p.radius = x.radius;
        for (int t = 0; t <= 2 * x.radius; ++t) p.taps[t] = side ? x.taps[2 * x.radius - t] : x.taps[t];
      } else {
        p.kind = PK_DENSE;
        std::vector<double> M(size_t(x.n) * x.n);
        for (int i2 = 0; i2 < x.n; ++i2)
          for (int j2 = 0; j2 < x.n; ++j2)
            M[i2 + size_t(x.n) * j2] = side ? x.dense[j2 + size_t(x.n) * i2] : x.dense[i2 + size_t(x.n) * j2];
        auto buf = std::make_unique<DevBuf>();
        RK(buf->ensure(M.size() * sizeof(double)));
        CK(cudaMemcpy(buf->p, M.data(), M.size() * sizeof(double), cudaMemcpyHostToDevice));
        p.dense = static_cast<const double*>(buf->p);
        H.dense.push_back(std::move(buf));
        // keep a host copy for the fused kernel's mode-3 matrix
        if (p.mode == 2 && x.n <= kMaxMix)
          for (size_t q = 0; q < M.size(); ++q) op.M3[q] = M[q];
      }
    }
  }
  // fused pattern: <= 1 banded pass on modes 1 and 2, <= 1 pass on mode 3
  // (dense or banded, size <= kMaxMix unless absent), none above
  int cnt[kMaxOrder] = {0, 0, 0, 0};
  bool ok = true;
  for (int p = 0; p < op.npass; ++p) {
    const Pass& ps = op.pass[p];
    cnt[ps.mode]++;
    if (ps.mode >= 3) ok = false;
    if (ps.mode <= 1 && ps.kind != PK_BAND) ok = false;
    if (ps.mode == 2 && ps.n > kMaxMix) ok = false;
  }
  for (int k = 0; k < 3; ++k)
    if (cnt[k] > 1) ok = false;
  int64_t nslab = 1;
  for (int k = 2; k < op.order; ++k) nslab *= op.dims[k];
  if (op.order >= 2 && op.dims[1] > 65535LL * 16) ok = false;
  op.fused = ok;
  if (ok) {
    op.r1 = op.r2 = 0;
    op.t1[0] = op.t2[0] = 1.0;
    op.mix = 0;
    for (int p = 0; p < op.npass; ++p) {
      const Pass& ps = op.pass[p];
      if (ps.mode == 0) {
        op.r1 = ps.radius;
        for (int t = 0; t <= 2 * ps.radius; ++t) op.t1[t] = ps.taps[t];
      } else if (ps.mode == 1) {
        op.r2 = ps.radius;
        for (int t = 0; t <= 2 * ps.radius; ++t) op.t2[t] = ps.taps[t];
      } else {
        const int nn = ps.n;
        op.mix = nn;
        if (ps.kind == PK_BAND) {
          for (int pp = 0; pp < nn; ++pp)
            for (int c = 0; c < nn; ++c) {
              const int t = c - pp;
              op.M3[pp + nn * c] = (t >= -ps.radius && t <= ps.radius) ? ps.taps[ps.radius + t] : 0.0;
            }
        }
      }
    }
  }
  (void)nslab;
  // spatio-temporal pattern: banded modes 1-2 (<= 1 pass each), <= 1 pass on
  // mode 3 mixing 1 or 3 channels, <= 1 banded pass of radius <= 2 on mode 4
  {
    bool st = op.order <= 4;
    int c4[kMaxOrder] = {0, 0, 0, 0};
    op.st_nc = 1;
    op.r4 = 0;
    op.t4[0] = 1.0;
    op.st_M[0] = 1.0;
    for (int p = 0; p < op.npass && st; ++p) {
      const Pass& ps = op.pass[p];
      if (++c4[ps.mode] > 1) st = false;
      if (ps.mode <= 1 && ps.kind != PK_BAND) st = false;
      if (ps.mode == 2) {
        if (ps.n != 1 && ps.n != 3) {
          st = false;
        } else {
          const int nn = ps.n;
          op.st_nc = nn;
          for (int pp = 0; pp < nn; ++pp)
            for (int c = 0; c < nn; ++c) {
              if (ps.kind == PK_BAND) {
                const int t = c - pp;
                op.st_M[pp + nn * c] = (t >= -ps.radius && t <= ps.radius) ? ps.taps[ps.radius + t] : 0.0;
              } else {
                op.st_M[pp + nn * c] = op.M3[pp + nn * c];
              }
            }
        }
      }
      if (ps.mode == 3) {
        if (ps.kind != PK_BAND || ps.radius > 2) {
          st = false;
        } else {
          op.r4 = ps.radius;
          for (int t = 0; t <= 2 * ps.radius; ++t) op.t4[t] = ps.taps[t];
        }
      }
    }
    if (op.order >= 2 && op.dims[1] > 65535LL * 16) st = false;
    if (op.order >= 1 && op.dims[0] > 65535LL * 64) st = false;
    // the fused image kernel's fields carry the spatial taps
    if (st && !op.fused) {
      op.r1 = op.r2 = 0;
      op.t1[0] = op.t2[0] = 1.0;
      for (int p = 0; p < op.npass; ++p) {
        const Pass& ps = op.pass[p];
        if (ps.mode == 0) {
          op.r1 = ps.radius;
          for (int t = 0; t <= 2 * ps.radius; ++t) op.t1[t] = ps.taps[t];
        } else if (ps.mode == 1) {
          op.r2 = ps.radius;
          for (int t = 0; t <= 2 * ps.radius; ++t) op.t2[t] = ps.taps[t];
        }
      }
    }
    op.st = st;
  }
  return RTG_OK;
}

// ------------------------------------------------------------------ sketch plans

rtg_status build_sketch(const rtg_shape& sh, const int64_t* sdims, uint64_t seed, uint64_t pid,
                        int dtype, SketchPlan& sp) {
  const char* err = make_sketch_plan(sh.order, sh.dims, sdims, seed, pid, dtype, sp);
  if (err != nullptr) return fail(RTG_ERR_INVALID_ARG, "%s", err);
  return RTG_OK;
}

bool is_device_ptr(const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes a{};
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool overlaps(const void* a, const void* b, size_t bytes) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + bytes && y < x + bytes;
}

// ------------------------------------------------------------------ workspace

struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += count * sizeof(T);
    return p;
  }
};

// Lays out (and, with mem != null, points) every buffer of an Arnoldi workspace.
size_t carve_work(void* mem, int dtype, int64_t n, const SketchPlan& sp, int m, int tk_blocks,
                  int64_t apply_elems, Work& w, void** tA, void** tB, SketchScratch* sk,
                  int vdtype = -1, int nU = 0) {
  Carver c(mem);
  const size_t e = elt_size(dtype);
  if (vdtype < 0) vdtype = dtype;
  const size_t ev = elt_size(vdtype);
  const int64_t d = sp.d;
  w = Work{};
  w.dtype = dtype;
  w.vdtype = vdtype;
  w.n = n;
  w.d = static_cast<int>(d);
  w.m = m;
  int64_t G = gs_grid(d);
  if (sp.dots_blocks > G) G = sp.dots_blocks;
  if (nU > 0 && G < 1024) G = 1024;   // Golub-Kahan norm reductions
  w.V = c.take<char>(size_t(m + 1) * n * ev);
  w.W = c.take<char>(size_t(n) * ev);
  w.U = nU > 0 ? c.take<char>(size_t(nU) * n * ev) : nullptr;
  w.S = c.take<char>(size_t(d) * e);
  w.Spart = c.take<char>(size_t(d) * e);
  w.nparts = 1;
  void* skmem = c.take<char>(sketch_scratch_bytes(sp));
  *sk = carve_sketch_scratch(sp, skmem);
  w.tmp0 = sk->tmp0;
  w.tmp1 = sk->tmp1;
  w.Q = c.take<char>(size_t(m + 1) * d * e);
  w.part = c.take<double>(size_t(G) * (2 * m + 4));
  w.part_rows = static_cast<int>(G);
  w.counter = c.take<unsigned>(8);
  w.ctl = c.take<Ctl>(1);
  w.H = c.take<double>(size_t(m + 1) * m);
  w.R = c.take<double>(size_t(m + 1) * m);
  w.cs = c.take<double>(m);
  w.sn = c.take<double>(m);
  w.g = c.take<double>(m + 1);
  w.G = c.take<double>(size_t(gram_ld(m)) * (m + 1));
  w.rho_hist = c.take<double>(kMaxK);
  w.y = c.take<double>(m);
  w.gcv = c.take<double>(kMaxMu);
  w.ysel = c.take<double>(size_t(kMaxMu) * m + size_t(tk_blocks) * size_t(tk_scratch_doubles(m)));
  *tA = c.take<char>(size_t(apply_elems) * e);
  *tB = c.take<char>(size_t(apply_elems) * e);
  if (mem == nullptr) *sk = SketchScratch{};
  return c.off + 256;
}

}  // namespace

void rtg::record_error(const char* msg) { g_err = msg; }

cudaError_t rtg::raise_smem(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> set;   // (device, kernel) -> bytes set
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto it = set.find({dev, kernel});
  if (it != set.end() && it->second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  set[{dev, kernel}] = bytes;
  return cudaSuccess;
}

// ------------------------------------------------------------------ handle

struct rtg_context;

struct SolvePlan {
  OpHolder op;
  OpHolder opT;           // Golub-Kahan: the adjoint operator
  int method = 0;         // 0 RTG-GMRES, 1 sketched Golub-Kahan
  SketchPlan sp{};
  DevBuf mem;
  Work w{};
  void* tA = nullptr;
  void* tB = nullptr;
  SketchScratch sk;
  SolveDesc* desc_dev = nullptr;
  InfoDev* info_dev = nullptr;
  SolveDesc* desc_host = nullptr;
  InfoDev* info_host = nullptr;
  DevBuf small;           // desc + info
  DevBuf Cst, X0st, Xst;  // staging of host arrays
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int mode = 0;           // 0 LS, 1 fixed mu, 2 GCV
  int n_mu = 0;
  bool has_x0 = false;
  bool use_graph = true;
  bool true_resid = false;
  int dtype = RTG_F32;
  int vdtype = RTG_F32;                                           // storage of V and W
  int launches_pro = 0, launches_step = 0, launches_epi = 0;   // kernels per phase
  int launches_setup = 0;                                         // reset + Theta, part of the prologue
  int launches_restart = 0;   // one restart sequence (graph: per restart; direct: every step)
  int direct_steps = 0;                                           // steps launched by the last direct solve
  int* stop_host = nullptr;                                       // pinned: ctl->stop read back per direct step
  bool ext_desc = false;  // desc/info live in a batch's buffers (not owned)
  // lock-step batch (w.b.n problems in one launch per kernel): the problems'
  // blocks of `mem` each start with their descriptor and info record
  unsigned* group_left = nullptr;   // device counter of problems still running
  ~SolvePlan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (desc_host && !ext_desc) cudaFreeHost(desc_host);
    if (info_host && !ext_desc) cudaFreeHost(info_host);
    if (stop_host) cudaFreeHost(stop_host);
  }
};

// A batch of independent solves replayed as one CUDA graph.  Problems that
// share every structural parameter (shape, operator, sketch sizes, m,
// regularisation mode, X0 or not) form a lock-step group: one plan whose
// kernels each serve the whole group (problem = slowest part of blockIdx.z)
// and one device-side loop that runs while any of them does.  Each group is
// one branch of the graph (its prologue, loop and epilogue).
struct BatchPlan {
  std::vector<std::shared_ptr<SolvePlan>> plans;   // one per group
  std::vector<int> group_of, slot_of;              // per problem: its group, its place in the host records
  std::vector<int> gfirst;                         // per group: first host record
  std::vector<int> gcount;                         // per group: its problems
  std::vector<int> gplan;                          // per group: its first plan in `plans`
  char* desc_host = nullptr;     // pinned: nprob descriptors, then nprob info records, in group order
  // work-queue batch (opts.queue_slots > 0): a group is a class of problems of
  // equal structure served by several one-problem plans (graph branches) that
  // take the class's problems from a device queue; qmem holds every problem's
  // descriptor and info record (group order), a counter per class and a
  // current-problem word per branch
  bool queued = false;
  DevBuf qmem;
  size_t q_info = 0, q_ctr = 0, q_cur = 0;   // byte offsets in qmem
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  ~BatchPlan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    plans.clear();
    if (desc_host) cudaFreeHost(desc_host);
  }
};

// Phase timing (RTG_FLAG_PHASE_TIMES): on the direct-launch path every
// kernel group is bracketed by CUDA events on the solve's stream.  Each
// group is preceded by a gate kernel that holds the stream until the host
// has queued the group, so host launch latency never lands between two
// events; the device then runs the group back to back as it would in the
// graph.  A group belongs to a step; groups of steps at or after the stop
// (whose kernels return at once) are dropped when the results are read.
struct PhaseTimer {
  cudaStream_t s = nullptr;
  unsigned* host = nullptr;      // [0] flag written by the host, [1] gate status
  unsigned* dev = nullptr;
  unsigned gen = 0;
  struct Rec {
    cudaEvent_t a, b;
    int phase, step, launches;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  cudaEvent_t a_open = nullptr;

  ~PhaseTimer() {
    for (auto e : pool) cudaEventDestroy(e);
    if (host) cudaFreeHost(host);
  }
  cudaError_t init() {
    if (host) return cudaSuccess;
    void* p = nullptr;
    cudaError_t e = cudaHostAlloc(&p, 2 * sizeof(unsigned), cudaHostAllocMapped);
    if (e != cudaSuccess) return e;
    host = static_cast<unsigned*>(p);
    host[0] = 0;
    host[1] = 0;
    return cudaHostGetDevicePointer(reinterpret_cast<void**>(&dev), host, 0);
  }
  cudaEvent_t next_event() {
    if (used == pool.size()) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      pool.push_back(e);
    }
    return pool[used++];
  }
  void reset(cudaStream_t st) {
    s = st;
    recs.clear();
    used = 0;
    host[1] = 0;
  }
  cudaError_t hold() { return launch_gate(dev, ++gen, dev + 1, s); }
  void release() { __atomic_store_n(host, gen, __ATOMIC_RELEASE); }
  void begin() {
    a_open = next_event();
    if (a_open) cudaEventRecord(a_open, s);
  }
  void end(int phase, int step, int launches) {
    cudaEvent_t b = next_event();
    if (!a_open || !b) return;
    cudaEventRecord(b, s);
    recs.push_back(Rec{a_open, b, phase, step, launches});
    a_open = nullptr;
  }
  // after the stream has been synchronised
  void collect(int iters, rtg_info* info) {
    for (const Rec& r : recs) {
      if (r.step >= iters) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) continue;
      info->phase_ms[r.phase] += ms;
      info->phase_launches[r.phase] += r.launches;
    }
  }
};

// Brackets one kernel group when a timer is given.
struct PhaseScope {
  PhaseTimer* t;
  int phase, step, launches;
  PhaseScope(PhaseTimer* t_, int ph, int st, int l) : t(t_), phase(ph), step(st), launches(l) {
    if (t) t->begin();
  }
  ~PhaseScope() {
    if (t) t->end(phase, step, launches);
  }
};

// Scratch of rtg_sketch for one (shape, sketch sizes, problem id, dtype,
// stream): the packed signs, Theta operand images and chain intermediates, and
// the seed the signs were last drawn for (they are drawn again when a call
// brings another seed).
struct SketchCache {
  DevBuf buf;
  uint64_t seed = 0;
  bool drawn = false;
};

// Scratch of rtg_operator_apply's unfused path on one stream.
struct ApplyScratch {
  DevBuf tA, tB;
};

struct rtg_context {
  int device = 0;
  std::map<std::string, std::unique_ptr<OpHolder>> ops;
  // keyed by stream too, so that calls on different streams never share scratch
  std::map<std::string, std::unique_ptr<SketchCache>> sketches;
  std::map<cudaStream_t, std::unique_ptr<ApplyScratch>> apply_scratch;
  // autotuned basis-update ring geometry per (tensor size, sketch size, storage, problems per group)
  std::map<std::string, int> tuned;
  // rtg_ws_solve: R_0 of the prediction, S(R_0), S(C), log lambda and the decision
  DevBuf ws_work;
  WsDecision* ws_dec_host = nullptr;   // pinned
  ~rtg_context() {
    if (ws_dec_host) cudaFreeHost(ws_dec_host);
  }
  std::map<std::string, std::shared_ptr<SolvePlan>> plans;
  std::map<std::string, std::unique_ptr<BatchPlan>> batches;
  std::unique_ptr<PhaseTimer> timer;
  // per workspace slot: the plan and call state of the last submitted solve
  struct Pending {
    std::shared_ptr<SolvePlan> plan;
    cudaStream_t stream = nullptr;
    int m = 0, n_mu = 0, mode = 0;
    bool use_graph = true, phase_times = false, active = false;
  };
  Pending pending[RTG_MAX_SLOTS];
};

struct rtg_krylov_state {
  rtg_context* ctx = nullptr;
  OpHolder op;
  SketchPlan sp{};
  DevBuf mem;
  Work w{};
  void* tA = nullptr;
  void* tB = nullptr;
  SketchScratch sk;
  int dtype = RTG_F32;
  int m = 0;
  bool started = false;
};

namespace {

rtg_status get_op(rtg_context* h, const rtg_factor* A, int nA, const rtg_factor* B, int nB,
                  const rtg_shape& sh, OpHolder** out) {
  std::string key = op_key(A, nA, B, nB, sh);
  auto it = h->ops.find(key);
  if (it != h->ops.end()) {
    *out = it->second.get();
    return RTG_OK;
  }
  if (h->ops.size() > 64) {
    cudaDeviceSynchronize();
    h->ops.clear();
  }
  auto H = std::make_unique<OpHolder>();
  RK(build_op(A, nA, B, nB, sh, *H));
  *out = H.get();
  h->ops[key] = std::move(H);
  return RTG_OK;
}



StepOpts solve_step_opts(const SolvePlan& P, int use_cond, cudaGraphConditionalHandle hnd) {
  StepOpts o{};
  o.desc_tol = &P.desc_dev->tol;
  o.desc_bd_tol = &P.desc_dev->bd_tol;
  o.solve_mode = 1;
  o.use_cond = use_cond;
  o.cond = static_cast<unsigned long long>(hnd);
  o.group_left = P.group_left;
  return o;
}

PtrRef desc_ref(const void* const* field) {
  PtrRef r;
  r.ind = field;
  return r;
}

rtg_status enqueue_prologue(SolvePlan& P, const StepOpts& so, cudaStream_t s,
                            PhaseTimer* pt = nullptr) {
  Work& w = P.w;
  {
    PhaseScope ps(pt, RTG_PHASE_SETUP, -1, P.launches_setup);
    CK(launch_reset(w, 0, s, P.group_left));
    CK(launch_theta(P.sp, P.sk.bits, P.sk.frags, s, P.desc_dev->key, w.b));
  }
  PhaseScope ps(pt, RTG_PHASE_INIT, -1, P.launches_pro - P.launches_setup);
  PtrRef C = desc_ref(reinterpret_cast<const void* const*>(&P.desc_dev->C));
  PtrRef src = C;
  int sdt = P.dtype;
  if (P.has_x0) {   // R_0 = C - Phi(X_0) into the V_0 slot
    PtrRef X0 = desc_ref(reinterpret_cast<const void* const*>(&P.desc_dev->X0));
    CK(launch_apply(P.op.op, P.dtype, X0, ref(w.V), -1.0, 1.0, C, P.tA, P.tB, nullptr, s, P.dtype, P.vdtype, w.b));
    src = ref(w.V);
    sdt = P.vdtype;
  }
  const bool fused = P.sp.fused_dots != 0;
  SketchDots dots{&w, 0, so};
  CK(launch_sketch(P.sp, P.sk, src, fused ? w.S : w.Spart, fused ? &dots : nullptr, nullptr, s, sdt, w.b));
  CK(launch_start(w, src, so, fused, s, sdt));
  return RTG_OK;
}

rtg_status enqueue_step(const OpHolder& op, const SketchPlan& sp, const Work& w, int dtype,
                        void* tA, void* tB, const SketchScratch& sk, const StepOpts& so,
                        cudaStream_t s, PhaseTimer* pt = nullptr, int step = 0) {
  PtrRef vj;
  vj.base = w.V;
  vj.jidx = &w.ctl->j;
  vj.stride = w.n;
  vj.nslot = w.m + 1;
  const int* stop = &w.ctl->stop;
  {
    PhaseScope ps(pt, RTG_PHASE_APPLY, step, apply_launches(op.op, false, dtype, w.vdtype, w.vdtype));
    CK(launch_apply(op.op, dtype, vj, ref(w.W), 1.0, 0.0, PtrRef{}, tA, tB, stop, s, w.vdtype, w.vdtype, w.b));
  }
  const bool fused = sp.fused_dots != 0;
  {
    PhaseScope ps(pt, RTG_PHASE_SKETCH, step, sketch_launches(sp));
    SketchDots dots{&w, 1, so};
    CK(launch_sketch(sp, sk, ref(w.W), fused ? w.S : w.Spart, fused ? &dots : nullptr, stop, s, w.vdtype, w.b));
  }
  if (!fused) {
    PhaseScope ps(pt, RTG_PHASE_GS, step, 1);
    CK(launch_pass1(w, so, s));
  }
  PhaseScope ps(pt, RTG_PHASE_UPDATE, step, 1);
  CK(launch_update(w, so, s));
  return RTG_OK;
}

// Restart sequence at the end of the step body of a plan with restarts
// (GMRES restarted from the least-squares iterate): every kernel returns at
// once unless the body's Givens block ended a cycle with cycles left
// (ctl->rs_skip == 0).  y = argmin ||beta e1 - Hbar y|| (Eq. 11S), X = X_0 + V y,
// R_0 = C - Phi(X) into the V_0 slot, a new cycle (reset, beta = ||R_0||_Theta,
// V_0 = R_0 / beta, the first sketched column), and rs_skip = 1 again.
rtg_status enqueue_restart(SolvePlan& P, const StepOpts& so, cudaStream_t s) {
  Work& w = P.w;
  const int* gate = &w.ctl->rs_skip;
  FinishOpts f{};
  f.desc = P.desc_dev;
  f.n_mu = 0;
  f.mode = 0;
  CK(launch_tikhonov(w, f, s, gate));
  PtrRef X0 = P.has_x0 ? desc_ref(reinterpret_cast<const void* const*>(&P.desc_dev->X0)) : PtrRef{};
  PtrRef X = desc_ref(reinterpret_cast<const void* const*>(&P.desc_dev->X));
  PtrRef C = desc_ref(reinterpret_cast<const void* const*>(&P.desc_dev->C));
  CK(launch_assemble(w, X0, X, s, gate));
  CK(launch_apply(P.op.op, P.dtype, X, ref(w.V), -1.0, 1.0, C, P.tA, P.tB, gate, s, P.dtype, P.vdtype, w.b));
  CK(launch_reset(w, 1, s, nullptr, gate));
  const bool fused = P.sp.fused_dots != 0;
  SketchDots dots{&w, 0, so};
  CK(launch_sketch(P.sp, P.sk, ref(w.V), fused ? w.S : w.Spart, fused ? &dots : nullptr, gate, s, P.vdtype, w.b));
  CK(launch_start(w, ref(w.V), so, fused, s, P.vdtype, gate));
  CK(launch_restart_done(w, so, s));
  return RTG_OK;
}

// The restart sequence as the body of an IF node appended to the capture on
// cs (so.rs_cond is the node's condition handle).
rtg_status capture_restart_if(SolvePlan& P, const StepOpts& so, cudaStream_t cs) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t gcap = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &gcap, &deps, nullptr, &nd));
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = static_cast<cudaGraphConditionalHandle>(so.rs_cond);
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  CK(cudaGraphAddNode(&node, gcap, deps, nullptr, nd, &cp));
  CK(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaStream_t c3 = nullptr;
  CK(cudaStreamCreateWithFlags(&c3, cudaStreamNonBlocking));
  rtg_status st = RTG_OK;
  cudaError_t e = cudaStreamBeginCaptureToGraph(c3, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamBeginCaptureToGraph(restart)");
  if (st == RTG_OK) {
    st = enqueue_restart(P, so, c3);
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(c3, &out);
    if (st == RTG_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamEndCapture(restart)");
  }
  cudaStreamDestroy(c3);
  return st;
}

int restart_launches(const OpPlan& op, const SketchPlan& sp, int dtype, int vdtype) {
  return 2 + apply_launches(op, true, dtype, dtype, vdtype) + 1 + sketch_launches(sp) + (sp.fused_dots ? 1 : 2) + 1;
}

// Sketched Golub-Kahan (Algorithm 4): prologue U_0, alpha_0, V_0 and one step
// (forward half: beta_{j+1}, U_{j+1}, Givens; backward half: alpha_{j+1}, V_{j+1}).
rtg_status enqueue_gk_prologue(SolvePlan& P, const StepOpts& so, cudaStream_t s, PhaseTimer* pt = nullptr) {
  Work& w = P.w;
  {
    PhaseScope ps(pt, RTG_PHASE_SETUP, -1, P.launches_setup);
    CK(launch_reset(w, 0, s));
    CK(launch_theta(P.sp, P.sk.bits, P.sk.frags, s, P.desc_dev->key));
  }
  PhaseScope ps(pt, RTG_PHASE_INIT, -1, P.launches_pro - P.launches_setup);
  PtrRef C = desc_ref(reinterpret_cast<const void* const*>(&P.desc_dev->C));
  PtrRef src = C;
  if (P.has_x0) {   // R_0 = C - Phi(X_0) into W
    PtrRef X0 = desc_ref(reinterpret_cast<const void* const*>(&P.desc_dev->X0));
    CK(launch_apply(P.op.op, P.dtype, X0, ref(w.W), -1.0, 1.0, C, P.tA, P.tB, nullptr, s));
    src = ref(w.W);
  }
  CK(launch_sketch(P.sp, P.sk, src, w.S, nullptr, nullptr, s));
  CK(launch_gk_norm(w, 0, so, s));
  CK(launch_gk_update(w, 0, src, so, s));
  const int* stop = &w.ctl->stop;
  CK(launch_apply(P.opT.op, P.dtype, ref(w.U), ref(w.W), 1.0, 0.0, PtrRef{}, P.tA, P.tB, stop, s));
  CK(launch_sketch(P.sp, P.sk, ref(w.W), w.S, nullptr, stop, s));
  CK(launch_gk_norm(w, 1, so, s));
  CK(launch_gk_update(w, 1, PtrRef{}, so, s));
  return RTG_OK;
}

rtg_status enqueue_gk_step(SolvePlan& P, const StepOpts& so, cudaStream_t s, PhaseTimer* pt = nullptr,
                           int step = 0) {
  Work& w = P.w;
  const int* stop = &w.ctl->stop;
  PtrRef vj;   // V_j, j = ctl->j
  vj.base = w.V;
  vj.jidx = &w.ctl->j;
  vj.stride = w.n;
  PtrRef uj;   // U_{j+1} after the forward half advanced j: ring slot j % 2
  uj.base = w.U;
  uj.jidx = &w.ctl->j;
  uj.stride = w.n;
  uj.mod = 2;
  const int al = apply_launches(P.op.op, false, P.dtype, P.dtype, P.dtype);
  const int alT = apply_launches(P.opT.op, false, P.dtype, P.dtype, P.dtype);
  {
    PhaseScope ps(pt, RTG_PHASE_APPLY, step, al);
    CK(launch_apply(P.op.op, P.dtype, vj, ref(w.W), 1.0, 0.0, PtrRef{}, P.tA, P.tB, stop, s));
  }
  {
    PhaseScope ps(pt, RTG_PHASE_SKETCH, step, sketch_launches(P.sp));
    CK(launch_sketch(P.sp, P.sk, ref(w.W), w.S, nullptr, stop, s));
  }
  {
    PhaseScope ps(pt, RTG_PHASE_GS, step, 1);
    CK(launch_gk_norm(w, 2, so, s));
  }
  {
    PhaseScope ps(pt, RTG_PHASE_UPDATE, step, 1);
    CK(launch_gk_update(w, 2, PtrRef{}, so, s));
  }
  {
    PhaseScope ps(pt, RTG_PHASE_APPLY, step, alT);
    CK(launch_apply(P.opT.op, P.dtype, uj, ref(w.W), 1.0, 0.0, PtrRef{}, P.tA, P.tB, stop, s));
  }
  {
    PhaseScope ps(pt, RTG_PHASE_SKETCH, step, sketch_launches(P.sp));
    CK(launch_sketch(P.sp, P.sk, ref(w.W), w.S, nullptr, stop, s));
  }
  {
    PhaseScope ps(pt, RTG_PHASE_GS, step, 1);
    CK(launch_gk_norm(w, 3, so, s));
  }
  PhaseScope ps(pt, RTG_PHASE_UPDATE, step, 1);
  CK(launch_gk_update(w, 3, PtrRef{}, so, s));
  return RTG_OK;
}

rtg_status enqueue_epilogue(SolvePlan& P, cudaStream_t s, PhaseTimer* pt = nullptr) {
  FinishOpts f{};
  f.desc = P.desc_dev;
  f.n_mu = P.n_mu;
  f.mode = P.mode;
  {
    PhaseScope ps(pt, RTG_PHASE_TIKHONOV, -1, 1);
    CK(launch_tikhonov(P.w, f, s));
  }
  PhaseScope ps(pt, RTG_PHASE_ASSEMBLE, -1, P.launches_epi - 1);
  PtrRef X0 = P.has_x0 ? desc_ref(reinterpret_cast<const void* const*>(&P.desc_dev->X0)) : PtrRef{};
  PtrRef X = desc_ref(reinterpret_cast<const void* const*>(&P.desc_dev->X));
  CK(launch_assemble(P.w, X0, X, s));
  if (P.true_resid) {   // R = C - Phi(X) into the V_0 slot (the basis is no longer needed), S(R), norms
    PtrRef C = desc_ref(reinterpret_cast<const void* const*>(&P.desc_dev->C));
    CK(launch_apply(P.op.op, P.dtype, X, ref(P.w.V), -1.0, 1.0, C, P.tA, P.tB, nullptr, s, P.dtype, P.dtype,
                    P.w.b));
    CK(launch_sketch(P.sp, P.sk, ref(P.w.V), P.w.Spart, nullptr, nullptr, s, P.dtype, P.w.b));
    CK(launch_true_resid(P.w, C, s));
  }
  CK(launch_finalize(P.w, P.info_dev, s));
  return RTG_OK;
}

// Appends a conditional node of `type` on handle `hnd` to the capture on
// `cs` (after everything captured so far) and returns its body graph.
rtg_status add_conditional(cudaStream_t cs, cudaGraphConditionalHandle hnd, cudaGraphConditionalNodeType type,
                           cudaGraph_t* body) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t gcap = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &gcap, &deps, nullptr, &nd);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamGetCaptureInfo");
  cudaGraphNode_t cnode = nullptr;
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hnd;
  cp.conditional.type = type;
  cp.conditional.size = 1;
  e = cudaGraphAddNode(&cnode, gcap, deps, nullptr, nd, &cp);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphAddNode(conditional)");
  e = cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamUpdateCaptureDependencies");
  *body = cp.conditional.phGraph_out[0];
  return RTG_OK;
}

// Captures P's solve (prologue, a WHILE node over one Arnoldi step, epilogue)
// on `cs`, which is capturing into graph g; cs2 captures the loop's body.
// The loop's condition handle goes to *loop when loop is not null.
rtg_status capture_solve(SolvePlan& P, cudaGraph_t g, cudaStream_t cs, cudaStream_t cs2,
                         cudaGraphConditionalHandle* loop = nullptr) {
  cudaGraphConditionalHandle hnd;
  CK(cudaGraphConditionalHandleCreate(&hnd, g, 1, cudaGraphCondAssignDefault));
  if (loop) *loop = hnd;
  StepOpts so = solve_step_opts(P, 1, hnd);
  RK(P.method == 1 ? enqueue_gk_prologue(P, so, cs) : enqueue_prologue(P, so, cs));
  cudaGraph_t body = nullptr;
  RK(add_conditional(cs, hnd, cudaGraphCondTypeWhile, &body));
  // restarts: an IF node at the end of the body holds the restart
  // sequence; the Givens block that ends a cycle sets its condition
  if (P.w.cycles > 1) {
    cudaGraphConditionalHandle rh;
    CK(cudaGraphConditionalHandleCreate(&rh, body, 0, cudaGraphCondAssignDefault));
    so.use_rs_cond = 1;
    so.rs_cond = static_cast<unsigned long long>(rh);
  }
  CK(cudaStreamBeginCaptureToGraph(cs2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  rtg_status st = P.method == 1 ? enqueue_gk_step(P, so, cs2)
                                : enqueue_step(P.op, P.sp, P.w, P.dtype, P.tA, P.tB, P.sk, so, cs2);
  if (st == RTG_OK && P.w.cycles > 1) st = capture_restart_if(P, so, cs2);
  cudaGraph_t bodyout = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs2, &bodyout);
  RK(st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture(body)");
  return enqueue_epilogue(P, cs);
}

struct CaptureStreams {
  cudaStream_t s[3] = {nullptr, nullptr, nullptr};
  rtg_status create() {
    for (auto& x : s) CK(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
    return RTG_OK;
  }
  ~CaptureStreams() {
    for (auto x : s)
      if (x) cudaStreamDestroy(x);
  }
};

// Ends the capture on cs whatever happened before, and returns the first error.
rtg_status end_capture(cudaStream_t cs, rtg_status st) {
  cudaGraph_t gout = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs, &gout);
  if (st == RTG_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamEndCapture");
  if (st != RTG_OK) cudaGetLastError();
  return st;
}

// Place of a branch in a chain of branches (a batch with a bounded number of
// branches in flight): `after` holds the nodes its first node waits for
// (none: it starts with the graph), `tail` receives its last nodes.
struct ChainLink {
  const std::vector<cudaGraphNode_t>* after = nullptr;
  std::vector<cudaGraphNode_t>* tail = nullptr;
};

rtg_status begin_branch(cudaStream_t cs, cudaGraph_t g, const ChainLink& ch) {
  const bool dep = ch.after != nullptr && !ch.after->empty();
  CK(cudaStreamBeginCaptureToGraph(cs, g, dep ? ch.after->data() : nullptr, nullptr, dep ? ch.after->size() : 0,
                                   cudaStreamCaptureModeThreadLocal));
  return RTG_OK;
}

// Records the capture's current last nodes (what the next captured node
// would depend on) as the branch's tail.
rtg_status branch_tail(cudaStream_t cs, const ChainLink& ch, rtg_status st) {
  if (st != RTG_OK || ch.tail == nullptr) return st;
  cudaStreamCaptureStatus cst;
  cudaGraph_t gcap = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  const cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &gcap, &deps, nullptr, &nd);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamGetCaptureInfo(tail)");
  ch.tail->assign(deps, deps + nd);
  return RTG_OK;
}

// Captures P's solve into g as a branch (after ch.after, if given).
rtg_status build_branch(SolvePlan& P, cudaGraph_t g, const ChainLink& ch = ChainLink{}) {
  CaptureStreams cs;
  RK(cs.create());
  RK(begin_branch(cs.s[0], g, ch));
  return end_capture(cs.s[0], branch_tail(cs.s[0], ch, capture_solve(P, g, cs.s[0], cs.s[1])));
}

// A branch of a work-queue batch: it takes a problem of its class, then
// loops (a WHILE node) over solve + hand back + take the next, until the
// class's queue is empty.  P is a one-problem plan; q names the class's
// queue and P's descriptor, info record and current-problem word.
rtg_status build_queue_branch(SolvePlan& P, cudaGraph_t g, QueueArgs q, const ChainLink& ch = ChainLink{}) {
  CaptureStreams cs;
  RK(cs.create());
  cudaGraphConditionalHandle oh;
  CK(cudaGraphConditionalHandleCreate(&oh, g, 0, cudaGraphCondAssignDefault));
  q.cond = static_cast<unsigned long long>(oh);
  RK(begin_branch(cs.s[0], g, ch));
  rtg_status st = RTG_OK;
  cudaGraph_t body = nullptr;
  if (const cudaError_t e = launch_queue_next(q, 0, cs.s[0]); e != cudaSuccess) st = cuda_fail(e, "queue take");
  if (st == RTG_OK) st = add_conditional(cs.s[0], oh, cudaGraphCondTypeWhile, &body);
  if (st == RTG_OK) {
    if (const cudaError_t e =
            cudaStreamBeginCaptureToGraph(cs.s[1], body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        e != cudaSuccess) {
      st = cuda_fail(e, "cudaStreamBeginCaptureToGraph(queue body)");
    } else {
      cudaGraphConditionalHandle inner{};
      st = capture_solve(P, body, cs.s[1], cs.s[2], &inner);
      q.inner = static_cast<unsigned long long>(inner);
      q.use_inner = 1;
      if (st == RTG_OK)
        if (const cudaError_t e2 = launch_queue_next(q, 1, cs.s[1]); e2 != cudaSuccess) st = cuda_fail(e2, "queue next");
      st = end_capture(cs.s[1], st);
    }
  }
  return end_capture(cs.s[0], branch_tail(cs.s[0], ch, st));
}

rtg_status build_graph(SolvePlan& P) {
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  const rtg_status st = build_branch(P, g);
  if (st != RTG_OK) {
    cudaGraphDestroy(g);
    return st;
  }
  P.graph = g;
  CK(cudaGraphInstantiate(&P.exec, g, 0));
  return RTG_OK;
}

}  // namespace

static rtg_status sketch_scratch_for(rtg_handle h, const SketchPlan& sp, uint64_t seed, uint64_t pid,
                                     cudaStream_t s, SketchScratch* out);

// ================================================================== C ABI

// Everything a solve plan is built from.
struct PlanSpec {
  const rtg_factor* A;
  int nA;
  const rtg_factor* B;
  int nB;
  rtg_shape shape;
  int dtype, vdtype;
  int64_t n;
  int m;
  SketchPlan sp;
  int mode, n_mu;
  bool has_x0, use_graph;
  int method = 0;   // 0 RTG-GMRES, 1 sketched Golub-Kahan
  bool true_resid = false;   // epilogue computes C - Phi(X) and its norms
  int cycles = 1;            // restarts + 1
};

// Factors of the adjoint operator: every mode matrix transposed (banded:
// taps reversed; dense: the matrix transposed).
struct TransposedFactors {
  std::vector<rtg_factor> f;
  std::vector<std::vector<double>> data;
  TransposedFactors(const rtg_factor* in, int nf) {
    f.assign(in, in + nf);
    data.resize(nf);
    for (int i = 0; i < nf; ++i) {
      const rtg_factor& x = in[i];
      if (x.kind == RTG_FACTOR_BANDED_TOEPLITZ) {
        data[i].assign(x.taps, x.taps + 2 * x.radius + 1);
        std::reverse(data[i].begin(), data[i].end());
        f[i].taps = data[i].data();
      } else if (x.kind == RTG_FACTOR_DENSE) {
        data[i].resize(size_t(x.n) * x.n);
        for (int a = 0; a < x.n; ++a)
          for (int b = 0; b < x.n; ++b) data[i][a + size_t(x.n) * b] = x.dense[b + size_t(x.n) * a];
        f[i].dense = data[i].data();
      }
    }
  }
};

// Autotuner of the basis update's tiles (a project-written timing search):
// the shared-memory ring's slot size (the chunk of the tensor one CTA
// streams) and depth.  Every geometry gives the same results bit for bit,
// so the choice only changes speed.  Each candidate runs on the plan's own
// workspace and grid (all problems of a lock-step group) from synthetic
// step states (j = 4, 16, 40 bounded by m - 1: the update reads j + 1
// tensors), five timed launches each after one untimed; the smallest sum of
// the medians wins and is cached per (n, d, storage, problems per launch)
// in the handle.  The workspace is cleared afterwards (every solve starts
// by resetting its state anyway).
constexpr int kConcurrentBranches = 4;

// RTG_NO_AUTOTUNE=1 in the environment keeps the default geometry;
// RTG_TILE_CONFIG=k fixes geometry k.
// branches: graph branches of a batched solve that run at once.  With
// several, the search (which times one problem alone, where more and
// smaller CTAs win) is skipped for the geometry with the fewest CTAs, the
// largest slots: measured the fastest under concurrent branches.
static rtg_status tune_update(SolvePlan& P, std::map<std::string, int>* cache, int branches) {
  Work& w = P.w;
  w.upcfg = 0;
  if (cache == nullptr || !update_uses_ring(w)) return RTG_OK;
  const char* off = std::getenv("RTG_NO_AUTOTUNE");
  if (off != nullptr && off[0] == '1') return RTG_OK;
  const char* force = std::getenv("RTG_TILE_CONFIG");   // a fixed geometry (tests, measurements)
  if (force != nullptr && force[0] >= '0' && force[0] < '0' + update_configs() && force[1] == 0) {
    w.upcfg = force[0] - '0';
    return RTG_OK;
  }
  if (branches >= kConcurrentBranches) {
    w.upcfg = update_configs() - 1;
    return RTG_OK;
  }
  std::string key;
  append_bytes(key, &w.n, sizeof w.n);
  append_bytes(key, &w.d, sizeof w.d);
  append_bytes(key, &w.vdtype, sizeof w.vdtype);
  append_bytes(key, &w.b.n, sizeof w.b.n);
  auto hit = cache->find(key);
  if (hit != cache->end()) {
    w.upcfg = hit->second;
    return RTG_OK;
  }
  cudaStream_t s = nullptr;
  CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  struct Cleanup {
    cudaStream_t s;
    cudaEvent_t e[2] = {nullptr, nullptr};
    ~Cleanup() {
      for (auto x : e)
        if (x) cudaEventDestroy(x);
      cudaStreamDestroy(s);
    }
  } cl{s};
  CK(cudaEventCreate(&cl.e[0]));
  CK(cudaEventCreate(&cl.e[1]));
  // the median of five launches at step indices 4, 16 and 40 (bounded by
  // m - 1), summed: early steps whose tensors sit in L2 and a late one whose
  // basis exceeds it
  const int ncfg = update_configs();
  float tot[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int js[3] = {4, 16, 40}, nj = 0;
  for (int q = 0; q < 3; ++q) {
    const int j = js[q] < w.m - 1 ? js[q] : w.m - 1;
    if (nj == 0 || js[nj - 1] != j) js[nj++] = j;
  }
  StepOpts o{};   // no graph condition, no lock-step count
  for (int q = 0; q < nj; ++q) {
    Ctl c{};
    c.j = js[q];
    c.hnext = 1.0;
    c.rs_skip = 1;
    for (int p = 0; p < w.b.n; ++p)
      CK(cudaMemcpyAsync(reinterpret_cast<char*>(w.ctl) + int64_t(p) * w.b.stride, &c, sizeof(Ctl),
                         cudaMemcpyHostToDevice, s));
    for (int cfg = 0; cfg < ncfg && cfg < 8; ++cfg) {
      w.upcfg = cfg;
      CK(launch_update(w, o, s));
      float t[5];
      for (int r = 0; r < 5; ++r) {
        CK(cudaEventRecord(cl.e[0], s));
        CK(launch_update(w, o, s));
        CK(cudaEventRecord(cl.e[1], s));
        CK(cudaEventSynchronize(cl.e[1]));
        CK(cudaEventElapsedTime(&t[r], cl.e[0], cl.e[1]));
      }
      std::sort(t, t + 5);
      tot[cfg] += t[2];
    }
  }
  int best = 0;
  for (int cfg = 1; cfg < ncfg && cfg < 8; ++cfg)
    if (tot[cfg] < tot[best]) best = cfg;
  CK(cudaMemsetAsync(P.mem.p, 0, P.mem.bytes, s));
  CK(cudaStreamSynchronize(s));
  w.upcfg = best;
  (*cache)[key] = best;
  return RTG_OK;
}

// Builds a plan: operator, workspace, descriptor / info record (in the
// given batch buffers, or its own), launch counts and, for a stand-alone
// graph solve, its CUDA graph.  Builds only while nothing of the handle runs.
rtg_status make_plan(const PlanSpec& ps, SolveDesc* ddev, InfoDev* idev, SolveDesc* dhost, InfoDev* ihost,
                     std::shared_ptr<SolvePlan>* out, int nbatch = 0,
                     std::map<std::string, int>* tune_cache = nullptr, int branches = 1) {
  const rtg_factor* A = ps.A;
  const rtg_factor* B = ps.B;
  const int nA = ps.nA, nB = ps.nB, dtype = ps.dtype, vdtype = ps.vdtype, m = ps.m, mode = ps.mode;
  const int n_mu = ps.n_mu;
  const bool has_x0 = ps.has_x0, use_graph = ps.use_graph;
  const rtg_shape& shape = ps.shape;
  const int64_t n = ps.n;
  const SketchPlan& sp = ps.sp;
  auto np = std::make_shared<SolvePlan>();
  SolvePlan* P = np.get();
  P->dtype = dtype;
  P->mode = mode;
  P->n_mu = n_mu;
  P->has_x0 = has_x0;
  P->use_graph = use_graph;
  P->sp = sp;
  P->method = ps.method;
  P->true_resid = ps.true_resid;
  RK(build_op(A, nA, B, nB, shape, P->op));
  if (ps.method == 1) {
    TransposedFactors tA(A, nA), tB(B, nB);
    RK(build_op(tA.f.data(), nA, tB.f.data(), nB, shape, P->opT));
  }
  P->vdtype = vdtype;
  if (vdtype == RTG_BF16 && !st_supported(P->op.op, RTG_BF16))
    return fail(RTG_ERR_UNSUPPORTED, "RTG_FLAG_BF16_BASIS needs banded modes 1-2 (radius <= 9), a mode-3 mix "
                                     "of 1 or 3 channels, a mode-4 band of radius <= 2 and dims[0] %% 8 == 0");
  int64_t ae = apply_scratch_elems(P->op.op);
  if (ps.method == 1 && apply_scratch_elems(P->opT.op) > ae) ae = apply_scratch_elems(P->opT.op);
  const int tkb = mode == 2 ? n_mu : 1;
  const int nU = ps.method == 1 ? 2 : 0;
  Work tmpw;
  void *ta, *tb;
  SketchScratch tsk;
  const size_t bytes = carve_work(nullptr, dtype, n, sp, m, tkb, ae, tmpw, &ta, &tb, &tsk, vdtype, nU);
  if (nbatch > 0) {
    // lock-step batch: one block per problem (descriptor, info record,
    // workspace), every block laid out alike, `bs` bytes apart; the host
    // records (dhost, ihost) hold nbatch entries each, contiguous
    const size_t dsz = (sizeof(SolveDesc) + 255) & ~size_t(255);
    const size_t isz = (sizeof(InfoDev) + 255) & ~size_t(255);
    const size_t bs = (dsz + isz + bytes + 255) & ~size_t(255);
    RK(P->mem.ensure(bs * size_t(nbatch)));
    CK(cudaMemset(P->mem.p, 0, bs * size_t(nbatch)));
    char* b0 = static_cast<char*>(P->mem.p);
    carve_work(b0 + dsz + isz, dtype, n, sp, m, tkb, ae, P->w, &P->tA, &P->tB, &P->sk, vdtype, nU);
    P->w.b.n = nbatch;
    P->w.b.stride = static_cast<int64_t>(bs);
    P->ext_desc = true;
    P->desc_dev = reinterpret_cast<SolveDesc*>(b0);
    P->info_dev = reinterpret_cast<InfoDev*>(b0 + dsz);
    P->desc_host = dhost;
    P->info_host = ihost;
    RK(P->small.ensure(256));
    CK(cudaMemset(P->small.p, 0, 256));
    P->group_left = static_cast<unsigned*>(P->small.p);
  } else {
    RK(P->mem.ensure(bytes));
    CK(cudaMemset(P->mem.p, 0, bytes));
    carve_work(P->mem.p, dtype, n, sp, m, tkb, ae, P->w, &P->tA, &P->tB, &P->sk, vdtype, nU);
  }
  P->w.cycles = ps.cycles;
  RK(tune_update(*P, tune_cache, branches));
  if (nbatch > 0) {
  } else if (ddev != nullptr) {   // descriptor and info record in a batch's buffers
    P->ext_desc = true;
    P->desc_dev = ddev;
    P->info_dev = idev;
    P->desc_host = dhost;
    P->info_host = ihost;
  } else {
    RK(P->small.ensure(sizeof(SolveDesc) + sizeof(InfoDev) + 512));
    P->desc_dev = static_cast<SolveDesc*>(P->small.p);
    P->info_dev = reinterpret_cast<InfoDev*>(static_cast<char*>(P->small.p) + ((sizeof(SolveDesc) + 255) & ~size_t(255)));
    CK(cudaMallocHost(&P->desc_host, sizeof(SolveDesc)));
    CK(cudaMallocHost(&P->info_host, sizeof(InfoDev)));
    std::memset(P->desc_host, 0, sizeof(SolveDesc));
    CK(cudaMemset(P->small.p, 0, P->small.bytes));
  }
  CK(cudaMallocHost(&P->stop_host, sizeof(int)));
  CK(cudaEventCreate(&P->ev0));
  CK(cudaEventCreate(&P->ev1));
  {
    int nsk = 0;
    for (int k = 0; k < sp.order; ++k) nsk += sp.sketched[k];
    const int gs = sp.fused_dots ? 0 : 1;
    P->launches_setup = 1 + (nsk > 0 ? (dtype == RTG_F32 ? 2 : 1) : 0);
    P->launches_pro = P->launches_setup +
                      (has_x0 ? apply_launches(P->op.op, true, dtype, dtype, vdtype) : 0) +
                      sketch_launches(sp) + gs + 1;
    P->launches_step = apply_launches(P->op.op, false, dtype, vdtype, vdtype) + sketch_launches(sp) + gs + 1;
    P->launches_restart = ps.cycles > 1 ? restart_launches(P->op.op, sp, dtype, vdtype) : 0;
    P->launches_epi = 3 + (ps.true_resid ? apply_launches(P->op.op, true, dtype, dtype, dtype) +
                                               sketch_launches(sp) + 1 : 0);
    if (ps.method == 1) {
      const int al = apply_launches(P->op.op, false, dtype, dtype, dtype);
      const int alT = apply_launches(P->opT.op, false, dtype, dtype, dtype);
      P->launches_pro = P->launches_setup + (has_x0 ? apply_launches(P->op.op, true, dtype, dtype, dtype) : 0) +
                        2 * sketch_launches(sp) + alT + 4;
      P->launches_step = al + alT + 2 * sketch_launches(sp) + 4;
    }
  }
  if (use_graph && ddev == nullptr) RK(build_graph(*P));
  *out = std::move(np);
  return RTG_OK;
}

// Host summary of a finished solve from its info record.
void fill_info(const SolvePlan& P, const InfoDev& I, int mode, int n_mu, bool use_graph, float ms,
               rtg_info* info) {
  info->iters = I.iters;
  info->restarts = I.restarts;
  info->breakdown = I.breakdown;
  info->converged = I.converged;
  info->beta = I.beta;
  info->mu = I.mu;
  info->rho_final = I.rho_final;
  if (info->rho_hist)
    for (int i = 0; i < I.iters && i < kMaxK; ++i) info->rho_hist[i] = I.rho_hist[i];
  if (info->gcv && mode == 2)
    for (int i = 0; i < n_mu; ++i) info->gcv[i] = I.gcv[i];
  info->true_rel_resid = P.true_resid ? I.true_rel_resid : -1.0;
  info->true_rel_resid_theta = P.true_resid ? I.true_rel_resid_theta : -1.0;
  info->elapsed_ms = ms;
  info->device_status = I.status;
  info->tile_config = P.w.upcfg;
  info->launches = P.launches_pro + P.launches_epi + (use_graph ? I.iters : P.direct_steps) * P.launches_step +
                   (use_graph ? I.restarts : P.direct_steps) * P.launches_restart;
  for (int k = 0; k < RTG_PHASE_COUNT; ++k) {
    info->phase_ms[k] = 0.0;
    info->phase_launches[k] = 0;
  }
}

// Per-call descriptor of a solve.
void fill_desc(SolveDesc& D, const void* C, const void* X0, void* X, uint64_t seed, double tol,
               double bd_tol, int dtype, double lambda, int n_mu, const double* mu_grid) {
  D.C = C;
  D.X0 = X0;
  D.X = X;
  D.key[0] = seed;
  D.key[1] = 0;
  D.tol = tol;
  D.bd_tol = bd_tol > 0 ? bd_tol : (dtype == RTG_F64 ? 1e-12 : 1e-6);
  D.lambda = lambda;
  D.n_mu = n_mu;
  for (int i = 0; i < n_mu; ++i) D.mu_grid[i] = mu_grid[i];
}

extern "C" {

const char* rtg_last_error(void) { return g_err.c_str(); }

const char* rtg_status_string(rtg_status s) {
  switch (s) {
    case RTG_OK: return "RTG_OK";
    case RTG_ERR_INVALID_ARG: return "RTG_ERR_INVALID_ARG";
    case RTG_ERR_UNSUPPORTED: return "RTG_ERR_UNSUPPORTED";
    case RTG_ERR_CUDA: return "RTG_ERR_CUDA";
    case RTG_ERR_ALLOC: return "RTG_ERR_ALLOC";
    case RTG_ERR_TIMEOUT: return "RTG_ERR_TIMEOUT";
    case RTG_ERR_NONFINITE: return "RTG_ERR_NONFINITE";
  }
  return "RTG_UNKNOWN_STATUS";
}

int32_t rtg_version(void) { return 100; }

rtg_status rtg_create(rtg_handle* handle, int device) {
  if (handle == nullptr) return fail(RTG_ERR_INVALID_ARG, "handle is NULL");
  *handle = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "cudaGetDeviceCount");
  }
  if (device < 0 || device >= count) return fail(RTG_ERR_INVALID_ARG, "device %d not in 0..%d", device, count - 1);
  DeviceGuard dg(device);
  CK(cudaFree(nullptr));   // make sure the context exists
  auto* ctx = new rtg_context();
  ctx->device = device;
  *handle = ctx;
  return RTG_OK;
}

rtg_status rtg_destroy(rtg_handle handle) {
  if (handle == nullptr) return RTG_OK;
  DeviceGuard dg(handle->device);
  cudaDeviceSynchronize();
  delete handle;
  return RTG_OK;
}

rtg_status rtg_philox_words(rtg_handle h, uint64_t seed, uint64_t pid, int64_t n_words,
                            uint64_t* out, rtg_stream stream) {
  if (h == nullptr) return fail(RTG_ERR_INVALID_ARG, "handle is NULL");
  if (n_words < 0) return fail(RTG_ERR_INVALID_ARG, "n_words < 0");
  if (n_words == 0) return RTG_OK;
  DeviceGuard dg(h->device);
  if (!is_device_ptr(out)) return fail(RTG_ERR_INVALID_ARG, "out is not a device pointer");
  CK(launch_philox_words(seed, pid, n_words, out, reinterpret_cast<cudaStream_t>(stream)));
  return RTG_OK;
}

rtg_status rtg_operator_apply(rtg_handle h, const rtg_factor* A, int32_t nA, const rtg_factor* B,
                              int32_t nB, rtg_shape shape, rtg_dtype dtype, const void* X,
                              void* Y, rtg_stream stream) {
  if (h == nullptr) return fail(RTG_ERR_INVALID_ARG, "handle is NULL");
  int64_t n = 0;
  RK(check_shape(shape, &n));
  RK(check_dtype(dtype, true));
  RK(check_factors(A, nA, shape, "A_factors"));
  RK(check_factors(B, nB, shape, "B_factors"));
  DeviceGuard dg(h->device);
  if (!is_device_ptr(X) || !is_device_ptr(Y)) return fail(RTG_ERR_INVALID_ARG, "X and Y must be device pointers");
  if (overlaps(X, Y, size_t(n) * elt_size(dtype))) return fail(RTG_ERR_INVALID_ARG, "Y overlaps X");
  OpHolder* op = nullptr;
  RK(get_op(h, A, nA, B, nB, shape, &op));
  if (dtype == RTG_BF16) {
    if (!st_supported(op->op, RTG_BF16))
      return fail(RTG_ERR_UNSUPPORTED, "BF16 apply needs banded modes 1-2 (radius <= 9), a mode-3 mix of 1 or 3 "
                                       "channels, a mode-4 band of radius <= 2 and dims[0] %% 8 == 0");
    if (reinterpret_cast<uintptr_t>(X) % 16 != 0) return fail(RTG_ERR_INVALID_ARG, "BF16 X must be 16-byte aligned");
    CK(launch_apply(op->op, RTG_F32, ref(X), ref(Y), 1.0, 0.0, PtrRef{}, nullptr, nullptr, nullptr,
                    reinterpret_cast<cudaStream_t>(stream), RTG_BF16, RTG_BF16));
    return RTG_OK;
  }
  if (apply_uses_st(op->op, dtype, dtype, dtype) && reinterpret_cast<uintptr_t>(X) % 16 != 0)
    return fail(RTG_ERR_INVALID_ARG, "X must be 16-byte aligned for this operator");
  const int64_t sc = apply_scratch_elems(op->op);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void *ta = nullptr, *tb = nullptr;
  if (sc > 0) {   // the unfused path's intermediates, owned per stream
    std::unique_ptr<ApplyScratch>& as = h->apply_scratch[s];
    if (!as) as = std::make_unique<ApplyScratch>();
    RK(as->tA.ensure(size_t(sc) * elt_size(dtype)));
    RK(as->tB.ensure(size_t(sc) * elt_size(dtype)));
    ta = as->tA.p;
    tb = as->tB.p;
  }
  CK(launch_apply(op->op, dtype, ref(X), ref(Y), 1.0, 0.0, PtrRef{}, ta, tb, nullptr, s));
  return RTG_OK;
}

rtg_status rtg_sketch(rtg_handle h, rtg_shape shape, rtg_dtype dtype, const int64_t* sketch_dims,
                      uint64_t seed, uint64_t pid, const void* X, void* SX, rtg_stream stream) {
  if (h == nullptr) return fail(RTG_ERR_INVALID_ARG, "handle is NULL");
  int64_t n = 0;
  RK(check_shape(shape, &n));
  RK(check_dtype(dtype, true));
  const rtg_dtype pdt = dtype == RTG_BF16 ? RTG_F32 : dtype;   // BF16 input: FP32 plan and output
  SketchPlan sp;
  RK(build_sketch(shape, sketch_dims, seed, pid, pdt, sp));
  if (dtype == RTG_BF16 && (sp.nstage == 0 || !sp.stage_first[0]))
    return fail(RTG_ERR_UNSUPPORTED, "a BF16 sketch needs mode 1 sketched (sketch_dims[0] < dims[0])");
  DeviceGuard dg(h->device);
  if (!is_device_ptr(X) || !is_device_ptr(SX)) return fail(RTG_ERR_INVALID_ARG, "X and SX must be device pointers");
  if (overlaps(X, SX, size_t(std::min<int64_t>(n, sp.d)) * elt_size(pdt)))
    return fail(RTG_ERR_INVALID_ARG, "SX must not overlap X");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SketchScratch sc;
  RK(sketch_scratch_for(h, sp, seed, pid, s, &sc));
  CK(launch_sketch(sp, sc, ref(X), SX, nullptr, nullptr, s, dtype));
  return RTG_OK;
}

}  // extern "C"

// The signs depend on (seed, problem id); the scratch of rtg_sketch is kept
// per shape, sketch sizes, problem id, dtype and stream, and its signs are
// drawn again (on s) whenever the seed differs from the one they were drawn for.
static rtg_status sketch_scratch_for(rtg_handle h, const SketchPlan& sp, uint64_t seed, uint64_t pid,
                                     cudaStream_t s, SketchScratch* out) {
  std::string key;
  append_bytes(key, &sp.order, sizeof sp.order);
  append_bytes(key, sp.dims, sizeof sp.dims);
  append_bytes(key, sp.sdims, sizeof sp.sdims);
  append_bytes(key, &pid, sizeof pid);
  append_bytes(key, &sp.dtype, sizeof sp.dtype);
  append_bytes(key, &s, sizeof s);
  auto it = h->sketches.find(key);
  SketchCache* ce = nullptr;
  if (it == h->sketches.end()) {
    if (h->sketches.size() > 16) {
      cudaDeviceSynchronize();
      h->sketches.clear();
    }
    auto b = std::make_unique<SketchCache>();
    RK(b->buf.ensure(sketch_scratch_bytes(sp)));
    ce = b.get();
    h->sketches[key] = std::move(b);
  } else {
    ce = it->second.get();
  }
  const SketchScratch sc = carve_sketch_scratch(sp, ce->buf.p);
  if (!ce->drawn || ce->seed != seed) {
    CK(launch_theta(sp, sc.bits, sc.frags, s));
    ce->seed = seed;
    ce->drawn = true;
  }
  *out = sc;
  return RTG_OK;
}

extern "C" {

rtg_status rtg_krylov_create(rtg_handle h, const rtg_factor* A, int32_t nA, const rtg_factor* B,
                             int32_t nB, rtg_shape shape, rtg_dtype dtype, int32_t m,
                             const int64_t* sketch_dims, uint64_t seed, uint64_t pid,
                             rtg_krylov* out) {
  if (h == nullptr || out == nullptr) return fail(RTG_ERR_INVALID_ARG, "handle or krylov is NULL");
  *out = nullptr;
  int64_t n = 0;
  RK(check_shape(shape, &n));
  RK(check_dtype(dtype));
  RK(check_factors(A, nA, shape, "A_factors"));
  RK(check_factors(B, nB, shape, "B_factors"));
  if (m < 1 || m > kMaxK) return fail(RTG_ERR_INVALID_ARG, "m=%d not in 1..%d", m, kMaxK);
  DeviceGuard dg(h->device);
  auto K = std::make_unique<rtg_krylov_state>();
  K->ctx = h;
  K->dtype = dtype;
  K->m = m;
  RK(build_op(A, nA, B, nB, shape, K->op));
  RK(build_sketch(shape, sketch_dims, seed, pid, dtype, K->sp));
  const int64_t ae = apply_scratch_elems(K->op.op);
  Work tmpw;
  void *ta, *tb;
  SketchScratch tsk;
  const size_t bytes = carve_work(nullptr, dtype, n, K->sp, m, 1, ae, tmpw, &ta, &tb, &tsk);
  RK(K->mem.ensure(bytes));
  CK(cudaMemset(K->mem.p, 0, bytes));
  carve_work(K->mem.p, dtype, n, K->sp, m, 1, ae, K->w, &K->tA, &K->tB, &K->sk);
  CK(launch_theta(K->sp, K->sk.bits, K->sk.frags, nullptr));
  CK(cudaDeviceSynchronize());
  *out = K.release();
  return RTG_OK;
}

rtg_status rtg_krylov_destroy(rtg_krylov K) {
  if (K == nullptr) return RTG_OK;
  DeviceGuard dg(K->ctx->device);
  cudaDeviceSynchronize();
  delete K;
  return RTG_OK;
}

rtg_status rtg_krylov_start(rtg_handle h, rtg_krylov K, const void* C, const void* X0,
                            rtg_stream stream) {
  if (h == nullptr || K == nullptr) return fail(RTG_ERR_INVALID_ARG, "handle or krylov is NULL");
  DeviceGuard dg(h->device);
  if (!is_device_ptr(C)) return fail(RTG_ERR_INVALID_ARG, "C must be a device pointer");
  if (X0 != nullptr && !is_device_ptr(X0)) return fail(RTG_ERR_INVALID_ARG, "X0 must be a device pointer or NULL");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Work& w = K->w;
  CK(launch_reset(w, 0, s));
  PtrRef src = ref(C);
  if (X0 != nullptr) {
    CK(launch_apply(K->op.op, K->dtype, ref(X0), ref(w.V), -1.0, 1.0, ref(C), K->tA, K->tB, nullptr, s));
    src = ref(w.V);
  }
  StepOpts o{};
  o.tol = 0.0;
  o.bd_tol = K->dtype == RTG_F64 ? 1e-12 : 1e-6;
  const bool fused = K->sp.fused_dots != 0;
  SketchDots dots{&w, 0, o};
  CK(launch_sketch(K->sp, K->sk, src, fused ? w.S : w.Spart, fused ? &dots : nullptr, nullptr, s));
  CK(launch_start(w, src, o, fused, s));
  K->started = true;
  return RTG_OK;
}

rtg_status rtg_arnoldi_step(rtg_handle h, rtg_krylov K, rtg_stream stream) {
  if (h == nullptr || K == nullptr) return fail(RTG_ERR_INVALID_ARG, "handle or krylov is NULL");
  if (!K->started) return fail(RTG_ERR_INVALID_ARG, "rtg_krylov_start has not been called");
  DeviceGuard dg(h->device);
  StepOpts o{};
  o.tol = 0.0;
  o.bd_tol = K->dtype == RTG_F64 ? 1e-12 : 1e-6;
  o.solve_mode = 0;
  return enqueue_step(K->op, K->sp, K->w, K->dtype, K->tA, K->tB, K->sk, o,
                      reinterpret_cast<cudaStream_t>(stream));
}

rtg_status rtg_krylov_query(rtg_handle h, rtg_krylov K, rtg_krylov_view* view, double* H,
                            rtg_stream stream) {
  if (h == nullptr || K == nullptr || view == nullptr) return fail(RTG_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard dg(h->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Ctl c{};
  CK(cudaMemcpyAsync(&c, K->w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  if (H != nullptr)
    CK(cudaMemcpyAsync(H, K->w.H, sizeof(double) * size_t(K->m + 1) * K->m, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  view->j = c.j;
  view->m = K->m;
  view->breakdown = c.breakdown;
  view->sketch_size = K->w.d;
  view->n = K->w.n;
  view->beta = c.beta;
  view->rho = c.rho;
  view->V = K->w.V;
  view->Q = K->w.Q;
  return RTG_OK;
}

}  // extern "C"

// Called after the solve's descriptor has been uploaded and before its
// graph (or first kernel) is queued, on the solve's stream.
struct PreLaunch {
  rtg_status (*fn)(SolvePlan& P, cudaStream_t s, void* ctx);
  void* ctx;
};

// method 0: RTG-GMRES; 1: sketched Golub-Kahan.
static rtg_status submit_impl(int method, rtg_handle h, const rtg_factor* A, int32_t nA, const rtg_factor* B,
                              int32_t nB, rtg_shape shape, rtg_dtype dtype, const void* C, int32_t m,
                              const int64_t* sketch_dims, uint64_t seed, double lambda, const void* X0,
                              void* X, const rtg_opts* opts_in, rtg_stream stream,
                              const PreLaunch* pre = nullptr) {
  if (h == nullptr) return fail(RTG_ERR_INVALID_ARG, "handle is NULL");
  int64_t n = 0;
  RK(check_shape(shape, &n));
  RK(check_dtype(dtype));
  RK(check_factors(A, nA, shape, "A_factors"));
  RK(check_factors(B, nB, shape, "B_factors"));
  if (m < 1 || m > kMaxK) return fail(RTG_ERR_INVALID_ARG, "m=%d not in 1..%d", m, kMaxK);
  if (C == nullptr || X == nullptr) return fail(RTG_ERR_INVALID_ARG, "C and X must not be NULL");
  if (!std::isfinite(lambda)) return fail(RTG_ERR_INVALID_ARG, "lambda is not finite");
  rtg_opts opts{};
  if (opts_in) opts = *opts_in;
  if (!(opts.tol >= 0.0) || !std::isfinite(opts.tol)) return fail(RTG_ERR_INVALID_ARG, "opts.tol must be finite and >= 0");
  if (opts.max_restarts < 0) return fail(RTG_ERR_INVALID_ARG, "opts.max_restarts=%d must be >= 0", opts.max_restarts);
  if (opts.max_restarts > 0 && method == 1)
    return fail(RTG_ERR_UNSUPPORTED, "restarts are for rtg_gmres_solve (max_restarts=%d)", opts.max_restarts);
  if (int64_t(m) * (opts.max_restarts + 1) > kMaxK)
    return fail(RTG_ERR_INVALID_ARG, "m * (max_restarts + 1) = %lld exceeds %d steps",
                (long long)m * (opts.max_restarts + 1), kMaxK);
  if (!(opts.breakdown_tol >= 0.0)) return fail(RTG_ERR_INVALID_ARG, "opts.breakdown_tol must be >= 0");
  if (opts.slot < 0 || opts.slot >= RTG_MAX_SLOTS) return fail(RTG_ERR_INVALID_ARG, "opts.slot=%d not in 0..%d", opts.slot, RTG_MAX_SLOTS - 1);
  const int mode = lambda > 0 ? 1 : (lambda == 0 ? 0 : 2);
  if (mode == 2) {
    if (opts.n_mu < 1 || opts.n_mu > kMaxMu || opts.mu_grid == nullptr)
      return fail(RTG_ERR_INVALID_ARG, "lambda < 0 needs opts.mu_grid with 1..%d values", kMaxMu);
    for (int i = 0; i < opts.n_mu; ++i)
      if (!(opts.mu_grid[i] > 0.0) || !std::isfinite(opts.mu_grid[i])) return fail(RTG_ERR_INVALID_ARG, "mu_grid[%d] must be finite and > 0", i);
  }
  DeviceGuard dg(h->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t bytes_t = size_t(n) * elt_size(dtype);
  const bool C_dev = is_device_ptr(C), X_dev = is_device_ptr(X);
  const bool X0_dev = X0 != nullptr && is_device_ptr(X0);
  if (X0 != nullptr && X0 != X && overlaps(X0, X, bytes_t)) return fail(RTG_ERR_INVALID_ARG, "X partially overlaps X0");
  if (overlaps(C, X, bytes_t)) return fail(RTG_ERR_INVALID_ARG, "X overlaps C");

  SketchPlan sp;
  RK(build_sketch(shape, sketch_dims, seed, 0, dtype, sp));
  const bool phase_times = (opts.flags & RTG_FLAG_PHASE_TIMES) != 0;
  const int vdtype = (opts.flags & RTG_FLAG_BF16_BASIS) ? RTG_BF16 : dtype;
  if (vdtype == RTG_BF16 && method == 1)
    return fail(RTG_ERR_UNSUPPORTED, "RTG_FLAG_BF16_BASIS is for rtg_gmres_solve");
  if (vdtype == RTG_BF16) {
    if (dtype != RTG_F32) return fail(RTG_ERR_UNSUPPORTED, "RTG_FLAG_BF16_BASIS needs dtype RTG_F32");
    if (sp.nstage == 0 || !sp.stage_first[0])
      return fail(RTG_ERR_UNSUPPORTED, "RTG_FLAG_BF16_BASIS needs mode 1 sketched (sketch_dims[0] < dims[0])");
  }
  const bool use_graph = !(opts.flags & RTG_FLAG_NO_GRAPH) && !phase_times;
  std::string key = op_key(A, nA, B, nB, shape);
  append_bytes(key, &dtype, sizeof dtype);
  append_bytes(key, &m, sizeof m);
  append_bytes(key, sp.sdims, sizeof sp.sdims);
  const int nmu_key = mode == 2 ? opts.n_mu : 0;
  append_bytes(key, &mode, sizeof mode);
  append_bytes(key, &nmu_key, sizeof nmu_key);
  const bool has_x0 = X0 != nullptr;
  key.push_back(has_x0 ? '1' : '0');
  key.push_back(use_graph ? 'g' : 'd');
  append_bytes(key, &opts.slot, sizeof opts.slot);
  append_bytes(key, &vdtype, sizeof vdtype);
  append_bytes(key, &method, sizeof method);
  const bool true_resid = (opts.flags & RTG_FLAG_TRUE_RESIDUAL) != 0;
  key.push_back(true_resid ? 't' : '-');
  const int cycles = opts.max_restarts + 1;
  append_bytes(key, &cycles, sizeof cycles);

  rtg_context::Pending& pend = h->pending[opts.slot];
  if (pend.active) return fail(RTG_ERR_INVALID_ARG, "slot %d has a submitted solve that was not waited for", opts.slot);
  if (phase_times)
    for (const auto& q : h->pending)
      if (q.active && q.phase_times) return fail(RTG_ERR_INVALID_ARG, "another phase-timed solve is pending");
  auto it = h->plans.find(key);
  SolvePlan* P = nullptr;
  std::shared_ptr<SolvePlan> hold;
  if (it == h->plans.end()) {
    // the plan cache holds many shapes (a loop of solves over a set of uneven
    // problems keeps each plan); it is emptied when it would exceed 1024 plans
    // or a quarter of the device memory
    size_t held = 0;
    for (const auto& q : h->plans) held += q.second->mem.bytes;
    size_t freeb = 0, totalb = 0;
    if (cudaMemGetInfo(&freeb, &totalb) != cudaSuccess) {
      cudaGetLastError();
      totalb = 0;
    }
    if (h->plans.size() >= 1024 || (totalb > 0 && held > totalb / 4)) {
      // plans of other slots may still run on their streams: wait for the device
      cudaDeviceSynchronize();
      for (auto& q : h->pending)
        if (!q.active) q.plan.reset();
      h->plans.clear();
    }
    // Building a plan allocates memory and instantiates a CUDA graph; it
    // does so only while no other solve of this handle is in flight.
    for (const auto& q : h->pending)
      if (q.active) CK(cudaStreamSynchronize(q.stream));
    PlanSpec ps{A, nA, B, nB, shape, dtype, vdtype, n, m, sp, mode, nmu_key, has_x0, use_graph, method,
                true_resid, cycles};
    std::shared_ptr<SolvePlan> np;
    RK(make_plan(ps, nullptr, nullptr, nullptr, nullptr, &np, 0, &h->tuned));
    P = np.get();
    h->plans[key] = np;
    hold = np;
  } else {
    hold = it->second;
    P = hold.get();
  }
  // per-call descriptor (host arrays are staged through plan buffers)
  SolveDesc& D = *P->desc_host;
  D.C = C;
  D.X0 = X0;
  D.X = X;
  if (!C_dev) {
    RK(P->Cst.ensure(bytes_t));
    CK(cudaMemcpyAsync(P->Cst.p, C, bytes_t, cudaMemcpyHostToDevice, s));
    D.C = P->Cst.p;
  }
  if (has_x0 && !X0_dev) {
    RK(P->X0st.ensure(bytes_t));
    CK(cudaMemcpyAsync(P->X0st.p, X0, bytes_t, cudaMemcpyHostToDevice, s));
    D.X0 = P->X0st.p;
  }
  if (!X_dev) {
    RK(P->Xst.ensure(bytes_t));
    D.X = P->Xst.p;
    if (has_x0 && X0 == X) D.X0 = D.X;
    if (has_x0 && X0 == X && !X0_dev) {
      CK(cudaMemcpyAsync(P->Xst.p, X0, bytes_t, cudaMemcpyHostToDevice, s));
    }
  }
  {   // the 16-byte loads of the spatio-temporal apply and of the BF16 start kernel
    const bool x0_st = has_x0 && apply_uses_st(P->op.op, dtype, dtype, P->vdtype);
    if (x0_st && reinterpret_cast<uintptr_t>(D.X0) % 16 != 0)
      return fail(RTG_ERR_INVALID_ARG, "X0 must be 16-byte aligned for this operator");
    if (P->vdtype == RTG_BF16 && reinterpret_cast<uintptr_t>(D.C) % 16 != 0)
      return fail(RTG_ERR_INVALID_ARG, "C must be 16-byte aligned with RTG_FLAG_BF16_BASIS");
    if ((P->true_resid || P->w.cycles > 1) && apply_uses_st(P->op.op, dtype, dtype, P->vdtype) &&
        reinterpret_cast<uintptr_t>(D.X) % 16 != 0)
      return fail(RTG_ERR_INVALID_ARG, "X must be 16-byte aligned for this operator with "
                                       "RTG_FLAG_TRUE_RESIDUAL or restarts");
  }
  D.key[0] = seed;
  D.key[1] = 0;
  D.tol = opts.tol;
  D.bd_tol = opts.breakdown_tol > 0 ? opts.breakdown_tol : (dtype == RTG_F64 ? 1e-12 : 1e-6);
  D.lambda = lambda;
  D.n_mu = mode == 2 ? opts.n_mu : 0;
  for (int i = 0; i < D.n_mu; ++i) D.mu_grid[i] = opts.mu_grid[i];
  CK(cudaMemcpyAsync(P->desc_dev, P->desc_host, sizeof(SolveDesc), cudaMemcpyHostToDevice, s));
  if (pre != nullptr) RK(pre->fn(*P, s, pre->ctx));
  CK(cudaEventRecord(P->ev0, s));
  if (use_graph) {
    CK(cudaGraphLaunch(P->exec, s));
  } else {
    const StepOpts so = solve_step_opts(*P, 0, 0);
    PhaseTimer* pt = nullptr;
    if (phase_times) {
      if (!h->timer) h->timer = std::make_unique<PhaseTimer>();
      CK(h->timer->init());
      pt = h->timer.get();
      pt->reset(s);
    }
    // each group is queued behind a gate that the host opens once the group is queued
    auto group = [&](auto&& body) -> rtg_status {
      if (pt) CK(pt->hold());
      rtg_status st = body();
      if (pt) pt->release();
      return st;
    };
    // The host waits for each step and stops launching once the device has
    // stopped the solve, so the launch sequence is the one the graph runs.
    auto stopped = [&]() -> rtg_status {
      CK(cudaMemcpyAsync(P->stop_host, &P->w.ctl->stop, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      return RTG_OK;
    };
    RK(group([&] { return P->method == 1 ? enqueue_gk_prologue(*P, so, s, pt) : enqueue_prologue(*P, so, s, pt); }));
    RK(stopped());
    int steps = 0;
    while (steps < m * P->w.cycles && *P->stop_host == 0) {
      const int j = steps++;
      RK(group([&] {
        if (P->method == 1) return enqueue_gk_step(*P, so, s, pt, j);
        RK(enqueue_step(P->op, P->sp, P->w, dtype, P->tA, P->tB, P->sk, so, s, pt, j));
        if (P->w.cycles > 1) {
          PhaseScope rs(pt, RTG_PHASE_INIT, j, restart_launches(P->op.op, P->sp, dtype, P->vdtype));
          RK(enqueue_restart(*P, so, s));
        }
        return RTG_OK;
      }));
      RK(stopped());
    }
    P->direct_steps = steps;
    RK(group([&] { return enqueue_epilogue(*P, s, pt); }));
  }
  CK(cudaEventRecord(P->ev1, s));
  if (!X_dev) CK(cudaMemcpyAsync(X, P->Xst.p, bytes_t, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(P->info_host, P->info_dev, sizeof(InfoDev), cudaMemcpyDeviceToHost, s));
  pend.plan = hold;
  pend.stream = s;
  pend.m = m;
  pend.n_mu = mode == 2 ? opts.n_mu : 0;
  pend.mode = mode;
  pend.use_graph = use_graph;
  pend.phase_times = phase_times;
  pend.active = true;
  return RTG_OK;
}

extern "C" {

rtg_status rtg_gmres_submit(rtg_handle h, const rtg_factor* A, int32_t nA, const rtg_factor* B,
                            int32_t nB, rtg_shape shape, rtg_dtype dtype, const void* C, int32_t m,
                            const int64_t* sketch_dims, uint64_t seed, double lambda, const void* X0,
                            void* X, const rtg_opts* opts_in, rtg_stream stream) {
  return submit_impl(0, h, A, nA, B, nB, shape, dtype, C, m, sketch_dims, seed, lambda, X0, X, opts_in, stream);
}

rtg_status rtg_gk_solve(rtg_handle h, const rtg_factor* A, int32_t nA, const rtg_factor* B,
                        int32_t nB, rtg_shape shape, rtg_dtype dtype, const void* C, int32_t m,
                        const int64_t* sketch_dims, uint64_t seed, double lambda, const void* X0,
                        void* X, const rtg_opts* opts_in, rtg_info* info, rtg_stream stream) {
  RK(submit_impl(1, h, A, nA, B, nB, shape, dtype, C, m, sketch_dims, seed, lambda, X0, X, opts_in, stream));
  return rtg_gmres_wait(h, opts_in ? opts_in->slot : 0, info);
}

rtg_status rtg_gmres_wait(rtg_handle h, int32_t slot, rtg_info* info) {
  if (h == nullptr) return fail(RTG_ERR_INVALID_ARG, "handle is NULL");
  if (slot < 0 || slot >= RTG_MAX_SLOTS) return fail(RTG_ERR_INVALID_ARG, "slot=%d not in 0..%d", slot, RTG_MAX_SLOTS - 1);
  rtg_context::Pending& pend = h->pending[slot];
  if (!pend.active) return fail(RTG_ERR_INVALID_ARG, "slot %d has no submitted solve", slot);
  pend.active = false;
  DeviceGuard dg(h->device);
  SolvePlan* P = pend.plan.get();
  const int mode = pend.mode;
  const bool use_graph = pend.use_graph, phase_times = pend.phase_times;
  CK(cudaStreamSynchronize(pend.stream));
  const InfoDev& I = *P->info_host;
  if (info) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, P->ev0, P->ev1);
    fill_info(*P, I, mode, pend.n_mu, use_graph, ms, info);
    if (phase_times) h->timer->collect(I.iters, info);
  }
  if (phase_times && h->timer->host[1] != 0) {
    return fail(RTG_ERR_TIMEOUT, "phase timing: a gate waited 10 s for the host to queue its group");
  }
  return RTG_OK;
}

rtg_status rtg_gmres_solve_batched(rtg_handle h, int32_t nprob, const rtg_problem* probs,
                                   rtg_dtype dtype, const rtg_opts* opts_in, rtg_info* infos,
                                   rtg_stream stream) {
  if (h == nullptr) return fail(RTG_ERR_INVALID_ARG, "handle is NULL");
  rtg_opts opts{};
  if (opts_in) opts = *opts_in;
  if (opts.queue_slots < 0) return fail(RTG_ERR_INVALID_ARG, "opts.queue_slots must be >= 0");
  const bool queued = opts.queue_slots > 0;
  if (queued && opts.group_max > 1)
    return fail(RTG_ERR_INVALID_ARG, "opts.queue_slots and opts.group_max > 1 exclude each other");
  if (queued && (opts.flags & RTG_FLAG_PHASE_TIMES))
    return fail(RTG_ERR_UNSUPPORTED, "RTG_FLAG_PHASE_TIMES is not available with opts.queue_slots");
  const int max_prob = queued ? RTG_MAX_QUEUE : RTG_MAX_BATCH;
  if (nprob < 1 || nprob > max_prob) return fail(RTG_ERR_INVALID_ARG, "nprob=%d not in 1..%d", nprob, max_prob);
  if (probs == nullptr) return fail(RTG_ERR_INVALID_ARG, "probs is NULL");
  RK(check_dtype(dtype));
  if (opts.max_restarts < 0) return fail(RTG_ERR_INVALID_ARG, "opts.max_restarts=%d must be >= 0", opts.max_restarts);
  const bool use_graph = !(opts.flags & (RTG_FLAG_NO_GRAPH | RTG_FLAG_PHASE_TIMES));
  const bool phase_times = (opts.flags & RTG_FLAG_PHASE_TIMES) != 0;
  if (!(opts.breakdown_tol >= 0.0)) return fail(RTG_ERR_INVALID_ARG, "opts.breakdown_tol must be >= 0");
  const int vdtype = (opts.flags & RTG_FLAG_BF16_BASIS) ? RTG_BF16 : dtype;
  if (vdtype == RTG_BF16 && dtype != RTG_F32) return fail(RTG_ERR_UNSUPPORTED, "RTG_FLAG_BF16_BASIS needs dtype RTG_F32");
  DeviceGuard dg(h->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // validate every problem and form its structural key (problems with equal
  // keys run in lock step; the sequence of keys names the batch plan)
  std::vector<PlanSpec> specs(nprob);
  std::vector<std::string> keys(nprob);
  std::string bkey;
  if (opts.group_max < 0) return fail(RTG_ERR_INVALID_ARG, "opts.group_max must be >= 0");
  append_bytes(bkey, &opts.group_max, sizeof opts.group_max);
  append_bytes(bkey, &opts.queue_slots, sizeof opts.queue_slots);
  const int bflags = opts.flags & RTG_FLAG_TRUE_RESIDUAL;
  append_bytes(bkey, &bflags, sizeof bflags);
  append_bytes(bkey, &opts.max_restarts, sizeof opts.max_restarts);
  append_bytes(bkey, &dtype, sizeof dtype);
  append_bytes(bkey, &vdtype, sizeof vdtype);
  for (int i = 0; i < nprob; ++i) {
    const rtg_problem& q = probs[i];
    int64_t n = 0;
    RK(check_shape(q.shape, &n));
    RK(check_factors(q.A_factors, q.nA, q.shape, "A_factors"));
    RK(check_factors(q.B_factors, q.nB, q.shape, "B_factors"));
    if (q.m < 1 || q.m > kMaxK) return fail(RTG_ERR_INVALID_ARG, "problem %d: m=%d not in 1..%d", i, q.m, kMaxK);
    if (int64_t(q.m) * (opts.max_restarts + 1) > kMaxK)
      return fail(RTG_ERR_INVALID_ARG, "problem %d: m * (max_restarts + 1) exceeds %d steps", i, kMaxK);
    if (q.C == nullptr || q.X == nullptr) return fail(RTG_ERR_INVALID_ARG, "problem %d: C and X must not be NULL", i);
    if (!is_device_ptr(q.C) || !is_device_ptr(q.X) || (q.X0 && !is_device_ptr(q.X0)))
      return fail(RTG_ERR_INVALID_ARG, "problem %d: batched solves take device pointers", i);
    const size_t bytes_t = size_t(n) * elt_size(dtype);
    if (q.X0 != nullptr && q.X0 != q.X && overlaps(q.X0, q.X, bytes_t)) return fail(RTG_ERR_INVALID_ARG, "problem %d: X partially overlaps X0", i);
    if (overlaps(q.C, q.X, bytes_t)) return fail(RTG_ERR_INVALID_ARG, "problem %d: X overlaps C", i);
    if (!std::isfinite(q.lam) || !(q.tol >= 0.0) || !std::isfinite(q.tol))
      return fail(RTG_ERR_INVALID_ARG, "problem %d: lambda and tol must be finite, tol >= 0", i);
    const int mode = q.lam > 0 ? 1 : (q.lam == 0 ? 0 : 2);
    if (mode == 2) {
      if (opts.n_mu < 1 || opts.n_mu > kMaxMu || opts.mu_grid == nullptr)
        return fail(RTG_ERR_INVALID_ARG, "lambda < 0 needs opts.mu_grid with 1..%d values", kMaxMu);
      for (int k = 0; k < opts.n_mu; ++k)
        if (!(opts.mu_grid[k] > 0.0) || !std::isfinite(opts.mu_grid[k])) return fail(RTG_ERR_INVALID_ARG, "mu_grid[%d] must be finite and > 0", k);
    }
    SketchPlan sp;
    RK(build_sketch(q.shape, q.sketch_dims, q.seed, 0, dtype, sp));
    if (vdtype == RTG_BF16 && (sp.nstage == 0 || !sp.stage_first[0]))
      return fail(RTG_ERR_UNSUPPORTED, "problem %d: RTG_FLAG_BF16_BASIS needs mode 1 sketched", i);
    const int nmu = mode == 2 ? opts.n_mu : 0;
    specs[i] = PlanSpec{q.A_factors, q.nA, q.B_factors, q.nB, q.shape, dtype, vdtype, n, q.m, sp, mode, nmu,
                        q.X0 != nullptr, true, 0, (opts.flags & RTG_FLAG_TRUE_RESIDUAL) != 0,
                        opts.max_restarts + 1};
    std::string key = op_key(q.A_factors, q.nA, q.B_factors, q.nB, q.shape);
    append_bytes(key, &q.m, sizeof q.m);
    append_bytes(key, sp.sdims, sizeof sp.sdims);
    append_bytes(key, &mode, sizeof mode);
    append_bytes(key, &nmu, sizeof nmu);
    key.push_back(q.X0 ? '1' : '0');
    const uint32_t len = static_cast<uint32_t>(key.size());
    append_bytes(bkey, &len, sizeof len);
    bkey += key;
    keys[i] = std::move(key);
  }
  auto it = h->batches.find(bkey);
  BatchPlan* BP = nullptr;
  if (it == h->batches.end()) {
    // building allocates and instantiates: nothing of this handle may run
    CK(cudaDeviceSynchronize());
    if (h->batches.size() >= 4) h->batches.clear();
    auto nb = std::make_unique<BatchPlan>();
    BP = nb.get();
    // groups in order of first appearance; problems keep their order inside a group
    std::map<std::string, int> gid;
    std::vector<std::vector<int>> members;
    BP->group_of.resize(nprob);
    for (int i = 0; i < nprob; ++i) {
      auto g = gid.find(keys[i]);
      int k = 0;
      const int cap = queued ? nprob : (opts.group_max > 1 ? opts.group_max : 1);
      if (g == gid.end() || int(members[g->second].size()) >= cap) {
        k = static_cast<int>(members.size());
        gid[keys[i]] = k;
        members.emplace_back();
      } else {
        k = g->second;
      }
      members[k].push_back(i);
      BP->group_of[i] = k;
    }
    BP->slot_of.resize(nprob);
    int pos = 0;
    for (size_t k = 0; k < members.size(); ++k) {
      BP->gfirst.push_back(pos);
      BP->gcount.push_back(static_cast<int>(members[k].size()));
      for (int i : members[k]) BP->slot_of[i] = pos++;
    }
    // branches: one per group, or (queue) up to queue_slots per class
    std::vector<int> nbr(members.size(), 1);
    int branches = 0;
    for (size_t k = 0; k < members.size(); ++k) {
      if (queued) nbr[k] = std::min(opts.queue_slots, BP->gcount[k]);
      branches += nbr[k];
    }
    if (branches > RTG_MAX_BATCH)
      return fail(RTG_ERR_INVALID_ARG, "%d graph branches (classes x queue_slots) exceed %d", branches, RTG_MAX_BATCH);
    const size_t total = size_t(nprob) * (sizeof(SolveDesc) + sizeof(InfoDev));
    CK(cudaMallocHost(&BP->desc_host, total));
    std::memset(BP->desc_host, 0, total);
    SolveDesc* dh = reinterpret_cast<SolveDesc*>(BP->desc_host);
    InfoDev* ih = reinterpret_cast<InfoDev*>(BP->desc_host + size_t(nprob) * sizeof(SolveDesc));
    BP->queued = queued;
    if (queued) {
      BP->q_info = (size_t(nprob) * sizeof(SolveDesc) + 255) & ~size_t(255);
      BP->q_ctr = (BP->q_info + size_t(nprob) * sizeof(InfoDev) + 255) & ~size_t(255);
      BP->q_cur = (BP->q_ctr + members.size() * sizeof(unsigned) + 255) & ~size_t(255);
      RK(BP->qmem.ensure(BP->q_cur + size_t(branches) * sizeof(int)));
      CK(cudaMemset(BP->qmem.p, 0, BP->qmem.bytes));
    }
    char* qb = static_cast<char*>(BP->qmem.p);
    CK(cudaGraphCreate(&BP->graph, 0));
    // the plans (one per branch), each branch's class and estimated cost
    // (tensor entries x Krylov dimension x problems it serves)
    std::vector<int> cls_of;
    std::vector<double> cost;
    for (size_t k = 0; k < members.size(); ++k) {
      BP->gplan.push_back(static_cast<int>(BP->plans.size()));
      const int first = BP->gfirst[k];
      const PlanSpec& ps = specs[members[k][0]];
      for (int r = 0; r < nbr[k]; ++r) {
        std::shared_ptr<SolvePlan> pl;
        RK(make_plan(ps, nullptr, nullptr, dh + first, ih + first, &pl, queued ? 1 : BP->gcount[k], &h->tuned,
                     branches));
        BP->plans.push_back(std::move(pl));
        cls_of.push_back(static_cast<int>(k));
        cost.push_back(double(ps.n) * ps.m * BP->gcount[k] / nbr[k]);
      }
    }
    // queue batch with more branches than queue_slots (classes of few
    // problems): the branches form queue_slots chains, at most one branch of
    // a chain in flight; longest first, each to the chain with the least work
    // so far
    const int nchain = (queued && branches > opts.queue_slots) ? opts.queue_slots : branches;
    std::vector<std::vector<int>> chains(nchain);
    {
      std::vector<int> order(branches);
      for (int b = 0; b < branches; ++b) order[b] = b;
      if (nchain < branches)
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
      std::vector<double> load(nchain, 0.0);
      for (int b : order) {
        const int c = nchain < branches ? int(std::min_element(load.begin(), load.end()) - load.begin()) : b;
        chains[c].push_back(b);
        load[c] += cost[b];
      }
    }
    for (const auto& chain : chains) {
      std::vector<cudaGraphNode_t> prev, tail;
      for (int b : chain) {
        SolvePlan& P = *BP->plans[b];
        const int k = cls_of[b];
        const ChainLink link{prev.empty() ? nullptr : &prev, &tail};
        if (queued) {
          const int first = BP->gfirst[k];
          QueueArgs q{};
          q.desc = reinterpret_cast<const SolveDesc*>(qb) + first;
          q.info = reinterpret_cast<InfoDev*>(qb + BP->q_info) + first;
          q.counter = reinterpret_cast<unsigned*>(qb + BP->q_ctr) + k;
          q.n = BP->gcount[k];
          q.my_desc = P.desc_dev;
          q.my_info = P.info_dev;
          q.cur = reinterpret_cast<int*>(qb + BP->q_cur) + b;
          RK(build_queue_branch(P, BP->graph, q, link));
        } else {
          RK(build_branch(P, BP->graph, link));
        }
        prev.swap(tail);
      }
    }
    CK(cudaGraphInstantiate(&BP->exec, BP->graph, 0));
    CK(cudaEventCreate(&BP->ev0));
    CK(cudaEventCreate(&BP->ev1));
    h->batches[bkey] = std::move(nb);
  } else {
    BP = it->second.get();
  }
  SolveDesc* dh = reinterpret_cast<SolveDesc*>(BP->desc_host);
  InfoDev* ih = reinterpret_cast<InfoDev*>(BP->desc_host + size_t(nprob) * sizeof(SolveDesc));
  auto plan_of = [&](int i) -> SolvePlan& { return *BP->plans[BP->gplan[BP->group_of[i]]]; };
  for (int i = 0; i < nprob; ++i) {
    const rtg_problem& q = probs[i];
    const SolvePlan& P = plan_of(i);
    if (q.X0 && apply_uses_st(P.op.op, dtype, dtype, vdtype) && reinterpret_cast<uintptr_t>(q.X0) % 16 != 0)
      return fail(RTG_ERR_INVALID_ARG, "problem %d: X0 must be 16-byte aligned for this operator", i);
    if (vdtype == RTG_BF16 && reinterpret_cast<uintptr_t>(q.C) % 16 != 0)
      return fail(RTG_ERR_INVALID_ARG, "problem %d: C must be 16-byte aligned with RTG_FLAG_BF16_BASIS", i);
    if ((P.true_resid || P.w.cycles > 1) && apply_uses_st(P.op.op, dtype, dtype, vdtype) &&
        reinterpret_cast<uintptr_t>(q.X) % 16 != 0)
      return fail(RTG_ERR_INVALID_ARG, "problem %d: X must be 16-byte aligned for this operator with "
                                       "RTG_FLAG_TRUE_RESIDUAL", i);
    fill_desc(dh[BP->slot_of[i]], q.C, q.X0, q.X, q.seed, q.tol, opts.breakdown_tol, dtype, q.lam,
              P.mode == 2 ? opts.n_mu : 0, opts.mu_grid);
  }
  const size_t ngroups = BP->gfirst.size();
  char* qb = static_cast<char*>(BP->qmem.p);
  if (BP->queued && use_graph) {
    // the whole queue in one copy; the class counters start at zero
    CK(cudaMemcpyAsync(qb, dh, size_t(nprob) * sizeof(SolveDesc), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(qb + BP->q_ctr, 0, ngroups * sizeof(unsigned), s));
  } else if (!BP->queued) {
    // one strided copy per group each way: host records are contiguous, device
    // records sit at the start of each problem's block
    for (size_t k = 0; k < ngroups; ++k) {
      const SolvePlan& P = *BP->plans[BP->gplan[k]];
      CK(cudaMemcpy2DAsync(P.desc_dev, size_t(P.w.b.stride), dh + BP->gfirst[k], sizeof(SolveDesc),
                           sizeof(SolveDesc), size_t(P.w.b.n), cudaMemcpyHostToDevice, s));
    }
  }
  CK(cudaEventRecord(BP->ev0, s));
  std::vector<rtg_info> gph(ngroups);   // phase times per group (direct launches)
  std::vector<int> dsteps(nprob, 0);    // steps launched per problem (direct launches)
  if (use_graph) {
    CK(cudaGraphLaunch(BP->exec, s));
  } else {
    // Direct launches, one group after another.  The host reads the group's
    // count of running problems after each step and stops launching when it
    // reaches zero, so the launch sequence is the one the graph runs.  A
    // queued class runs its problems one after another on its first plan.
    PhaseTimer* pt = nullptr;
    if (phase_times) {
      if (!h->timer) h->timer = std::make_unique<PhaseTimer>();
      CK(h->timer->init());
      pt = h->timer.get();
    }
    for (size_t k = 0; k < ngroups; ++k) {
      SolvePlan& P = *BP->plans[BP->gplan[k]];
      auto group = [&](auto&& body) -> rtg_status {
        if (pt) CK(pt->hold());
        rtg_status st = body();
        if (pt) pt->release();
        return st;
      };
      auto left = [&]() -> rtg_status {
        CK(cudaMemcpyAsync(P.stop_host, P.group_left, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return RTG_OK;
      };
      const StepOpts so = solve_step_opts(P, 0, 0);
      const int runs = BP->queued ? BP->gcount[k] : 1;
      for (int r = 0; r < runs; ++r) {
        const int rec = BP->gfirst[k] + r;
        if (BP->queued) CK(cudaMemcpyAsync(P.desc_dev, dh + rec, sizeof(SolveDesc), cudaMemcpyHostToDevice, s));
        if (pt) pt->reset(s);
        RK(group([&] { return enqueue_prologue(P, so, s, pt); }));
        RK(left());
        int steps = 0;
        while (steps < P.w.m * P.w.cycles && *P.stop_host != 0) {
          const int j = steps++;
          RK(group([&] {
            RK(enqueue_step(P.op, P.sp, P.w, dtype, P.tA, P.tB, P.sk, so, s, pt, j));
            if (P.w.cycles > 1) {
              PhaseScope rs(pt, RTG_PHASE_INIT, j, restart_launches(P.op.op, P.sp, dtype, vdtype));
              RK(enqueue_restart(P, so, s));
            }
            return RTG_OK;
          }));
          RK(left());
        }
        P.direct_steps = steps;
        for (int q = 0; q < (BP->queued ? 1 : BP->gcount[k]); ++q) dsteps[rec + q] = steps;
        RK(group([&] { return enqueue_epilogue(P, s, pt); }));
        if (BP->queued) CK(cudaMemcpyAsync(ih + rec, P.info_dev, sizeof(InfoDev), cudaMemcpyDeviceToHost, s));
        if (pt) {
          CK(cudaStreamSynchronize(s));
          rtg_info& gi = gph[k];
          for (int q = 0; q < RTG_PHASE_COUNT; ++q) {
            gi.phase_ms[q] = 0.0;
            gi.phase_launches[q] = 0;
          }
          pt->collect(steps, &gi);
        }
      }
    }
  }
  CK(cudaEventRecord(BP->ev1, s));
  if (BP->queued && use_graph) {
    CK(cudaMemcpyAsync(ih, qb + BP->q_info, size_t(nprob) * sizeof(InfoDev), cudaMemcpyDeviceToHost, s));
  } else if (!BP->queued) {
    for (size_t k = 0; k < ngroups; ++k) {
      const SolvePlan& P = *BP->plans[BP->gplan[k]];
      CK(cudaMemcpy2DAsync(ih + BP->gfirst[k], sizeof(InfoDev), P.info_dev, size_t(P.w.b.stride),
                           sizeof(InfoDev), size_t(P.w.b.n), cudaMemcpyDeviceToHost, s));
    }
  }
  CK(cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, BP->ev0, BP->ev1);
  if (infos)
    for (int i = 0; i < nprob; ++i) {
      SolvePlan& P = plan_of(i);
      P.direct_steps = dsteps[BP->slot_of[i]];
      fill_info(P, ih[BP->slot_of[i]], P.mode, P.n_mu, use_graph, ms, &infos[i]);
      // the queue kernel that handed the problem back and took the next
      // (each branch's first take is not counted)
      if (BP->queued && use_graph) infos[i].launches += 1;
      if (phase_times)   // the phase times of the problem's whole group
        for (int q = 0; q < RTG_PHASE_COUNT; ++q) {
          infos[i].phase_ms[q] = gph[BP->group_of[i]].phase_ms[q];
          infos[i].phase_launches[q] = gph[BP->group_of[i]].phase_launches[q];
        }
    }
  return RTG_OK;
}

rtg_status rtg_gmres_solve(rtg_handle h, const rtg_factor* A, int32_t nA, const rtg_factor* B,
                           int32_t nB, rtg_shape shape, rtg_dtype dtype, const void* C, int32_t m,
                           const int64_t* sketch_dims, uint64_t seed, double lambda, const void* X0,
                           void* X, const rtg_opts* opts_in, rtg_info* info, rtg_stream stream) {
  RK(rtg_gmres_submit(h, A, nA, B, nB, shape, dtype, C, m, sketch_dims, seed, lambda, X0, X,
                      opts_in, stream));
  return rtg_gmres_wait(h, opts_in ? opts_in->slot : 0, info);
}

}  // extern "C"

// ================================================================== learned warm start

namespace {
struct WsHook {
  WsDecision* dec;
};
rtg_status ws_hook(SolvePlan& P, cudaStream_t s, void* ctx) {
  CK(launch_ws_write_desc(static_cast<WsHook*>(ctx)->dec, P.desc_dev, s));
  return RTG_OK;
}
}  // namespace

extern "C" rtg_status rtg_ws_solve(rtg_ws ws, rtg_handle h, const rtg_factor* A, int32_t nA, const rtg_factor* B,
                                   int32_t nB, rtg_shape shape, const float* C, int32_t m,
                                   const int64_t* sketch_dims, uint64_t seed, float* X, const rtg_opts* opts_in,
                                   rtg_info* info, rtg_ws_result* result, rtg_stream stream) {
  if (ws == nullptr || h == nullptr) return fail(RTG_ERR_INVALID_ARG, "warm-start or solver handle is NULL");
  int64_t n = 0;
  RK(check_shape(shape, &n));
  if (shape.order != 3 || shape.dims[2] != 3)
    return fail(RTG_ERR_INVALID_ARG, "the warm start takes I1 x I2 x 3 images");
  if (shape.dims[0] % 8 || shape.dims[1] % 8 || shape.dims[0] < 8 || shape.dims[1] < 8)
    return fail(RTG_ERR_INVALID_ARG, "the warm start needs image sides that are multiples of 8");
  RK(check_factors(A, nA, shape, "A_factors"));
  RK(check_factors(B, nB, shape, "B_factors"));
  if (C == nullptr || X == nullptr) return fail(RTG_ERR_INVALID_ARG, "C and X must not be NULL");
  rtg_opts opts{};
  if (opts_in) opts = *opts_in;
  if (opts.n_mu < 1 || opts.mu_grid == nullptr)
    return fail(RTG_ERR_INVALID_ARG, "rtg_ws_solve needs opts.mu_grid (the fallback chooses mu by GCV)");
  if (!(opts.tol >= 0.0) || !std::isfinite(opts.tol)) return fail(RTG_ERR_INVALID_ARG, "opts.tol must be finite and >= 0");
  if (opts.flags & (RTG_FLAG_PHASE_TIMES | RTG_FLAG_BF16_BASIS))
    return fail(RTG_ERR_UNSUPPORTED, "rtg_ws_solve takes neither RTG_FLAG_PHASE_TIMES nor RTG_FLAG_BF16_BASIS");
  DeviceGuard dg(h->device);
  if (!is_device_ptr(C) || !is_device_ptr(X)) return fail(RTG_ERR_INVALID_ARG, "C and X must be device pointers");
  if (overlaps(C, X, size_t(n) * 4)) return fail(RTG_ERR_INVALID_ARG, "X overlaps C");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SketchPlan sp;
  RK(build_sketch(shape, sketch_dims, seed, 0, RTG_F32, sp));
  OpHolder* op = nullptr;
  RK(get_op(h, A, nA, B, nB, shape, &op));
  if (apply_uses_st(op->op, RTG_F32, RTG_F32, RTG_F32) &&
      (reinterpret_cast<uintptr_t>(X) % 16 != 0 || reinterpret_cast<uintptr_t>(C) % 16 != 0))
    return fail(RTG_ERR_INVALID_ARG, "C and X must be 16-byte aligned for this operator");
  // workspace: R_0 (n), S(R_0) and S(C) (d each), log lambda, the decision
  const size_t off_sr = (size_t(n) * 4 + 255) & ~size_t(255);
  const size_t off_sc = off_sr + ((size_t(sp.d) * 4 + 255) & ~size_t(255));
  const size_t off_ll = off_sc + ((size_t(sp.d) * 4 + 255) & ~size_t(255));
  const size_t off_dec = off_ll + 256;
  RK(h->ws_work.ensure(off_dec + 256));
  if (h->ws_dec_host == nullptr) CK(cudaMallocHost(&h->ws_dec_host, sizeof(WsDecision)));
  char* base = static_cast<char*>(h->ws_work.p);
  float* R0 = reinterpret_cast<float*>(base);
  float* SR = reinterpret_cast<float*>(base + off_sr);
  float* SC = reinterpret_cast<float*>(base + off_sc);
  float* loglam = reinterpret_cast<float*>(base + off_ll);
  WsDecision* dec = reinterpret_cast<WsDecision*>(base + off_dec);
  // X_0 = C + net(C) and log lambda (the network's forward kernels, into X)
  RK(rtg_ws_predict(ws, 1, static_cast<int32_t>(shape.dims[0]), static_cast<int32_t>(shape.dims[1]), C, X, loglam,
                    stream));
  // R_0 = C - Phi(X_0), ||S(R_0)|| and ||S(C)||, the decision, X_0 = 0 on fallback
  const int64_t sc_el = apply_scratch_elems(op->op);
  void *ta = nullptr, *tb = nullptr;
  if (sc_el > 0) {
    std::unique_ptr<ApplyScratch>& as = h->apply_scratch[s];
    if (!as) as = std::make_unique<ApplyScratch>();
    RK(as->tA.ensure(size_t(sc_el) * 4));
    RK(as->tB.ensure(size_t(sc_el) * 4));
    ta = as->tA.p;
    tb = as->tB.p;
  }
  CK(launch_apply(op->op, RTG_F32, ref(X), ref(R0), -1.0, 1.0, ref(C), ta, tb, nullptr, s));
  SketchScratch skc;
  RK(sketch_scratch_for(h, sp, seed, 0, s, &skc));
  CK(launch_sketch(sp, skc, ref(R0), SR, nullptr, nullptr, s, RTG_F32));
  CK(launch_sketch(sp, skc, ref(C), SC, nullptr, nullptr, s, RTG_F32));
  CK(launch_ws_decide(SR, SC, sp.d, loglam, opts.tol, dec, s));
  CK(launch_ws_zero_if(dec, X, n, s));
  // the solve: X_0 = X (aliased), a GCV plan whose descriptor gets the decided
  // lambda (> 0: fixed mu) and stop level on the device, right before its graph
  WsHook hk{dec};
  PreLaunch pre{ws_hook, &hk};
  const int slot = opts.slot;
  RK(submit_impl(0, h, A, nA, B, nB, shape, RTG_F32, C, m, sketch_dims, seed, -1.0, X, X, &opts, stream, &pre));
  CK(cudaMemcpyAsync(h->ws_dec_host, dec, sizeof(WsDecision), cudaMemcpyDeviceToHost, s));
  RK(rtg_gmres_wait(h, slot, info));
  if (result != nullptr) {
    static_assert(sizeof(rtg_ws_result) == sizeof(WsDecision), "rtg_ws_result mirrors the device decision");
    std::memcpy(result, h->ws_dec_host, sizeof(WsDecision));
  }
  if (info != nullptr && h->ws_dec_host->lambda > 0.0) info->mu = h->ws_dec_host->lambda;
  return RTG_OK;
}

// ================================================================== diagnostics

extern "C" rtg_status rtg_selftest_bounded_wait(int32_t device, int32_t limit_ms, int32_t* status_out) {
  if (status_out == nullptr) return fail(RTG_ERR_INVALID_ARG, "status_out is NULL");
  if (limit_ms < 1 || limit_ms > 10000) return fail(RTG_ERR_INVALID_ARG, "limit_ms=%d not in 1..10000", limit_ms);
  int count = 0;
  CK(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) return fail(RTG_ERR_INVALID_ARG, "device %d not in 0..%d", device, count - 1);
  DeviceGuard dg(device);
  void* p = nullptr;
  CK(cudaHostAlloc(&p, 2 * sizeof(unsigned), cudaHostAllocMapped));
  struct Free {
    void* p;
    ~Free() { cudaFreeHost(p); }
  } fr{p};
  unsigned* host = static_cast<unsigned*>(p);
  host[0] = 0;   // the flag: nothing sets it
  host[1] = 0;   // the status the kernel writes
  unsigned* dev = nullptr;
  CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&dev), host, 0));
  cudaStream_t s = nullptr;
  CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  // the wait on a flag nothing sets, then a wait whose flag is already met
  // (the stream and the context stay usable after the expiry)
  cudaError_t e = launch_gate(dev, 1u, dev + 1, s, static_cast<unsigned long long>(limit_ms) * 1000000ull);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  const unsigned first = __atomic_load_n(host + 1, __ATOMIC_ACQUIRE);
  __atomic_store_n(host + 1, 0u, __ATOMIC_RELEASE);
  if (e == cudaSuccess) e = launch_gate(dev, 0u, dev + 1, s, 1000000000ull);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (e != cudaSuccess) return cuda_fail(e, "bounded-wait self-test");
  if (__atomic_load_n(host + 1, __ATOMIC_ACQUIRE) != 0u)
    return fail(RTG_ERR_CUDA, "a wait on a flag that was already set reported a timeout");
  *status_out = static_cast<int32_t>(first);
  return RTG_OK;
}
