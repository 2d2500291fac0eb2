// Internal declarations shared by the translation units of librtg.
// Tensors are column-major (mode 1 fastest), the ivec order of Section 4.1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rtg.h"

namespace rtg {

constexpr int kMaxOrder = RTG_MAX_ORDER;
constexpr int kMaxRadius = RTG_MAX_RADIUS;
constexpr int kMaxTaps = 2 * kMaxRadius + 1;
constexpr int kMaxK = RTG_MAX_KRYLOV;
constexpr int kMaxMu = RTG_MAX_MU;
constexpr int kMaxPasses = 8;
constexpr int kMaxMix = 4;          // channel-mixing size handled inside the fused blur kernel

// Lock-step batch: one launch serves n problems of identical shape.  Every
// pointer a kernel receives is problem 0's; problem p's memory (workspace,
// descriptor, info record, sketch scratch) sits `stride` bytes further per
// problem.  The problem is the slowest part of blockIdx.z (z = p * nz + local
// z, nz = gridDim.z / n).  n = 1, stride = 0 for a single solve.
struct Batch {
  int n = 1;
  int64_t stride = 0;
};
#ifdef __CUDACC__
struct BIdx {
  int p;          // problem
  unsigned z;     // local blockIdx.z
  unsigned nz;    // local gridDim.z
  int64_t off;    // byte offset of the problem's memory
};
__device__ __forceinline__ BIdx bidx(const Batch& b) {
  BIdx r;
  r.nz = gridDim.z / static_cast<unsigned>(b.n);
  r.p = static_cast<int>(blockIdx.z / r.nz);
  r.z = blockIdx.z % r.nz;
  r.off = static_cast<int64_t>(r.p) * b.stride;
  return r;
}
template <typename T>
__device__ __forceinline__ T* bsh(T* p, int64_t off) {
  return p == nullptr ? p : reinterpret_cast<T*>(reinterpret_cast<uintptr_t>(p) + off);
}
#endif
// grid z of a batched launch: local z, capped so that n * z fits the limit
inline unsigned batch_z(int64_t local, const Batch& b) {
  int64_t cap = 65535 / (b.n > 0 ? b.n : 1);
  if (local > cap) local = cap;
  if (local < 1) local = 1;
  return static_cast<unsigned>(local * b.n);
}

enum PassKind : int { PK_BAND = 1, PK_DENSE = 2 };

// One mode product of the separable operator Phi (Eq. 56-57): either a
// banded Toeplitz matrix (taps) or a dense matrix (device, column-major).
struct Pass {
  int mode;          // 0-based
  int kind;          // PK_BAND / PK_DENSE
  int n;             // mode size
  int radius;        // PK_BAND
  double taps[kMaxTaps];
  const double* dense;   // PK_DENSE: device pointer, n*n column-major
};

// Operator as the list of mode products, in application order, plus the
// parameters of the fused kernel when the list matches its pattern:
// banded/identity on modes 1 and 2, and on mode 3 identity or a dense
// (or banded) matrix of size <= kMaxMix; higher modes untouched.
struct OpPlan {
  int order;
  int64_t dims[kMaxOrder];
  int npass;
  Pass pass[kMaxPasses];
  bool fused;
  int r1, r2;                // fused: radii on modes 1 and 2 (0 with a unit tap = identity)
  double t1[kMaxTaps], t2[kMaxTaps];
  int mix;                   // fused: 0 = no channel mixing, else mix size (= dims[2])
  double M3[kMaxMix * kMaxMix];   // fused: mode-3 matrix, M3[p + mix*c] = M(p, c)
  // spatio-temporal path: banded modes 1-2, mode-3 mix of st_nc (1 or 3)
  // channels, banded mode 4 of radius r4 <= 2 (t4: 2 r4 + 1 taps)
  bool st;
  int st_nc;
  double st_M[kMaxMix * kMaxMix];
  int r4;
  double t4[5];
};

// Control block of one sketched Arnoldi process (device resident).
struct Ctl {
  int j;            // completed steps in this cycle
  int stop;         // no further steps
  int breakdown;
  int converged;
  int status;       // rtg_status seen on the device
  int skip_update;  // do not form V_{j+1} (stopped by convergence inside a solve)
  int iters_total;  // steps over all cycles
  int cycle;
  int loops;        // executions of the step body since the reset (hard cap m+1)
  int givens;       // a finished Hessenberg column awaits its Givens update
  int counted;      // lock-step batch: this problem's stop has been counted
  int rs_skip;      // 1 unless a restart is pending: the body's restart kernels return at once
  double beta;      // ||R_0||_Theta of this cycle
  double beta0;     // of the first cycle (scale of rho)
  double rho;       // last rho_j
  double pre2;      // ||S(Phi V_j)||^2 before orthogonalisation
  double hnext;     // h_{j+1,j}
  double mu;        // chosen regularisation
  double gcv_best;
  double gk_scale;  // Golub-Kahan: the norm the next update divides by
  double true_rr;   // ||C - Phi(X)||_F / ||C||_F of the returned X (true-residual epilogue)
  double true_th;   // ||C - Phi(X)||_Theta / ||R_0||_Theta of the first cycle
};

// Per-call parameters of a solve, read by the graph's kernels.
struct SolveDesc {
  const void* C;
  const void* X0;   // may be null
  void* X;
  double tol;
  double bd_tol;
  double lambda;    // > 0 fixed, 0 least squares, < 0 GCV
  int n_mu;
  int pad;
  double mu_grid[kMaxMu];
  uint64_t key[2];  // Philox seed and problem id of the sketch signs
};

// Learned warm start (rtg_ws_solve): the device-side decision taken from
// ||S(R_0)|| and ||S(C)|| before the solve's graph runs.  Same layout as
// rtg_ws_result.
struct WsDecision {
  int fell_back;    // 1: ||S(C - Phi(X_0))|| >= ||S(C)||: X_0 = 0, GCV
  int pad;
  double lambda;    // > 0: exp(predicted log lambda); < 0: GCV over the grid
  double tol;       // stop level of rho (relative to ||R_0||_Theta of the solve)
  double sC, sR;    // ||S(C)||, ||S(C - Phi(X_0))|| of the prediction
};

// Host-visible summary written at the end of a solve (one D2H copy).
struct InfoDev {
  int iters, restarts, breakdown, converged, status, k, pad0, pad1;
  double beta, mu, rho_final, true_rel_resid, true_rel_resid_theta;
  double rho_hist[kMaxK];
  double gcv[kMaxMu];
};

// Leading dimension of the Gram matrix G of the stored sketched basis: even,
// so that every column starts on a 16-byte boundary (the step finish stages
// it in shared memory with 16-byte copies that bypass L1).
__host__ __device__ inline int gram_ld(int m) { return (m + 2) & ~1; }

// Workspace of one Arnoldi process.  T is the data type (double / float).
// Doubles of the reduced solve's per-CTA working set: two (m+1) x (m+1)
// matrices and two vectors of m+1.
__host__ __device__ inline int64_t tk_scratch_doubles(int m) {
  return 2 * static_cast<int64_t>(m + 1) * (m + 1) + 2 * static_cast<int64_t>(m + 1);
}

struct Work {
  int dtype;                   // RTG_F64 / RTG_F32: C, X, S, Q and the arithmetic
  int vdtype;                  // storage of V and W: dtype, or RTG_BF16 for an FP32 solve
  int64_t n;                   // elements per tensor
  int d;                       // sketch size prod(s'_k)
  int m;                       // Krylov dimension
  int cycles = 1;              // most Arnoldi cycles of a solve (restarts + 1)
  int upcfg = 0;               // basis-update ring geometry (index into the autotuner's list)
  void* V;                     // (m+1) * n
  void* W;                     // n
  void* U;                     // Golub-Kahan: ring of 2 left-basis tensors (else null)
  void* S;                     // d   (sketch of W, then s after the first GS pass)
  void* Spart;                 // nparts * d partial sketches written by the chain
  int nparts;
  void* tmp0;                  // sketch chain intermediates
  void* tmp1;
  void* Q;                     // (m+1) * d sketched basis
  double* part;                // partial sums: blocks x (2m+4)
  unsigned* counter;           // last-block counters (several)
  Ctl* ctl;
  double* H;                   // (m+1) x m Hessenberg, column-major
  double* R;                   // (m+1) x m rotated Hessenberg (upper triangular part)
  double* cs;                  // Givens cosines (m)
  double* sn;                  // Givens sines (m)
  double* g;                   // rotated right-hand side (m+1)
  double* G;                   // (m+1) x (m+1) Gram matrix of the stored sketched basis, leading
                               // dimension gram_ld(m)
  double* rho_hist;            // (m) per cycle
  double* y;                   // solution coefficients (m)
  double* gcv;                 // GCV values (kMaxMu)
  double* ysel;                // per-mu coefficient candidates (kMaxMu * m)
  int part_rows;               // rows available in part
  Batch b;                     // lock-step batch of identical workspaces
#ifdef __CUDACC__
  // this workspace moved to the problem `off` bytes further
  __device__ __forceinline__ Work at(int64_t off) const {
    Work r = *this;
    r.V = bsh(V, off);
    r.W = bsh(W, off);
    r.U = bsh(U, off);
    r.S = bsh(S, off);
    r.Spart = bsh(Spart, off);
    r.tmp0 = bsh(tmp0, off);
    r.tmp1 = bsh(tmp1, off);
    r.Q = bsh(Q, off);
    r.part = bsh(part, off);
    r.counter = bsh(counter, off);
    r.ctl = bsh(ctl, off);
    r.H = bsh(H, off);
    r.R = bsh(R, off);
    r.cs = bsh(cs, off);
    r.sn = bsh(sn, off);
    r.g = bsh(g, off);
    r.G = bsh(G, off);
    r.rho_hist = bsh(rho_hist, off);
    r.y = bsh(y, off);
    r.gcv = bsh(gcv, off);
    r.ysel = bsh(ysel, off);
    return r;
  }
#endif
};

// Sketch description: modes with s_k < I_k carry Theta_k as packed sign
// bits (row-major rows of ceil(I_k/32) words), and the contraction chain
// (one stage per sketched mode, in increasing mode order).
struct SketchPlan {
  int order;
  int dtype;                   // data type of the chain (RTG_F64 / RTG_F32)
  int64_t dims[kMaxOrder];
  int64_t sdims[kMaxOrder];    // s'_k
  int sketched[kMaxOrder];
  int64_t bit_off[kMaxOrder];  // offset of Theta_k in the Philox sign stream
  int64_t word_off[kMaxOrder]; // offset of Theta_k in the packed device array
  int wpr[kMaxOrder];          // 32-bit words per row
  int64_t total_words;         // packed device array size (uint32 words)
  int64_t d;                   // prod(s'_k)
  int64_t tmp_elems;           // elements of one scratch tensor
  double scale;                // prod 1/sqrt(s_k) over sketched modes
  uint64_t seed, pid;
  // contraction stages
  int nstage;
  int stage_mode[kMaxOrder];
  int stage_first[kMaxOrder];  // 1: L == 1 (first-mode tensor-core kernel)
  int stage_split[kMaxOrder];  // K split (partial outputs)
  int stage_kt[kMaxOrder];     // K tiles of 16
  int stage_ntile[kMaxOrder];  // 128-row tiles (L == 1 stages, tcgen05) or n8 tiles (later stages) of the sketch size
  int stage_kb[kMaxOrder];     // K blocks of 64 (tcgen05 stages)
  int stage_umma[kMaxOrder];   // an L == 1 stage of the FP32 chain that runs on tcgen05
  int64_t stage_L[kMaxOrder], stage_I[kMaxOrder], stage_R[kMaxOrder], stage_s[kMaxOrder];
  int64_t stage_out[kMaxOrder];   // elements of one stage output
  // FP32 chain layouts: an inner stage reads its input either in the
  // natural (column-major) order or blocked for it: block (r, l/16) holds
  // I rows of 20 floats (16 values of l, 4 pad).  A stage that is not last
  // writes its output blocked for the next stage, whose view of the
  // tensor is (L', I', R') with M = product of the unsketched dims between
  // the two modes: (l, q, r) -> l' = l + L q + L s (r % M), i' = (r / M) % I',
  // r' = r / (M I').
  int stage_in_blocked[kMaxOrder];
  int64_t next_M[kMaxOrder], next_L[kMaxOrder], next_I[kMaxOrder], next_LT[kMaxOrder];
  int64_t stage_out_alloc[kMaxOrder];   // floats the stage output buffer needs
  int64_t frag_off[kMaxOrder];    // uint32 offset of the stage's Theta images (tcgen05) or fragments (mma.sync)
  int64_t frag_words;
  int64_t part_elems;             // elements of each scratch tensor
  int last_split;                 // partial copies of the final sketch (1)
  int fused_dots;                 // the last stage can run the first Gram-Schmidt pass
  int64_t dots_blocks;            // CTAs of that last stage (rows of partial sums)
};

// Scratch of one sketch chain: signs, Theta images / fragments, two tensors.
struct SketchScratch {
  uint32_t* bits = nullptr;
  uint32_t* frags = nullptr;
  void* tmp0 = nullptr;
  void* tmp1 = nullptr;
};

// Fills sp; returns an error message or nullptr (k_sketch.cu).
const char* make_sketch_plan(int order, const int64_t* dims, const int64_t* sketch_dims,
                             uint64_t seed, uint64_t pid, int dtype, SketchPlan& sp);
size_t sketch_scratch_bytes(const SketchPlan& sp);
SketchScratch carve_sketch_scratch(const SketchPlan& sp, void* base);

// A tensor pointer resolved on the device: an explicit base, or a base read
// from device memory (per-call descriptors of a captured graph), optionally
// advanced by (*jidx) * stride elements (the current basis vector V_j).
struct PtrRef {
  const void* base = nullptr;
  const void* const* ind = nullptr;
  const int* jidx = nullptr;
  int64_t stride = 0;
  int joff = 0;
  int mod = 0;      // > 0: slot (*jidx + joff) % mod of a ring
  int nslot = 0;    // host: slots of the buffer `base` (slot indexing without a ring), 0 unknown
#ifdef __CUDACC__
  __device__ __forceinline__ PtrRef at(int64_t off) const {
    PtrRef r = *this;
    r.base = bsh(base, off);
    r.ind = bsh(ind, off);
    r.jidx = bsh(jidx, off);
    return r;
  }
  template <typename T>
  __device__ __forceinline__ T* get() const {
    const void* b = ind ? *ind : base;
    T* p = static_cast<T*>(const_cast<void*>(b));
    if (jidx) {
      const int slot = mod > 0 ? (*jidx + joff) % mod : *jidx + joff;
      p += static_cast<int64_t>(slot) * stride;
    }
    return p;
  }
#endif
};
inline PtrRef ref(const void* p) { PtrRef r; r.base = p; return r; }

// Raises a kernel's largest dynamic shared memory on the current device to
// at least `bytes` (never lowers it: graphs captured earlier may launch the
// kernel with a larger size than the current call needs) and gives the
// unified L1 / shared array to shared memory as far as it goes.  Every kernel
// of a solve asks for the same split, so an SM never drains to re-partition
// it between launches.  Thread-safe (rtg_api.cu).
cudaError_t raise_smem(const void* kernel, size_t bytes);
template <typename K>
inline cudaError_t set_smem(K* kernel, size_t bytes) {
  return raise_smem(reinterpret_cast<const void*>(kernel), bytes);
}

// Sets the thread-local message rtg_last_error() returns (rtg_api.cu).
void record_error(const char* msg);

// ---------------------------------------------------------------- launchers
// k_philox.cu
cudaError_t launch_philox_words(uint64_t seed, uint64_t pid, int64_t n_words, uint64_t* out,
                                cudaStream_t s);
// key_dev (optional): device array {seed, problem_id} read when the kernel runs,
// so one captured graph serves every seed; otherwise sp.seed / sp.pid.
cudaError_t launch_theta_bits(const SketchPlan& sp, uint32_t* bits, cudaStream_t s,
                              const uint64_t* key_dev = nullptr, Batch b = Batch{});
// signs, then (FP32 chain) the Theta images and fragments of every stage
cudaError_t launch_theta(const SketchPlan& sp, uint32_t* bits, uint32_t* frags, cudaStream_t s,
                         const uint64_t* key_dev = nullptr, Batch b = Batch{});

// k_apply.cu: Y = alpha * Phi(X) + beta * Z (Z may be null when beta == 0).
// tmp: scratch of n elements for the unfused path (may be null if unused).
// tin / tout: storage type of X and Y when they differ from dtype (RTG_BF16
// runs the spatio-temporal kernel, FP32 arithmetic); Z has type dtype.
cudaError_t launch_apply(const OpPlan& op, int dtype, PtrRef X, PtrRef Y, double alpha,
                         double beta, PtrRef Z, void* tmp, void* tmp2, const int* stop,
                         cudaStream_t s, int tin = -1, int tout = -1, Batch b = Batch{});
// The spatio-temporal kernel can apply op to X stored as tin.
bool st_supported(const OpPlan& op, int tin);
int st_bucket(int r);
// Scratch elements the unfused path needs (0 when fused).
int64_t apply_scratch_elems(const OpPlan& op);
// Kernels one launch_apply issues (combine: alpha != 1 or a Z term).
int apply_launches(const OpPlan& op, bool combine, int dtype = RTG_F32, int tin = -1, int tout = -1);
// launch_apply takes the spatio-temporal kernel for these types.
bool apply_uses_st(const OpPlan& op, int dtype, int tin, int tout);

// k_sketch.cu: S(X) into `out` (d elements).  With dots != null and
// sp.fused_dots, the last contraction also runs Gram-Schmidt pass
// dots->pass (0: beta, 1: h1) on the sketch it writes (out must be w.S).
struct Work;
struct StepOpts;
struct SketchDots;
// xdtype: storage type of X (default sp.dtype); RTG_BF16 needs an FP32 plan whose
// first stage contracts mode 1.
cudaError_t launch_sketch(const SketchPlan& sp, const SketchScratch& sc, PtrRef X, void* out,
                          const SketchDots* dots, const int* stop, cudaStream_t s, int xdtype = -1,
                          Batch b = Batch{});
int sketch_launches(const SketchPlan& sp);

// k_arnoldi.cu: the sketched Arnoldi process on a Work.
//   start:  beta = ||S||, V_0 = src / beta, Q_0 = S / beta  (src = R_0)
//   pass1:  one reduction (Q^T S, ||S||^2, Gram row), then h (CGS2 through
//           the Gram matrix), h_{j+1,j}, Givens and the stop rule
//   update: V_{j+1} = (W - V h)/h_{j+1,j}, Q_{j+1} = (S - Q h)/h_{j+1,j}
struct StepOpts {
  double tol;            // rho stop level (read from desc when desc_tol is set)
  double bd_tol;
  const double* desc_tol;    // optional device pointer overriding tol
  const double* desc_bd_tol; // optional device pointer overriding bd_tol
  int solve_mode;        // 1: skip V_{j+1} once the solve stops
  int use_cond;
  unsigned long long cond;   // cudaGraphConditionalHandle
  // restarts in a graph: the IF node around the body's restart sequence
  // (set to 1 by the Givens block that ends a cycle, back to 0 by the
  // sequence's last kernel)
  int use_rs_cond;
  unsigned long long rs_cond;
  // lock-step batch: problems still running (the loop ends when it reaches 0);
  // shared by the batch, not moved with a problem's memory
  unsigned* group_left;
#ifdef __CUDACC__
  __device__ __forceinline__ StepOpts at(int64_t off) const {
    StepOpts r = *this;
    r.desc_tol = bsh(desc_tol, off);
    r.desc_bd_tol = bsh(desc_bd_tol, off);
    return r;
  }
#endif
};
struct SketchDots {
  const Work* w;
  int pass;
  StepOpts o;
};
// pass 0 on w.Spart (unless the sketch already ran it) and the scaling V_0, Q_0
// src has type sdtype (dtype, or vdtype when it is the V_0 slot).
// gate (optional): device flag; the kernels return at once while it is nonzero
// (the restart sequence passes &ctl->rs_skip)
cudaError_t launch_start(const Work& w, PtrRef src, const StepOpts& o, bool fused, cudaStream_t s,
                         int sdtype = -1, const int* gate = nullptr);
cudaError_t launch_pass1(const Work& w, const StepOpts& o, cudaStream_t s);
int gs_grid(int64_t d);
cudaError_t launch_update(const Work& w, const StepOpts& o, cudaStream_t s);
// the update streams the basis through the shared-memory ring (w.upcfg applies)
bool update_uses_ring(const Work& w);
// number of ring geometries (w.upcfg in 0..count-1)
int update_configs();
// group_left (lock-step batch): set to the number of problems
cudaError_t launch_reset(const Work& w, int new_cycle, cudaStream_t s, unsigned* group_left = nullptr,
                         const int* gate = nullptr);
// end of a restart sequence: rs_skip = 1 again (and the IF node's condition 0)
cudaError_t launch_restart_done(const Work& w, const StepOpts& o, cudaStream_t s);

// k_solve.cu: projected Tikhonov / GCV, assembly and the info summary.
struct FinishOpts {
  const SolveDesc* desc;     // lambda, mu grid
  int n_mu;                  // structural: GCV blocks (lambda < 0)
  int mode;                  // 0: least squares, 1: fixed mu, 2: GCV
};
cudaError_t launch_tikhonov(const Work& w, const FinishOpts& f, cudaStream_t s, const int* gate = nullptr);
// X = X0 + sum_j y_j V_j; after a restart (ctl->cycle > 0) X itself is the X0 (it holds the
// accumulated iterate)
cudaError_t launch_assemble(const Work& w, PtrRef X0, PtrRef X, cudaStream_t s, const int* gate = nullptr);
cudaError_t launch_finalize(const Work& w, InfoDev* info, cudaStream_t s);
// The final residual of the Block GMRES algorithm: with R = C - Phi(X) in the
// V_0 slot (type dtype) and S(R) in w.Spart, ||R||_F / ||C||_F and
// ||S(R)|| / beta_0 into the control block (deterministic reduction).
cudaError_t launch_true_resid(const Work& w, PtrRef C, cudaStream_t s);
// k_gk.cu: sketched Golub-Kahan (Algorithm 4).  phase 0: beta_0 = ||S(R_0)||;
// 1: alpha_0 = ||S(Phi^T U_0)||; 2: beta_{j+1} = ||S(Phi V_j) - alpha_j S(U_j)||;
// 3: alpha_{j+1} = ||S(Phi^T U_{j+1}) - beta_{j+1} S(V_j)||.  The sketch of the
// product is in w.S, S(U_j) in Q slot 0, S(V_j) in Q slot 1.
cudaError_t launch_gk_norm(const Work& w, int phase, const StepOpts& o, cudaStream_t s);
// phase 0: U_0 = src / beta_0; 1: V_0 = W / alpha_0; 2: U_{j+1} = (W - alpha_j U_j) / beta_{j+1}
// (and the Givens step of column j beside it); 3: V_{j+1} = (W - beta_{j+1} V_j) / alpha_{j+1};
// the sketched vectors follow the same recurrences.
cudaError_t launch_gk_update(const Work& w, int phase, PtrRef src, const StepOpts& o, cudaStream_t s);

// k_solve.cu, learned warm start: decision from the sketches S(R_0) (SR) and
// S(C) (SC) of d entries and the predicted log lambda; tol is the stop level
// relative to ||S(C)||.
cudaError_t launch_ws_decide(const float* SR, const float* SC, int64_t d, const float* loglam, double tol,
                             WsDecision* dec, cudaStream_t s);
// X = 0 when the decision fell back
cudaError_t launch_ws_zero_if(const WsDecision* dec, float* X, int64_t n, cudaStream_t s);
// the decided lambda and tol into the solve's descriptor (after its upload)
cudaError_t launch_ws_write_desc(const WsDecision* dec, SolveDesc* desc, cudaStream_t s);

// Phase timing: bounded wait of the stream on a host-written flag.
cudaError_t launch_gate(const unsigned* flag, unsigned want, unsigned* status, cudaStream_t s,
                        unsigned long long limit_ns = 10000000000ull);
}  // namespace rtg
