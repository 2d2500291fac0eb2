/*
 * rtg.h -- C ABI of the GB300 (sm_103a) Randomized Tensor Global GMRES library.
 *
 * Method: A. Badahmane, "Randomized Tensor Krylov Subspace Methods via
 * Sketched Einstein Product with Applications to Image and Video
 * Restoration".  The library solves Phi(X) = C for a separable blur
 * operator Phi(X) = A *_N X (*_M B) (Section 1; Eq. 56-57) by RTG-GMRES:
 * sketched global Arnoldi (Section 4.3 and the algorithm "Block GMRES via
 * Sketched Einstein Product"), the Hessenberg least-squares problem
 * (Eq. 11S) and the projected Tikhonov problem (Eq. 12S-14S, Eq. 13) with
 * mu chosen by GCV (Section 3, "Parameter selection via GCV").
 *
 * Conventions shared by every entry point
 *  - Tensors are dense, contiguous and column-major: mode 1 varies fastest
 *    (the ivec ordering of Section 4.1).  Order 1..4.
 *  - Device pointers are caller-owned; the library never frees them.
 *    rtg_gmres_solve also accepts host pointers (pageable or pinned) for
 *    C, X0 and X and stages them through its own device buffers.
 *  - Host arrays inside structs (taps, dense factors, mu grids) are read
 *    during the call only.
 *  - All work is ordered on the given stream (NULL = legacy default
 *    stream).  rtg_gmres_solve and rtg_krylov_query synchronise that stream
 *    once, at the end, to return host-side results; the other calls are
 *    asynchronous.
 *  - Errors: every call returns an rtg_status; arguments are validated
 *    before anything is launched, and rtg_last_error() returns a
 *    thread-local message for the last failing call.  No call aborts the
 *    process or traps the GPU; device-side anomalies (non-finite values,
 *    breakdown) are reported through rtg_info.
 *  - A handle is bound to one device and is not thread-safe: use one
 *    handle per host thread.  Calls of one handle on different streams
 *    may overlap on the GPU: rtg_operator_apply and rtg_sketch keep their
 *    scratch per stream, and solves in flight at once use different
 *    workspace slots (rtg_opts.slot).
 */
#ifndef RTG_H
#define RTG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RTG_MAX_ORDER 4
#define RTG_MAX_RADIUS 32      /* banded factors: taps of length 2r+1, r <= 32 */
#define RTG_MAX_KRYLOV 256     /* largest Krylov dimension m */
#define RTG_MAX_MU 32          /* largest GCV grid */

typedef enum rtg_status {
    RTG_OK = 0,
    RTG_ERR_INVALID_ARG = 1,   /* bad pointer, shape, size or option */
    RTG_ERR_UNSUPPORTED = 2,   /* valid but not implemented (e.g. dtype for that call) */
    RTG_ERR_CUDA = 3,          /* a CUDA runtime call failed; see rtg_last_error() */
    RTG_ERR_ALLOC = 4,         /* device or pinned allocation failed */
    RTG_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
    RTG_ERR_NONFINITE = 6      /* NaN/Inf met in the data (reported by rtg_gmres_solve) */
} rtg_status;

typedef enum rtg_dtype {
    RTG_F64 = 0,               /* double data, double arithmetic */
    RTG_F32 = 1,               /* float data, float arithmetic with FP64 small solves */
    RTG_BF16 = 2               /* bfloat16 storage, FP32 arithmetic (apply, sketch; the
                                  solve's basis with RTG_FLAG_BF16_BASIS) */
} rtg_dtype;

typedef enum rtg_factor_kind {
    RTG_FACTOR_IDENTITY = 0,
    RTG_FACTOR_BANDED_TOEPLITZ = 1,  /* (M x)_i = sum_{|t|<=r} taps[r+t] x_{i+t}, zero outside */
    RTG_FACTOR_DENSE = 2             /* dense n x n matrix M, column-major (M(i,j) at i + n*j) */
} rtg_factor_kind;

typedef struct rtg_shape {
    int32_t order;                   /* 1..RTG_MAX_ORDER */
    int64_t dims[RTG_MAX_ORDER];     /* I_1..I_order, each >= 1; unused entries ignored */
} rtg_shape;

/*
 * One factor of the separable operator (Eq. 56-57; Section 1).
 * A left factor ("A factor") acts as the mode product X x_mode M: the
 * 4th-order blurring tensor of Eq. 56 is A[i,j,i',j'] = A_1[i,i'] A_2[j,j'],
 * so A *_2 X = X x_1 A_1 x_2 A_2.  A right factor ("B factor") is the
 * Einstein right product X *_1 B, i.e. (X *_1 B)[..,c'] = sum_c X[..,c] B[c,c'],
 * applied as X x_mode B^T.  For a banded right factor, B is the banded
 * Toeplitz matrix built from its taps.
 */
typedef struct rtg_factor {
    int32_t mode;                    /* 1-based mode the factor acts on */
    int32_t kind;                    /* rtg_factor_kind */
    int32_t n;                       /* must equal dims[mode-1] */
    int32_t radius;                  /* banded: r (0..RTG_MAX_RADIUS) */
    const double* taps;              /* banded: host array of 2r+1 taps */
    const double* dense;             /* dense: host array n*n, column-major */
} rtg_factor;

/* Options of rtg_gmres_solve.  A zero-initialised struct is valid. */
typedef struct rtg_opts {
    double tol;                      /* stop at the first j with rho_j <= tol (0: run m steps) */
    const double* mu_grid;           /* host array of n_mu GCV candidates (lambda < 0) */
    int32_t n_mu;                    /* 1..RTG_MAX_MU when lambda < 0 */
    int32_t max_restarts;            /* restarted cycles (>= 0; rtg_gmres_solve and the batched
                                        solve): a cycle that reaches j = m without meeting tol
                                        restarts from its least-squares iterate;
                                        m * (max_restarts + 1) <= RTG_MAX_KRYLOV */
    double breakdown_tol;            /* breakdown if h_{j+1,j} <= breakdown_tol * ||S(Phi V_j)||;
                                        0 selects 1e-12 (F64) / 1e-6 (F32) */
    int32_t flags;                   /* RTG_FLAG_* */
    int32_t slot;                    /* workspace slot, 0..RTG_MAX_SLOTS-1: solves that may be
                                        in flight at the same time on different streams must use
                                        different slots (each slot owns its own basis, sketch and
                                        graph); calls on one slot are ordered by their stream */
    int32_t group_max;               /* batched solves: most problems in one lock-step group;
                                        0 or 1: every problem its own graph branch */
    int32_t queue_slots;             /* batched solves: > 0 serves each class of problems of
                                        equal structure by at most this many graph branches that
                                        take the class's problems from a device work queue
                                        (memory: one workspace per branch, not per problem);
                                        0: off.  Excludes group_max > 1 */
} rtg_opts;

#define RTG_MAX_SLOTS 64

#define RTG_FLAG_NO_GRAPH      1     /* launch kernels directly instead of a CUDA graph */
#define RTG_FLAG_TRUE_RESIDUAL 2     /* the final residual of the Block GMRES algorithm
                                        (Section 4.4, its last steps): after the assembly,
                                        R = C - Phi(X) for the returned X, then
                                        info->true_rel_resid = ||R||_F / ||C||_F and
                                        info->true_rel_resid_theta = ||R||_Theta / ||R_0||_Theta
                                        (one more apply, sketch and reduction; with an operator
                                        that takes the spatio-temporal kernel X must be 16-byte
                                        aligned) */
#define RTG_FLAG_PHASE_TIMES   4     /* time every kernel group with CUDA events into
                                        info->phase_ms (implies RTG_FLAG_NO_GRAPH); see below */
#define RTG_FLAG_BF16_BASIS    8     /* precision form (dtype RTG_F32 only): the basis V_i and
                                        W = Phi(V_j) are stored in BF16, half the bytes of the
                                        basis update; every sum is accumulated in FP32, the
                                        sketches S(W) and Q in FP32, the Gram-Schmidt
                                        coefficients, Givens and Tikhonov in FP64.  Needs the
                                        spatio-temporal operator form (banded modes 1-2 of
                                        radius <= 9, a mode-3 mix of 1 or 3 channels, a mode-4
                                        band of radius <= 2), dims[0] % 8 == 0, mode 1
                                        sketched, and C / X0 16-byte aligned. */

/* Kernel groups of one solve, the index of rtg_info.phase_ms / phase_launches.
 *   SETUP     workspace reset and the sketch signs / Theta operand images (Section 2, Theta_k)
 *   INIT      R_0 = C - Phi(X_0), S(R_0), beta, V_1 and its sketch (Algorithm 2 start)
 *   APPLY     W = Phi(V_j)                                  (Eq. 57 operator)
 *   SKETCH    S(W) and, where fused, the sketched dots and Gram-Schmidt finish
 *   GS        sketched dots and Gram-Schmidt finish when not fused into SKETCH
 *   UPDATE    V_{j+1} = (W - sum_i h_ij V_i) / h_{j+1,j}, sketched basis column
 *   TIKHONOV  projected Tikhonov / GCV (Eq. 13)
 *   ASSEMBLE  X = X_0 + sum_j y_j V_j and the info record
 * Steps after the stop are not counted. */
enum {
    RTG_PHASE_SETUP = 0, RTG_PHASE_INIT, RTG_PHASE_APPLY, RTG_PHASE_SKETCH, RTG_PHASE_GS,
    RTG_PHASE_UPDATE, RTG_PHASE_TIKHONOV, RTG_PHASE_ASSEMBLE, RTG_PHASE_COUNT
};

typedef struct rtg_info {
    int32_t iters;                   /* Arnoldi steps taken, all cycles */
    int32_t restarts;
    int32_t breakdown;               /* 1: h_{j+1,j} fell below the breakdown level (exact in K_j) */
    int32_t converged;               /* 1: rho <= tol (or breakdown) */
    double beta;                     /* ||R_0||_Theta of the first cycle */
    double mu;                       /* regularisation used (GCV choice, fixed lambda, or 0) */
    double rho_final;                /* last rho_j */
    double* rho_hist;                /* optional caller host array of length >= m*(max_restarts+1) */
    double* gcv;                     /* optional caller host array of length n_mu (GCV values) */
    double true_rel_resid;           /* ||C - Phi(X)||_F / ||C||_F with RTG_FLAG_TRUE_RESIDUAL, else -1 */
    double elapsed_ms;               /* device time of the solve (CUDA events) */
    int32_t device_status;           /* rtg_status seen on the device (NONFINITE, ...) */
    int32_t launches;                /* kernels this library launched for the solve */
    int32_t tile_config;             /* basis-update tile geometry the autotuner chose for this
                                        plan (0: the default; see the solve's description) */
    /* With RTG_FLAG_PHASE_TIMES: device time (ms) and kernel launches of each
     * RTG_PHASE_* group, summed over the solve.  Each group is bracketed by
     * CUDA events on the solve's stream, and the GPU is held at a gate until
     * the host has queued the whole group, so no host launch latency falls
     * between the events.  Zero without the flag. */
    double phase_ms[RTG_PHASE_COUNT];
    int32_t phase_launches[RTG_PHASE_COUNT];
    double true_rel_resid_theta;     /* ||C - Phi(X)||_Theta / ||R_0||_Theta with RTG_FLAG_TRUE_RESIDUAL,
                                        else -1 */
} rtg_info;

typedef struct rtg_context* rtg_handle;
typedef struct rtg_krylov_state* rtg_krylov;
typedef struct CUstream_st* rtg_stream;   /* same type as cudaStream_t */

/* Create a handle on CUDA device `device`.  The handle owns all workspace
 * (basis, sketches, Hessenberg data, graphs) and grows it on demand. */
rtg_status rtg_create(rtg_handle* handle, int device);
/* Free the handle and everything it owns.  NULL is accepted. */
rtg_status rtg_destroy(rtg_handle handle);
/* Thread-local description of the last error (never NULL). */
const char* rtg_last_error(void);
const char* rtg_status_string(rtg_status status);
int32_t rtg_version(void);

/*
 * Y = Phi(X): the Einstein-product operator of Section 1 with separable
 * factors (Eq. 56-57, zero boundary conditions).  Modes without a factor
 * are untouched.  Several factors on one mode compose (right factors after
 * left ones).  X and Y: device arrays of prod(dims) elements of `dtype`;
 * Y must not overlap X.  F64 / F32: any factors.  BF16: X and Y in BF16,
 * FP32 arithmetic, one rounding of each output; needs the spatio-temporal
 * form (banded modes 1-2 of radius <= 9, a mode-3 mix of 1 or 3 channels,
 * a mode-4 band of radius <= 2), dims[0] % 8 == 0 and X 16-byte aligned.
 * The video operator (order 4 with a mode-4 band) also runs as one pass
 * in F32, with X 16-byte aligned.
 * Errors: INVALID_ARG (shape, factor mode/size/radius, NULL, alignment),
 * UNSUPPORTED (BF16 with another operator form), CUDA.
 */
rtg_status rtg_operator_apply(rtg_handle handle,
                              const rtg_factor* A_factors, int32_t nA,
                              const rtg_factor* B_factors, int32_t nB,
                              rtg_shape shape, rtg_dtype dtype,
                              const void* X, void* Y, rtg_stream stream);

/*
 * SX = S(X) = X x_1 Theta_1 x_2 ... x_d Theta_d (Section 3, the global
 * tensor sketching operator; Section 3.1, the compressed tensor).
 * Theta_k is s_k x I_k with Rademacher entries +-1/sqrt(s_k) drawn from
 * Philox4x64-10 keyed (seed, problem_id): signs of the sketched modes in
 * increasing mode order, each Theta_k row-major, sign e = bit e%64 of
 * output word e/64 (set bit = -1), output word w from counter (w/4+1,0,0,0).
 * A mode with s_k >= I_k is not sketched (Theta_k = I, s'_k = I_k).
 * SX: device array of prod(s'_k) elements of `dtype`, column-major; for
 * dtype BF16 (X in BF16, exact in one tensor-core limb) SX is FP32, and
 * mode 1 must be sketched.  The handle keeps the signs and the chain's
 * intermediates per (shape, sketch sizes, problem_id, dtype, stream) and
 * draws the signs again whenever a call brings another seed.  The bounded
 * device-side waits of the FP32 chain never fail in normal operation; if
 * one gave up, the entries of SX that its thread block computes are NaN.
 * Errors: INVALID_ARG (s_k < 1, shape), UNSUPPORTED (BF16 with mode 1 not
 * sketched), CUDA.
 */
rtg_status rtg_sketch(rtg_handle handle, rtg_shape shape, rtg_dtype dtype,
                      const int64_t* sketch_dims, uint64_t seed, uint64_t problem_id,
                      const void* X, void* SX, rtg_stream stream);

/*
 * Raw Philox4x64-10 stream behind the sketch (see rtg_sketch): out[w] for
 * w < n_words, device array of uint64.  Exposed so the signs can be checked
 * bit for bit.
 */
rtg_status rtg_philox_words(rtg_handle handle, uint64_t seed, uint64_t problem_id,
                            int64_t n_words, uint64_t* out, rtg_stream stream);

/*
 * Caller-held sketched Arnoldi state (Section 4.3): basis V_1..V_{m+1}
 * (full space), their sketches Q = [S(V_1) .. S(V_{m+1})], the Hessenberg
 * matrix Hbar_m and the Givens QR used for rho_j.  rtg_krylov_create
 * allocates it for one operator, shape, dtype (F64/F32), Krylov dimension m
 * and sketch; the factors are copied.
 */
rtg_status rtg_krylov_create(rtg_handle handle,
                             const rtg_factor* A_factors, int32_t nA,
                             const rtg_factor* B_factors, int32_t nB,
                             rtg_shape shape, rtg_dtype dtype, int32_t m,
                             const int64_t* sketch_dims, uint64_t seed, uint64_t problem_id,
                             rtg_krylov* krylov);
rtg_status rtg_krylov_destroy(rtg_krylov krylov);

/*
 * Start the process: R_0 = C - Phi(X_0) (X0 may be NULL for X_0 = 0),
 * beta = ||R_0||_Theta, V_1 = R_0/beta, S(V_1) (first steps of the Block
 * GMRES algorithm).  C, X0: device arrays.  Asynchronous.
 */
rtg_status rtg_krylov_start(rtg_handle handle, rtg_krylov krylov,
                            const void* C, const void* X0, rtg_stream stream);

/*
 * One sketched Arnoldi step j -> j+1: W = Phi(V_j); h_ij = <V_i, W>_Theta
 * for i <= j, computed as classical Gram-Schmidt with one
 * re-orthogonalisation pass in the sketch space (equal to the paper's
 * modified Gram-Schmidt in exact arithmetic); h_{j+1,j} = ||W - sum h_ij V_i||_Theta;
 * V_{j+1} and S(V_{j+1}); Givens update of the least-squares residual
 * rho_j = ||beta e1 - Hbar_j y_j|| / beta (Eq. 11S).  After a breakdown
 * or once j = m the call is a no-op.  Asynchronous.
 */
rtg_status rtg_arnoldi_step(rtg_handle handle, rtg_krylov krylov, rtg_stream stream);

/* Host view of a Krylov state (filled by rtg_krylov_query, which synchronises the stream). */
typedef struct rtg_krylov_view {
    int32_t j;                       /* number of completed steps */
    int32_t m;
    int32_t breakdown;
    int32_t sketch_size;             /* d = prod(s'_k) */
    int64_t n;                       /* prod(dims) */
    double beta;
    double rho;                      /* last rho_j (1.0 before the first step) */
    const void* V;                   /* device: (m+1) tensors of n elements, V_i at V + i*n */
    const void* Q;                   /* device: (m+1) sketches of d elements (dtype of the state) */
} rtg_krylov_view;

/* H: optional host array of (m+1)*m doubles, column-major, receives Hbar. */
rtg_status rtg_krylov_query(rtg_handle handle, rtg_krylov krylov, rtg_krylov_view* view,
                            double* H, rtg_stream stream);

/*
 * RTG-GMRES for Phi(X) = C (the algorithm "Block GMRES via Sketched
 * Einstein Product" with the projected Tikhonov problem of Eq. 12S/13):
 *   R_0 = C - Phi(X_0), beta = ||R_0||_Theta; up to m sketched Arnoldi
 *   steps, stopping at the first j with rho_j <= opts->tol or on breakdown;
 *   then y = argmin ||beta e1 - Hbar y||^2 + mu ||y||^2 with
 *     lambda > 0: mu = lambda;  lambda == 0: mu = 0 (Eq. 11S);
 *     lambda < 0: mu = argmin GCV(mu) over opts->mu_grid (ties: larger mu);
 *   X = X_0 + sum_j y_j V_j (Eq. 10S).
 * With opts->max_restarts = R > 0, a cycle that ends at j = m with
 * rho_j > tol (no breakdown) restarts: y = argmin ||beta e1 - Hbar y||
 * (Eq. 11S), X_0 <- X_0 + sum_j y_j V_j, R_0 = C - Phi(X_0), and a new
 * sketched Arnoldi cycle, at most R times; rho_j stays relative to the
 * first cycle's ||R_0||_Theta, and the regularised solve above is taken on
 * the last cycle.  The whole sequence stays inside the solve's CUDA graph
 * (its restart kernels return at once in steps that do not restart).
 * info->rho_hist then needs m * (R + 1) entries.
 * Tiles: when a plan (one per shape, operator, sizes, options and slot) is
 * first built, a timing search picks the basis update's tile geometry
 * (slot size and depth of its shared-memory ring) on the plan's own
 * workspace; every geometry gives identical results.  The environment
 * variable RTG_NO_AUTOTUNE=1 keeps the default geometry and RTG_TILE_CONFIG=k
 * (k = 0..4) fixes geometry k; both are read when a plan is built.
 * C, X0 (may be NULL), X: device or host arrays of prod(dims) elements of
 * dtype (F64 or F32); X may alias X0.  info may be NULL.  The call
 * synchronises `stream` once at the end; it equals rtg_gmres_submit
 * followed by rtg_gmres_wait on opts->slot.
 * Errors: INVALID_ARG, UNSUPPORTED, ALLOC, CUDA; numeric trouble is
 * reported in info->device_status (RTG_ERR_NONFINITE) with RTG_OK returned.
 */
rtg_status rtg_gmres_solve(rtg_handle handle,
                           const rtg_factor* A_factors, int32_t nA,
                           const rtg_factor* B_factors, int32_t nB,
                           rtg_shape shape, rtg_dtype dtype,
                           const void* C, int32_t m, const int64_t* sketch_dims,
                           uint64_t seed, double lambda, const void* X0, void* X,
                           const rtg_opts* opts, rtg_info* info, rtg_stream stream);

/*
 * The same solve in two halves, so that one host thread can keep several
 * independent solves in flight on different streams (each on its own
 * workspace slot, opts->slot).  rtg_gmres_submit validates the arguments
 * and queues the whole solve on `stream` (staging copies, the solve's CUDA
 * graph, the copy-back of X when X is a host array) and returns without
 * waiting; host arrays C, X0 and X must stay valid until the matching
 * rtg_gmres_wait.  rtg_gmres_wait(slot) synchronises the stream of the last
 * solve submitted on `slot` and fills `info` (may be NULL).  A slot holds
 * one submitted solve at a time: submitting on a slot that was not waited
 * for returns RTG_ERR_INVALID_ARG.  Phase timing (RTG_FLAG_PHASE_TIMES)
 * uses one timer per handle, so at most one such solve may be pending.
 */
rtg_status rtg_gmres_submit(rtg_handle handle,
                            const rtg_factor* A_factors, int32_t nA,
                            const rtg_factor* B_factors, int32_t nB,
                            rtg_shape shape, rtg_dtype dtype,
                            const void* C, int32_t m, const int64_t* sketch_dims,
                            uint64_t seed, double lambda, const void* X0, void* X,
                            const rtg_opts* opts, rtg_stream stream);
rtg_status rtg_gmres_wait(rtg_handle handle, int32_t slot, rtg_info* info);

/*
 * Sketched Golub-Kahan (Algorithm 4, "Block Golub-Kahan via Sketched
 * Einstein Product") for the same problem and with the same arguments as
 * rtg_gmres_solve: R_0 = C - Phi(X_0), beta_1 = ||R_0||_Theta,
 * U_1 = R_0 / beta_1, alpha_1 V_1 = Phi^T(U_1); for k = 1, 2, ...:
 * beta_{k+1} U_{k+1} = Phi(V_k) - alpha_k U_k,
 * alpha_{k+1} V_{k+1} = Phi^T(U_{k+1}) - beta_{k+1} V_k, with Theta-norms
 * (only norms are sketched; short recurrences, no re-orthogonalisation).
 * Phi^T is the adjoint of Phi (every mode matrix transposed).  The lower
 * bidiagonal Btilde_k takes the place of Hbar_k: rho_k, the stop rule, the
 * projected Tikhonov / GCV solve (Eq. 13) and X = X_0 + sum y_k V_k are as
 * for RTG-GMRES.  Stops also when alpha_{k+1} falls to the breakdown level.
 * Memory: m+1 tensors V plus two U.  RTG_FLAG_BF16_BASIS and restarts are
 * not available (UNSUPPORTED).
 * Errors: as rtg_gmres_solve.
 */
rtg_status rtg_gk_solve(rtg_handle handle,
                        const rtg_factor* A_factors, int32_t nA,
                        const rtg_factor* B_factors, int32_t nB,
                        rtg_shape shape, rtg_dtype dtype,
                        const void* C, int32_t m, const int64_t* sketch_dims,
                        uint64_t seed, double lambda, const void* X0, void* X,
                        const rtg_opts* opts, rtg_info* info, rtg_stream stream);

/*
 * Learned warm start (no paper counterpart: the form this library adds).
 * A convolutional encoder-decoder with base width c (four levels: c, 2c,
 * 4c, 4c channels; 3x3 convolutions, stride-2 down-sampling, nearest x2
 * up-sampling with additive skips) maps an observation C to
 * X_0 = C + net(C) and log(lambda) = w . mean_pixels(bottleneck) + b.
 * Images are I1 x I2 x 3 in the solver's layout (mode 1 fastest), I1 and
 * I2 multiples of 8; a batch is n_img such images back to back.  BF16
 * tensor-core products with FP32 accumulation; FP32 master parameters.
 * Flat parameter order: per layer e1, e2, e3, e4, d3, d2, d1, out the
 * weights (c_out, 3, 3, c_in) then the biases, then the head's 4c weights
 * and its bias (rtg_ws_num_params entries).
 */
typedef struct rtg_warmstart* rtg_ws;
/* params: host array of the initial parameters (rtg_ws_num_params of a
 * network of this base; the caller draws them). */
rtg_status rtg_ws_create(int32_t device, int32_t base, const float* params, rtg_ws* ws);
rtg_status rtg_ws_destroy(rtg_ws ws);
int64_t rtg_ws_num_params(rtg_ws ws);
/* Copies the parameters and / or the gradients of the last training step
 * to host arrays (either may be NULL). */
rtg_status rtg_ws_get(rtg_ws ws, float* params, float* grads);
/* X0 (device, same layout as C) and loglam (device, n_img floats). */
rtg_status rtg_ws_predict(rtg_ws ws, int32_t n_img, int32_t I1, int32_t I2, const float* C, float* X0,
                          float* loglam, rtg_stream stream);
/* One training step on a batch: forward, loss
 *   mean over images of ||X_0 - X*||^2 / ||X*||^2 + (log lambda - log mu*)^2,
 * backward, and (lr > 0) one Adam step (beta 0.9 / 0.999, eps 1e-8).
 * Xstar, logmu: device targets (solver solutions and log regularisation);
 * X0_scratch: device array like C; loss_out: host (may be NULL; when given
 * the call synchronises the stream). */
rtg_status rtg_ws_train_step(rtg_ws ws, int32_t n_img, int32_t I1, int32_t I2, const float* C,
                             const float* Xstar, const float* logmu, float lr, float* X0_scratch,
                             double* loss_out, rtg_stream stream);

/* Decision record of rtg_ws_solve. */
typedef struct rtg_ws_result {
    int32_t fell_back;               /* 1: ||S(C - Phi(X_0))|| >= ||S(C)||: solved from X_0 = 0 with GCV */
    int32_t pad;
    double lambda;                   /* exp(predicted log lambda), or -1 when GCV chose mu (fallback) */
    double tol;                      /* stop level handed to the solve: tol ||S(C)|| / ||S(R_0)|| */
    double sketch_norm_C;            /* ||S(C)|| */
    double sketch_norm_R0;           /* ||S(C - Phi(X_0))|| of the prediction */
} rtg_ws_result;

/*
 * Warm-started RTG-GMRES (no paper counterpart: the solve path of the
 * learned warm start).  On `stream`, with no host round trip until the
 * solve has finished:
 *   X_0 = C + net(C) and log lambda (rtg_ws_predict, into X);
 *   R_0 = C - Phi(X_0); s_R = ||S(R_0)||, s_C = ||S(C)|| (the solve's sketch);
 *   if s_R >= s_C (or non-finite): X_0 = 0 and mu by GCV over opts->mu_grid
 *   (the plain cold solve, the fallback); else mu = exp(log lambda) and the
 *   stop level becomes opts->tol * s_C / s_R, so that both paths stop at
 *   ||S(C - Phi X)|| <= opts->tol ||S(C)|| (the rho of the solve is relative
 *   to its own ||S(R_0)||);
 *   then rtg_gmres_solve with X_0 as the initial guess (opts->max_restarts
 *   and RTG_FLAG_TRUE_RESIDUAL apply; a warm start that already meets the
 *   stop level returns X_0 after no step).
 * C, X: device FP32 arrays of an I1 x I2 x 3 image (mode 1 fastest), I1 and
 * I2 multiples of 8; X receives the solution.  opts->mu_grid is required.
 * The call synchronises `stream` once at the end; info as for
 * rtg_gmres_solve (info->mu: the mu used); result (may be NULL): the decision.
 * Errors: as rtg_gmres_solve and rtg_ws_predict.
 */
rtg_status rtg_ws_solve(rtg_ws ws, rtg_handle handle,
                        const rtg_factor* A_factors, int32_t nA,
                        const rtg_factor* B_factors, int32_t nB,
                        rtg_shape shape, const float* C, int32_t m, const int64_t* sketch_dims,
                        uint64_t seed, float* X, const rtg_opts* opts, rtg_info* info,
                        rtg_ws_result* result, rtg_stream stream);

/*
 * One 3x3 convolution layer of the warm-start network with the same
 * kernels (zero padding 1, stride 1 or 2, channels-last FP32 activations
 * x (N, H, W, cin), weights w (cout, 3, 3, cin) FP32 rounded to BF16 for
 * the tensor-core product, FP32 accumulation).  Forward: y = conv(x) + b
 * (y: N, H/stride, W/stride, cout).  Backward (dy given): dx, dw, db (each
 * may be NULL); dy is rounded to BF16 for the products, db sums dy in FP32.
 * All pointers are device arrays; workspace is allocated per call and the
 * stream is synchronised before returning.
 */
rtg_status rtg_nn_conv3x3(int32_t device, int32_t N, int32_t H, int32_t W, int32_t cin, int32_t cout,
                          int32_t stride, const float* x, const float* w, const float* b, float* y,
                          const float* dy, float* dx, float* dw, float* db, rtg_stream stream);

/* One problem of a batched solve: the arguments of rtg_gmres_solve. */
typedef struct rtg_problem {
    const rtg_factor* A_factors;
    int32_t nA;
    const rtg_factor* B_factors;
    int32_t nB;
    rtg_shape shape;
    const void* C;                   /* device, prod(dims) elements of the batch dtype */
    const void* X0;                  /* device or NULL */
    void* X;                         /* device; may alias X0 */
    int32_t m;
    int32_t pad;
    int64_t sketch_dims[RTG_MAX_ORDER];
    uint64_t seed;
    double lam;                      /* lambda: > 0 fixed, 0 least squares, < 0 GCV over opts->mu_grid */
    double tol;                      /* stop level of rho_j */
} rtg_problem;

#define RTG_MAX_BATCH 1024          /* problems of a batch, or graph branches of a queued batch */
#define RTG_MAX_QUEUE 65536         /* problems of a batch with opts->queue_slots > 0 */

/*
 * Batched form: nprob independent RTG-GMRES solves, of any mix of shapes,
 * operators, Krylov dimensions and sketch sizes.  By default every problem
 * is its own group.  With opts->group_max = g > 1, problems of the same
 * structure (shape, factor list and values, m, sketch sizes, kind of
 * regularisation -- fixed, least squares or GCV -- and whether X0 is given)
 * form lock-step groups of up to g problems: every kernel launch serves the
 * whole group, each problem keeps its own stop decision (a stopped
 * problem's blocks return at once), and the group's device-side loop runs
 * while any of its problems does.  Lock step pays when single problems are
 * too small to fill the GPU and converge alike; separate groups pay when
 * convergence varies.  Each result equals, bit for bit, the same problem
 * solved alone.  The groups are independent branches of one CUDA graph, built on
 * the first call for a given list of problem structures and replayed
 * afterwards; descriptors go up in one strided copy per group and the info
 * records come back the same way.
 * Work queue (opts->queue_slots = K > 0): the problems of each class of equal
 * structure (the lock-step key above) go into a device queue, and the class
 * gets min(K, its problems) graph branches, each with one workspace.  A
 * branch takes the next problem with an atomic increment of the class's
 * counter, solves it, returns its info record and takes the next, until the
 * queue is empty (a device-side WHILE loop around the solve's own), so a
 * branch whose problem stops early goes on to another, and the device memory
 * grows with the branches, not the problems: up to RTG_MAX_QUEUE problems,
 * at most RTG_MAX_BATCH branches in all.  When the classes together have
 * more than K branches (many classes of few problems), the branches run as
 * K chains (a branch starts when the one before it in its chain has ended):
 * largest estimated work first (tensor entries x m x problems per branch),
 * each to the chain with the least estimated work so far.  Descriptors go
 * up in one copy and the info records come back in one.  Which branch
 * solves which problem depends on timing; the result does not (each equals
 * the same problem solved alone, bit for bit).  RTG_FLAG_NO_GRAPH runs each
 * class's problems in order on one workspace; RTG_FLAG_PHASE_TIMES is
 * UNSUPPORTED here, and group_max > 1 with queue_slots > 0 is INVALID_ARG.
 * opts (may be NULL) is shared: GCV grid,
 * breakdown level, RTG_FLAG_BF16_BASIS, and RTG_FLAG_NO_GRAPH /
 * RTG_FLAG_PHASE_TIMES (direct launches, one group after another; with
 * PHASE_TIMES each problem's phase_ms / phase_launches are those of its
 * whole group); slot does not apply.  infos: NULL or nprob records
 * (elapsed_ms is the whole batch's).  The call synchronises `stream`.
 * Errors: as rtg_gmres_solve, per problem (the message names it); host
 * pointers are INVALID_ARG.
 */
rtg_status rtg_gmres_solve_batched(rtg_handle handle, int32_t nprob, const rtg_problem* probs,
                                   rtg_dtype dtype, const rtg_opts* opts, rtg_info* infos,
                                   rtg_stream stream);

/*
 * rtg_sketch_noalloc -- the paper has no counterpart; this is a service of
 * the library.  Same result as rtg_sketch (same kernels, same Philox
 * signs) for callers that cannot call cudaMalloc: code that runs next to a
 * framework which has already reserved the device memory for its own pool,
 * or latency-critical code that cannot afford the implicit device
 * synchronisation of cudaMalloc/cudaFree.  It takes no handle and
 * allocates nothing: its scratch (packed signs and the contraction
 * intermediates) lives in one 16 MiB array of the library's static device
 * memory, which every GPU that loads the library holds until the process
 * exits.  Sizes whose scratch (signs, Theta operand images and two partial-sum
 * intermediates) exceeds 16 MiB are rejected with RTG_ERR_INVALID_ARG and a message in rtg_last_error(),
 * and so are tensors of more than 2^40 elements and an SX that overlaps X (as for rtg_sketch).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array and it keeps
 * the last call's contents (each call writes every scratch byte it reads,
 * so nothing needs clearing); calls that overlap on the GPU (different
 * streams, or different host threads) race on it.  X, SX: device arrays as
 * for rtg_sketch; the call is asynchronous on `stream`, and a bounded
 * device-side wait that gave up leaves NaN in SX as for rtg_sketch.
 */
rtg_status rtg_sketch_noalloc(rtg_shape shape, rtg_dtype dtype, const int64_t* sketch_dims,
                              uint64_t seed, uint64_t problem_id, const void* X, void* SX,
                              rtg_stream stream);

/*
 * Diagnostics (no paper counterpart).  Every device-side wait of the
 * library on a flag that another agent sets (the host-opened gates of phase
 * timing) is bounded by globaltimer and, on expiry, records RTG_ERR_TIMEOUT
 * where the host reads it and returns, leaving the context usable.  This
 * call exercises that path on `device`: a wait of limit_ms (1..10000) on a
 * flag in mapped host memory that nothing sets, then a wait whose flag is
 * already met on the same stream.  *status_out receives the status the first
 * wait recorded (RTG_ERR_TIMEOUT expected); the call returns RTG_ERR_CUDA if
 * the stream did not come back or the second wait reported a timeout.
 * Synchronous; allocates a few bytes of pinned host memory.
 */
rtg_status rtg_selftest_bounded_wait(int32_t device, int32_t limit_ms, int32_t* status_out);

#ifdef __cplusplus
}
#endif
#endif /* RTG_H */
