"""Python binding of librtg: argument marshalling only.

Every computation runs in the CUDA kernels behind the C ABI; this module
converts Python objects into the ABI's structs and pointers.  PyTorch
provides device memory and streams.  Tensors are column-major (mode 1
fastest, the ivec order of Section 4.1 of the paper): use
:func:`empty` / :func:`to_device` to make them.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import _lib as L

__all__ = ["Handle", "Factor", "banded", "dense", "identity", "empty", "to_device",
           "colmajor_strides", "SolveResult", "Krylov"]


def _torch():
    import torch
    return torch


def colmajor_strides(dims: Sequence[int]) -> Tuple[int, ...]:
    s, out = 1, []
    for d in dims:
        out.append(s)
        s *= int(d)
    return tuple(out)


def empty(dims: Sequence[int], dtype=None, device="cuda"):
    """Uninitialised column-major tensor of shape ``dims`` on ``device``."""
    torch = _torch()
    dtype = dtype or torch.float32
    rev = tuple(int(d) for d in reversed(dims))
    return torch.empty(rev, dtype=dtype, device=device).permute(*reversed(range(len(dims))))


def to_device(a: np.ndarray, dtype=None, device="cuda"):
    """Copy a numpy array (any order) into a new column-major tensor on ``device``."""
    torch = _torch()
    t = torch.from_numpy(np.asfortranarray(a))
    out = empty(a.shape, dtype or t.dtype, device)
    out.copy_(t)
    return out


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float64:
        return L.F64
    if t.dtype == torch.float32:
        return L.F32
    if t.dtype == torch.bfloat16:
        return L.BF16
    raise TypeError(f"unsupported dtype {t.dtype}")


def _check_tensor(t, dims: Sequence[int], name: str) -> None:
    if tuple(t.shape) != tuple(dims):
        raise ValueError(f"{name}: shape {tuple(t.shape)} != {tuple(dims)}")
    if t.numel() > 1 and tuple(t.stride()) != colmajor_strides(dims):
        raise ValueError(f"{name}: not column-major dense (strides {t.stride()})")


def _shape(dims: Sequence[int]) -> L.Shape:
    if not 1 <= len(dims) <= L.MAX_ORDER:
        raise ValueError("order must be 1..4")
    s = L.Shape()
    s.order = len(dims)
    for k, d in enumerate(dims):
        s.dims[k] = int(d)
    return s


@dataclasses.dataclass
class Factor:
    """One factor of the separable operator: ``mode`` is 1-based."""
    mode: int
    kind: int
    n: int
    taps: Optional[np.ndarray] = None
    matrix: Optional[np.ndarray] = None

    @property
    def radius(self) -> int:
        return 0 if self.taps is None else (len(self.taps) - 1) // 2


def banded(mode: int, n: int, taps) -> Factor:
    taps = np.ascontiguousarray(taps, dtype=np.float64)
    assert len(taps) % 2 == 1
    return Factor(mode, L.FACTOR_BANDED_TOEPLITZ, n, taps=taps)


def dense(mode: int, M) -> Factor:
    M = np.asarray(M, dtype=np.float64)
    return Factor(mode, L.FACTOR_DENSE, M.shape[0], matrix=np.asfortranarray(M))


def identity(mode: int, n: int) -> Factor:
    return Factor(mode, L.FACTOR_IDENTITY, n)


def _factor_array(fs: Sequence[Factor]):
    arr = (L.Factor * max(len(fs), 1))()
    keep = []
    for i, f in enumerate(fs):
        arr[i].mode, arr[i].kind, arr[i].n, arr[i].radius = f.mode, f.kind, f.n, f.radius
        if f.taps is not None:
            arr[i].taps = f.taps.ctypes.data_as(C.POINTER(C.c_double))
            keep.append(f.taps)
        if f.matrix is not None:
            m = np.ascontiguousarray(f.matrix.ravel(order="F"))
            keep.append(m)
            arr[i].dense = m.ctypes.data_as(C.POINTER(C.c_double))
    return (arr if fs else None), len(fs), keep


def _stream(stream) -> Optional[int]:
    if stream is None:
        return _torch().cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


@dataclasses.dataclass
class SolveResult:
    iters: int
    restarts: int
    breakdown: bool
    converged: bool
    beta: float
    mu: float
    rho_final: float
    rho: np.ndarray
    gcv: Optional[np.ndarray]
    elapsed_ms: float
    device_status: int
    launches: int
    phase_ms: Optional[dict] = None        # group -> device ms (phase_times=True)
    phase_launches: Optional[dict] = None  # group -> kernel launches (phase_times=True)
    tile_config: int = 0                   # basis-update tile geometry chosen by the autotuner
    true_rel_resid: float = -1.0           # ||C - Phi(X)||_F / ||C||_F (true_residual=True)
    true_rel_resid_theta: float = -1.0     # ||C - Phi(X)||_Theta / ||R_0||_Theta (true_residual=True)


class Handle:
    """A librtg handle bound to one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = L.load()
        h = C.c_void_p()
        L.check(self.lib.rtg_create(C.byref(h), int(device)))
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.rtg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- K0
    def philox_words(self, seed: int, problem_id: int, n_words: int, stream=None):
        """Raw Philox4x64-10 stream behind the sketch signs (uint64 as int64 tensor)."""
        torch = _torch()
        out = torch.empty(n_words, dtype=torch.int64, device=f"cuda:{self.device}")
        L.check(self.lib.rtg_philox_words(self._h, C.c_uint64(seed), C.c_uint64(problem_id),
                                          n_words, out.data_ptr(), _stream(stream)))
        return out

    # ---------------------------------------------------------------- K1
    def operator_apply(self, X, A_factors: Sequence[Factor] = (), B_factors: Sequence[Factor] = (),
                       Y=None, stream=None):
        """Y = Phi(X) for the separable Einstein-product operator."""
        dims = tuple(X.shape)
        _check_tensor(X, dims, "X")
        if Y is None:
            Y = empty(dims, X.dtype, X.device)
        _check_tensor(Y, dims, "Y")
        a, na, ka = _factor_array(A_factors)
        b, nb, kb = _factor_array(B_factors)
        L.check(self.lib.rtg_operator_apply(self._h, a, na, b, nb, _shape(dims), _dtype_code(X),
                                            X.data_ptr(), Y.data_ptr(), _stream(stream)))
        return Y

    # ---------------------------------------------------------------- K3
    def sketch(self, X, sketch_dims: Sequence[int], seed: int, problem_id: int = 0, SX=None,
               stream=None):
        """SX = S(X) with mode-wise Rademacher sketches (modes with s_k >= I_k untouched)."""
        dims = tuple(X.shape)
        _check_tensor(X, dims, "X")
        sd = tuple(int(min(s, d)) for s, d in zip(sketch_dims, dims))
        if SX is None:   # a BF16 input gives an FP32 sketch
            SX = empty(sd, _torch().float32 if X.dtype == _torch().bfloat16 else X.dtype, X.device)
        _check_tensor(SX, sd, "SX")
        sk = (C.c_int64 * len(dims))(*[int(s) for s in sketch_dims])
        L.check(self.lib.rtg_sketch(self._h, _shape(dims), _dtype_code(X), sk, C.c_uint64(seed),
                                    C.c_uint64(problem_id), X.data_ptr(), SX.data_ptr(),
                                    _stream(stream)))
        return SX

    # ---------------------------------------------------------------- solve
    def gmres_solve(self, C_obs, m: int, sketch_dims: Sequence[int], seed: int, lam: float,
                    A_factors: Sequence[Factor] = (), B_factors: Sequence[Factor] = (),
                    X0=None, X=None, tol: float = 0.0, mu_grid=None, max_restarts: int = 0,
                    breakdown_tol: float = 0.0, use_graph: bool = True, phase_times: bool = False,
                    slot: int = 0, bf16_basis: bool = False, true_residual: bool = False, stream=None):
        """RTG-GMRES; C_obs, X0, X may be device tensors or host numpy arrays (Fortran order).

        phase_times=True launches directly and times each kernel group with
        CUDA events (result.phase_ms / result.phase_launches).  bf16_basis=True
        stores the Krylov basis in BF16 (the precision form).  Returns (X, SolveResult)."""
        pend = self.gmres_submit(C_obs, m, sketch_dims, seed, lam, A_factors, B_factors, X0=X0, X=X,
                                 tol=tol, mu_grid=mu_grid, max_restarts=max_restarts,
                                 breakdown_tol=breakdown_tol, use_graph=use_graph,
                                 phase_times=phase_times, slot=slot, bf16_basis=bf16_basis,
                                 true_residual=true_residual, stream=stream)
        return self.gmres_wait(pend)

    def gk_solve(self, C_obs, m: int, sketch_dims: Sequence[int], seed: int, lam: float,
                 A_factors: Sequence[Factor] = (), B_factors: Sequence[Factor] = (),
                 X0=None, X=None, tol: float = 0.0, mu_grid=None, breakdown_tol: float = 0.0,
                 use_graph: bool = True, phase_times: bool = False, slot: int = 0,
                 true_residual: bool = False, stream=None):
        """Sketched Golub-Kahan (rtg_gk_solve): same problem and arguments as
        gmres_solve (device tensors).  Returns (X, SolveResult)."""
        dims = tuple(C_obs.shape)
        _check_tensor(C_obs, dims, "C")
        if X is None:
            X = empty(dims, C_obs.dtype, C_obs.device)
        a, na, ka = _factor_array(A_factors)
        b, nb, kb = _factor_array(B_factors)
        sk = (C.c_int64 * len(dims))(*[int(s) for s in sketch_dims])
        opts = L.Opts()
        opts.tol = float(tol)
        grid = None
        if mu_grid is not None:
            grid = np.ascontiguousarray(mu_grid, dtype=np.float64)
            opts.mu_grid = grid.ctypes.data_as(C.POINTER(C.c_double))
            opts.n_mu = len(grid)
        opts.breakdown_tol = float(breakdown_tol)
        opts.flags = ((0 if use_graph else L.FLAG_NO_GRAPH) | (L.FLAG_PHASE_TIMES if phase_times else 0)
                      | (L.FLAG_TRUE_RESIDUAL if true_residual else 0))
        opts.slot = int(slot)
        info = L.Info()
        rho = np.zeros(m + 1)
        info.rho_hist = rho.ctypes.data_as(C.POINTER(C.c_double))
        gcv = np.zeros(L.MAX_MU)
        info.gcv = gcv.ctypes.data_as(C.POINTER(C.c_double))
        L.check(self.lib.rtg_gk_solve(self._h, a, na, b, nb, _shape(dims), _dtype_code(C_obs), _ptr(C_obs),
                                      int(m), sk, C.c_uint64(seed), float(lam), _ptr(X0), _ptr(X),
                                      C.byref(opts), C.byref(info), _stream(stream)))
        res = _solve_result(info, rho, gcv, grid, lam)
        if phase_times:
            res.phase_ms = {k: info.phase_ms[i] for i, k in enumerate(L.PHASES)}
            res.phase_launches = {k: info.phase_launches[i] for i, k in enumerate(L.PHASES)}
        return X, res

    def gmres_submit(self, C_obs, m: int, sketch_dims: Sequence[int], seed: int, lam: float,
                     A_factors: Sequence[Factor] = (), B_factors: Sequence[Factor] = (),
                     X0=None, X=None, tol: float = 0.0, mu_grid=None, max_restarts: int = 0,
                     breakdown_tol: float = 0.0, use_graph: bool = True, phase_times: bool = False,
                     slot: int = 0, bf16_basis: bool = False, true_residual: bool = False,
                     stream=None) -> "PendingSolve":
        """Queue a solve on `stream` without waiting (rtg_gmres_submit).  Solves
        in flight at once on different streams need different workspace slots;
        gmres_wait(pending) returns (X, SolveResult)."""
        dims = tuple(C_obs.shape)
        host = isinstance(C_obs, np.ndarray)
        if host:
            if C_obs.dtype not in (np.float32, np.float64) or not C_obs.flags.f_contiguous:
                raise ValueError("host C must be a Fortran-ordered float32/float64 array")
            dt = L.F64 if C_obs.dtype == np.float64 else L.F32
            if X is None:
                X = np.empty(dims, dtype=C_obs.dtype, order="F")
        else:
            _check_tensor(C_obs, dims, "C")
            dt = _dtype_code(C_obs)
            if X is None:
                X = empty(dims, C_obs.dtype, C_obs.device)
        a, na, ka = _factor_array(A_factors)
        b, nb, kb = _factor_array(B_factors)
        sk = (C.c_int64 * len(dims))(*[int(s) for s in sketch_dims])
        opts = L.Opts()
        opts.tol = float(tol)
        grid = None
        if mu_grid is not None:
            grid = np.ascontiguousarray(mu_grid, dtype=np.float64)
            opts.mu_grid = grid.ctypes.data_as(C.POINTER(C.c_double))
            opts.n_mu = len(grid)
        opts.max_restarts = int(max_restarts)
        opts.breakdown_tol = float(breakdown_tol)
        opts.flags = ((0 if use_graph else L.FLAG_NO_GRAPH) | (L.FLAG_PHASE_TIMES if phase_times else 0)
                      | (L.FLAG_BF16_BASIS if bf16_basis else 0)
                      | (L.FLAG_TRUE_RESIDUAL if true_residual else 0))
        opts.slot = int(slot)
        L.check(self.lib.rtg_gmres_submit(self._h, a, na, b, nb, _shape(dims), dt, _ptr(C_obs), int(m),
                                          sk, C.c_uint64(seed), float(lam), _ptr(X0), _ptr(X),
                                          C.byref(opts), _stream(stream)))
        # the host arrays (C, X0, X) and factor arrays stay referenced until the wait
        return PendingSolve(int(slot), X, m, max_restarts, grid, lam, phase_times,
                            (C_obs, X0, a, b, ka, kb, sk))

    def gmres_solve_batched(self, problems: Sequence[dict], mu_grid=None, breakdown_tol: float = 0.0,
                            bf16_basis: bool = False, use_graph: bool = True, phase_times: bool = False,
                            group_max: int = 0, true_residual: bool = False, max_restarts: int = 0,
                            queue_slots: int = 0, stream=None):
        """Batched form (rtg_gmres_solve_batched): every problem is a dict with
        C (device tensor), m, sketch_dims, seed, lam, and optionally A, B
        (factor lists), tol, X0, X.  All problems share C's dtype; each may
        have its own shape; problems of equal structure run in lock step.
        use_graph=False / phase_times=True launch directly, one group after
        another (phase_ms: the problem's whole group).  group_max > 1 runs
        problems of equal structure in lock-step groups of up to that many
        (default: one graph branch per problem).  queue_slots = K > 0 serves
        each class of equal structure by at most K graph branches that take
        its problems from a device work queue (one workspace per branch);
        more than K branches in all (many classes) run as K chains.
        Returns ([X], [SolveResult])."""
        if not problems:
            raise ValueError("no problems")
        arr = (L.Problem * len(problems))()
        keep = []
        Xs = []
        dt = _dtype_code(problems[0]["C"])
        for i, q in enumerate(problems):
            Cq = q["C"]
            dims = tuple(Cq.shape)
            _check_tensor(Cq, dims, "C")
            if _dtype_code(Cq) != dt:
                raise ValueError("all problems of a batch share one dtype")
            X = q.get("X")
            if X is None:
                X = empty(dims, Cq.dtype, Cq.device)
            _check_tensor(X, dims, "X")
            a, na, ka = _factor_array(q.get("A", ()))
            b, nb, kb = _factor_array(q.get("B", ()))
            keep.append((a, b, ka, kb, q.get("X0")))
            pr = arr[i]
            pr.A_factors, pr.nA, pr.B_factors, pr.nB = a, na, b, nb
            pr.shape = _shape(dims)
            pr.C, pr.X0, pr.X = _ptr(Cq), _ptr(q.get("X0")), _ptr(X)
            pr.m = int(q["m"])
            for k, sdim in enumerate(q["sketch_dims"]):
                pr.sketch_dims[k] = int(sdim)
            pr.seed = int(q["seed"])
            pr.lam = float(q["lam"])
            pr.tol = float(q.get("tol", 0.0))
            Xs.append(X)
        opts = L.Opts()
        grid = None
        if mu_grid is not None:
            grid = np.ascontiguousarray(mu_grid, dtype=np.float64)
            opts.mu_grid = grid.ctypes.data_as(C.POINTER(C.c_double))
            opts.n_mu = len(grid)
        opts.breakdown_tol = float(breakdown_tol)
        opts.group_max = int(group_max)
        opts.queue_slots = int(queue_slots)
        opts.max_restarts = int(max_restarts)
        opts.flags = ((L.FLAG_BF16_BASIS if bf16_basis else 0) | (0 if use_graph else L.FLAG_NO_GRAPH) |
                      (L.FLAG_PHASE_TIMES if phase_times else 0) | (L.FLAG_TRUE_RESIDUAL if true_residual else 0))
        infos = (L.Info * len(problems))()
        bufs = []
        for i, q in enumerate(problems):
            rho = np.zeros(int(q["m"]) * (int(max_restarts) + 1) + 1)
            gcv = np.zeros(L.MAX_MU)
            infos[i].rho_hist = rho.ctypes.data_as(C.POINTER(C.c_double))
            infos[i].gcv = gcv.ctypes.data_as(C.POINTER(C.c_double))
            bufs.append((rho, gcv))
        L.check(self.lib.rtg_gmres_solve_batched(self._h, len(problems), arr, dt, C.byref(opts), infos,
                                                 _stream(stream)))
        res = [_solve_result(infos[i], bufs[i][0], bufs[i][1], grid, float(q["lam"]))
               for i, q in enumerate(problems)]
        if phase_times:
            for i, r in enumerate(res):
                r.phase_ms = {k: infos[i].phase_ms[j] for j, k in enumerate(L.PHASES)}
                r.phase_launches = {k: infos[i].phase_launches[j] for j, k in enumerate(L.PHASES)}
        return Xs, res

    def gmres_wait(self, pend: "PendingSolve"):
        """Wait for a submitted solve (rtg_gmres_wait); returns (X, SolveResult)."""
        info = L.Info()
        rho = np.zeros(pend.m * (pend.max_restarts + 1) + 1)
        info.rho_hist = rho.ctypes.data_as(C.POINTER(C.c_double))
        gcv = np.zeros(L.MAX_MU)
        info.gcv = gcv.ctypes.data_as(C.POINTER(C.c_double))
        L.check(self.lib.rtg_gmres_wait(self._h, pend.slot, C.byref(info)))
        res = _solve_result(info, rho, gcv, pend.grid, pend.lam)
        if pend.phase_times:
            res.phase_ms = {k: info.phase_ms[i] for i, k in enumerate(L.PHASES)}
            res.phase_launches = {k: info.phase_launches[i] for i, k in enumerate(L.PHASES)}
        return pend.X, res


def _solve_result(info, rho, gcv, grid, lam):
    return SolveResult(info.iters, info.restarts, bool(info.breakdown), bool(info.converged),
                       info.beta, info.mu, info.rho_final, rho[:info.iters].copy(),
                       gcv[:len(grid)].copy() if (grid is not None and lam < 0) else None,
                       info.elapsed_ms, info.device_status, info.launches, tile_config=info.tile_config,
                       true_rel_resid=info.true_rel_resid, true_rel_resid_theta=info.true_rel_resid_theta)


@dataclasses.dataclass
class PendingSolve:
    """A solve queued by Handle.gmres_submit and not yet waited for."""
    slot: int
    X: object
    m: int
    max_restarts: int
    grid: Optional[np.ndarray]
    lam: float
    phase_times: bool
    keep: tuple


class Krylov:
    """Caller-held sketched Arnoldi state (rtg_krylov_*)."""

    def __init__(self, handle: Handle, dims: Sequence[int], dtype, m: int,
                 sketch_dims: Sequence[int], seed: int, A_factors: Sequence[Factor] = (),
                 B_factors: Sequence[Factor] = (), problem_id: int = 0):
        torch = _torch()
        self.h = handle
        self.dims = tuple(dims)
        self.dtype = dtype
        self.m = m
        code = L.F64 if dtype == torch.float64 else L.F32
        a, na, ka = _factor_array(A_factors)
        b, nb, kb = _factor_array(B_factors)
        sk = (C.c_int64 * len(dims))(*[int(s) for s in sketch_dims])
        k = C.c_void_p()
        L.check(handle.lib.rtg_krylov_create(handle._h, a, na, b, nb, _shape(dims), code, int(m), sk,
                                             C.c_uint64(seed), C.c_uint64(problem_id), C.byref(k)))
        self._k = k
        self.sdims = tuple(int(min(s, d)) for s, d in zip(sketch_dims, dims))

    def close(self):
        if getattr(self, "_k", None) is not None and self._k.value:
            self.h.lib.rtg_krylov_destroy(self._k)
            self._k = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def start(self, C_obs, X0=None, stream=None):
        _check_tensor(C_obs, self.dims, "C")
        L.check(self.h.lib.rtg_krylov_start(self.h._h, self._k, C_obs.data_ptr(),
                                            None if X0 is None else X0.data_ptr(), _stream(stream)))

    def step(self, stream=None):
        L.check(self.h.lib.rtg_arnoldi_step(self.h._h, self._k, _stream(stream)))

    def query(self, stream=None):
        """(view, Hbar as (m+1) x m numpy array)."""
        v = L.KrylovView()
        H = np.zeros((self.m + 1) * self.m)
        L.check(self.h.lib.rtg_krylov_query(self.h._h, self._k, C.byref(v),
                                            H.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream)))
        return v, H.reshape((self.m + 1, self.m), order="F")

    def basis(self, count: Optional[int] = None):
        """Views of the device basis V_0..V_{count-1} and sketches Q_0..Q_{count-1}."""
        torch = _torch()
        v, _ = self.query()
        count = v.j + 1 if count is None else count
        elt = 8 if self.dtype == torch.float64 else 4
        n, d = v.n, v.sketch_size
        Vs, Qs = [], []
        for i in range(count):
            Vs.append(_wrap(v.V + i * n * elt, self.dims, self.dtype, self.h.device))
            Qs.append(_wrap(v.Q + i * d * elt, self.sdims, self.dtype, self.h.device))
        return Vs, Qs


class _DeviceRange:
    """Minimal __cuda_array_interface__ exporter for a range of library memory."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def _wrap(ptr: int, dims, dtype, device):
    """Copy a device range into a new column-major tensor (no aliasing of library memory)."""
    torch = _torch()
    n = int(np.prod(dims))
    typestr = "<f8" if dtype == torch.float64 else "<f4"
    flat = torch.as_tensor(_DeviceRange(ptr, n, typestr), device=f"cuda:{device}").clone()
    return flat.reshape(tuple(reversed(dims))).permute(*reversed(range(len(dims))))


class WarmStart:
    """The learned warm start (rtg_ws_*): X_0 = C + net(C) and log(lambda).

    params: flat initial parameters in the library's order (e.g. from
    workloads.warmstart_params).  Batches are device tensors of shape
    (n, I1, I2, 3)... given as a list-free contiguous float32 buffer of
    n images in the solver layout: use stack_images / unstack_images."""

    def __init__(self, base: int, params: np.ndarray, device: int = 0):
        self.lib = L.load()
        flat = np.ascontiguousarray(params, dtype=np.float32)
        h = C.c_void_p()
        L.check(self.lib.rtg_ws_create(int(device), int(base), flat.ctypes.data_as(C.POINTER(C.c_float)),
                                       C.byref(h)))
        self._h = h
        self.base = base
        self.n = int(self.lib.rtg_ws_num_params(h))
        if self.n != flat.size:
            raise ValueError(f"expected {self.n} parameters, got {flat.size}")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.rtg_ws_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get(self):
        p = np.zeros(self.n, dtype=np.float32)
        g = np.zeros(self.n, dtype=np.float32)
        L.check(self.lib.rtg_ws_get(self._h, p.ctypes.data_as(C.POINTER(C.c_float)),
                                    g.ctypes.data_as(C.POINTER(C.c_float))))
        return p, g

    def predict(self, Cb, I1: int, I2: int, stream=None):
        """Cb: device float32 buffer of n images (solver layout, back to back)."""
        torch = _torch()
        n = Cb.numel() // (I1 * I2 * 3)
        X0 = torch.empty_like(Cb)
        ll = torch.empty(n, dtype=torch.float32, device=Cb.device)
        L.check(self.lib.rtg_ws_predict(self._h, n, I1, I2, Cb.data_ptr(), X0.data_ptr(), ll.data_ptr(),
                                        _stream(stream)))
        return X0, ll

    def solve(self, handle: "Handle", C_obs, m: int, sketch_dims: Sequence[int], seed: int,
              A_factors: Sequence[Factor] = (), B_factors: Sequence[Factor] = (), X=None, tol: float = 0.0,
              mu_grid=None, max_restarts: int = 0, true_residual: bool = False, slot: int = 0, stream=None):
        """Warm-started RTG-GMRES (rtg_ws_solve): prediction, fallback test and
        stop-level rescale on the device, then the solve.  Returns
        (X, SolveResult, decision dict)."""
        dims = tuple(C_obs.shape)
        _check_tensor(C_obs, dims, "C")
        if X is None:
            X = empty(dims, C_obs.dtype, C_obs.device)
        a, na, ka = _factor_array(A_factors)
        b, nb, kb = _factor_array(B_factors)
        sk = (C.c_int64 * len(dims))(*[int(s) for s in sketch_dims])
        opts = L.Opts()
        opts.tol = float(tol)
        grid = np.ascontiguousarray(mu_grid, dtype=np.float64)
        opts.mu_grid = grid.ctypes.data_as(C.POINTER(C.c_double))
        opts.n_mu = len(grid)
        opts.max_restarts = int(max_restarts)
        opts.flags = L.FLAG_TRUE_RESIDUAL if true_residual else 0
        opts.slot = int(slot)
        info = L.Info()
        rho = np.zeros(m * (max_restarts + 1) + 1)
        info.rho_hist = rho.ctypes.data_as(C.POINTER(C.c_double))
        gcv = np.zeros(L.MAX_MU)
        info.gcv = gcv.ctypes.data_as(C.POINTER(C.c_double))
        dec = L.WsResult()
        L.check(self.lib.rtg_ws_solve(self._h, handle._h, a, na, b, nb, _shape(dims), C_obs.data_ptr(), int(m), sk,
                                      C.c_uint64(seed), X.data_ptr(), C.byref(opts), C.byref(info), C.byref(dec),
                                      _stream(stream)))
        res = _solve_result(info, rho, gcv, grid, -1.0 if dec.fell_back else 1.0)
        return X, res, {"fell_back": bool(dec.fell_back), "lam": dec.lam, "tol": dec.tol,
                        "sketch_norm_C": dec.sketch_norm_C, "sketch_norm_R0": dec.sketch_norm_R0}

    def train_step(self, Cb, Xs, logmu, I1: int, I2: int, lr: float, stream=None):
        torch = _torch()
        n = Cb.numel() // (I1 * I2 * 3)
        X0 = torch.empty_like(Cb)
        loss = C.c_double()
        L.check(self.lib.rtg_ws_train_step(self._h, n, I1, I2, Cb.data_ptr(), Xs.data_ptr(), logmu.data_ptr(),
                                           float(lr), X0.data_ptr(), C.byref(loss), _stream(stream)))
        return float(loss.value)


def stack_images(images) -> "object":
    """Column-major (I1, I2, 3) device tensors -> one contiguous buffer in the solver layout."""
    torch = _torch()
    return torch.cat([im.permute(2, 1, 0).reshape(-1) for im in images])


def unstack_images(buf, n: int, I1: int, I2: int):
    return [buf[i * I1 * I2 * 3:(i + 1) * I1 * I2 * 3].view(3, I2, I1).permute(2, 1, 0) for i in range(n)]


def conv3x3(x, w, b=None, stride: int = 1, dy=None, device: int = 0):
    """One warm-start convolution layer (rtg_nn_conv3x3) on channels-last device tensors.
    Forward (dy None): returns y.  Backward: returns (dx, dw, db)."""
    torch = _torch()
    lib = L.load()
    N, H, W, cin = x.shape
    cout = w.shape[0]
    p = lambda t: 0 if t is None else t.data_ptr()
    if dy is None:
        y = torch.empty((N, H // stride, W // stride, cout), dtype=torch.float32, device=x.device)
        L.check(lib.rtg_nn_conv3x3(device, N, H, W, cin, cout, stride, x.data_ptr(), w.data_ptr(), p(b),
                                   y.data_ptr(), 0, 0, 0, 0, _stream(None)))
        return y
    dx = torch.empty_like(x)
    dw = torch.empty_like(w)
    db = torch.empty(cout, dtype=torch.float32, device=x.device)
    L.check(lib.rtg_nn_conv3x3(device, N, H, W, cin, cout, stride, x.data_ptr(), w.data_ptr(), 0, 0,
                               dy.data_ptr(), dx.data_ptr(), dw.data_ptr(), db.data_ptr(), _stream(None)))
    return dx, dw, db
