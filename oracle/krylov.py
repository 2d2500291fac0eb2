"""Sketched and classical tensor global Arnoldi / GMRES (oracle; test infrastructure only).

The sketched process follows Section 4.3 and the algorithm "Block GMRES
via Sketched Einstein Product" (Section 4.4): R_0 = C - Phi(X_0),
beta = ||R_0||_Theta, V_1 = R_0/beta; for each j, W = Phi(V_j) in the full
space, then for i = 1..j h_ij = <V_i, W>_Theta and W <- W - h_ij V_i
(modified Gram-Schmidt, the sketch of the updated W recomputed before each
inner product), h_{j+1,j} = ||W||_Theta, V_{j+1} = W/h_{j+1,j}.  Only inner
products and norms are sketched (Section 5.4), so the Krylov space is the
ordinary K_m(Phi, R_0).

The classical tensor global GMRES (Eq. 8-11, whose Arnoldi process the
paper calls Algorithm 1 without printing it) is the same process with
Frobenius inner products; it is written out separately below.

The least-squares problem (Eq. 11S) is solved with a library solver after
every step; rho_j = ||beta e1 - Hbar_j y_j||_2 / beta_0 is the relative
residual in the Theta-norm (the identity of Section 4.4).  The iteration
stops at the first j with rho_j <= tol, on a breakdown
h_{j+1,j} <= breakdown_tol * ||S(Phi(V_j))||, or at j = m.  The returned
X uses the Tikhonov solution of Eq. 13 with mu fixed (lam > 0), GCV over a
grid (lam < 0) or plain least squares (lam == 0).  With max_restarts > 0 an
unconverged cycle restarts from its least-squares iterate.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional, Sequence

import numpy as np

from .einstein import frobenius_inner, frobenius_norm
from .operator import apply_operator
from .sketch import sketch
from .tikhonov import gcv_choose, tikhonov_stacked


@dataclasses.dataclass
class ArnoldiResult:
    V: List[np.ndarray]        # basis tensors V_1..V_{k+1} (V_{k+1} absent after a stop/breakdown)
    H: np.ndarray              # (k+1) x k Hessenberg matrix Hbar_k
    beta: float
    rho: List[float]           # relative LS residual after each step
    breakdown: bool
    k: int


def ls_residual(Hbar: np.ndarray, beta: float):
    """min_y ||beta e1 - Hbar y||_2 and its minimiser (Eq. 11S), library least squares."""
    b = np.zeros(Hbar.shape[0])
    b[0] = beta
    y = np.linalg.lstsq(Hbar, b, rcond=None)[0]
    return float(np.linalg.norm(b - Hbar @ y)), y


def sketched_arnoldi(apply_phi: Callable, R0: np.ndarray, m: int, S: Callable,
                     tol: float = 0.0, breakdown_tol: float = 1e-12,
                     rho_scale: Optional[float] = None) -> ArnoldiResult:
    """Sketched global Arnoldi with literal MGS (Section 4.3; Block GMRES algorithm, steps 1-15)."""
    sR0 = S(R0)
    beta = float(np.sqrt(frobenius_inner(sR0, sR0)))
    if beta == 0.0:
        return ArnoldiResult([], np.zeros((1, 0)), 0.0, [], False, 0)
    scale = beta if rho_scale is None else rho_scale
    V = [R0 / beta]
    SV = [S(V[0])]
    H = np.zeros((m + 1, m))
    rho: List[float] = []
    breakdown = False
    k = m
    for j in range(m):
        W = apply_phi(V[j])
        sW = S(W)
        pre = frobenius_norm(sW)
        for i in range(j + 1):
            H[i, j] = frobenius_inner(SV[i], sW)      # h_ij = <V_i, W>_Theta
            W = W - H[i, j] * V[i]
            sW = S(W)
        hn = frobenius_norm(sW)                       # h_{j+1,j} = ||W||_Theta
        breakdown = hn <= breakdown_tol * pre
        H[j + 1, j] = 0.0 if breakdown else hn
        res, _ = ls_residual(H[:j + 2, :j + 1], beta)
        rho.append(res / scale)
        if breakdown:
            k = j + 1
            break
        V.append(W / hn)
        SV.append(S(V[-1]))
        if rho[-1] <= tol:
            k = j + 1
            break
    return ArnoldiResult(V, H[:k + 1, :k].copy(), beta, rho, breakdown, k)


def frobenius_arnoldi(apply_phi: Callable, R0: np.ndarray, m: int, tol: float = 0.0,
                      breakdown_tol: float = 1e-12,
                      rho_scale: Optional[float] = None) -> ArnoldiResult:
    """Classical tensor global Arnoldi with Frobenius inner products (Eq. 7-11), MGS order."""
    beta = frobenius_norm(R0)
    if beta == 0.0:
        return ArnoldiResult([], np.zeros((1, 0)), 0.0, [], False, 0)
    scale = beta if rho_scale is None else rho_scale
    V = [R0 / beta]
    H = np.zeros((m + 1, m))
    rho: List[float] = []
    breakdown = False
    k = m
    for j in range(m):
        W = apply_phi(V[j])
        pre = frobenius_norm(W)
        for i in range(j + 1):
            H[i, j] = float(np.vdot(V[i].ravel(), W.ravel()))
            W = W - H[i, j] * V[i]
        hn = frobenius_norm(W)
        breakdown = hn <= breakdown_tol * pre
        H[j + 1, j] = 0.0 if breakdown else hn
        res, _ = ls_residual(H[:j + 2, :j + 1], beta)
        rho.append(res / scale)
        if breakdown:
            k = j + 1
            break
        V.append(W / hn)
        if rho[-1] <= tol:
            k = j + 1
            break
    return ArnoldiResult(V, H[:k + 1, :k].copy(), beta, rho, breakdown, k)


def _combine(X0: np.ndarray, V: Sequence[np.ndarray], y: np.ndarray) -> np.ndarray:
    """X_0 + sum_j V_j y_j (Eq. 10S; final update of the Block GMRES algorithm)."""
    X = X0.copy()
    for j in range(len(y)):
        X = X + y[j] * V[j]
    return X


def _gmres(arnoldi: Callable, apply_phi: Callable, C: np.ndarray, X0: Optional[np.ndarray],
           m: int, tol: float, lam: float, mu_grid, max_restarts: int) -> dict:
    X0 = np.zeros_like(C, dtype=np.float64) if X0 is None else np.array(X0, dtype=np.float64)
    rho_all: List[float] = []
    beta0 = None
    restarts = 0
    iters = 0
    while True:
        R0 = C - apply_phi(X0)
        arn = arnoldi(R0, rho_scale=beta0)
        if beta0 is None:
            beta0 = arn.beta
        if arn.k == 0:            # zero residual: X0 already solves the problem
            break
        rho_all.extend(arn.rho)
        iters += arn.k
        converged = arn.breakdown or arn.rho[-1] <= tol
        if converged or restarts >= max_restarts:
            break
        _, y = ls_residual(arn.H, arn.beta)
        X0 = _combine(X0, arn.V, y)
        restarts += 1
    if arn.k == 0:
        return dict(X=X0, rho=[], iters=0, k=0, mu=float(max(lam, 0.0)), gcv=None, beta=0.0,
                    H=np.zeros((1, 0)), y=np.zeros(0), breakdown=False, converged=True,
                    restarts=restarts, V=[], X0=X0)
    gcv = None
    if lam > 0:
        mu = float(lam)
    elif lam == 0:
        mu = 0.0
    else:
        mu, gcv = gcv_choose(arn.H, arn.beta, mu_grid)
    y = tikhonov_stacked(arn.H, arn.beta, mu) if mu > 0 else ls_residual(arn.H, arn.beta)[1]
    X = _combine(X0, arn.V, y)
    return dict(X=X, rho=rho_all, iters=iters, k=arn.k, mu=mu, gcv=gcv, beta=beta0, H=arn.H,
                y=y, breakdown=arn.breakdown,
                converged=bool(arn.breakdown or rho_all[-1] <= tol), restarts=restarts,
                V=arn.V, X0=X0)


def rtg_gmres(mats, C: np.ndarray, m: int, thetas, X0: Optional[np.ndarray] = None,
              tol: float = 0.0, lam: float = 0.0, mu_grid=None, breakdown_tol: float = 1e-12,
              max_restarts: int = 0) -> dict:
    """RTG-GMRES: sketched Arnoldi, least squares (Eq. 11S), projected Tikhonov (Eq. 12S/13)."""
    apply_phi = lambda X: apply_operator(X, mats)
    S = lambda X: sketch(X, thetas)
    arnoldi = lambda R0, rho_scale=None: sketched_arnoldi(apply_phi, R0, m, S, tol,
                                                          breakdown_tol, rho_scale)
    return _gmres(arnoldi, apply_phi, np.asarray(C, dtype=np.float64), X0, m, tol, lam,
                  mu_grid, max_restarts)


def tg_gmres(mats, C: np.ndarray, m: int, X0: Optional[np.ndarray] = None, tol: float = 0.0,
             lam: float = 0.0, mu_grid=None, breakdown_tol: float = 1e-12,
             max_restarts: int = 0) -> dict:
    """Classical TG-GMRES (Eq. 8-11) with Frobenius inner products; same solve and stop rule."""
    apply_phi = lambda X: apply_operator(X, mats)
    arnoldi = lambda R0, rho_scale=None: frobenius_arnoldi(apply_phi, R0, m, tol, breakdown_tol,
                                                           rho_scale)
    return _gmres(arnoldi, apply_phi, np.asarray(C, dtype=np.float64), X0, m, tol, lam,
                  mu_grid, max_restarts)
