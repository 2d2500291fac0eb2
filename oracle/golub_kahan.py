"""Sketched Golub-Kahan bidiagonalisation and its regularised solve (oracle; test infrastructure only).

Follows the algorithm "Block Golub-Kahan via Sketched Einstein Product"
(Section 4.5), step by step, in FP64:

    beta_1 = ||R_0||_Theta,  U_1 = R_0 / beta_1,
    W = Phi^T(U_1),  alpha_1 = ||W||_Theta,  V_1 = W / alpha_1,
    for k = 1, 2, ..., m:
        W = Phi(V_k) - alpha_k U_k,          beta_{k+1} = ||W||_Theta,  U_{k+1} = W / beta_{k+1}
        Z = Phi^T(U_{k+1}) - beta_{k+1} V_k, alpha_{k+1} = ||Z||_Theta, V_{k+1} = Z / alpha_{k+1}

with the lower-bidiagonal (k+1) x k matrix Btilde_k (alpha_i on the
diagonal, beta_{i+1} below it), y = argmin ||beta_1 e_1 - Btilde_k y||^2 +
mu ||y||^2 and X = X_0 + sum_i y_i V_i.  Only norms are sketched; the
recurrences are the short ones of the listing (no re-orthogonalisation).

Readings (the listing is garbled in places): the forward product, written
A *_M V and A *_P X, is Phi; the transposed product A^T *_N U is the
adjoint of Phi in the Frobenius inner product, i.e. every mode matrix
transposed.  R_0 = C - Phi(X_0) (the listing starts from C, i.e. X_0 = 0).
rho_k = ||beta_1 e_1 - Btilde_k y_k||_2 / beta_1 (least-squares residual
of the projected problem), evaluated once beta_{k+1} is known; the process
stops at the first k with rho_k <= tol, when beta_{k+1} or alpha_{k+1}
falls to breakdown_tol times the sketched norm of the product before the
subtraction (the listing's "= 0"), or at k = m.  mu: fixed (lam > 0), 0
(lam == 0) or by GCV over a grid (lam < 0), as for RTG-GMRES.
"""
from __future__ import annotations

from typing import Callable, List, Optional

import numpy as np

from .einstein import frobenius_norm
from .krylov import ls_residual
from .operator import apply_operator
from .sketch import sketch
from .tikhonov import gcv_choose, tikhonov_stacked


def transpose_mats(mats):
    """Mode matrices of the adjoint operator Phi^T (each transposed)."""
    return [None if M is None else np.ascontiguousarray(M.T) for M in mats]


def sketched_golub_kahan(apply_phi: Callable, apply_phit: Callable, R0: np.ndarray, m: int,
                         S: Callable, tol: float = 0.0, breakdown_tol: float = 1e-12) -> dict:
    """The bidiagonalisation of the algorithm above; returns the bases, Btilde and rho."""
    snorm = lambda X: frobenius_norm(S(X))
    beta1 = snorm(R0)
    if beta1 == 0.0:
        return dict(U=[], V=[], B=np.zeros((1, 0)), beta=0.0, rho=[], breakdown=False, k=0)
    U = [R0 / beta1]
    W = apply_phit(U[0])
    pre = snorm(W)
    alpha = pre
    V: List[np.ndarray] = []
    B = np.zeros((m + 1, m))
    rho: List[float] = []
    breakdown = alpha <= breakdown_tol * beta1 if beta1 > 0 else True
    if breakdown:
        return dict(U=U, V=[], B=np.zeros((1, 0)), beta=beta1, rho=[], breakdown=True, k=0)
    V.append(W / alpha)
    k = m
    for j in range(m):                       # 0-based step j builds column j of Btilde
        B[j, j] = alpha
        PW = apply_phi(V[j])
        pre = snorm(PW)
        W = PW - alpha * U[j]
        beta = snorm(W)
        breakdown = beta <= breakdown_tol * pre
        B[j + 1, j] = 0.0 if breakdown else beta
        res, _ = ls_residual(B[:j + 2, :j + 1], beta1)
        rho.append(res / beta1)
        if not breakdown:
            U.append(W / beta)
        if breakdown or rho[-1] <= tol or j + 1 == m:
            k = j + 1
            break
        PZ = apply_phit(U[j + 1])
        pre = snorm(PZ)
        Z = PZ - beta * V[j]
        alpha = snorm(Z)
        if alpha <= breakdown_tol * pre:
            breakdown = True
            k = j + 1
            break
        V.append(Z / alpha)
    return dict(U=U, V=V[:k], B=B[:k + 1, :k].copy(), beta=beta1, rho=rho, breakdown=breakdown, k=k)


def sketched_gk_solve(mats, C: np.ndarray, m: int, thetas, X0: Optional[np.ndarray] = None,
                      tol: float = 0.0, lam: float = 0.0, mu_grid=None,
                      breakdown_tol: float = 1e-12) -> dict:
    """Sketched Golub-Kahan least squares / projected Tikhonov (GCV as for RTG-GMRES)."""
    C = np.asarray(C, dtype=np.float64)
    X0 = np.zeros_like(C) if X0 is None else np.array(X0, dtype=np.float64)
    matsT = transpose_mats(mats)
    phi = lambda X: apply_operator(X, mats)
    phit = lambda X: apply_operator(X, matsT)
    S = lambda X: sketch(X, thetas)
    R0 = C - phi(X0)
    gk = sketched_golub_kahan(phi, phit, R0, m, S, tol, breakdown_tol)
    if gk["k"] == 0:
        return dict(X=X0, rho=[], iters=0, k=0, mu=float(max(lam, 0.0)), gcv=None, beta=gk["beta"],
                    B=gk["B"], y=np.zeros(0), breakdown=gk["breakdown"], converged=True, V=[])
    Bt = gk["B"]
    gcv = None
    if lam > 0:
        mu = float(lam)
    elif lam == 0:
        mu = 0.0
    else:
        mu, gcv = gcv_choose(Bt, gk["beta"], mu_grid)
    y = tikhonov_stacked(Bt, gk["beta"], mu) if mu > 0 else ls_residual(Bt, gk["beta"])[1]
    X = X0.copy()
    for i in range(len(y)):
        X = X + y[i] * gk["V"][i]
    return dict(X=X, rho=gk["rho"], iters=gk["k"], k=gk["k"], mu=mu, gcv=gcv, beta=gk["beta"],
                B=Bt, y=y, breakdown=gk["breakdown"],
                converged=bool(gk["breakdown"] or gk["rho"][-1] <= tol), V=gk["V"], U=gk["U"])
