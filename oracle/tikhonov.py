"""Projected Tikhonov problem and GCV (oracle; test infrastructure only).

Section 3, "Sketched projected Tikhonov problem" (Eq. 12S, 14S) and
"Sketched Tikhonov regularization" (Eq. 12-14), "Parameter selection via
GCV".  Hbar is the (k+1) x k Hessenberg matrix, beta the (sketched) norm
of the initial residual.
"""
from __future__ import annotations

from typing import Sequence, Tuple

import numpy as np


def _rhs(Hbar: np.ndarray, beta: float) -> np.ndarray:
    b = np.zeros(Hbar.shape[0])
    b[0] = beta
    return b


def tikhonov_stacked(Hbar: np.ndarray, beta: float, mu: float) -> np.ndarray:
    """y_mu = argmin || [Hbar; sqrt(mu) I] y - [beta e1; 0] ||_2 (Eq. 13), by a library least-squares solve."""
    k = Hbar.shape[1]
    A = np.vstack([Hbar, np.sqrt(mu) * np.eye(k)])
    b = np.concatenate([_rhs(Hbar, beta), np.zeros(k)])
    return np.linalg.lstsq(A, b, rcond=None)[0]


def tikhonov_normal(Hbar: np.ndarray, beta: float, mu: float) -> np.ndarray:
    """Normal equations (Hbar^T Hbar + mu I) y = Hbar^T beta e1 (Eq. 14 / 14S)."""
    k = Hbar.shape[1]
    return np.linalg.solve(Hbar.T @ Hbar + mu * np.eye(k), Hbar.T @ _rhs(Hbar, beta))


def tikhonov_svd(Hbar: np.ndarray, beta: float, mu: float) -> np.ndarray:
    """Filter-factor form through the SVD of Hbar ("for small m ... SVD", Section 3)."""
    U, s, Vt = np.linalg.svd(Hbar, full_matrices=False)
    c = U.T @ _rhs(Hbar, beta)
    return Vt.T @ (s * c / (s * s + mu))


def gcv_value(Hbar: np.ndarray, beta: float, mu: float) -> float:
    """GCV(mu) = ||Hbar y_mu - beta e1||^2 / [tr(I - Hbar Hbar_mu^{-1} Hbar^T)]^2, Hbar_mu = Hbar^T Hbar + mu I.

    The numerator uses the stacked solution (Eq. 13); the trace is formed
    from the explicit (k+1) x (k+1) matrix, as the definition reads.
    """
    k1, k = Hbar.shape
    b = _rhs(Hbar, beta)
    y = tikhonov_stacked(Hbar, beta, mu)
    num = float(np.sum((Hbar @ y - b) ** 2))
    Hmu = Hbar.T @ Hbar + mu * np.eye(k)
    T = np.eye(k1) - Hbar @ np.linalg.solve(Hmu, Hbar.T)
    return num / float(np.trace(T)) ** 2


def gcv_choose(Hbar: np.ndarray, beta: float, grid: Sequence[float]) -> Tuple[float, np.ndarray]:
    """mu in ``grid`` minimising GCV; among equal values the larger mu wins."""
    vals = np.array([gcv_value(Hbar, beta, float(mu)) for mu in grid])
    best = None
    for mu, v in zip(grid, vals):
        if best is None or v < best[1] or (v == best[1] and mu > best[0]):
            best = (float(mu), float(v))
    return best[0], vals
