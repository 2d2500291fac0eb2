"""Observation model and quality measures of Section 5 (oracle; test infrastructure only)."""
from __future__ import annotations

import numpy as np

from .einstein import frobenius_norm
from .operator import apply_operator


def make_observation(x_true: np.ndarray, mats, E: np.ndarray, nu: float):
    """C = C_hat + N with C_hat = Phi(X_hat) and N = nu ||C_hat||_F E/||E||_F (Eq. 59).

    The scaling makes the noise level ||N||/||C_hat|| (Section 5.3) exactly nu.
    Returns (C, C_hat, nu_C) with nu_C = ||N||_F / ||C||_F.
    """
    C_hat = apply_operator(x_true, mats)
    N = nu * frobenius_norm(C_hat) * E / frobenius_norm(E)
    C = C_hat + N
    return C, C_hat, frobenius_norm(N) / frobenius_norm(C)


def relative_error(x_true: np.ndarray, x: np.ndarray) -> float:
    """RE = ||X_hat - X_restored||_F / ||X_hat||_F (Section 5.5)."""
    return frobenius_norm(x_true - x) / frobenius_norm(x_true)


def psnr(x_true: np.ndarray, x: np.ndarray) -> float:
    """PSNR as Section 5.5 defines it: 10 log10(||X_hat - mean(X_hat)||^2 / ||X_restored - X_hat||^2)."""
    num = frobenius_norm(x_true - np.mean(x_true)) ** 2
    den = frobenius_norm(x - x_true) ** 2
    return 10.0 * np.log10(num / den)


def rho_star(nu_C: float) -> float:
    """Stop level on the relative sketched residual: 1e-3, raised to 1.01 nu_C
    when the noise floor of the observation lies above it (discrepancy principle)."""
    return max(1e-3, 1.01 * nu_C)
