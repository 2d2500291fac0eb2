"""Tensor algebra of Section 2 and Section 4.1 (oracle; test infrastructure only)."""
from __future__ import annotations

import numpy as np


def einstein_product(A: np.ndarray, B: np.ndarray, N: int) -> np.ndarray:
    """Einstein product A *_N B (Section 2.1).

    Sums over the last N modes of A and the first N modes of B; the
    result has A's leading modes followed by B's trailing modes.
    """
    assert A.shape[A.ndim - N:] == B.shape[:N], (A.shape, B.shape, N)
    return np.tensordot(A, B, axes=(list(range(A.ndim - N, A.ndim)), list(range(N))))


def mode_product(X: np.ndarray, M: np.ndarray, k: int) -> np.ndarray:
    """Mode-k product X x_k M (0-based k): (X x_k M)[.., p, ..] = sum_i M[p, i] X[.., i, ..].

    Used by the compressed tensor of Section 3.1 and by the separable
    operator (a mode product with a banded Toeplitz matrix).
    """
    assert M.shape[1] == X.shape[k]
    Y = np.tensordot(M, X, axes=([1], [k]))
    return np.moveaxis(Y, 0, k)


def unfold(X: np.ndarray, n_row_modes: int) -> np.ndarray:
    """Unfolding Psi_IJ of Section 4.1.

    Rows are indexed by ivec over the first ``n_row_modes`` modes and
    columns by ivec over the rest, ivec being the column-major (mode 1
    fastest) linear index; Fortran-order reshape is exactly that map.
    """
    rows = int(np.prod(X.shape[:n_row_modes]))
    cols = int(np.prod(X.shape[n_row_modes:]))
    return np.reshape(X, (rows, cols), order="F")


def frobenius_inner(X: np.ndarray, Y: np.ndarray) -> float:
    """Frobenius inner product of Section 2.2: sum of elementwise products."""
    return float(np.sum(X * Y))


def frobenius_norm(X: np.ndarray) -> float:
    """Induced norm ||X||_F = sqrt(<X, X>_F) (Section 2.2)."""
    return float(np.sqrt(frobenius_inner(X, X)))
