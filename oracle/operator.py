"""The blur operator Phi of Sections 1 and 5 (oracle; test infrastructure only).

Phi(X) = A *_N X (*_M B) with A separable: A[i1..iN, i1'..iN'] =
prod_k A_k[i_k, i_k'].  Each A_k is a banded Toeplitz matrix built from
1-D PSF taps with zero boundary conditions (Eq. 57 and the boundary
conditions that follow it), so Phi(X) = X x_1 A_1 x_2 A_2 ... and the
Einstein right product with B is X x_mode B^T.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np

from .einstein import mode_product


def banded_toeplitz(n: int, taps: np.ndarray) -> np.ndarray:
    """n x n matrix with (A x)_i = sum_{|t|<=r} taps[r+t] x_{i+t}, zero outside [0, n)."""
    taps = np.asarray(taps, dtype=np.float64)
    r = (len(taps) - 1) // 2
    A = np.zeros((n, n))
    for i in range(n):
        for t in range(-r, r + 1):
            if 0 <= i + t < n:
                A[i, i + t] = taps[r + t]
    return A


def _factor_matrix(n: int, kind: str, data) -> Optional[np.ndarray]:
    if kind == "identity":
        return None
    if kind == "banded":
        return banded_toeplitz(n, data)
    if kind == "dense":
        M = np.asarray(data, dtype=np.float64)
        assert M.shape == (n, n)
        return M
    raise ValueError(kind)


def factor_matrices(dims: Sequence[int], factors: Sequence[Tuple[int, str, object]],
                    right_factors: Sequence[Tuple[int, str, object]] = ()) -> List[Optional[np.ndarray]]:
    """Per-mode matrices M_k with Phi(X) = X x_1 M_1 ... x_d M_d (None = identity).

    ``factors`` (mode 1-based, kind, data) are left factors A_k.
    ``right_factors`` are Einstein right-product matrices B; since
    (X *_1 B)[.., c'] = sum_c X[.., c] B[c, c'], the mode matrix is B^T.
    """
    mats: List[Optional[np.ndarray]] = [None] * len(dims)
    for mode, kind, data in factors:
        M = _factor_matrix(dims[mode - 1], kind, data)
        mats[mode - 1] = M if mats[mode - 1] is None or M is None else M @ mats[mode - 1]
    for mode, kind, data in right_factors:
        B = _factor_matrix(dims[mode - 1], kind, data)
        if B is None:
            continue
        M = B.T
        mats[mode - 1] = M if mats[mode - 1] is None else M @ mats[mode - 1]
    return mats


def apply_operator(X: np.ndarray, mats: Sequence[Optional[np.ndarray]]) -> np.ndarray:
    """Phi(X) as successive mode products with the per-mode matrices."""
    Y = np.asarray(X, dtype=np.float64)
    for k, M in enumerate(mats):
        if M is not None:
            Y = mode_product(Y, M, k)
    return Y


def blur_tensor(A1: np.ndarray, A2: np.ndarray) -> np.ndarray:
    """Fourth-order blurring tensor of Eq. 56: A[i, j, i', j'] = A1[i, i'] A2[j, j']."""
    return np.einsum("ab,cd->acbd", A1, A2)


def psf_convolve(X: np.ndarray, P: np.ndarray) -> np.ndarray:
    """Spatially invariant 2-D convolution with zero boundary, Eq. 57 widened to radius r.

    C[i, j, k] = sum_{a,b=-r..r} P[r - a, r - b] X[i + a, j + b, k], with X
    zero outside the image (the flipped PSF index of Eq. 57).  Plain loops.
    """
    r = (P.shape[0] - 1) // 2
    I1, I2 = X.shape[:2]
    C = np.zeros_like(X, dtype=np.float64)
    for i in range(I1):
        for j in range(I2):
            acc = np.zeros(X.shape[2:])
            for a in range(-r, r + 1):
                for b in range(-r, r + 1):
                    if 0 <= i + a < I1 and 0 <= j + b < I2:
                        acc = acc + P[r - a, r - b] * X[i + a, j + b]
            C[i, j] = acc
    return C


def dense_operator_matrix(dims: Sequence[int], mats: Sequence[Optional[np.ndarray]]) -> np.ndarray:
    """Matrix of Phi acting on ivec-vectorised tensors: M_d kron ... kron M_1."""
    out = np.ones((1, 1))
    for k in range(len(dims)):
        M = mats[k] if mats[k] is not None else np.eye(dims[k])
        out = np.kron(M, out)
    return out
