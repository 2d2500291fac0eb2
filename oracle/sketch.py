"""Mode-wise Rademacher sketch S of Section 3 (oracle; test infrastructure only)."""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np

from .einstein import mode_product
from .philox import rademacher_signs


def sketch_matrices(dims: Sequence[int], sketch_dims: Sequence[int], seed: int,
                    problem_id: int = 0) -> List[Optional[np.ndarray]]:
    """Theta_k in R^{s_k x I_k} with entries +-1/sqrt(s_k) (Section 3, "Let Theta_k ...").

    A mode whose sketch size is at least its dimension is not sketched
    (Theta_k = I; a square Rademacher matrix is neither orthogonal nor
    reliably invertible).  Signs come from one Philox stream: the sketched
    modes in increasing order, each Theta_k flattened row-major.
    """
    assert len(dims) == len(sketch_dims)
    total = sum(s * I for s, I in zip(sketch_dims, dims) if s < I)
    signs = rademacher_signs(seed, problem_id, total) if total else np.zeros(0)
    out: List[Optional[np.ndarray]] = []
    off = 0
    for s, I in zip(sketch_dims, dims):
        if s >= I:
            out.append(None)
            continue
        out.append(signs[off:off + s * I].reshape(s, I) / np.sqrt(s))
        off += s * I
    return out


def sketch(X: np.ndarray, thetas: Sequence[Optional[np.ndarray]]) -> np.ndarray:
    """S(X) = X x_1 Theta_1 x_2 Theta_2 ... x_d Theta_d (global sketching operator, Section 3)."""
    Y = np.asarray(X, dtype=np.float64)
    for k, T in enumerate(thetas):
        if T is not None:
            Y = mode_product(Y, T, k)
    return Y


def sketch_dense_matrix(dims: Sequence[int], thetas: Sequence[Optional[np.ndarray]]) -> np.ndarray:
    """Theta_d kron ... kron Theta_1, the vectorised form of S (Section 3, "Equivalent Vectorized Form")."""
    out = np.ones((1, 1))
    for k in range(len(dims)):
        T = thetas[k] if thetas[k] is not None else np.eye(dims[k])
        out = np.kron(T, out)
    return out
