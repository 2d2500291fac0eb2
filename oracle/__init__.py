"""FP64 CPU oracle for Randomized Tensor Global GMRES (RTG-GMRES).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously
correct numpy implementation of what the GPU path computes, written from
the paper (Badahmane, "Randomized Tensor Krylov Subspace Methods via
Sketched Einstein Product with Applications to Image and Video
Restoration").  Only the test-suite, the package-level smoke check and
the benchmark's CPU-baseline leg may import it; the product path never
does, and this package imports nothing from the product.

Every function cites the passage it follows.  The arithmetic is FP64 and
follows the paper's steps in its order and notation: successive mode
products for the sketch (Section 3.1), literal modified Gram-Schmidt with
the sketch of the updated tensor recomputed after every subtraction
(Algorithm "Block GMRES via Sketched Einstein Product"), least squares by
a library solver (Eq. 11S), the stacked Tikhonov problem (Eq. 13) and the
GCV function as defined in Section 3 ("Parameter selection via GCV").

Pins (what ties each part to something other than itself) live in
tests/test_oracle_*.py.  Parity unpinned: the statistical embedding
property of the Rademacher sketch (Definition of the tensor
epsilon-subspace embedding) is only checked in distribution, not pinned.
"""
from .einstein import einstein_product, mode_product, unfold, frobenius_inner, frobenius_norm
from .operator import (banded_toeplitz, factor_matrices, apply_operator, blur_tensor,
                       psf_convolve, dense_operator_matrix)
from .philox import philox4x64_10, philox_words, rademacher_signs
from .sketch import sketch_matrices, sketch, sketch_dense_matrix
from .krylov import (sketched_arnoldi, frobenius_arnoldi, rtg_gmres, tg_gmres,
                     ls_residual)
from .tikhonov import (tikhonov_stacked, tikhonov_normal, tikhonov_svd, gcv_value,
                       gcv_choose)
from .metrics import make_observation, relative_error, psnr, rho_star
from .golub_kahan import transpose_mats, sketched_golub_kahan, sketched_gk_solve
from . import warmstart

__all__ = [n for n in dir() if not n.startswith("_")]
