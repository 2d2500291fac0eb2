"""Pins for the oracle's tensor algebra, operator and sketch (CPU only).

Each test ties the oracle to something other than itself: the paper's
identities (unfolding, Kronecker form of the sketch), brute-force loops
written from the definitions, numpy's own Philox generator, and closed
forms.
"""
import numpy as np
import pytest

import oracle
from oracle import einstein as E


def _rng(s=0):
    return np.random.default_rng(s)


def ivec(idx1, dims):
    """Section 4.1, 1-based: i_1 + sum_{r>=2} (i_r - 1) prod_{u<r} I_u."""
    out = idx1[0]
    stride = 1
    for r in range(1, len(dims)):
        stride *= dims[r - 1]
        out += (idx1[r] - 1) * stride
    return out


def test_unfold_matches_ivec_definition():
    X = _rng().standard_normal((3, 4, 2, 5))
    U = E.unfold(X, 2)
    for i1 in range(3):
        for i2 in range(4):
            for j1 in range(2):
                for j2 in range(5):
                    r = ivec((i1 + 1, i2 + 1), (3, 4)) - 1
                    c = ivec((j1 + 1, j2 + 1), (2, 5)) - 1
                    assert U[r, c] == X[i1, i2, j1, j2]


def test_einstein_product_brute_force():
    rng = _rng(1)
    A = rng.standard_normal((2, 3, 4, 3))
    B = rng.standard_normal((4, 3, 5))
    C = E.einstein_product(A, B, 2)
    ref = np.zeros((2, 3, 5))
    for i1 in range(2):
        for i2 in range(3):
            for j in range(5):
                s = 0.0
                for k1 in range(4):
                    for k2 in range(3):
                        s += A[i1, i2, k1, k2] * B[k1, k2, j]
                ref[i1, i2, j] = s
    assert np.allclose(C, ref, rtol=0, atol=1e-13)


def test_einstein_product_is_unfolded_matmul():
    """Psi_IJ(A *_N B) = Psi_IK(A) Psi_KJ(B) (Section 4.1)."""
    rng = _rng(2)
    A = rng.standard_normal((3, 4, 5, 2))
    B = rng.standard_normal((5, 2, 3, 2))
    lhs = E.unfold(E.einstein_product(A, B, 2), 2)
    rhs = E.unfold(A, 2) @ E.unfold(B, 2)
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-12)


def test_mode_product_brute_force():
    rng = _rng(3)
    X = rng.standard_normal((3, 4, 2))
    M = rng.standard_normal((5, 4))
    Y = E.mode_product(X, M, 1)
    assert Y.shape == (3, 5, 2)
    for a in range(3):
        for p in range(5):
            for c in range(2):
                assert abs(Y[a, p, c] - sum(M[p, i] * X[a, i, c] for i in range(4))) < 1e-13


def test_banded_toeplitz_definition():
    taps = np.array([0.1, 0.2, 0.4, 0.2, 0.1, 0.0, 0.0][:5])
    A = oracle.banded_toeplitz(6, taps)
    x = np.arange(1.0, 7.0)
    for i in range(6):
        s = sum(taps[2 + t] * x[i + t] for t in range(-2, 3) if 0 <= i + t < 6)
        assert abs((A @ x)[i] - s) < 1e-14


def test_operator_equals_einstein_with_blur_tensor():
    """Phi(X) = A *_2 X *_1 B with A[i,j,i',j'] = A1[i,i'] A2[j,j'] (Eq. 56, Section 1)."""
    rng = _rng(4)
    dims = (7, 6, 3)
    t1, t2 = rng.standard_normal(5), rng.standard_normal(3)
    B = rng.standard_normal((3, 3))
    mats = oracle.factor_matrices(dims, [(1, "banded", t1), (2, "banded", t2)], [(3, "dense", B)])
    X = rng.standard_normal(dims)
    A4 = oracle.blur_tensor(oracle.banded_toeplitz(7, t1), oracle.banded_toeplitz(6, t2))
    ref = E.einstein_product(E.einstein_product(A4, X, 2), B, 1)
    assert np.allclose(oracle.apply_operator(X, mats), ref, rtol=0, atol=1e-12)


def test_operator_equals_psf_convolution_eq57():
    """Separable PSF P = p1 p2^T with zero boundary (Eq. 57): the Toeplitz taps are the flipped PSF."""
    rng = _rng(5)
    p1, p2 = rng.uniform(0, 1, 5), rng.uniform(0, 1, 5)   # non-symmetric on purpose
    X = rng.standard_normal((8, 7, 3))
    C = oracle.psf_convolve(X, np.outer(p1, p2))
    mats = oracle.factor_matrices(X.shape, [(1, "banded", p1[::-1]), (2, "banded", p2[::-1])])
    assert np.allclose(oracle.apply_operator(X, mats), C, rtol=0, atol=1e-12)


def test_operator_dense_kronecker_matrix():
    rng = _rng(6)
    dims = (5, 4, 3, 2)
    mats = oracle.factor_matrices(dims, [(1, "banded", rng.standard_normal(3)),
                                         (2, "banded", rng.standard_normal(5)),
                                         (4, "banded", rng.standard_normal(3))],
                                  [(3, "dense", rng.standard_normal((3, 3)))])
    X = rng.standard_normal(dims)
    M = oracle.dense_operator_matrix(dims, mats)
    lhs = oracle.apply_operator(X, mats).ravel(order="F")
    assert np.allclose(M @ X.ravel(order="F"), lhs, rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed,pid", [(0, 0), (1, 0), (12345, 7), (2**63 + 5, 2**40 + 3)])
def test_philox_matches_numpy_philox(seed, pid):
    """The oracle's Philox4x64-10 (written from its published definition) against numpy's generator."""
    ref = np.random.Philox(key=seed + (pid << 64)).random_raw(37)
    got = oracle.philox_words(seed, pid, 37)
    assert [int(v) for v in ref] == got


def test_rademacher_bit_order():
    words = np.array(oracle.philox_words(3, 1, 4), dtype=np.uint64)
    bits = np.unpackbits(words.view(np.uint8), bitorder="little")   # bit e%64 of word e//64
    signs = oracle.rademacher_signs(3, 1, 256)
    assert np.array_equal(signs, np.where(bits == 1, -1.0, 1.0))


def test_sketch_matrices_shape_scale_identity():
    th = oracle.sketch_matrices((64, 48, 3), (16, 8, 3), seed=0)
    assert th[0].shape == (16, 64) and th[1].shape == (8, 48) and th[2] is None
    assert np.allclose(np.abs(th[0]), 1 / 4.0) and np.allclose(np.abs(th[1]), 1 / np.sqrt(8))
    # modes draw consecutive bits of one stream, row-major within each Theta_k
    s = oracle.rademacher_signs(0, 0, 16 * 64 + 8 * 48)
    assert np.array_equal(np.sign(th[0]).ravel(), s[:1024])
    assert np.array_equal(np.sign(th[1]).ravel(), s[1024:])


def test_sketch_equals_kronecker_form():
    """vec(S(X)) = (Theta_d kron ... kron Theta_1) vec(X) (Section 3, vectorised form)."""
    dims, sk = (6, 5, 3, 4), (3, 2, 3, 2)
    th = oracle.sketch_matrices(dims, sk, seed=9)
    X = _rng(7).standard_normal(dims)
    lhs = oracle.sketch(X, th).ravel(order="F")
    rhs = oracle.sketch_dense_matrix(dims, th) @ X.ravel(order="F")
    assert lhs.shape == (3 * 2 * 3 * 2,)
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-12)


def test_sketch_embedding_in_expectation():
    """E ||S(X)||^2 = ||X||^2 for Rademacher +-1/sqrt(s) sketches (norm-form embedding,
    Section 3.2): checked statistically over seeds; only the distribution is pinned."""
    X = _rng(8).standard_normal((32, 24, 3))
    ratios = []
    for seed in range(200):
        th = oracle.sketch_matrices(X.shape, (8, 8, 3), seed=seed)
        ratios.append(oracle.frobenius_norm(oracle.sketch(X, th)) ** 2 / oracle.frobenius_norm(X) ** 2)
    ratios = np.array(ratios)
    assert abs(ratios.mean() - 1.0) < 4 * ratios.std() / np.sqrt(len(ratios))
    # larger sketches concentrate better
    r2 = []
    for seed in range(60):
        th = oracle.sketch_matrices(X.shape, (24, 20, 3), seed=seed)
        r2.append(oracle.frobenius_norm(oracle.sketch(X, th)) ** 2 / oracle.frobenius_norm(X) ** 2)
    assert np.std(r2) < ratios.std()


def test_noise_level_exact():
    import workloads as w
    x = w.piecewise_image(16, 16, 3, seed=1)
    mats = oracle.factor_matrices(x.shape, [(1, "banded", w.gaussian_taps(1.0, 2))])
    C, Ch, nuC = oracle.make_observation(x, mats, w.noise_draw(x.shape, 1), 1e-2)
    assert abs(oracle.frobenius_norm(C - Ch) / oracle.frobenius_norm(Ch) - 1e-2) < 1e-14
    assert abs(nuC - oracle.frobenius_norm(C - Ch) / oracle.frobenius_norm(C)) < 1e-15


def test_psnr_re_definitions():
    x = np.array([0.0, 1.0, 2.0, 3.0])
    y = x + np.array([0.1, -0.1, 0.0, 0.0])
    assert abs(oracle.relative_error(x, y) - np.sqrt(0.02) / np.sqrt(14.0)) < 1e-15
    # ||x - mean||^2 = 5, ||y - x||^2 = 0.02
    assert abs(oracle.psnr(x, y) - 10 * np.log10(5 / 0.02)) < 1e-12
