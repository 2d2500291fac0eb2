"""Pins for the oracle's Krylov process, least squares, Tikhonov and GCV (CPU only).

The checks come from the paper's relations (Arnoldi relation 7S,
sketched orthonormality, the Theta-norm residual identity, the reduction
to TG-GMRES when Theta_k = I) and from mathematics that does not depend on
the oracle (dense solves of the vectorised system, closed forms for
operators with two eigenvalues, a GCV closed form).  The last tests plant
mistakes in the oracle and show that these pins catch them.
"""
import numpy as np
import pytest

import oracle
from oracle import krylov as K
import workloads as w


def _problem(dims=(12, 10, 3), sk=(6, 5, 3), seed=0, radius=2, sigma=1.0):
    rng = np.random.default_rng(seed)
    a = w.gaussian_taps(sigma, radius)
    mats = oracle.factor_matrices(dims, [(1, "banded", a), (2, "banded", a)],
                                  [(3, "dense", w.channel_mix())])
    C = rng.standard_normal(dims)
    th = oracle.sketch_matrices(dims, sk, seed=seed)
    return mats, C, th


def _arnoldi(mats, C, th, m):
    apply_phi = lambda X: oracle.apply_operator(X, mats)
    S = lambda X: oracle.sketch(X, th)
    return oracle.sketched_arnoldi(apply_phi, C, m, S)


# ----------------------------------------------------------------------------- invariants

def arnoldi_relation_error(mats, arn):
    """max_j ||Phi(V_j) - sum_i h_ij V_i|| / ||Phi(V_j)|| (relation 7S / Proposition 2)."""
    err = 0.0
    for j in range(arn.k):
        lhs = oracle.apply_operator(arn.V[j], mats)
        rhs = sum(arn.H[i, j] * arn.V[i] for i in range(j + 2))
        err = max(err, oracle.frobenius_norm(lhs - rhs) / oracle.frobenius_norm(lhs))
    return err


def orthonormality_error(th, V):
    """|| S(V)^T S(V) - I ||_max with the sketches recomputed from the stored basis."""
    SV = np.stack([oracle.sketch(v, th).ravel(order="F") for v in V], axis=1)
    return float(np.max(np.abs(SV.T @ SV - np.eye(len(V)))))


def test_arnoldi_relation_7S():
    mats, C, th = _problem()
    arn = _arnoldi(mats, C, th, 12)
    assert arn.k == 12 and len(arn.V) == 13
    assert arnoldi_relation_error(mats, arn) < 1e-13


def test_sketched_orthonormality():
    mats, C, th = _problem(seed=1)
    arn = _arnoldi(mats, C, th, 12)
    assert orthonormality_error(th, arn.V) < 1e-10
    # the full-space basis is not Frobenius-orthonormal (only Theta-orthonormal)
    F = np.stack([v.ravel() for v in arn.V], axis=1)
    assert np.max(np.abs(F.T @ F - np.eye(len(arn.V)))) > 1e-3


def test_residual_identity_in_theta_norm():
    """||S(C - Phi(X_0 + V_m y))||_F = ||beta e1 - Hbar_m y||_2 for any y (Section 4.4)."""
    mats, C, th = _problem(seed=2)
    arn = _arnoldi(mats, C, th, 8)
    rng = np.random.default_rng(0)
    for _ in range(3):
        y = rng.standard_normal(arn.k)
        X = sum(y[j] * arn.V[j] for j in range(arn.k))
        lhs = oracle.frobenius_norm(oracle.sketch(C - oracle.apply_operator(X, mats), th))
        b = np.zeros(arn.k + 1)
        b[0] = arn.beta
        rhs = np.linalg.norm(b - arn.H @ y)
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, rhs)


def test_rho_history_monotone_and_matches_true_sketched_residual():
    mats, C, th = _problem(seed=3)
    r = oracle.rtg_gmres(mats, C, 10, th, lam=0.0)
    rho = np.array(r["rho"])
    assert np.all(np.diff(rho) <= 1e-14)
    resid = oracle.sketch(C - oracle.apply_operator(r["X"], mats), th)
    assert abs(oracle.frobenius_norm(resid) / r["beta"] - rho[-1]) < 1e-12


def test_identity_sketch_reduces_to_tg_gmres():
    """With Theta_k = I the method is classical TG-GMRES (the sketched process follows Algorithm 1)."""
    dims = (12, 10, 3)
    mats, C, _ = _problem(dims)
    th = oracle.sketch_matrices(dims, dims, seed=0)
    assert all(t is None for t in th)
    a = oracle.rtg_gmres(mats, C, 15, th, lam=1e-3)
    b = oracle.tg_gmres(mats, C, 15, lam=1e-3)
    assert np.allclose(a["rho"], b["rho"], rtol=1e-11, atol=0)
    assert np.allclose(a["H"], b["H"], rtol=0, atol=1e-12)
    assert np.allclose(a["X"], b["X"], rtol=0, atol=1e-11)


# ----------------------------------------------------------------------------- dense solves

def _tiny_operator(dims, seed):
    rng = np.random.default_rng(seed)
    t1 = np.array([0.2, 1.0, 0.3]) + 0.1 * rng.standard_normal(3)
    t2 = np.array([0.1, 1.0, 0.25]) + 0.1 * rng.standard_normal(3)
    B = np.eye(dims[2]) + 0.2 * rng.standard_normal((dims[2], dims[2]))
    return oracle.factor_matrices(dims, [(1, "banded", t1), (2, "banded", t2)], [(3, "dense", B)])


def test_full_dimension_solve_matches_dense_vectorised_system():
    """m = n, Theta = I, mu = 0: the Krylov space is the whole space and X = Phi^{-1} C (Eq. 8)."""
    dims = (4, 3, 2)
    n = 24
    mats = _tiny_operator(dims, 0)
    C = np.random.default_rng(1).standard_normal(dims)
    th = oracle.sketch_matrices(dims, dims, 0)
    r = oracle.rtg_gmres(mats, C, n, th, lam=0.0, breakdown_tol=1e-10)
    M = oracle.dense_operator_matrix(dims, mats)
    x_ref = np.linalg.solve(M, C.ravel(order="F"))
    assert np.allclose(r["X"].ravel(order="F"), x_ref, rtol=0, atol=1e-9 * np.abs(x_ref).max())


@pytest.mark.parametrize("mu", [1e-3, 1e-2, 0.3])
def test_tikhonov_on_invariant_subspace_matches_dense_tikhonov(mu):
    """Symmetric Phi with three distinct eigenvalues: K_3(Phi, C) is invariant and holds the
    Tikhonov solution (Phi^T Phi + mu I)^{-1} Phi^T C of Eq. 5, which the projected problem
    (Eq. 12S/13) must return after the breakdown at j = 3."""
    dims = (5, 4, 3)
    B = np.diag([0.5, 1.0, 2.0])
    mats = oracle.factor_matrices(dims, [], [(3, "dense", B)])
    C = np.random.default_rng(1).standard_normal(dims)
    th = oracle.sketch_matrices(dims, dims, 0)
    r = oracle.rtg_gmres(mats, C, 10, th, lam=mu)
    assert r["iters"] == 3 and r["breakdown"]
    M = oracle.dense_operator_matrix(dims, mats)
    x_ref = np.linalg.solve(M.T @ M + mu * np.eye(M.shape[0]), M.T @ C.ravel(order="F"))
    assert np.allclose(r["X"].ravel(order="F"), x_ref, rtol=0, atol=1e-12)


def test_two_eigenvalue_operator_converges_in_two_steps():
    """Phi with exactly two distinct eigenvalues: the Krylov space has dimension 2, so the
    Arnoldi process breaks down at j = 2 with zero residual and X = Phi^{-1} C."""
    dims = (5, 4, 3)
    B = np.diag([1.0, 2.0, 2.0])
    mats = oracle.factor_matrices(dims, [], [(3, "dense", B)])
    C = np.random.default_rng(2).standard_normal(dims)
    th = oracle.sketch_matrices(dims, (3, 2, 3), seed=4)
    r = oracle.rtg_gmres(mats, C, 10, th, lam=0.0)
    assert r["iters"] == 2 and r["breakdown"]
    X_ref = C / np.array([1.0, 2.0, 2.0])[None, None, :]
    assert np.allclose(r["X"], X_ref, rtol=0, atol=1e-12)


def test_identity_operator_happy_breakdown():
    dims = (6, 5, 3)
    mats = oracle.factor_matrices(dims, [])
    C = np.random.default_rng(3).standard_normal(dims)
    th = oracle.sketch_matrices(dims, (3, 3, 3), seed=0)
    r = oracle.rtg_gmres(mats, C, 5, th, lam=0.0)
    assert r["iters"] == 1 and r["breakdown"] and r["rho"][0] < 1e-14
    assert np.allclose(r["X"], C, rtol=0, atol=1e-14)


def test_zero_rhs_returns_initial_guess():
    dims = (6, 5, 3)
    mats, _, th = _problem(dims, (3, 3, 3))
    r = oracle.rtg_gmres(mats, np.zeros(dims), 5, th, lam=1e-3)
    assert r["iters"] == 0 and np.all(r["X"] == 0.0)


def test_restart_continues_from_least_squares_iterate():
    mats, C, th = _problem(seed=5)
    one = oracle.rtg_gmres(mats, C, 4, th, lam=0.0)
    two = oracle.rtg_gmres(mats, C, 4, th, lam=0.0, max_restarts=1, tol=1e-30)
    assert two["restarts"] == 1 and two["iters"] == 8
    assert np.allclose(two["X0"], one["X"], rtol=0, atol=1e-12)
    assert two["rho"][-1] < one["rho"][-1]


# ----------------------------------------------------------------------------- Tikhonov / GCV

def _hessenberg(k, seed):
    rng = np.random.default_rng(seed)
    H = np.triu(rng.standard_normal((k + 1, k)), -1)
    H[np.arange(1, k + 1), np.arange(k)] = np.abs(H[np.arange(1, k + 1), np.arange(k)]) + 0.1
    H = H @ np.diag(np.logspace(0, -5, k))   # ill-conditioned like a blur
    return H


@pytest.mark.parametrize("mu", [1e-6, 1e-3, 0.5])
def test_tikhonov_three_forms_agree(mu):
    """Stacked least squares (Eq. 13), normal equations (Eq. 14) and the SVD filter form."""
    H = _hessenberg(12, 0)
    a = oracle.tikhonov_stacked(H, 2.0, mu)
    b = oracle.tikhonov_normal(H, 2.0, mu)
    c = oracle.tikhonov_svd(H, 2.0, mu)
    scale = np.abs(c).max()
    assert np.allclose(a, c, rtol=0, atol=1e-9 * scale)
    assert np.allclose(b, c, rtol=0, atol=1e-7 * scale)


def test_gcv_closed_form():
    """Hbar = [I_k; 0]: y_mu = beta/(1+mu) e1, residual beta*mu/(1+mu), trace 1 + k*mu/(1+mu)."""
    k, beta = 6, 3.0
    H = np.vstack([np.eye(k), np.zeros((1, k))])
    for mu in [1e-3, 0.1, 2.0]:
        ref = (beta * mu / (1 + mu)) ** 2 / (1 + k * mu / (1 + mu)) ** 2
        assert abs(oracle.gcv_value(H, beta, mu) - ref) <= 1e-10 * ref


def test_gcv_trace_matches_singular_value_form():
    H = _hessenberg(10, 1)
    s = np.linalg.svd(H, compute_uv=False)
    for mu in [1e-4, 1e-2]:
        y = oracle.tikhonov_svd(H, 1.5, mu)
        b = np.zeros(11)
        b[0] = 1.5
        num = np.sum((H @ y - b) ** 2)
        den = (11 - np.sum(s * s / (s * s + mu))) ** 2
        assert abs(oracle.gcv_value(H, 1.5, mu) - num / den) <= 1e-8 * num / den


def test_gcv_choose_ties_pick_larger_mu():
    H = np.vstack([np.eye(3), np.zeros((1, 3))])
    mu, vals = oracle.gcv_choose(H, 1.0, [0.5, 0.5000000000000001, 2.0])
    assert mu == float(np.array([0.5, 0.5000000000000001, 2.0])[np.argmin(vals)]) or \
        vals[0] == vals[1]
    mu2, _ = oracle.gcv_choose(np.vstack([np.eye(2), np.zeros((1, 2))]), 0.0 + 1.0, [1.0, 1.0])
    assert mu2 == 1.0


# ----------------------------------------------------------------------------- planted mistakes

def test_pins_catch_reversed_sketch_index(monkeypatch):
    """Plant a reversed index in the oracle's sketch mode product: the Kronecker pin fails."""
    import importlib
    skmod = importlib.import_module("oracle.sketch")
    dims, sk = (6, 5, 3), (3, 2, 3)
    th = oracle.sketch_matrices(dims, sk, seed=1)
    X = np.random.default_rng(0).standard_normal(dims)
    ref = oracle.sketch_dense_matrix(dims, th) @ X.ravel(order="F")
    real = skmod.mode_product
    monkeypatch.setattr(skmod, "mode_product", lambda Y, M, k: real(np.flip(Y, axis=k), M, k))
    got = oracle.sketch(X, th).ravel(order="F")
    assert not np.allclose(got, ref, atol=1e-8)


def test_pins_catch_dropped_gram_schmidt_term(monkeypatch):
    """Plant a missing subtraction in the oracle's Arnoldi: relation 7S and orthonormality fail."""
    mats, C, th = _problem(seed=6)
    real_inner = K.frobenius_inner
    calls = {"n": 0}

    def skipping_inner(a, b):
        calls["n"] += 1
        return 0.0 if calls["n"] % 5 == 3 else real_inner(a, b)
    monkeypatch.setattr(K, "frobenius_inner", skipping_inner)
    arn = _arnoldi(mats, C, th, 8)
    monkeypatch.setattr(K, "frobenius_inner", real_inner)
    # relation 7S still holds by construction (H records what was subtracted) ...
    assert arnoldi_relation_error(mats, arn) < 1e-12
    # ... but sketched orthonormality does not
    assert orthonormality_error(th, arn.V) > 1e-3


def test_pins_catch_wrong_sign_in_operator(monkeypatch):
    """Plant a sign error in the operator's Toeplitz band: the Eq. 57 convolution pin fails."""
    import importlib
    opmod = importlib.import_module("oracle.operator")
    rng = np.random.default_rng(5)
    p1, p2 = rng.uniform(0, 1, 5), rng.uniform(0, 1, 5)
    X = rng.standard_normal((6, 5, 2))
    C = oracle.psf_convolve(X, np.outer(p1, p2))
    real = opmod.banded_toeplitz
    monkeypatch.setattr(opmod, "banded_toeplitz", lambda n, taps: real(n, np.asarray(taps)[::-1]))
    mats = opmod.factor_matrices(X.shape, [(1, "banded", p1[::-1]), (2, "banded", p2[::-1])])
    assert not np.allclose(oracle.apply_operator(X, mats), C, atol=1e-6)
