"""Pins for the oracle's sketched Golub-Kahan process (CPU only).

What fixes the oracle here is mathematics it does not contain: the
adjoint identity <Phi X, Y> = <X, Phi^T Y> for the transposed mode
matrices; with Theta = I, the orthonormality of both Golub-Kahan bases
(a property of the bidiagonalisation, not of the code's construction) and
the equality of the least-squares iterate with the minimiser of
||C - Phi(X)|| over X_0 + K_k(Phi^T Phi, Phi^T R_0), computed from an
explicit Krylov basis of the dense vectorised operator; at full dimension
the exact least-squares solution.  A planted mistake (Phi in place of
Phi^T with a non-symmetric operator) fails the orthonormality pin.
"""
import numpy as np
import pytest

import oracle
from oracle import golub_kahan as GK
import workloads as w


def _nonsym_problem(dims=(7, 6, 3), seed=0):
    rng = np.random.default_rng(seed)
    t1 = rng.uniform(0.1, 1.0, 5)          # asymmetric taps
    t2 = rng.uniform(0.1, 1.0, 3)
    M3 = rng.standard_normal((3, 3)) + 3 * np.eye(3)
    mats = oracle.factor_matrices(dims, [(1, "banded", t1), (2, "banded", t2)], [(3, "dense", M3)])
    C = rng.standard_normal(dims)
    return mats, C


def _identity_thetas(dims):
    return oracle.sketch_matrices(dims, dims, seed=0)   # s_k = I_k: no mode sketched


def test_transposed_mats_give_the_adjoint():
    mats, _ = _nonsym_problem()
    rng = np.random.default_rng(1)
    X = rng.standard_normal((7, 6, 3))
    Y = rng.standard_normal((7, 6, 3))
    lhs = np.vdot(oracle.apply_operator(X, mats).ravel(), Y.ravel())
    rhs = np.vdot(X.ravel(), oracle.apply_operator(Y, GK.transpose_mats(mats)).ravel())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _gk(mats, C, th, m, phit_mats=None):
    phi = lambda X: oracle.apply_operator(X, mats)
    tm = GK.transpose_mats(mats) if phit_mats is None else phit_mats
    phit = lambda X: oracle.apply_operator(X, tm)
    S = lambda X: oracle.sketch(X, th)
    return GK.sketched_golub_kahan(phi, phit, C, m, S)


def _gram(vs):
    M = np.stack([v.ravel() for v in vs], axis=1)
    return M.T @ M


def test_identity_sketch_bases_are_orthonormal():
    mats, C = _nonsym_problem()
    gk = _gk(mats, C, _identity_thetas(C.shape), 6)
    for basis in (gk["U"], gk["V"]):
        G = _gram(basis)
        assert np.max(np.abs(G - np.eye(len(basis)))) < 1e-10


def test_forward_and_backward_relations():
    mats, C = _nonsym_problem()
    th = oracle.sketch_matrices(C.shape, (4, 3, 3), seed=2)      # sketched: relations still hold
    gk = _gk(mats, C, th, 5)
    B, U, V = gk["B"], gk["U"], gk["V"]
    tm = GK.transpose_mats(mats)
    for j in range(gk["k"]):
        lhs = oracle.apply_operator(V[j], mats)
        rhs = B[j, j] * U[j] + B[j + 1, j] * U[j + 1]
        assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(lhs)
    for j in range(gk["k"] - 1):
        lhs = oracle.apply_operator(U[j + 1], tm)
        rhs = B[j + 1, j] * V[j] + B[j + 1, j + 1] * V[j + 1]
        assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(lhs)
    for x in U + V:   # unit Theta-norm
        assert abs(np.linalg.norm(oracle.sketch(x, th)) - 1.0) < 1e-12


def _dense_op(mats, dims):
    n = int(np.prod(dims))
    A = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        A[:, i] = oracle.apply_operator(e.reshape(dims, order="F"), mats).ravel(order="F")
    return A


@pytest.mark.parametrize("k", [1, 3, 5, 8])
def test_identity_sketch_iterate_is_the_krylov_least_squares_minimiser(k):
    mats, C = _nonsym_problem()
    dims = C.shape
    A = _dense_op(mats, dims)
    res = GK.sketched_gk_solve(mats, C, k, _identity_thetas(dims), tol=0.0, lam=0.0)
    c = C.ravel(order="F")
    # explicit Krylov basis of A^T A on A^T c, orthonormalised
    K = [A.T @ c]
    for _ in range(k - 1):
        K.append(A.T @ (A @ K[-1]))
    Q, _ = np.linalg.qr(np.stack(K, axis=1))
    z = np.linalg.lstsq(A @ Q, c, rcond=None)[0]
    x = Q @ z
    got = res["X"].ravel(order="F")
    assert np.linalg.norm(got - x) <= 1e-8 * np.linalg.norm(x)


def test_full_dimension_gives_the_solution_of_a_well_conditioned_system():
    """n steps on an n-dimensional, well-conditioned (cond ~ 2.8) non-symmetric
    operator reach the exact solution: with few steps the short recurrences
    keep their orthogonality (on ill-conditioned operators they lose it after
    some ten steps, as Golub-Kahan without re-orthogonalisation does)."""
    dims = (4, 3, 2)
    mats = oracle.factor_matrices(dims, [(1, "banded", np.array([0.1, 1.0, 0.25])),
                                         (2, "banded", np.array([0.2, 1.0, 0.05]))],
                                  [(3, "dense", np.array([[1.0, 0.3], [-0.2, 1.0]]))])
    C = np.random.default_rng(0).standard_normal(dims)
    A = _dense_op(mats, dims)
    res = GK.sketched_gk_solve(mats, C, 24, _identity_thetas(dims), tol=0.0, lam=0.0)
    x = np.linalg.solve(A, C.ravel(order="F"))
    assert np.linalg.norm(res["X"].ravel(order="F") - x) <= 1e-10 * np.linalg.norm(x)


def test_rho_is_the_projected_least_squares_residual():
    mats, C = _nonsym_problem()
    th = oracle.sketch_matrices(C.shape, (4, 3, 3), seed=3)
    res = GK.sketched_gk_solve(mats, C, 5, th, tol=0.0, lam=0.0)
    r, _ = oracle.ls_residual(res["B"], res["beta"])
    assert abs(res["rho"][-1] - r / res["beta"]) <= 1e-12


def test_gcv_and_fixed_mu_run_on_the_bidiagonal():
    p = w.image_config(1)
    mats = oracle.factor_matrices(p.dims, p.factors, p.right_factors)
    C, _, nu_c = oracle.make_observation(p.x_true, mats, p.noise, p.nu)
    th = oracle.sketch_matrices(p.dims, p.sketch_dims, 0, 0)
    r1 = GK.sketched_gk_solve(mats, C, 8, th, lam=1e-3)
    r2 = GK.sketched_gk_solve(mats, C, 8, th, lam=-1.0, mu_grid=w.mu_grid())
    assert r1["mu"] == 1e-3 and r2["mu"] in list(w.mu_grid())
    y = oracle.tikhonov_stacked(r1["B"], r1["beta"], 1e-3)
    assert np.allclose(y, r1["y"])


def test_pin_catches_forward_operator_in_the_backward_step():
    mats, C = _nonsym_problem()
    gk = _gk(mats, C, _identity_thetas(C.shape), 6, phit_mats=mats)   # planted: Phi instead of Phi^T
    G = _gram(gk["V"])
    assert np.max(np.abs(G - np.eye(len(gk["V"])))) > 1e-3
