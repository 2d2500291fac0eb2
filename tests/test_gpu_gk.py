"""Sketched Golub-Kahan on the GPU (rtg_gk_solve) against the FP64 oracle.

Same tolerances as RTG-GMRES: 1e-9 relative in FP64 (the arithmetic
differs from the oracle's only in summation order), 1e-4 in FP32 (the
sketch sums and the basis in FP32).  A non-symmetric operator (asymmetric
taps, non-symmetric channel matrix) checks that the adjoint Phi^T is used
where the algorithm asks for it.
"""
import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_00839_gb300 import api
    return api.Handle(0)


def _api():
    from paper_2603_00839_gb300 import api
    return api


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _factors(factors, right, dims):
    api = _api()
    A = [api.banded(m, dims[m - 1], t) if k == "banded" else api.dense(m, t) for m, k, t in factors]
    B = [api.banded(m, dims[m - 1], t) if k == "banded" else api.dense(m, t) for m, k, t in right]
    return A, B


def test_gk_image64_f64_matches_oracle(h):
    api = _api()
    p = w.image_config(1)
    mats = oracle.factor_matrices(p.dims, p.factors, p.right_factors)
    C, _, nu_c = oracle.make_observation(p.x_true, mats, p.noise, p.nu)
    th = oracle.sketch_matrices(p.dims, p.sketch_dims, 0, 0)
    ref = oracle.sketched_gk_solve(mats, C, p.m, th, tol=1e-3, lam=p.lam)
    A, B = _factors(p.factors, p.right_factors, p.dims)
    X, info = h.gk_solve(api.to_device(C, torch.float64), p.m, p.sketch_dims, 0, p.lam, A, B, tol=1e-3)
    assert info.iters == ref["iters"] and info.device_status == 0
    assert np.max(np.abs(info.rho - np.array(ref["rho"])) / np.array(ref["rho"])) < 1e-9
    assert _rel(X.cpu().numpy(), ref["X"]) < 1e-9


def test_gk_nonsymmetric_operator_f64(h):
    api = _api()
    rng = np.random.default_rng(7)
    dims = (40, 36, 3)
    t1 = rng.uniform(0.1, 1.0, 7)
    t2 = rng.uniform(0.1, 1.0, 5)
    M3 = rng.standard_normal((3, 3)) + 3 * np.eye(3)
    f = [(1, "banded", t1), (2, "banded", t2)]
    r = [(3, "dense", M3)]
    mats = oracle.factor_matrices(dims, f, r)
    C = rng.standard_normal(dims)
    sk = (16, 12, 3)
    th = oracle.sketch_matrices(dims, sk, 3, 0)
    ref = oracle.sketched_gk_solve(mats, C, 12, th, tol=0.0, lam=0.0)
    A, B = _factors(f, r, dims)
    X, info = h.gk_solve(api.to_device(C, torch.float64), 12, sk, 3, 0.0, A, B, tol=0.0)
    assert info.iters == ref["iters"]
    assert np.max(np.abs(info.rho - np.array(ref["rho"])) / np.array(ref["rho"])) < 1e-9
    assert _rel(X.cpu().numpy(), ref["X"]) < 1e-9


def test_gk_image512_f32_gcv_matches_oracle(h):
    api = _api()
    p = w.image_config(2)
    mats = oracle.factor_matrices(p.dims, p.factors, p.right_factors)
    C, _, nu_c = oracle.make_observation(p.x_true, mats, p.noise, p.nu)
    th = oracle.sketch_matrices(p.dims, p.sketch_dims, p.seed, 0)
    tol = max(1e-3, 1.01 * nu_c)
    ref = oracle.sketched_gk_solve(mats, C, p.m, th, tol=tol, lam=-1.0, mu_grid=p.mu_grid)
    A, B = _factors(p.factors, p.right_factors, p.dims)
    X, info = h.gk_solve(api.to_device(C, torch.float32), p.m, p.sketch_dims, p.seed, -1.0, A, B,
                         tol=tol, mu_grid=p.mu_grid)
    assert info.iters == ref["iters"]
    assert info.mu == ref["mu"]
    assert np.max(np.abs(info.rho - np.array(ref["rho"])) / np.array(ref["rho"])) < 1e-4
    assert _rel(X.cpu().double().numpy(), ref["X"]) < 1e-4


def test_gk_graph_direct_and_initial_guess(h):
    api = _api()
    p = w.image_config(1)
    mats = oracle.factor_matrices(p.dims, p.factors, p.right_factors)
    C, _, nu_c = oracle.make_observation(p.x_true, mats, p.noise, p.nu)
    A, B = _factors(p.factors, p.right_factors, p.dims)
    Cd = api.to_device(C, torch.float64)
    Xg, ig = h.gk_solve(Cd, 10, p.sketch_dims, 0, 1e-2, A, B, tol=0.0)
    Xd, idr = h.gk_solve(Cd, 10, p.sketch_dims, 0, 1e-2, A, B, tol=0.0, use_graph=False)
    assert ig.iters == idr.iters == 10
    assert np.array_equal(Xg.cpu().numpy(), Xd.cpu().numpy())
    X0 = 0.5 * p.x_true
    th = oracle.sketch_matrices(p.dims, p.sketch_dims, 0, 0)
    ref = oracle.sketched_gk_solve(mats, C, 10, th, X0=X0, tol=0.0, lam=1e-2)
    X, info = h.gk_solve(Cd, 10, p.sketch_dims, 0, 1e-2, A, B, X0=api.to_device(X0, torch.float64), tol=0.0)
    assert _rel(X.cpu().numpy(), ref["X"]) < 1e-9


def test_gk_zero_rhs_returns_initial_guess(h):
    api = _api()
    p = w.image_config(1)
    A, B = _factors(p.factors, p.right_factors, p.dims)
    C = api.to_device(np.zeros(p.dims), torch.float64)
    X0 = api.to_device(np.ones(p.dims), torch.float64)
    Y = h.operator_apply(X0, A, B)       # C = Phi(X0): R_0 = 0
    X, info = h.gk_solve(Y, 8, p.sketch_dims, 0, 0.0, A, B, X0=X0, tol=0.0)
    assert info.converged and info.iters == 0
    assert np.array_equal(X.cpu().numpy(), X0.cpu().numpy())


def test_gk_video_f32_matches_oracle(h):
    api = _api()
    p = w.video_config(seed=2, I=64, frames=8)
    mats = oracle.factor_matrices(p.dims, p.factors, p.right_factors)
    C, _, nu_c = oracle.make_observation(p.x_true, mats, p.noise, p.nu)
    th = oracle.sketch_matrices(p.dims, p.sketch_dims, p.seed, 0)
    ref = oracle.sketched_gk_solve(mats, C, 15, th, tol=0.0, lam=1e-3)
    A, B = _factors(p.factors, p.right_factors, p.dims)
    X, info = h.gk_solve(api.to_device(C, torch.float32), 15, p.sketch_dims, p.seed, 1e-3, A, B, tol=0.0)
    assert info.iters == ref["iters"]
    assert np.max(np.abs(info.rho - np.array(ref["rho"])) / np.array(ref["rho"])) < 1e-4
    assert _rel(X.cpu().double().numpy(), ref["X"]) < 1e-4
