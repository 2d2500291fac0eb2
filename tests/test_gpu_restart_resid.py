"""GPU parity of restarted RTG-GMRES, the final true residual and the
non-finite checks.

Restarts (the Block GMRES algorithm run again from its least-squares
iterate) are compared with the oracle's restarted solve: the concatenated
rho history, the restart count and X (FP64: 1e-9; FP32: 1e-4).  The true
residual of the algorithm's last steps (R_m = C - A *_N X_m, Section 4.4)
is compared with its definition evaluated in FP64 on the GPU's own X, and
with the oracle's.  Non-finite data must end the solve with
RTG_ERR_NONFINITE in info.device_status, never a fault.
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


def _relnorm(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _small_problem(dims=(64, 48, 3), sk=(24, 16, 3), nu=5e-3, seed=4):
    a = w.gaussian_taps(1.5, 4)
    fac = [(1, "banded", a), (2, "banded", a)]
    rfac = [(3, "dense", w.channel_mix())]
    mats = oracle.factor_matrices(dims, fac, rfac)
    x = w.piecewise_image(dims[0], dims[1], dims[2], seed=seed)
    C, _, nu_c = oracle.make_observation(x, mats, w.noise_draw(dims, seed), nu)
    th = oracle.sketch_matrices(dims, sk, 2)
    api = _api()
    A = [api.banded(1, dims[0], a), api.banded(2, dims[1], a)]
    B = [api.dense(3, w.channel_mix())]
    return mats, C, th, A, B, sk


# ------------------------------------------------------------------------ restarts

@pytest.mark.parametrize("lam", [0.0, 2e-3, -1.0])
def test_restarted_solve_matches_oracle_f64(h, lam):
    mats, C, th, A, B, sk = _small_problem()
    grid = w.mu_grid(8) if lam < 0 else None
    m, R = 4, 3
    ref = oracle.rtg_gmres(mats, C, m, th, tol=1e-6, lam=lam, mu_grid=grid, max_restarts=R)
    assert ref["restarts"] == R and ref["iters"] == m * (R + 1)
    api = _api()
    X, info = h.gmres_solve(api.to_device(C, torch.float64), m, sk, 2, lam, A, B, tol=1e-6,
                            mu_grid=grid, max_restarts=R)
    assert info.device_status == 0
    assert info.restarts == ref["restarts"] and info.iters == ref["iters"]
    assert np.allclose(info.rho, ref["rho"], rtol=1e-9, atol=0)
    assert info.mu == ref["mu"]
    assert _relnorm(X.cpu().numpy(), ref["X"]) < 1e-9


def test_restarted_solve_stops_in_a_later_cycle(h):
    """tol met in the second cycle: one restart, converged, and the same
    result through the direct-launch path and with X aliasing X0."""
    mats, C, th, A, B, sk = _small_problem()
    m = 4
    full = oracle.rtg_gmres(mats, C, m, th, tol=0.0, lam=0.0, max_restarts=2)
    tol = 0.5 * (full["rho"][m - 1] + full["rho"][2 * m - 1])   # between the two cycle ends
    ref = oracle.rtg_gmres(mats, C, m, th, tol=tol, lam=1e-3, max_restarts=2)
    assert ref["restarts"] == 1 and ref["converged"]
    api = _api()
    Cd = api.to_device(C, torch.float64)
    X, info = h.gmres_solve(Cd, m, sk, 2, 1e-3, A, B, tol=tol, max_restarts=2)
    assert info.restarts == 1 and info.converged and info.iters == ref["iters"]
    assert np.allclose(info.rho, ref["rho"], rtol=1e-9, atol=0)
    assert _relnorm(X.cpu().numpy(), ref["X"]) < 1e-9
    Xd, idr = h.gmres_solve(Cd, m, sk, 2, 1e-3, A, B, tol=tol, max_restarts=2, use_graph=False)
    assert idr.iters == info.iters and np.array_equal(Xd.cpu().numpy(), X.cpu().numpy())
    X0 = 0.25 * np.ones(C.shape)
    ref0 = oracle.rtg_gmres(mats, C, m, th, X0=X0, tol=0.0, lam=1e-3, max_restarts=2)
    Xa = api.to_device(X0, torch.float64)
    Xa, ia = h.gmres_solve(Cd, m, sk, 2, 1e-3, A, B, X0=Xa, X=Xa, max_restarts=2)
    assert ia.restarts == 2 and np.allclose(ia.rho, ref0["rho"], rtol=1e-9, atol=0)
    assert _relnorm(Xa.cpu().numpy(), ref0["X"]) < 1e-9


def test_restarted_solve_f32_and_batched(h):
    """FP32 restarted solve against the oracle (1e-4) and the batched form
    (one graph branch per problem and a lock-step group) against the single
    solve, bit for bit."""
    mats, C, th, A, B, sk = _small_problem(dims=(96, 80, 3), sk=(32, 24, 3), seed=6)
    m, R = 6, 2
    ref = oracle.rtg_gmres(mats, C, m, th, tol=1e-7, lam=2e-3, max_restarts=R)
    api = _api()
    Cd = api.to_device(C, torch.float32)
    X, info = h.gmres_solve(Cd, m, sk, 2, 2e-3, A, B, tol=1e-7, max_restarts=R)
    assert info.restarts == R == ref["restarts"] and info.device_status == 0
    assert np.allclose(info.rho, ref["rho"], rtol=1e-4, atol=0)
    assert _relnorm(X.cpu().double().numpy(), ref["X"]) < 1e-4
    probs = [dict(C=Cd, A=A, B=B, m=m, sketch_dims=sk, seed=2, lam=2e-3, tol=1e-7) for _ in range(3)]
    for gmax in (0, 3):
        Xs, res = h.gmres_solve_batched(probs, max_restarts=R, group_max=gmax)
        for Xb, rb in zip(Xs, res):
            assert rb.restarts == R and rb.iters == info.iters
            assert np.array_equal(rb.rho, info.rho)
            assert np.array_equal(Xb.cpu().numpy(), X.cpu().numpy())


# ------------------------------------------------------------------------ true residual

@pytest.mark.parametrize("dt,bar", [(torch.float64, 1e-10), (torch.float32, 1e-4)])
def test_true_residual_matches_definition(h, dt, bar):
    mats, C, th, A, B, sk = _small_problem()
    api = _api()
    X, info = h.gmres_solve(api.to_device(C, dt), 20, sk, 2, 2e-3, A, B, tol=0.0, true_residual=True)
    Xh = X.cpu().double().numpy()
    R = C - oracle.apply_operator(Xh, mats)
    assert info.true_rel_resid > 0
    assert abs(info.true_rel_resid - np.linalg.norm(R) / np.linalg.norm(C)) <= bar * info.true_rel_resid
    beta0 = np.linalg.norm(oracle.sketch(C, th))
    th_ref = np.linalg.norm(oracle.sketch(R, th)) / beta0
    assert abs(info.true_rel_resid_theta - th_ref) <= bar * th_ref
    # the oracle's own solve gives the same residuals within the bar of its iterate
    ref = oracle.rtg_gmres(mats, C, 20, th, tol=0.0, lam=2e-3)
    Rr = C - oracle.apply_operator(ref["X"], mats)
    assert abs(info.true_rel_resid - np.linalg.norm(Rr) / np.linalg.norm(C)) <= 10 * bar * info.true_rel_resid
    # without the flag the fields stay -1
    _, i2 = h.gmres_solve(api.to_device(C, dt), 20, sk, 2, 2e-3, A, B, tol=0.0)
    assert i2.true_rel_resid == -1.0 and i2.true_rel_resid_theta == -1.0


def test_true_residual_full_size_image512_and_batched(h):
    """512x512x3 FP32 workload (GCV, stop at rho*): the true residual of the
    returned X against its FP64 evaluation; the batched form gives the same
    values bit for bit."""
    p = w.image_config(2)
    mats = oracle.factor_matrices(p.dims, p.factors, p.right_factors)
    C, _, nu_c = oracle.make_observation(p.x_true, mats, p.noise, p.nu)
    api = _api()
    A = [api.banded(m, p.dims[m - 1], t) for m, _, t in p.factors]
    B = [api.dense(m, t) for m, _, t in p.right_factors]
    Cd = api.to_device(C, torch.float32)
    tol = oracle.rho_star(nu_c)
    X, info = h.gmres_solve(Cd, p.m, p.sketch_dims, p.seed, p.lam, A, B, tol=tol, mu_grid=p.mu_grid,
                            true_residual=True)
    R = C - oracle.apply_operator(X.cpu().double().numpy(), mats)
    ref = np.linalg.norm(R) / np.linalg.norm(C)
    assert abs(info.true_rel_resid - ref) <= 1e-4 * ref
    Xs, res = h.gmres_solve_batched([dict(C=Cd, A=A, B=B, m=p.m, sketch_dims=p.sketch_dims, seed=p.seed,
                                          lam=p.lam, tol=tol)], mu_grid=p.mu_grid, true_residual=True)
    assert res[0].true_rel_resid == info.true_rel_resid
    assert res[0].true_rel_resid_theta == info.true_rel_resid_theta


# ------------------------------------------------------------------------ non-finite data

@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_nan_observation_is_reported(h, dt):
    mats, C, th, A, B, sk = _small_problem()
    C = C.copy()
    C[3, 5, 1] = np.nan
    api = _api()
    X, info = h.gmres_solve(api.to_device(C, dt), 10, sk, 2, 1e-3, A, B, tol=1e-3)
    assert info.device_status == 6          # RTG_ERR_NONFINITE
    assert info.iters == 0 and not info.converged


def test_overflow_during_the_iteration_is_reported(h):
    """An operator whose output overflows FP32 in the first step: beta is
    finite, h_{1,0} is not, and the solve stops with RTG_ERR_NONFINITE."""
    dims, sk = (64, 48, 3), (24, 16, 3)
    C = np.random.default_rng(0).standard_normal(dims)
    api = _api()
    big = [api.dense(3, 1e30 * np.eye(3))]
    X, info = h.gmres_solve(api.to_device(C, torch.float32), 10, sk, 2, 1e-3, [], big, tol=1e-3)
    assert info.device_status == 6
    assert np.isfinite(info.beta) and info.iters <= 1


# ------------------------------------------------------------------------ bounded waits

def test_bounded_device_wait_times_out_and_the_context_stays_usable(h):
    """A device-side wait on a flag that nothing sets gives up after its
    limit with RTG_ERR_TIMEOUT (no trap, no fault), the same stream then runs
    a wait whose flag is met, and a solve afterwards is correct."""
    import ctypes
    import time
    from paper_2603_00839_gb300 import _lib as L
    st = ctypes.c_int32(-1)
    t0 = time.perf_counter()
    L.check(L.load().rtg_selftest_bounded_wait(0, 200, ctypes.byref(st)))
    el = time.perf_counter() - t0
    assert st.value == L.ERR_TIMEOUT
    assert 0.19 <= el < 5.0
    mats, C, th, A, B, sk = _small_problem()
    ref = oracle.rtg_gmres(mats, C, 8, th, tol=0.0, lam=1e-3)
    api = _api()
    X, info = h.gmres_solve(api.to_device(C, torch.float64), 8, sk, 2, 1e-3, A, B)
    assert info.device_status == 0 and _relnorm(X.cpu().numpy(), ref["X"]) < 1e-9
