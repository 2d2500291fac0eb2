"""Batched form on the GPU: many independent solves in one CUDA graph launch.

By default every problem is its own branch of the graph; with group_max > 1
problems of equal structure (shape, operator, sketch sizes, m,
regularisation mode, X0 or not) run in lock step: one launch per kernel
serves the group, each problem keeps its own device-side stop decision, and
the group's loop runs while any of them does.  Each result must equal, bit
for bit, the same problem solved alone (same kernels, same per-problem
launch shapes, deterministic reductions).  Problems of one batch differ in shape (square and not),
operator, Krylov dimension, sketch sizes, regularisation and stop level, as
in the batched workload (side lengths 64..1024, sigma 0.5..3, radius
ceil(3 sigma), m = 30, sketch min(I_k, 128)).
"""
import math

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


def _problem(h, cfg, dtype=torch.float32):
    """Observation built on the device with the library's operator (outside any timing)."""
    api = _api()
    I1, I2, _ = cfg["dims"]
    x = w.piecewise_image(I1, I2, 3, cfg["image_seed"])
    taps = w.gaussian_taps(cfg["sigma"], cfg["radius"])
    A = [api.banded(1, I1, taps), api.banded(2, I2, taps)]
    X = api.to_device(x, dtype)
    Ch = h.operator_apply(X, A, [])
    E = api.to_device(w.noise_draw(x.shape, cfg["image_seed"]), dtype)
    C = api.empty(cfg["dims"], dtype)
    C.copy_(Ch + E * (cfg["nu"] * torch.linalg.vector_norm(Ch) / torch.linalg.vector_norm(E)))
    return dict(C=C, A=A, B=[], m=cfg["m"], sketch_dims=cfg["sketch_dims"], seed=cfg["problem_id"],
                lam=cfg["mu"], tol=max(1e-3, 1.01 * cfg["nu"]))


def _single(h, q, mu_grid=None):
    return h.gmres_solve(q["C"], q["m"], q["sketch_dims"], q["seed"], q["lam"], q["A"], q["B"],
                         tol=q["tol"], mu_grid=mu_grid)


def _cfgs(n, lo=64, hi=320, seed=3):
    return w.batched_configs(n, seed=seed, side_lo=lo, side_hi=hi)


def test_batched_equals_single_solves_uneven_sizes(h):
    api = _api()
    probs = [_problem(h, c) for c in _cfgs(6)]
    probs[1]["lam"] = -1.0            # one problem chooses mu by GCV
    probs[2]["m"] = 12                # another runs a short process
    probs[3]["tol"] = 0.0             # and one runs all m steps
    grid = w.mu_grid()
    Xs, res = h.gmres_solve_batched(probs, mu_grid=grid)
    for i, (q, X, r) in enumerate(zip(probs, Xs, res)):
        Xr, rr = _single(h, q, mu_grid=grid)
        assert r.iters == rr.iters and r.converged == rr.converged and r.device_status == 0
        assert np.array_equal(r.rho, rr.rho), (i, tuple(q["C"].shape), r.rho - rr.rho)
        assert r.mu == rr.mu
        assert np.array_equal(X.cpu().numpy(), Xr.cpu().numpy())
    # replay with new data on the same shapes: still equal to single solves
    for q in probs:
        q["C"] = api.to_device(0.5 * q["C"].cpu().numpy(), torch.float32)
    Xs2, res2 = h.gmres_solve_batched(probs, mu_grid=grid)
    for q, X, r in zip(probs, Xs2, res2):
        Xr, rr = _single(h, q, mu_grid=grid)
        assert r.iters == rr.iters
        assert np.array_equal(X.cpu().numpy(), Xr.cpu().numpy())


def test_batched_problem_matches_the_oracle(h):
    api = _api()
    p = w.image_config(1)            # 64x64x3, run in FP64 as part of a batch of three
    A = [api.banded(m, p.dims[m - 1], t) for m, _, t in p.factors]
    mats = oracle.factor_matrices(p.dims, p.factors, p.right_factors)
    C, _, nu_c = oracle.make_observation(p.x_true, mats, p.noise, p.nu)
    th = oracle.sketch_matrices(p.dims, p.sketch_dims, 0, 0)
    ref = oracle.rtg_gmres(mats, C, p.m, th, tol=1e-3, lam=p.lam)
    Cd = api.to_device(C, torch.float64)
    q = dict(C=Cd, A=A, B=[], m=p.m, sketch_dims=p.sketch_dims, seed=0, lam=p.lam, tol=1e-3)
    q2 = dict(q, C=api.to_device(0.7 * C, torch.float64), seed=5)
    q3 = dict(q, C=api.to_device(C[:48, :40, :].copy(), torch.float64),
              A=[api.banded(1, 48, p.factors[0][2]), api.banded(2, 40, p.factors[1][2])], sketch_dims=(24, 20, 3))
    Xs, res = h.gmres_solve_batched([q2, q, q3])
    assert res[1].iters == ref["iters"]
    assert np.linalg.norm(Xs[1].cpu().numpy() - ref["X"]) / np.linalg.norm(ref["X"]) < 1e-10


def test_batched_bf16_basis(h):
    probs = [_problem(h, c) for c in _cfgs(3, lo=64, hi=200, seed=9)]
    for q in probs:   # the BF16 basis needs dims[0] % 8 == 0
        q["C"] = q["C"][: (q["C"].shape[0] // 8) * 8]
        q["C"] = _api().to_device(q["C"].cpu().numpy(), torch.float32)
        I1 = q["C"].shape[0]
        q["A"] = [_api().banded(1, I1, q["A"][0].taps), q["A"][1]]
        q["sketch_dims"] = (min(I1 // 2, 128),) + tuple(q["sketch_dims"][1:])   # mode 1 sketched
    Xs, res = h.gmres_solve_batched(probs, bf16_basis=True)
    for q, X, r in zip(probs, Xs, res):
        Xr, rr = h.gmres_solve(q["C"], q["m"], q["sketch_dims"], q["seed"], q["lam"], q["A"], q["B"],
                               tol=q["tol"], bf16_basis=True)
        assert r.iters == rr.iters
        assert np.array_equal(X.cpu().numpy(), Xr.cpu().numpy())


def test_batched_rejects_bad_arguments(h):
    from paper_2603_00839_gb300 import _lib as L
    api = _api()
    q = _problem(h, _cfgs(1)[0])
    with pytest.raises(ValueError):
        h.gmres_solve_batched([])
    with pytest.raises(L.RtgError, match="problem 1: m="):
        h.gmres_solve_batched([q, dict(q, m=0)])
    q64 = dict(q, C=q["C"].double())
    q64["C"] = api.to_device(q["C"].cpu().double().numpy(), torch.float64)
    with pytest.raises(ValueError, match="one dtype"):
        h.gmres_solve_batched([q, q64])


def _same_shape(h, n, dims=(96, 80, 3), m=20, sk=(48, 40, 3), seed0=0, dtype=torch.float32):
    """n problems of one structure (one lock-step group): own image, noise level, seed, mu, tol."""
    out = []
    for k in range(n):
        cfg = dict(dims=dims, image_seed=seed0 + k, sigma=1.5, radius=5, nu=0.005 * (k + 1), m=m,
                   sketch_dims=sk, problem_id=seed0 + 7 * k + 1, mu=1e-3 * (k + 1))
        out.append(_problem(h, cfg, dtype))
    return out


def _assert_same(h, probs, Xs, res, **kw):
    for q, X, r in zip(probs, Xs, res):
        Xr, rr = h.gmres_solve(q["C"], q["m"], q["sketch_dims"], q["seed"], q["lam"], q["A"], q["B"],
                               tol=q["tol"], X0=q.get("X0"), **kw)
        assert r.device_status == 0 and rr.device_status == 0
        assert r.iters == rr.iters and r.converged == rr.converged
        assert np.array_equal(r.rho, rr.rho)
        assert r.mu == rr.mu
        assert np.array_equal(X.cpu().numpy(), Xr.cpu().numpy())


def test_lockstep_group_equals_single_solves(h):
    """Five problems of one structure stopping at different steps: one runs all m
    steps (tol 0), one stops after the first step, the others at rho*."""
    probs = _same_shape(h, 5)
    probs[1]["tol"] = 0.0
    probs[3]["tol"] = 0.9
    Xs, res = h.gmres_solve_batched(probs, group_max=8)
    iters = [r.iters for r in res]
    assert iters[1] == 20 and iters[3] == 1 and len(set(iters)) >= 3
    _assert_same(h, probs, Xs, res)


def test_lockstep_group_gcv(h):
    grid = w.mu_grid()
    probs = _same_shape(h, 4, seed0=10)
    for q in probs:
        q["lam"] = -1.0
    Xs, res = h.gmres_solve_batched(probs, mu_grid=grid, group_max=4)
    _assert_same(h, probs, Xs, res, mu_grid=grid)


def test_interleaved_groups(h):
    """Problems of two structures given alternately: two groups, results in caller order."""
    a = _same_shape(h, 3, seed0=20)
    b = _same_shape(h, 2, dims=(64, 72, 3), m=15, sk=(32, 36, 3), seed0=30)
    probs = [a[0], b[0], a[1], b[1], a[2]]
    Xs, res = h.gmres_solve_batched(probs, group_max=16)
    _assert_same(h, probs, Xs, res)
    # a second call on the same plan with new data
    for q in probs:
        q["C"] = _api().to_device(0.25 * q["C"].cpu().numpy(), torch.float32)
    Xs, res = h.gmres_solve_batched(probs, group_max=16)
    _assert_same(h, probs, Xs, res)
    # capped groups: {a0, a1}, {a2}, {b0, b1}
    Xs, res = h.gmres_solve_batched(probs, group_max=2)
    _assert_same(h, probs, Xs, res)


def test_lockstep_group_with_initial_guesses(h):
    api = _api()
    probs = _same_shape(h, 3, seed0=40)
    rng = np.random.default_rng(0)
    for q in probs:
        q["X0"] = api.to_device(0.1 * rng.standard_normal(tuple(q["C"].shape)), torch.float32)
    Xs, res = h.gmres_solve_batched(probs, group_max=3)
    _assert_same(h, probs, Xs, res)


def test_lockstep_group_fp64(h):
    probs = _same_shape(h, 3, seed0=50, dtype=torch.float64)
    Xs, res = h.gmres_solve_batched(probs, group_max=3)
    _assert_same(h, probs, Xs, res)


def test_lockstep_group_bf16_basis(h):
    probs = _same_shape(h, 3, dims=(96, 80, 3), sk=(48, 40, 3), seed0=60)
    Xs, res = h.gmres_solve_batched(probs, bf16_basis=True, group_max=3)
    _assert_same(h, probs, Xs, res, bf16_basis=True)


def test_lockstep_direct_and_phase_timed_launches_equal_the_graph(h):
    """Direct launches (one group after another, host stops at the group's end)
    and phase-timed launches give the graph's results bit for bit."""
    probs = _same_shape(h, 3, seed0=70) + _same_shape(h, 2, dims=(64, 72, 3), m=15, sk=(32, 36, 3), seed0=80)
    probs[0]["tol"] = 0.0
    with pytest.raises(Exception):
        h.gmres_solve_batched(probs, group_max=-1)
    Xg, rg = h.gmres_solve_batched(probs, group_max=8)
    Xg = [X.cpu().numpy().copy() for X in Xg]
    for kw in (dict(use_graph=False), dict(phase_times=True)):
        Xd, rd = h.gmres_solve_batched(probs, group_max=8, **kw)
        for a, b, ra, rb in zip(Xg, Xd, rg, rd):
            assert ra.iters == rb.iters and np.array_equal(ra.rho, rb.rho)
            assert np.array_equal(a, b.cpu().numpy())
    # phase times: the group's own, shared by its problems; the apply group runs once per step
    assert rd[0].phase_ms == rd[1].phase_ms and rd[3].phase_ms == rd[4].phase_ms
    assert rd[0].phase_launches["apply"] == max(r.iters for r in rd[:3])
    assert rd[3].phase_launches["apply"] == max(r.iters for r in rd[3:])
    assert all(v >= 0 for v in rd[0].phase_ms.values()) and rd[0].phase_ms["sketch"] > 0


def test_many_identical_branches_equal_the_single_solve(h):
    """128 identical 512x512x3 FP32 problems as concurrent graph branches: every
    result equals the single solve bit for bit.  Regression test for the ring
    refill of the basis update: its bulk copies into shared memory need a proxy
    fence after the threads' reads of the slot, and without it a few of these
    copies (CTAs of other kernels sharing the SM) read corrupted slots."""
    api = _api()
    I1 = I2 = 512
    dims, sk = (I1, I2, 3), (128, 128, 3)
    a = w.gaussian_taps(2.0, 6)
    A = [api.banded(1, I1, a), api.banded(2, I2, a)]
    B = [api.dense(3, w.channel_mix())]
    x = w.piecewise_image(I1, I2, 3, 7)
    Xt = api.to_device(x, torch.float32)
    Ch = h.operator_apply(Xt, A, B)
    E = api.to_device(w.noise_draw(dims, 7), torch.float32)
    C = api.empty(dims, torch.float32)
    C.copy_(Ch + E * (1e-2 * torch.linalg.vector_norm(Ch) / torch.linalg.vector_norm(E)))
    Xs, rs = h.gmres_solve(C, 30, sk, 3, 1e-3, A, B, tol=0.0)
    Xs = Xs.cpu().numpy()
    probs = [dict(C=C, A=A, B=B, m=30, sketch_dims=sk, seed=3, lam=1e-3, tol=0.0) for _ in range(128)]
    for _ in range(2):
        Xb, rb = h.gmres_solve_batched(probs)
        bad = [i for i in range(len(probs)) if not np.array_equal(Xb[i].cpu().numpy(), Xs)]
        assert not bad, f"{len(bad)} of {len(probs)} branches differ from the single solve"


def test_every_tile_geometry_gives_the_same_solve(h):
    """The autotuner's candidates (slot size and depth of the basis update's
    ring) change only speed: a solve and a lock-step batch give the same
    results bit for bit with every geometry, and the tuned choice is one of
    them."""
    import os
    api = _api()
    cfgs = w.batched_configs(3, seed=5, side_lo=96, side_hi=320)
    for c in cfgs:   # whole 8-element groups: the ring update (whose tiles are tuned) applies
        I1, I2 = c["dims"][0] // 8 * 8, c["dims"][1] // 8 * 8
        c["dims"] = (I1, I2, 3)
        c["sketch_dims"] = (min(I1, 128), min(I2, 128), 3)
    probs = [_problem(h, c) for c in cfgs]
    results = []
    for k in range(5):
        os.environ["RTG_TILE_CONFIG"] = str(k)
        try:
            hk = api.Handle(0)
            X, info = _single(hk, probs[0])
            Xb, rb = hk.gmres_solve_batched([probs[1]] * 3, group_max=3)
            assert info.tile_config == k and rb[0].tile_config == k
            results.append((X.cpu().numpy(), [x.cpu().numpy() for x in Xb]))
        finally:
            del os.environ["RTG_TILE_CONFIG"]
    for X, Xb in results[1:]:
        assert np.array_equal(X, results[0][0])
        assert all(np.array_equal(a, b) for a, b in zip(Xb, results[0][1]))
    X, info = _single(api.Handle(0), probs[0])
    assert 0 <= info.tile_config < 5 and np.array_equal(X.cpu().numpy(), results[0][0])
