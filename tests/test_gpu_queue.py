"""Batched form with a device work queue (opts.queue_slots = K > 0).

Problems of equal structure form a class; the class gets min(K, its size)
graph branches with one workspace each, and every branch takes the class's
problems one after another from a device queue (an atomic counter) until it
is empty.  Which branch solves which problem depends on timing, the result
must not: each problem's result equals, bit for bit, the same problem solved
alone (same kernels, same launch shapes, deterministic reductions, and a
workspace that the solve's prologue resets).
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


def _problem(h, cfg, dtype=torch.float32):
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


def _class(h, cfg, n, first_seed):
    """n problems of one structure: the same shape and operator, other images, noise and signs."""
    out = []
    for k in range(n):
        c = dict(cfg, image_seed=cfg["image_seed"] + 7919 * (k + 1), problem_id=first_seed + k,
                 nu=cfg["nu"] * (1.0 + 0.5 * k))
        out.append(_problem(h, c))
    return out


def _single(h, q, mu_grid=None, max_restarts=0):
    return h.gmres_solve(q["C"], q["m"], q["sketch_dims"], q["seed"], q["lam"], q["A"], q["B"],
                         X0=q.get("X0"), tol=q["tol"], mu_grid=mu_grid, max_restarts=max_restarts)


def _assert_equal_to_single(h, probs, Xs, res, mu_grid=None, max_restarts=0):
    for i, (q, X, r) in enumerate(zip(probs, Xs, res)):
        Xr, rr = _single(h, q, mu_grid=mu_grid, max_restarts=max_restarts)
        assert r.device_status == 0, i
        assert r.iters == rr.iters and r.converged == rr.converged and r.restarts == rr.restarts, i
        assert np.array_equal(r.rho, rr.rho), (i, r.rho - rr.rho)
        assert r.mu == rr.mu, i
        assert np.array_equal(X.cpu().numpy(), Xr.cpu().numpy()), i


def _mixed_batch(h):
    cfgs = w.batched_configs(3, seed=17, side_lo=48, side_hi=160)
    a = _class(h, cfgs[0], 7, 100)        # seven problems of one structure
    b = _class(h, cfgs[1], 3, 200)        # three of another
    c = _class(h, cfgs[2], 1, 300)        # and a class of one, choosing mu by GCV
    c[0]["lam"] = -1.0
    a[2]["tol"] = 0.0                     # stop levels and lambda are per problem, not structure
    a[4]["lam"] = 0.5 * a[4]["lam"]
    # interleave the classes in the problem list
    return [a[0], b[0], a[1], c[0], a[2], a[3], b[1], a[4], a[5], b[2], a[6]]


def test_queue_equals_single_solves(h):
    api = _api()
    grid = w.mu_grid()
    probs = _mixed_batch(h)
    for slots in (3, 1, 16):
        Xs, res = h.gmres_solve_batched(probs, mu_grid=grid, queue_slots=slots)
        _assert_equal_to_single(h, probs, Xs, res, mu_grid=grid)
    # replay with new data on the same structures (the queue counters restart)
    for q in probs:
        q["C"] = api.to_device(0.5 * q["C"].cpu().numpy(), torch.float32)
    Xs, res = h.gmres_solve_batched(probs, mu_grid=grid, queue_slots=3)
    _assert_equal_to_single(h, probs, Xs, res, mu_grid=grid)


def test_queue_direct_launches_equal_the_graph(h):
    grid = w.mu_grid()
    probs = _mixed_batch(h)
    Xg, rg = h.gmres_solve_batched(probs, mu_grid=grid, queue_slots=2)
    Xd, rd = h.gmres_solve_batched(probs, mu_grid=grid, queue_slots=2, use_graph=False)
    for a, b, ra, rb in zip(Xg, Xd, rg, rd):
        assert ra.iters == rb.iters and np.array_equal(ra.rho, rb.rho)
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())


def test_queue_with_restarts_and_initial_guesses(h):
    api = _api()
    cfg = w.batched_configs(1, seed=23, side_lo=64, side_hi=96)[0]
    cfg = dict(cfg, m=6)                  # short cycles: most problems restart
    probs = _class(h, cfg, 5, 400)
    for k, q in enumerate(probs):
        q["tol"] = 2e-3
        if k % 2 == 0:                    # X0 is structural: these three form a class of their own
            q["X0"] = api.to_device(0.1 * np.ones(tuple(q["C"].shape)), torch.float32)
    Xs, res = h.gmres_solve_batched(probs, queue_slots=2, max_restarts=3)
    assert any(r.restarts > 0 for r in res)
    _assert_equal_to_single(h, probs, Xs, res, max_restarts=3)


def test_queued_fp64_problems_match_the_oracle(h):
    api = _api()
    p = w.image_config(1)                 # 64x64x3, FP64
    A = [api.banded(m, p.dims[m - 1], t) for m, _, t in p.factors]
    mats = oracle.factor_matrices(p.dims, p.factors, p.right_factors)
    C, _, _ = oracle.make_observation(p.x_true, mats, p.noise, p.nu)
    probs, refs = [], []
    for k, (scale, seed) in enumerate([(1.0, 0), (0.7, 5), (1.3, 9), (0.9, 11)]):
        Ck = scale * C
        th = oracle.sketch_matrices(p.dims, p.sketch_dims, seed, 0)
        refs.append(oracle.rtg_gmres(mats, Ck, p.m, th, tol=1e-3, lam=p.lam))
        probs.append(dict(C=api.to_device(Ck, torch.float64), A=A, B=[], m=p.m, sketch_dims=p.sketch_dims,
                          seed=seed, lam=p.lam, tol=1e-3))
    Xs, res = h.gmres_solve_batched(probs, queue_slots=2)
    for X, r, ref in zip(Xs, res, refs):
        assert r.iters == ref["iters"] and r.device_status == 0
        assert np.allclose(r.rho, ref["rho"], rtol=1e-10, atol=0)
        assert np.linalg.norm(X.cpu().numpy() - ref["X"]) / np.linalg.norm(ref["X"]) < 1e-10


def test_queue_serves_more_problems_than_a_batch_holds(h):
    from paper_2603_00839_gb300 import _lib as L
    api = _api()
    n = 1100                              # above the branch-per-problem limit of 1024
    rng = np.random.default_rng(5)
    taps = w.gaussian_taps(1.0, 3)
    A = [api.banded(1, 16, taps), api.banded(2, 16, taps)]
    base = rng.standard_normal((16, 16, 3))
    probs = [dict(C=api.to_device(base * (1.0 + 0.01 * k), torch.float32), A=A, B=[], m=6,
                  sketch_dims=(8, 8, 3), seed=k, lam=1e-2, tol=1e-3) for k in range(n)]
    with pytest.raises(L.RtgError, match="nprob"):
        h.gmres_solve_batched(probs)      # one branch per problem: too many
    Xs, res = h.gmres_solve_batched(probs, queue_slots=4)
    assert all(r.device_status == 0 for r in res)
    sample = list(range(0, n, 137)) + [n - 1]
    _assert_equal_to_single(h, [probs[k] for k in sample], [Xs[k] for k in sample], [res[k] for k in sample])


def test_queue_rejects_bad_arguments(h):
    from paper_2603_00839_gb300 import _lib as L
    probs = _mixed_batch(h)[:3]
    with pytest.raises(L.RtgError, match="queue_slots"):
        h.gmres_solve_batched(probs, queue_slots=-1)
    with pytest.raises(L.RtgError, match="exclude"):
        h.gmres_solve_batched(probs, queue_slots=2, group_max=2)
    with pytest.raises(L.RtgError, match="PHASE_TIMES"):
        h.gmres_solve_batched(probs, queue_slots=2, phase_times=True)


def test_chained_branches_equal_single_solves(h):
    """More branches than queue slots (classes of one problem each, and a
    class of four beside them): the branches run as queue_slots chains."""
    cfgs = w.batched_configs(5, seed=31, side_lo=40, side_hi=140)
    singles = [_problem(h, c) for c in cfgs]           # five structures
    four = _class(h, cfgs[0], 4, 500)                   # and a class of four of the first one's
    probs = [singles[0], four[0], singles[1], singles[2], four[1], singles[3], four[2], singles[4], four[3]]
    for slots in (2, 3):
        Xs, res = h.gmres_solve_batched(probs, queue_slots=slots)
        _assert_equal_to_single(h, probs, Xs, res)


def test_queue_bf16_basis_and_true_residual(h):
    """The work queue with the BF16 basis, and with the final true residual:
    each result equals the same problem solved alone with the same options."""
    cfg = w.batched_configs(1, seed=41, side_lo=64, side_hi=120)[0]
    I1 = (cfg["dims"][0] // 8) * 8                   # the BF16 basis needs dims[0] % 8 == 0
    cfg = dict(cfg, dims=(I1,) + tuple(cfg["dims"][1:]),
               sketch_dims=(min(I1 // 2, 128),) + tuple(cfg["sketch_dims"][1:]))
    probs = _class(h, cfg, 5, 600)
    Xs, res = h.gmres_solve_batched(probs, queue_slots=2, bf16_basis=True)
    for q, X, r in zip(probs, Xs, res):
        Xr, rr = h.gmres_solve(q["C"], q["m"], q["sketch_dims"], q["seed"], q["lam"], q["A"], q["B"],
                               tol=q["tol"], bf16_basis=True)
        assert r.device_status == 0 and r.iters == rr.iters and np.array_equal(r.rho, rr.rho)
        assert np.array_equal(X.cpu().numpy(), Xr.cpu().numpy())
    Xs, res = h.gmres_solve_batched(probs, queue_slots=2, true_residual=True)
    for q, X, r in zip(probs, Xs, res):
        Xr, rr = h.gmres_solve(q["C"], q["m"], q["sketch_dims"], q["seed"], q["lam"], q["A"], q["B"],
                               tol=q["tol"], true_residual=True)
        assert r.device_status == 0 and r.true_rel_resid > 0
        assert r.true_rel_resid == rr.true_rel_resid and r.true_rel_resid_theta == rr.true_rel_resid_theta
        assert np.array_equal(X.cpu().numpy(), Xr.cpu().numpy())


def test_queue_full_size_image512_as_the_benchmark_runs_it(h):
    """The benchmark's launch configuration at full size: 512x512x3 FP32
    problems (seeds 0..11, GCV over the grid, stop at rho*) through the
    work queue on eight branches.  Every result equals its single solve bit
    for bit, and the first problem matches the FP64 oracle (rho history, X
    at the mu the GPU picked) at the FP32 bar of 1e-4."""
    api = _api()
    probs, first = [], None
    for s in range(12):
        p = w.image_config(2, seed=s)
        mats = oracle.factor_matrices(p.dims, p.factors, p.right_factors)
        C, _, nu_c = oracle.make_observation(p.x_true, mats, p.noise, p.nu)
        A = [api.banded(m, p.dims[m - 1], t) if k == "banded" else api.dense(m, t) for m, k, t in p.factors]
        B = [api.banded(m, p.dims[m - 1], t) if k == "banded" else api.dense(m, t) for m, k, t in p.right_factors]
        probs.append(dict(C=api.to_device(C, torch.float32), A=A, B=B, m=p.m, sketch_dims=p.sketch_dims,
                          seed=p.seed, lam=p.lam, tol=oracle.rho_star(nu_c)))
        if s == 0:
            first = (p, mats, C, oracle.rho_star(nu_c))
    grid = w.image_config(2).mu_grid
    Xs, res = h.gmres_solve_batched(probs, mu_grid=grid, queue_slots=8)
    _assert_equal_to_single(h, probs, Xs, res, mu_grid=grid)
    p, mats, C, tol = first
    th = oracle.sketch_matrices(p.dims, p.sketch_dims, p.seed, p.problem_id)
    ref = oracle.rtg_gmres(mats, C, p.m, th, tol=tol, lam=p.lam, mu_grid=grid)
    r = res[0]
    assert r.iters == ref["iters"]
    assert np.allclose(r.rho, ref["rho"], rtol=1e-4, atol=0)
    y = oracle.tikhonov_stacked(ref["H"], ref["beta"], r.mu)
    X_mu = sum(y[i] * ref["V"][i] for i in range(r.iters))
    Xg = Xs[0].cpu().double().numpy()
    assert np.linalg.norm(Xg - X_mu) / np.linalg.norm(X_mu) < 1e-4
