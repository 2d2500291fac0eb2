"""Batched form on the GPU: many independent solves in one CUDA graph launch.

Every problem of a batch runs as its own branch of one graph with its own
device-side stop decision, so each result must equal, bit for bit, the same
problem solved alone (same kernels, same launch shapes, deterministic
reductions).  Problems of one batch differ in shape (square and not),
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
    for q, X, r in zip(probs, Xs, res):
        Xr, rr = _single(h, q, mu_grid=grid)
        assert r.iters == rr.iters and r.converged == rr.converged and r.device_status == 0
        assert np.array_equal(r.rho, rr.rho)
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
