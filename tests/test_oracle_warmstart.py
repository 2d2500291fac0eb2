"""Pins for the oracle's warm-start network (CPU only).

The backward pass is checked against central finite differences of the
loss for every parameter tensor (sampled entries), the convolution against
a direct per-pixel sum, the stride-2 geometry and nearest up-sampling
against their definitions, and the untrained network against its designed
start (X_0 = C, log lambda = 0).  A planted mistake (a dropped skip
connection in the backward pass) fails the finite-difference pin.
"""
import numpy as np
import pytest

from oracle import warmstart as WS


def _batch(N=2, H=16, W=8, seed=0):
    rng = np.random.default_rng(seed)
    C = rng.standard_normal((N, H, W, 3))
    Xs = C + 0.1 * rng.standard_normal((N, H, W, 3))
    return C, Xs, rng.standard_normal(N)


def _params(base=2, seed=1):
    P = WS.init_params(base, seed)
    rng = np.random.default_rng(seed + 10)
    for k in P:   # a non-degenerate point: the designed zero output layer would hide gradients
        P[k] = P[k] + 0.1 * rng.standard_normal(P[k].shape)
    return P


def test_conv_matches_direct_sum():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 6, 4, 2))
    w = rng.standard_normal((3, 3, 3, 2))
    b = rng.standard_normal(3)
    for s in (1, 2):
        y = WS.conv(x, w, b, s)
        for (n, i, j, o) in [(0, 0, 0, 0), (0, 2, 1, 2), (0, y.shape[1] - 1, y.shape[2] - 1, 1)]:
            v = b[o]
            for dy in range(3):
                for dx in range(3):
                    yy, xx = s * i + dy - 1, s * j + dx - 1
                    if 0 <= yy < 6 and 0 <= xx < 4:
                        v += w[o, dy, dx] @ x[n, yy, xx]
            assert abs(y[n, i, j, o] - v) < 1e-12


def test_up2_and_its_backward_are_adjoint():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 3, 4, 5))
    y = rng.standard_normal((2, 6, 8, 5))
    assert abs(np.vdot(WS.up2(x), y) - np.vdot(x, WS.up2_backward(y))) < 1e-10
    assert np.array_equal(WS.up2(x)[:, 1::2, ::2], x)


def test_untrained_network_returns_its_input():
    C, Xs, lm = _batch()
    P = WS.init_params(4, 0)
    X0, ll, _ = WS.forward(P, C, 4)
    assert np.array_equal(X0, C) and np.all(ll == 0.0)
    # 9 c_in c_out + c_out per layer, plus the 4c + 1 of the lambda head: about half a million
    assert sum(v.size for v in WS.init_params(32, 0).values()) == 481_668


@pytest.mark.parametrize("name", ["e1.w", "e2.w", "e4.w", "d3.w", "d2.b", "d1.w", "out.w", "out.b", "lam.w", "lam.b"])
def test_backward_matches_finite_differences(name):
    C, Xs, lm = _batch()
    P = _params()
    loss, G = WS.loss_and_grads(P, C, Xs, lm, 2)
    rng = np.random.default_rng(4)
    idxs = [tuple(int(rng.integers(0, d)) for d in P[name].shape) for _ in range(4)]
    h = 1e-6
    for ix in idxs:
        Pp = {k: v.copy() for k, v in P.items()}
        Pm = {k: v.copy() for k, v in P.items()}
        Pp[name][ix] += h
        Pm[name][ix] -= h
        fd = (WS.loss_and_grads(Pp, C, Xs, lm, 2)[0] - WS.loss_and_grads(Pm, C, Xs, lm, 2)[0]) / (2 * h)
        assert abs(G[name][ix] - fd) <= 1e-6 * max(1.0, abs(fd))


def test_pin_catches_a_dropped_skip_gradient(monkeypatch):
    C, Xs, lm = _batch()
    P = _params()
    orig = WS.up2_backward
    calls = {"n": 0}

    def drop_first(dy):   # planted: the gradient through the d3 -> d2 upsampling is lost
        calls["n"] += 1
        out = orig(dy)
        return out * 0.0 if calls["n"] == 2 else out

    monkeypatch.setattr(WS, "up2_backward", drop_first)
    loss, G = WS.loss_and_grads(P, C, Xs, lm, 2)
    monkeypatch.setattr(WS, "up2_backward", orig)
    h = 1e-6
    ix = (0, 1, 1, 0)
    Pp = {k: v.copy() for k, v in P.items()}
    Pm = {k: v.copy() for k, v in P.items()}
    Pp["e1.w"][ix] += h
    Pm["e1.w"][ix] -= h
    fd = (WS.loss_and_grads(Pp, C, Xs, lm, 2)[0] - WS.loss_and_grads(Pm, C, Xs, lm, 2)[0]) / (2 * h)
    assert abs(G["e1.w"][ix] - fd) > 1e-4 * max(1.0, abs(fd))
