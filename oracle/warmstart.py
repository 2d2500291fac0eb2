"""Learned warm start: the convolutional encoder-decoder, FP64 (oracle; test infrastructure only).

The network maps an observation C (H x W x 3, H and W multiples of 8) to
an initial guess X_0 = C + out and a regularisation log(lambda).  Layers
(3x3 convolutions, zero padding 1, channels last inside the network):

    e1 = relu(conv(C;  3 -> c))          H
    e2 = relu(conv_s2(e1; c -> 2c))      H/2
    e3 = relu(conv_s2(e2; 2c -> 4c))     H/4
    e4 = relu(conv_s2(e3; 4c -> 4c))     H/8   (four levels)
    d3 = relu(conv(up(e4); 4c -> 4c)) + e3
    d2 = relu(conv(up(d3); 4c -> 2c)) + e2
    d1 = relu(conv(up(d2); 2c -> c)) + e1
    out = conv(d1; c -> 3),  X_0 = C + out
    log_lambda = w_l . mean_pixels(e4) + b_l

up: nearest-neighbour x2; conv_s2: stride 2 (output pixel (i, j) centred
on input pixel (2i, 2j)).  Loss of a batch: mean over images of
||X_0 - X*||^2 / ||X*||^2 + (log_lambda - log mu*)^2 with X* and mu* the
solver's solution and regularisation.  Everything here is plain numpy:
convolutions by explicit sums over the 9 taps, backward passes written out
from the chain rule; checked against finite differences in the tests.
Not from the paper (it has no learned component): the form the build adds.
"""
from __future__ import annotations

from typing import Dict, List

import numpy as np

def layer_shapes(base: int):
    """(name, c_in, c_out, stride) per convolution, from the shared generator module."""
    import workloads
    return workloads.warmstart_layer_shapes(base)


def init_params(base: int, seed: int) -> Dict[str, np.ndarray]:
    """The seeded initial parameters the GPU network also starts from."""
    import workloads
    return workloads.warmstart_params(base, seed)


def conv(x: np.ndarray, w: np.ndarray, b: np.ndarray, stride: int) -> np.ndarray:
    """y[n, i, j, o] = b[o] + sum_{dy, dx, c} w[o, dy, dx, c] x[n, s i + dy - 1, s j + dx - 1, c]."""
    N, H, W, C = x.shape
    Ho, Wo = H // stride, W // stride
    xp = np.zeros((N, H + 2, W + 2, C))
    xp[:, 1:H + 1, 1:W + 1, :] = x
    y = np.zeros((N, Ho, Wo, w.shape[0])) + b
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, dy:dy + stride * Ho:stride, dx:dx + stride * Wo:stride, :]
            y += patch @ w[:, dy, dx, :].T
    return y


def conv_backward(x: np.ndarray, w: np.ndarray, dy: np.ndarray, stride: int):
    """Gradients of conv with respect to x, w and b."""
    N, H, W, C = x.shape
    Ho, Wo = H // stride, W // stride
    xp = np.zeros((N, H + 2, W + 2, C))
    xp[:, 1:H + 1, 1:W + 1, :] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, ky:ky + stride * Ho:stride, kx:kx + stride * Wo:stride, :]
            dw[:, ky, kx, :] = np.einsum("nijo,nijc->oc", dy, patch)
            dxp[:, ky:ky + stride * Ho:stride, kx:kx + stride * Wo:stride, :] += dy @ w[:, ky, kx, :]
    db = dy.sum(axis=(0, 1, 2))
    return dxp[:, 1:H + 1, 1:W + 1, :], dw, db


def up2(x: np.ndarray) -> np.ndarray:
    return x.repeat(2, axis=1).repeat(2, axis=2)


def up2_backward(dy: np.ndarray) -> np.ndarray:
    N, H, W, C = dy.shape
    return dy.reshape(N, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def forward(P: Dict[str, np.ndarray], Cimg: np.ndarray, base: int):
    """Cimg: (N, H, W, 3).  Returns X_0, log_lambda and the cache for backward."""
    cache = {}
    st = {name: s for name, _, _, s in layer_shapes(base)}

    def layer(name, x, relu=True):
        z = conv(x, P[name + ".w"], P[name + ".b"], st[name])
        cache[name] = (x, z)
        return np.maximum(z, 0.0) if relu else z

    e1 = layer("e1", Cimg)
    e2 = layer("e2", e1)
    e3 = layer("e3", e2)
    e4 = layer("e4", e3)
    d3 = layer("d3", up2(e4)) + e3
    d2 = layer("d2", up2(d3)) + e2
    d1 = layer("d1", up2(d2)) + e1
    out = layer("out", d1, relu=False)
    g = e4.mean(axis=(1, 2))
    loglam = g @ P["lam.w"] + P["lam.b"][0]
    cache["g"] = g
    cache["e4_act"] = e4
    return Cimg + out, loglam, cache


def loss_and_grads(P: Dict[str, np.ndarray], Cimg: np.ndarray, Xstar: np.ndarray, logmu: np.ndarray,
                   base: int):
    """Loss of the batch and the gradient of every parameter (chain rule, written out)."""
    X0, loglam, cache = forward(P, Cimg, base)
    N = Cimg.shape[0]
    nrm = (Xstar ** 2).sum(axis=(1, 2, 3))
    diff = X0 - Xstar
    loss = float(np.mean((diff ** 2).sum(axis=(1, 2, 3)) / nrm + (loglam - logmu) ** 2))
    G = {}
    dout = 2.0 * diff / (nrm[:, None, None, None] * N)
    dloglam = 2.0 * (loglam - logmu) / N
    G["lam.w"] = cache["g"].T @ dloglam
    G["lam.b"] = np.array([dloglam.sum()])
    st = {name: s for name, _, _, s in layer_shapes(base)}

    def back(name, dy, relu=True):
        x, z = cache[name]
        if relu:
            dy = dy * (z > 0)
        dx, G[name + ".w"], G[name + ".b"] = conv_backward(x, P[name + ".w"], dy, st[name])
        return dx

    dd1 = back("out", dout, relu=False)
    de1 = dd1.copy()
    dd2 = up2_backward(back("d1", dd1))
    de2 = dd2.copy()
    dd3 = up2_backward(back("d2", dd2))
    de3 = dd3.copy()
    de4 = up2_backward(back("d3", dd3))
    e4 = cache["e4_act"]
    de4 = de4 + (dloglam[:, None] * P["lam.w"][None, :])[:, None, None, :] / (e4.shape[1] * e4.shape[2])
    de3 = de3 + back("e4", de4)
    de2 = de2 + back("e3", de3)
    de1 = de1 + back("e2", de2)
    back("e1", de1)
    return loss, G
