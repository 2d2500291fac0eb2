"""Seeded synthetic workloads for RTG-GMRES image and video restoration.

This module only draws inputs: images, videos, raw Gaussian noise, the
blur taps and channel-mixing matrix that define the operator, the
regularisation grid and the per-problem parameters of a batch.  It holds
none of the method's arithmetic (no operator application, no sketch, no
Krylov step), so both the CPU oracle's tests and the GPU benchmark draw
identical inputs from it without sharing any code of the method.

The test image of the paper's Example 1 (Section 5, Table 1) is not
available; the generators below stand in for it with the structure the
paper's model describes (Section 5.1: an N x N x 3 RGB image with entries
in [0, 1]; Section 5.3: zero-mean iid Gaussian noise; Eq. 58: Gaussian
PSF).  Arrays use numpy shape (I1, I2, ...) and are meant to be flattened
with mode 1 fastest (Fortran order), the ivec ordering of Section 4.1.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "piecewise_image", "smooth_video", "gaussian_taps", "box_taps",
    "channel_mix", "noise_draw", "mu_grid", "Problem", "image_config",
    "video_config", "batched_configs", "CONFIGS",
]


def _rng(seed: int, stream: int) -> np.random.Generator:
    # Independent streams for image, noise, ... derived from one seed.
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, stream])))


def piecewise_image(I1: int, I2: int, channels: int = 3, seed: int = 0,
                    n_rect: int = 20) -> np.ndarray:
    """Piecewise-smooth colour image in [0, 1].

    Half weight: ``n_rect`` axis-aligned rectangles with uniform random
    corners, drawn in painter's order, each with one U[0,1] value per
    channel.  Half weight: the linear ramp (i1/I1 + i2/I2)/2 in every
    channel.
    """
    rng = _rng(seed, 1)
    rect = np.zeros((I1, I2, channels))
    for _ in range(n_rect):
        a1, b1 = np.sort(rng.integers(0, I1, size=2))
        a2, b2 = np.sort(rng.integers(0, I2, size=2))
        val = rng.uniform(0.0, 1.0, size=channels)
        rect[a1:b1 + 1, a2:b2 + 1, :] = val
    i1 = np.arange(I1)[:, None] / I1
    i2 = np.arange(I2)[None, :] / I2
    ramp = 0.5 * (i1 + i2)
    return 0.5 * rect + 0.5 * ramp[:, :, None]


def smooth_video(I1: int, I2: int, channels: int = 3, frames: int = 8,
                 seed: int = 0, n_bumps: int = 16) -> np.ndarray:
    """Smooth colour video translated by one pixel per frame along mode 2.

    Each channel of an I1 x (I2 + frames) canvas is a sum of ``n_bumps``
    isotropic Gaussian bumps (random centre, width in [I1/32, I1/6],
    amplitude in [0, 1]), rescaled to [0, 1].  Frame t is the window of
    columns [t, t + I2).  Returns shape (I1, I2, channels, frames).
    """
    rng = _rng(seed, 2)
    W = I2 + frames
    x = np.arange(I1)[:, None]
    y = np.arange(W)[None, :]
    canvas = np.zeros((I1, W, channels))
    for c in range(channels):
        for _ in range(n_bumps):
            cx = rng.uniform(0, I1)
            cy = rng.uniform(0, W)
            w = rng.uniform(I1 / 32.0, I1 / 6.0)
            amp = rng.uniform(0.0, 1.0)
            canvas[:, :, c] += amp * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * w * w))
        lo, hi = canvas[:, :, c].min(), canvas[:, :, c].max()
        canvas[:, :, c] = (canvas[:, :, c] - lo) / max(hi - lo, 1e-300)
    out = np.empty((I1, I2, channels, frames))
    for t in range(frames):
        out[:, :, :, t] = canvas[:, t:t + I2, :]
    return out


def gaussian_taps(sigma: float, radius: int) -> np.ndarray:
    """1-D taps of the separable Gaussian PSF of Eq. 58, normalised to sum 1.

    Eq. 58 is unnormalised; scaling the taps so the blur preserves the
    mean intensity fixes the operator's scale (a reading recorded in the
    design notes).  Entry ``radius + t`` is the weight of offset t.
    """
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    a = np.exp(-0.5 * (t / sigma) ** 2)
    return a / a.sum()


def box_taps(width: int) -> np.ndarray:
    """Temporal box blur of odd ``width``: weight 1/width on each offset."""
    assert width % 2 == 1
    return np.full(width, 1.0 / width)


def channel_mix() -> np.ndarray:
    """The 3 x 3 cross-channel mixing matrix of the colour workloads."""
    return np.array([[0.8, 0.1, 0.1], [0.1, 0.8, 0.1], [0.1, 0.1, 0.8]])


def noise_draw(shape: Sequence[int], seed: int) -> np.ndarray:
    """Raw iid N(0, 1) draws E; the noise of Eq. 59 is nu*||C_hat||*E/||E||."""
    return _rng(seed, 3).standard_normal(tuple(shape))


def mu_grid(n: int = 8, lo: float = 1e-4, hi: float = 1e-1) -> np.ndarray:
    """Log-spaced regularisation grid for GCV (n values in [lo, hi])."""
    return np.logspace(math.log10(lo), math.log10(hi), n)


@dataclasses.dataclass
class Problem:
    """One restoration problem: ground truth, operator factors, settings.

    ``factors`` is a list of (mode, kind, data) with mode 1-based, kind in
    {"banded", "dense", "identity"}; banded data are taps (length 2r+1),
    dense data are the matrix M applied as X x_mode M.
    ``right_factors`` holds Einstein right-product matrices B (applied as
    X x_mode B^T).
    """
    name: str
    x_true: np.ndarray
    noise: np.ndarray
    nu: float
    factors: List[Tuple[int, str, np.ndarray]]
    right_factors: List[Tuple[int, str, np.ndarray]]
    m: int
    sketch_dims: Tuple[int, ...]
    lam: float                      # > 0 fixed mu, <= 0: GCV over mu_grid
    mu_grid: Optional[np.ndarray]
    seed: int                       # Philox key word 0 for the sketch
    problem_id: int = 0             # Philox key word 1
    dtype: str = "f32"

    @property
    def dims(self) -> Tuple[int, ...]:
        return tuple(self.x_true.shape)


def image_config(which: int, seed: int = 0) -> Problem:
    """The two plain colour-image workloads.

    which=1: 64x64x3 FP64, sigma 1.5, radius 4, channels untouched,
             noise 1e-3, m=30, sketch (32,32,3), mu=1e-3, Philox seed 0.
    which=2: 512x512x3 FP32, sigma 2.5, radius 7, 3x3 channel mixing,
             noise 1e-2, m=50, sketch (128,128,3), mu by GCV over 8 values.
    """
    if which == 1:
        x = piecewise_image(64, 64, 3, seed)
        a = gaussian_taps(1.5, 4)
        return Problem("image64_f64", x, noise_draw(x.shape, seed), 1e-3,
                       [(1, "banded", a), (2, "banded", a)], [], 30,
                       (32, 32, 3), 1e-3, None, 0, 0, "f64")
    if which == 2:
        x = piecewise_image(512, 512, 3, seed)
        a = gaussian_taps(2.5, 7)
        return Problem("image512_f32", x, noise_draw(x.shape, seed), 1e-2,
                       [(1, "banded", a), (2, "banded", a)],
                       [(3, "dense", channel_mix())], 50,
                       (128, 128, 3), -1.0, mu_grid(), seed, 0, "f32")
    raise ValueError(which)


def video_config(seed: int = 0, I: int = 256, frames: int = 64) -> Problem:
    """Video workload: I x I x 3 x frames, spatial sigma 2 radius 6,
    channel mixing, temporal box of width 5, noise 5e-3, m=40,
    sketch (96, 96, 3, 32) scaled with I and frames."""
    x = smooth_video(I, I, 3, frames, seed)
    a = gaussian_taps(2.0, 6)
    s_sp = max(1, (96 * I) // 256)
    s_t = max(1, frames // 2)
    return Problem(f"video{I}x{frames}", x, noise_draw(x.shape, seed), 5e-3,
                   [(1, "banded", a), (2, "banded", a), (4, "banded", box_taps(5))],
                   [(3, "dense", channel_mix())], 40, (s_sp, s_sp, 3, s_t),
                   -1.0, mu_grid(), seed, 0, "bf16")


def batched_configs(n_problems: int = 256, seed: int = 0,
                    side_lo: int = 64, side_hi: int = 1024) -> List[dict]:
    """Per-problem parameters of the batched workload (no pixel data).

    Side lengths uniform in [side_lo, side_hi] (independently per mode),
    blur sigma uniform in [0.5, 3] with radius ceil(3 sigma), noise and
    mu log-uniform in [1e-3, 2e-2] and [1e-4, 1e-1], m=30, sketch
    min(I_k, 128) per spatial mode.
    """
    rng = _rng(seed, 4)
    out = []
    for p in range(n_problems):
        I1 = int(rng.integers(side_lo, side_hi + 1))
        I2 = int(rng.integers(side_lo, side_hi + 1))
        sigma = float(rng.uniform(0.5, 3.0))
        nu = float(10 ** rng.uniform(math.log10(1e-3), math.log10(2e-2)))
        mu = float(10 ** rng.uniform(-4, -1))
        out.append(dict(problem_id=p, dims=(I1, I2, 3), sigma=sigma,
                        radius=int(math.ceil(3 * sigma)), nu=nu, mu=mu, m=30,
                        sketch_dims=(min(I1, 128), min(I2, 128), 3),
                        image_seed=seed * 100003 + p))
    return out


CONFIGS = {
    "image64_f64": lambda seed=0: image_config(1, seed),
    "image512_f32": lambda seed=0: image_config(2, seed),
    "video256x64": lambda seed=0: video_config(seed),
}


def warmstart_layer_shapes(base: int):
    """(name, c_in, c_out, stride) of the warm-start network's 3x3 convolutions."""
    c = base
    return [("e1", 3, c, 1), ("e2", c, 2 * c, 2), ("e3", 2 * c, 4 * c, 2), ("e4", 4 * c, 4 * c, 2),
            ("d3", 4 * c, 4 * c, 1), ("d2", 4 * c, 2 * c, 1), ("d1", 2 * c, c, 1), ("out", c, 3, 1)]


def warmstart_params(base: int, seed: int) -> dict:
    """Seeded initial parameters of the warm-start network: He-normal
    convolution weights (c_out, 3, 3, c_in), zero biases, and a zero output
    layer and lambda head (so the untrained network returns X_0 = C,
    log lambda = 0).  Ordered as the flat parameter array."""
    rng = _rng(seed, 5)
    P = {}
    for name, cin, cout, _ in warmstart_layer_shapes(base):
        std = math.sqrt(2.0 / (9 * cin)) if name != "out" else 0.0
        P[name + ".w"] = rng.standard_normal((cout, 3, 3, cin)) * std
        P[name + ".b"] = np.zeros(cout)
    P["lam.w"] = np.zeros(4 * base)
    P["lam.b"] = np.zeros(1)
    return P


def flatten_params(P: dict) -> np.ndarray:
    return np.concatenate([np.asarray(v, dtype=np.float64).ravel() for v in P.values()])
