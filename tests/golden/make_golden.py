"""Write the oracle's results on the two plain image workloads to JSON fixtures.

Calls only oracle/ (and the seeded generators in workloads/).  The stored
values are regression fixtures of the FP64 oracle, not the paper's
numbers: the paper prints no worked example with reproducible inputs
(its Table 1 image and settings are not given).  Run from the repo root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402


def run(which):
    p = workloads.image_config(which)
    mats = oracle.factor_matrices(p.dims, p.factors, p.right_factors)
    C, _, nu_c = oracle.make_observation(p.x_true, mats, p.noise, p.nu)
    th = oracle.sketch_matrices(p.dims, p.sketch_dims, p.seed, p.problem_id)
    tol = oracle.rho_star(nu_c)
    r = oracle.rtg_gmres(mats, C, p.m, th, tol=tol, lam=p.lam, mu_grid=p.mu_grid)
    rng = np.random.default_rng(1234)
    idx = rng.integers(0, np.prod(p.dims), size=64)
    Xf = r["X"].ravel(order="F")
    return {
        "workload": p.name, "dims": list(p.dims), "nu_C": nu_c, "tol": tol,
        "iters": r["iters"], "rho": r["rho"], "mu": r["mu"], "beta": r["beta"],
        "gcv": None if r["gcv"] is None else list(map(float, r["gcv"])),
        "H": r["H"].tolist(), "sample_index": idx.tolist(),
        "sample_X": [float(Xf[i]) for i in idx],
        "X_norm": oracle.frobenius_norm(r["X"]),
        "RE": oracle.relative_error(p.x_true, r["X"]), "PSNR": oracle.psnr(p.x_true, r["X"]),
    }


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)))
    for which, name in [(1, "image64_f64.json"), (2, "image512_f32.json")]:
        with open(os.path.join(out, name), "w") as f:
            json.dump(run(which), f, indent=1)
        print("wrote", name)
