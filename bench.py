"""Benchmark: RTG-GMRES solves/s on the 512x512x3 FP32 colour-image workload.

One step = one complete RTG-GMRES solve (sketch signs, R_0 and beta,
sketched Arnoldi steps until rho <= rho*, projected Tikhonov with GCV over
8 values of mu, assembly of X) on a seeded synthetic blurred, noisy image.
Default: N=1 GPU, 20 timed steps after 5 warm-up steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own problems (replicas: the path has no
exchange step), value = all solves / max-over-ranks time.  The reference
arm (--impl reference) times the FP64 CPU oracle on this host's cores.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "RTG-GMRES solves/s at rel. residual 1e-3: chosen form vs plain FP32, same GB300"
WORKLOAD = "image512x512x3_f32"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--problems", type=int, default=256,
                    help="distinct seeded problems (the plain form cycles them, the batched form solves "
                         "them together)")
    ap.add_argument("--batch", type=int, default=256, help="problems per batched launch (chosen form)")
    ap.add_argument("--queue-slots", type=int, default=8,
                    help="batched form: graph branches that take the batch's problems from a device work "
                         "queue (0: one graph branch per problem)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-warm-start", action="store_true", help="skip the learned warm-start form")
    ap.add_argument("--direct", action="store_true",
                    help="launch every solve's kernels directly instead of replaying its CUDA graph "
                         "(for profilers that do not see kernels inside conditional graph nodes); "
                         "skips the phase-timed roofline pass")
    ap.add_argument("--group-max", type=int, default=0,
                    help="batched form: problems of one lock-step group (0: one graph branch per problem)")
    ap.add_argument("--only-batched", action="store_true",
                    help="run the batched form alone (no plain, Golub-Kahan or warm-start forms, no phase "
                         "passes, no end-to-end pass): for profiler captures of its kernels")
    ap.add_argument("--restarts", type=int, default=0,
                    help="restarted cycles allowed per solve in every form (a cycle that reaches j = m above "
                         "rho* restarts from its least-squares iterate); the restarted batched form is "
                         "reported beside the chosen one in any case")
    ap.add_argument("--no-extra-forms", action="store_true",
                    help="skip the video precision form, the batched BF16-basis form and the uneven "
                         "256-problem batch")
    ap.add_argument("--uneven", type=int, default=256, help="problems of the uneven batched workload")
    ap.add_argument("--ws-full", action="store_true",
                    help="learned warm start at its full configuration: 20k training pairs of 128x128x3, "
                         "evaluated on 512 held-out 512x512x3 problems (about two minutes more)")
    ap.add_argument("--cpu-leg", type=int, default=0,
                    help="internal: time the oracle alone with this many BLAS threads and print JSON")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def job_times(local, world: int, device: str):
    """The slowest rank's value of each of this rank's times (MAX all-reduce
    over the process group when world > 1); `device` holds the reduced
    tensor ("cuda" under NCCL, "cpu" under gloo)."""
    import torch
    t = torch.tensor([float(x) for x in local], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def job_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput of replicas: every rank's units over the slowest time."""
    return world * units_per_rank / seconds


def rho_star(nu_c: float) -> float:
    # stop level of the relative sketched residual: 1e-3, or the noise floor
    # of the observation when that lies above it (discrepancy principle)
    return max(1e-3, 1.01 * nu_c)


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """SM clock and clock-event (throttle) reasons during the timed region:
    read-only NVML queries every 10 ms from a thread (libnvidia-ml through
    ctypes), else nvidia-smi every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown",
               0x4: "sw_power_cap", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index: int):
        # NVML and nvidia-smi number the GPUs physically; CUDA numbers the visible ones
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [t.strip() for t in vis.split(",") if t.strip()]
        self.gpu = int(ids[cuda_index]) if cuda_index < len(ids) and ids[cuda_index].isdigit() else cuda_index
        self.proc = None
        self.lines = []
        self.samples = []       # (sm MHz, reason bits) from NVML
        self.max_mhz = None
        self.nvml = None
        self.stop = threading.Event()
        self.t = None

    def _start_nvml(self) -> bool:
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return False
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.gpu), ctypes.byref(h)) != 0:
                lib.nvmlShutdown()
                return False
            fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
        except (OSError, AttributeError):
            return False
        mx = ctypes.c_uint(0)
        if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:   # 1: the SM clock domain
            self.max_mhz = float(mx.value)

        def loop():
            c, r = ctypes.c_uint(0), ctypes.c_ulonglong(0)
            while not self.stop.is_set():
                if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(c)) == 0 and fn(h, ctypes.byref(r)) == 0:
                    self.samples.append((float(c.value), int(r.value)))
                self.stop.wait(0.01)
        self.nvml = lib
        self.t = threading.Thread(target=loop, daemon=True)
        self.t.start()
        return True

    def __enter__(self):
        if self._start_nvml():
            return self
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.nvml is not None:
            self.stop.set()
            self.t.join(timeout=2)
            self.nvml.nvmlShutdown()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.nvml is not None:
            sm = [c for c, _ in self.samples]
            reasons = sorted({nm for _, r in self.samples for bit, nm in self.REASONS.items() if r & bit})
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.max_mhz,
                    "reasons": reasons, "samples": len(sm), "source": "NVML, every 10 ms"}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi, every 200 ms"}


# ----------------------------------------------------------------------------- problems

def make_problems(h, api, torch, count: int, seed0: int):
    """Observations built on the device with the library's own operator (outside the timed region)."""
    probs = []
    for s in range(count):
        p = workloads.image_config(2, seed=seed0 + s)
        A = [api.banded(m, p.dims[m - 1], t) for m, _, t in p.factors]
        B = [api.dense(m, t) for m, _, t in p.right_factors]
        X = api.to_device(p.x_true, torch.float32)
        Ch = h.operator_apply(X, A, B)
        E = api.to_device(p.noise, torch.float32)
        N = E * (p.nu * torch.linalg.vector_norm(Ch) / torch.linalg.vector_norm(E))
        C = api.empty(p.dims, torch.float32)
        C.copy_(Ch + N)
        nu_c = float(torch.linalg.vector_norm(N) / torch.linalg.vector_norm(C))
        probs.append(dict(p=p, A=A, B=B, C=C, tol=rho_star(nu_c), nu_c=nu_c))
    return probs


USE_GRAPH = True


RESTARTS = 0


def solve(h, pr, X, stream=None, host=False, bf16=False):
    p = pr["p"]
    C = pr["C_host"] if host else pr["C"]
    return h.gmres_solve(C, p.m, p.sketch_dims, p.seed, p.lam, pr["A"], pr["B"], X=X, tol=pr["tol"],
                         mu_grid=p.mu_grid, use_graph=USE_GRAPH, max_restarts=RESTARTS, bf16_basis=bf16,
                         stream=stream)


# ----------------------------------------------------------------------------- roofline

# Kernel groups whose minimum traffic the byte model below covers, and the
# source files that define each (the recorded ncu traffic is dropped when
# one of them has changed since).
PHASE_FILES = {"apply": ["k_apply.cu"], "sketch": ["k_sketch.cu", "gs_common.cuh", "tma_common.cuh", "umma_common.cuh"],
               "gs": ["k_arnoldi.cu", "gs_common.cuh"],
               "update": ["k_arnoldi.cu", "gs_common.cuh", "tma_common.cuh"],
               "assemble": ["k_solve.cu"], "init": ["k_arnoldi.cu", "k_sketch.cu"]}
KERNEL_NAMES = {"apply": "k_apply_reg<float,3,7> (W = Phi(V_j))",
                "sketch": "k_sk_first_umma<float> (tcgen05) + k_sk_inner_tc<32> (S(W) with fused sketched dots)",
                "update": "k_update_ring<float, slot, depth> (V_{j+1} streamed through a shared-memory ring of "
                          "the autotuned geometry, its sketched column, Givens block)",
                "assemble": "k_assemble<float>", "init": "prologue group"}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.txt")


def source_sha(phase: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in PHASE_FILES.get(phase, []) + ["rtg_internal.cuh"]:
        with open(os.path.join(ROOT, "paper_2603_00839_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(phase: str, workload: str, bytes_per_launch: float):
    """DRAM bytes per launch: the ratio of DRAM to algorithmic bytes that the
    committed ncu summary measured for this kernel group and workload, times
    this run's algorithmic bytes per launch (the group's traffic grows with
    the tensors it reads); None when the kernel source changed since."""
    try:
        lines = open(TRAFFIC_FILE).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        if ln.startswith("#"):
            continue
        kv = dict(t.split("=", 1) for t in ln.split() if "=" in t)
        if kv.get("phase") == phase and kv.get("workload") == workload:
            if kv.get("source_sha") != source_sha(phase):
                return None
            return round(float(kv["dram_ratio"]) * bytes_per_launch)
    return None


def cycle_steps(k: int, m: int):
    """Per-cycle step counts of a solve of k Arnoldi steps in cycles of at most m."""
    out = [m] * (k // m)
    if k % m or not out:
        out.append(k % m)
    return out


def phase_bytes(phase: str, n: int, d: int, k: int, b: int, m: int = 10 ** 9) -> float:
    """Minimum (algorithmic) bytes of one kernel group summed over a solve of k
    Arnoldi steps (cycles of at most m steps: j restarts at 0 in each);
    n tensor entries, d sketch entries, b bytes per entry.  Step j
    (0-based) builds V_{j+1} from W = Phi(V_j) and V_0..V_j."""
    cyc = cycle_steps(k, m)
    if phase == "apply":      # read V_j, write W
        return k * 2 * n * b
    if phase == "sketch":     # read W, write S(W), read Q_0..Q_j for the fused dots
        return sum(n * b + d * b + (j + 1) * d * b for c in cyc for j in range(c))
    if phase == "update":     # read W and V_0..V_j, write V_{j+1}; Q column from S and Q_0..Q_j
        return sum((j + 3) * n * b + (j + 3) * d * b for c in cyc for j in range(c))
    if phase == "assemble":   # read V_0..V_{k-1}, write X (last cycle)
        return (cyc[-1] + 1) * n * b
    if phase == "init":       # read C, write V_0 (scaled), sketch read of C; per restart also X += V y
        return 3 * n * b + sum((c + 1) * n * b + 4 * n * b for c in cyc[:-1])
    return 0.0


def phase_report(h, probs, X, peaks, workload: str):
    """One direct-launch solve per problem with every kernel group timed by CUDA
    events on the solve's stream; returns the per-group table and the
    roofline of the byte-bound group with the largest device time."""
    tot_ms, tot_l, tot_bytes, iters = {}, {}, {}, []
    p0 = probs[0]["p"]
    n = int(np.prod(p0.dims))
    d = int(np.prod([min(s, i) for s, i in zip(p0.sketch_dims, p0.dims)]))
    for pr in probs:
        p = pr["p"]
        _, info = h.gmres_solve(pr["C"], p.m, p.sketch_dims, p.seed, p.lam, pr["A"], pr["B"], X=X,
                                tol=pr["tol"], mu_grid=p.mu_grid, phase_times=True, max_restarts=RESTARTS)
        iters.append(info.iters)
        for k, v in info.phase_ms.items():
            tot_ms[k] = tot_ms.get(k, 0.0) + v
            tot_l[k] = tot_l.get(k, 0) + info.phase_launches[k]
            tot_bytes[k] = tot_bytes.get(k, 0.0) + phase_bytes(k, n, d, info.iters, 4, p.m)
    solves = len(probs)
    table = {}
    for k in tot_ms:
        if tot_l[k] == 0:
            continue
        e = {"us_per_solve": round(1e3 * tot_ms[k] / solves, 2), "launches_per_solve": tot_l[k] / solves}
        if tot_bytes[k] > 0:
            e["gbs"] = round(tot_bytes[k] / (tot_ms[k] * 1e-3) / 1e9, 1)
        table[k] = e
    share_total = sum(tot_ms.values())
    for k in table:
        table[k]["share"] = round(tot_ms[k] / share_total, 3)
    cand = [k for k in table if tot_bytes.get(k, 0) > 0 and k in ("apply", "sketch", "update")]
    dom = max(cand, key=lambda k: tot_ms[k])
    launches = tot_l[dom]
    bytes_per_launch = tot_bytes[dom] / launches
    us_per_launch = 1e3 * tot_ms[dom] / launches
    ach = bytes_per_launch / (us_per_launch * 1e-6) / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    roof = {"kernel": KERNEL_NAMES.get(dom, dom), "phase": dom, "bound": "hbm", "achieved": round(ach, 1),
            "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
            "traffic": recorded_traffic(dom, workload, bytes_per_launch), "bytes_per_launch": round(bytes_per_launch),
            "us_per_launch": round(us_per_launch, 3), "launches": launches,
            "timing": "CUDA events around each kernel group of direct-launch solves, stream gated "
                      "until the group is queued",
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs, burst copy)",
            "mean_iters": float(np.mean(iters))}
    return roof, table


def batched_phase_report(h, batch, grid, peaks, workload: str):
    """The batch of the chosen form run once more as one lock-step group with
    direct launches and every kernel group timed by CUDA events (each launch
    serves all problems of the batch; a stopped problem's blocks return at
    once).  Returns the roofline of the byte-bound group with the largest
    device time and the per-group table: algorithmic bytes summed over the
    problems' own steps."""
    _, res = h.gmres_solve_batched(batch, mu_grid=grid, phase_times=True, group_max=len(batch),
                                   max_restarts=RESTARTS)
    C0 = batch[0]["C"]
    n = int(np.prod(C0.shape))
    d = int(np.prod([min(s, i) for s, i in zip(batch[0]["sketch_dims"], C0.shape)]))
    ms, launches = res[0].phase_ms, res[0].phase_launches
    tot_bytes = {k: sum(phase_bytes(k, n, d, r.iters, 4, batch[0]["m"]) for r in res) for k in ms}
    table = {}
    share_total = sum(ms.values())
    for k in ms:
        if launches[k] == 0:
            continue
        e = {"us_per_batch": round(1e3 * ms[k], 2), "launches_per_batch": launches[k],
             "share": round(ms[k] / share_total, 3)}
        if tot_bytes[k] > 0:
            e["gbs"] = round(tot_bytes[k] / (ms[k] * 1e-3) / 1e9, 1)
        table[k] = e
    cand = [k for k in table if tot_bytes.get(k, 0) > 0 and k in ("apply", "sketch", "update")]
    dom = max(cand, key=lambda k: ms[k])
    bytes_per_launch = tot_bytes[dom] / launches[dom]
    us_per_launch = 1e3 * ms[dom] / launches[dom]
    ach = bytes_per_launch / (us_per_launch * 1e-6) / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    roof = {"kernel": KERNEL_NAMES.get(dom, dom), "phase": dom, "bound": "hbm", "achieved": round(ach, 1),
            "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
            "traffic": recorded_traffic(dom, workload + "_lockstep16", bytes_per_launch),
            "bytes_per_launch": round(bytes_per_launch), "us_per_launch": round(us_per_launch, 3),
            "launches": launches[dom], "problems_per_launch": len(batch),
            "timing": "CUDA events around each kernel group of the batch run as one lock-step group "
                      "(direct launches, stream gated until the group is queued)",
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs, burst copy)" if "fallback" not in peaks
                           else "fallback 6800 GB/s",
            "iters": [r.iters for r in res]}
    return roof, table


# ----------------------------------------------------------------------------- warm start

def warm_start_form(h, api, torch, probs, train_n=512, steps=400, I=128, base=32, held_out=0):
    """Learned warm start: trained here on solver-labelled IxIx3 pairs of the
    workload's operator family (sigma U[0.5, 3], radius ceil(3 sigma), the 3x3
    channel mix, noise 2e-3..2e-2), then problems of the benchmark's workload
    solved cold (plain RTG-GMRES, GCV) and warm (rtg_ws_solve: prediction,
    fallback test and stop-level rescale on the device) to the same stop level
    ||S(C - Phi X)|| <= rho* ||S(C)||.  Wall clock per solve, one at a time,
    inference and the fallback test included.  held_out > 0 evaluates on that
    many fresh 512x512x3 problems instead of the benchmark's."""
    rng = np.random.default_rng(123)
    grid = workloads.mu_grid()
    sk = (64, 64, 3)
    train, Xs, mus = [], [], []
    t0 = time.perf_counter()
    Mix = [api.dense(3, workloads.channel_mix())]
    for i in range(train_n):
        x = workloads.piecewise_image(I, I, 3, 70000 + i)
        sig = float(rng.uniform(0.5, 3.0))
        taps = workloads.gaussian_taps(sig, int(np.ceil(3 * sig)))
        A = [api.banded(1, I, taps), api.banded(2, I, taps)]
        X = api.to_device(x, torch.float32)
        Ch = h.operator_apply(X, A, Mix)
        E = api.to_device(workloads.noise_draw(x.shape, 70000 + i), torch.float32)
        nu = float(10 ** rng.uniform(np.log10(2e-3), np.log10(2e-2)))
        C = api.empty(x.shape, torch.float32)
        C.copy_(Ch + E * (nu * torch.linalg.vector_norm(Ch) / torch.linalg.vector_norm(E)))
        train.append(dict(C=C, A=A, B=Mix, m=30, sketch_dims=sk, seed=5, lam=-1.0, tol=max(1e-3, 1.01 * nu)))
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    for k in range(0, train_n, 64):
        X, res = h.gmres_solve_batched(train[k:k + 64], mu_grid=grid, max_restarts=RESTARTS)
        Xs += X
        mus += [r.mu for r in res]
    torch.cuda.synchronize()
    label_s = time.perf_counter() - t0
    net = api.WarmStart(base, workloads.flatten_params(workloads.warmstart_params(base, 11)))
    t0 = time.perf_counter()
    losses = []
    for step in range(steps):
        idx = rng.choice(train_n, 16, replace=False)
        Cb = api.stack_images([train[i]["C"] for i in idx])
        Xb = api.stack_images([Xs[i] for i in idx])
        lm = torch.tensor(np.log([mus[i] for i in idx]), dtype=torch.float32, device="cuda")
        losses.append(net.train_step(Cb, Xb, lm, I, I, lr=2e-3 if step < steps * 3 // 4 else 5e-4))
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del train, Xs
    if held_out > 0:
        evalp = make_problems(h, api, torch, held_out, seed0=10000)
    else:
        evalp = probs
    Xo = api.empty(evalp[0]["p"].dims, torch.float32)

    def cold(pr):
        p = pr["p"]
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, info = h.gmres_solve(pr["C"], p.m, p.sketch_dims, p.seed, p.lam, pr["A"], pr["B"], X=Xo, tol=pr["tol"],
                                mu_grid=p.mu_grid, max_restarts=RESTARTS)
        return time.perf_counter() - t, info

    def warm(pr):
        p = pr["p"]
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, info, dec = net.solve(h, pr["C"], p.m, p.sketch_dims, p.seed, pr["A"], pr["B"], X=Xo, tol=pr["tol"],
                                 mu_grid=p.mu_grid, max_restarts=RESTARTS)
        return time.perf_counter() - t, info, dec

    for pr in evalp[:2]:
        cold(pr)
        warm(pr)
    tc, ic, tw, iw, fb, conv_c, conv_w = [], [], [], [], 0, 0, 0
    for pr in evalp:
        a, r = cold(pr)
        tc.append(a)
        ic.append(r.iters)
        conv_c += int(r.converged)
        a, r, dec = warm(pr)
        tw.append(a)
        iw.append(r.iters)
        fb += int(dec["fell_back"])
        conv_w += int(r.converged)
    return {"value": round(conv_w / sum(tw), 2), "unit": "solves/s reaching rho* (wall clock, one at a time)",
            "cold_value": round(conv_c / sum(tc), 2), "mean_iters_warm": float(np.mean(iw)),
            "mean_iters_cold": float(np.mean(ic)), "fallbacks": f"{fb}/{len(evalp)}",
            "reached_stop_level": {"warm": f"{conv_w}/{len(evalp)}", "cold": f"{conv_c}/{len(evalp)}"},
            "evaluated_on": (f"{held_out} held-out 512x512x3 problems (seeds 10000..)" if held_out else
                             "the benchmark's 512x512x3 problems"),
            "training": {"pairs": train_n, "image": [I, I, 3], "steps": steps, "batch": 16,
                         "loss_first": round(float(np.mean(losses[:5])), 4),
                         "loss_last": round(float(np.mean(losses[-20:])), 4),
                         "generate_s": round(gen_s, 2), "label_s": round(label_s, 2), "train_s": round(train_s, 2)},
            "path": "rtg_ws_solve (predict, ||S(R_0)|| vs ||S(C)||, fallback and tol rescale on the device)",
            "network": f"4-level conv encoder-decoder, base {base}, BF16 tensor-core kernels"}


# ----------------------------------------------------------------------------- CPU baseline

def oracle_solves(seconds: float, problems: int = 16):
    """FP64 CPU oracle as it stands on the 512x512x3 workload (observation,
    signs and a restarted solve to rho*), for about `seconds`; returns
    (solves, elapsed, mean steps)."""
    import oracle
    done, iters, t0 = 0, [], time.perf_counter()
    while True:
        p = workloads.image_config(2, seed=done % problems)
        mats = oracle.factor_matrices(p.dims, p.factors, p.right_factors)
        C, _, nu_c = oracle.make_observation(p.x_true, mats, p.noise, p.nu)
        th = oracle.sketch_matrices(p.dims, p.sketch_dims, p.seed, p.problem_id)
        r = oracle.rtg_gmres(mats, C, p.m, th, tol=rho_star(nu_c), lam=p.lam, mu_grid=p.mu_grid,
                             max_restarts=RESTARTS)
        iters.append(r["iters"])
        done += 1
        if time.perf_counter() - t0 >= seconds:
            break
    return done, time.perf_counter() - t0, float(np.mean(iters))


def cpu_leg_main(threads: int, seconds: float):
    """Entry of the single-thread leg (run in a child process whose BLAS
    thread count was fixed by its environment before numpy loaded)."""
    done, el, it = oracle_solves(seconds)
    print(json.dumps({"solves": done, "seconds": el, "mean_iters": it, "threads": threads}), flush=True)


def cpu_baseline(seconds: float):
    """The oracle timed twice on this host: BLAS threads = all cores (this
    process) and 1 thread (a child process started with the thread count set
    in its environment).  The headline value is the all-cores leg."""
    done, el, it = oracle_solves(seconds)
    one = None
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-leg", "1", "--cpu-seconds",
                            str(seconds)], capture_output=True, text=True, env=env, timeout=20 * seconds + 120)
        for ln in r.stdout.splitlines():
            if ln.startswith("{"):
                one = json.loads(ln)
    except (OSError, subprocess.SubprocessError, ValueError):
        one = None
    out = {"value": round(done / el, 4), "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"{done} full FP64 oracle solves of the 512x512x3 workload (observation, signs, "
                     f"restarted solve to rho*, mean {it:.1f} Arnoldi steps), numpy BLAS default threads"}
    if one is not None:
        out["single_thread"] = {"value": round(one["solves"] / one["seconds"], 4), "unit": "solves/s",
                                "cores": 1, "sample": f"{one['solves']} solves, mean {one['mean_iters']:.1f} "
                                                      "steps, BLAS threads = 1"}
    return out


# ----------------------------------------------------------------------------- arms

def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    probs = [dict(p=workloads.image_config(2, seed=s)) for s in range(args.problems)]
    import oracle
    times = []
    iters = []
    for step in range(args.warmup + args.steps):
        pr = probs[step % len(probs)]
        p = pr["p"]
        t0 = time.perf_counter()
        mats = oracle.factor_matrices(p.dims, p.factors, p.right_factors)
        C, _, nu_c = oracle.make_observation(p.x_true, mats, p.noise, p.nu)
        th = oracle.sketch_matrices(p.dims, p.sketch_dims, p.seed, p.problem_id)
        r = oracle.rtg_gmres(mats, C, p.m, th, tol=rho_star(nu_c), lam=p.lam, mu_grid=p.mu_grid,
                             max_restarts=RESTARTS)
        t = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(t)
            iters.append(r["iters"])
    tot = sum(times)
    val = args.steps / tot
    out = {"impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": "solves/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(1e3 * tot / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "dims": [512, 512, 3], "m": 50,
                      "sketch": [128, 128, 3], "gcv_grid": 8, "mean_iters": float(np.mean(iters)),
                      "stop": "rho <= max(1e-3, 1.01*nu_C)", "restarts": RESTARTS},
           "cpu_baseline": {"value": round(val, 4), "unit": "solves/s", "cores": os.cpu_count(),
                            "kind": "oracle",
                            "sample": f"{args.steps} timed FP64 oracle solves (observation build "
                                      "included), numpy BLAS default threads"},
           "e2e": {"value": round(val, 4), "unit": "solves/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def device_timed(fn, steps: int, stream, flush):
    """Runs fn(step) `steps` times, L2 flushed before each, each bracketed by
    CUDA events on `stream`; returns (mean ms, [fn results])."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    out = []
    torch.cuda.synchronize()
    for s in range(steps):
        flush.zero_()
        evs[s][0].record(stream)
        out.append(fn(s))
        evs[s][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / max(steps, 1), out


def reached(res) -> str:
    return f"{sum(bool(r.converged) for r in res)}/{len(res)}"


def video_form(h, api, torch, stream, flush, peaks, reps: int = 4):
    """Precision form on the video workload (256x256x3x64, spatial sigma 2
    radius 6, channel mix, temporal box of width 5, noise 5e-3, m = 40,
    sketch (96, 96, 3, 32), GCV): plain FP32 solves against the BF16 basis,
    solves/s at the same rho*, and the BF16 result's difference from the
    FP32 one and both relative errors to the true video."""
    p = workloads.video_config(0)
    A = [api.banded(mm, p.dims[mm - 1], t) for mm, _, t in p.factors]
    B = [api.dense(mm, t) for mm, _, t in p.right_factors]
    X = api.to_device(p.x_true, torch.float32)
    Ch = h.operator_apply(X, A, B)
    E = api.to_device(p.noise, torch.float32)
    C = api.empty(p.dims, torch.float32)
    C.copy_(Ch + E * (p.nu * torch.linalg.vector_norm(Ch) / torch.linalg.vector_norm(E)))
    nu_c = float(p.nu * torch.linalg.vector_norm(Ch) / torch.linalg.vector_norm(C))
    tol = rho_star(nu_c)
    out = {}
    Xs = {}
    for name, bf in (("fp32", False), ("bf16_basis", True)):
        Xo = api.empty(p.dims, torch.float32)

        def one(_):
            return h.gmres_solve(C, p.m, p.sketch_dims, p.seed, p.lam, A, B, X=Xo, tol=tol, mu_grid=p.mu_grid,
                                 max_restarts=RESTARTS, bf16_basis=bf)[1]
        for _ in range(2):
            one(0)
        ms, res = device_timed(one, reps, stream, flush)
        Xs[name] = Xo
        re = float(torch.linalg.vector_norm(Xo - X) / torch.linalg.vector_norm(X))
        out[name] = {"value": round(sum(bool(r.converged) for r in res) / len(res) * 1e3 / ms, 2),
                     "ms_per_solve": round(ms, 3),
                     "mean_iters": float(np.mean([r.iters for r in res])), "reached_stop_level": reached(res),
                     "rel_error_to_true_video": round(re, 5)}
        # the step's operator apply (k_apply_st: reads V_j, writes W, both in the
        # basis format) against HBM, from one phase-timed solve
        _, pi = h.gmres_solve(C, p.m, p.sketch_dims, p.seed, p.lam, A, B, X=Xo, tol=tol, mu_grid=p.mu_grid,
                              max_restarts=RESTARTS, bf16_basis=bf, phase_times=True)
        la = pi.phase_launches["apply"]
        if la > 0 and pi.phase_ms["apply"] > 0:
            n = int(np.prod(p.dims))
            bpl = 2 * n * (2 if bf else 4)
            us = 1e3 * pi.phase_ms["apply"] / la
            gbs = bpl / (us * 1e-6) / 1e9
            peak = peaks.get("hbm_gbs", 6800.0)
            out[name]["apply"] = {"kernel": "k_apply_st<%s> (blur 2D + channel mix + temporal box, one pass)"
                                            % ("bf16, bf16" if bf else "float, float"),
                                  "bytes_per_launch": bpl, "us_per_launch": round(us, 2), "gbs": round(gbs, 1),
                                  "frac_of_measured_hbm": round(gbs / peak, 3)}
    out["bf16_vs_fp32_rel_diff"] = round(float(torch.linalg.vector_norm(Xs["bf16_basis"] - Xs["fp32"]) /
                                               torch.linalg.vector_norm(Xs["fp32"])), 5)
    out["speedup_bf16_over_fp32"] = round(out["bf16_basis"]["value"] / out["fp32"]["value"], 3)
    out["workload"] = "video256x256x3x64: sigma 2 r 6, 3x3 mix, temporal box 5, noise 5e-3, m 40, sketch (96,96,3,32)"
    out["error_vs_fp64_oracle"] = ("tests/test_gpu_precision.py: 64x64x3x8 video, 20 steps, BF16 basis rho history "
                                   "within 10 %, X within 2 % of the FP64 oracle")
    del Xs
    return out


def uneven_form(h, api, torch, stream, flush, count: int, reps: int = 2):
    """Batched form on the uneven workload: `count` colour-image problems with
    sides drawn in [64, 1024], blur sigma in [0.5, 3] (radius ceil(3 sigma)),
    noise in [1e-3, 2e-2], fixed lambda in [1e-4, 1e-1], m = 30, sketch
    min(I_k, 128) per spatial mode, FP32, stop at rho*: one graph launch of
    all problems against a loop of single plain solves of the same problems."""
    cfgs = workloads.batched_configs(count, seed=0)
    probs = []
    elems = 0
    for c in cfgs:
        I1, I2, _ = c["dims"]
        taps = workloads.gaussian_taps(c["sigma"], c["radius"])
        A = [api.banded(1, I1, taps), api.banded(2, I2, taps)]
        x = workloads.piecewise_image(I1, I2, 3, c["image_seed"])
        Xt = api.to_device(x, torch.float32)
        Ch = h.operator_apply(Xt, A, [])
        E = api.to_device(workloads.noise_draw(x.shape, c["image_seed"]), torch.float32)
        C = api.empty(c["dims"], torch.float32)
        C.copy_(Ch + E * (c["nu"] * torch.linalg.vector_norm(Ch) / torch.linalg.vector_norm(E)))
        nu_c = float(c["nu"] * torch.linalg.vector_norm(Ch) / torch.linalg.vector_norm(C))
        probs.append(dict(C=C, A=A, B=[], m=c["m"], sketch_dims=c["sketch_dims"], seed=c["problem_id"],
                          lam=c["mu"], tol=rho_star(nu_c), X=api.empty(c["dims"], torch.float32)))
        elems += I1 * I2 * 3
        del Xt, Ch, E
    torch.cuda.synchronize()

    def batched(_):
        return h.gmres_solve_batched(probs, max_restarts=RESTARTS)[1]

    def loop(_):
        return [h.gmres_solve(q["C"], q["m"], q["sketch_dims"], q["seed"], q["lam"], q["A"], q["B"], X=q["X"],
                              tol=q["tol"], max_restarts=RESTARTS)[1] for q in probs]
    t0 = time.perf_counter()
    batched(0)
    build_b = time.perf_counter() - t0
    batched(0)
    t0 = time.perf_counter()
    loop(0)
    build_l = time.perf_counter() - t0
    ms_b, rb = device_timed(batched, reps, stream, flush)
    ms_l, rl = device_timed(loop, reps, stream, flush)
    rb, rl = rb[-1], rl[-1]
    same = all(a.iters == b.iters for a, b in zip(rb, rl))
    nb_r, nl_r = sum(bool(r.converged) for r in rb), sum(bool(r.converged) for r in rl)
    return {"value": round(nb_r / (ms_b / 1e3), 2), "unit": "solves/s (reaching rho*)",
            "ms_per_batch": round(ms_b, 3),
            "loop_of_single_solves": {"value": round(nl_r / (ms_l / 1e3), 2), "ms_per_pass": round(ms_l, 3),
                                      "reached_stop_level": reached(rl)},
            "speedup_over_loop": round(ms_l / ms_b, 3), "problems": count, "total_elements": elems,
            "mean_iters": float(np.mean([r.iters for r in rb])), "reached_stop_level": reached(rb),
            "iters_equal_to_single_solves": same, "first_call_s": {"batched": round(build_b, 2),
                                                                   "loop": round(build_l, 2)},
            "launch": "one CUDA graph, one branch per problem (device-side WHILE loops)",
            "workload": "256 colour images, sides U{64..1024}, sigma U[0.5,3], noise 1e-3..2e-2, "
                        "lambda 1e-4..1e-1, m 30, sketch min(I_k,128), FP32"}


def queue_form(api, torch, stream, flush, batch, grid, slots, reps: int = 3):
    """The chosen form's batch solved with other graph layouts: every problem
    its own branch with its own workspace (slots 0), or that many branches
    taking the problems from the device work queue; and the first 16 problems
    alone, one branch each (a batch of 16 per launch).  A fresh handle, so
    that the device memory each plan takes is the change in free memory
    around its first call."""
    hq = api.Handle(torch.cuda.current_device())
    out = {"problems": len(batch)}
    for name, bt, k in [(f"queue_{k}" if k else "branch_per_problem", batch, k) for k in slots] + \
                       [("batch_of_16_branch_per_problem", batch[:16], 0)]:
        def run(_):
            return hq.gmres_solve_batched(bt, mu_grid=grid, queue_slots=k, max_restarts=RESTARTS)[1]
        free0 = torch.cuda.mem_get_info()[0]
        t0 = time.perf_counter()
        run(0)
        first = time.perf_counter() - t0
        mem = free0 - torch.cuda.mem_get_info()[0]
        run(0)
        ms, res = device_timed(run, reps, stream, flush)
        res = res[-1]
        out[name] = {"value": round(sum(bool(r.converged) for r in res) / (ms / 1e3), 2),
                     "unit": "solves/s (reaching rho*)", "ms_per_batch": round(ms, 3), "problems": len(bt),
                     "branches": k if k else len(bt), "device_bytes": int(mem),
                     "first_call_s": round(first, 2), "reached_stop_level": reached(res),
                     "mean_iters": float(np.mean([r.iters for r in res]))}
    hq.close()
    torch.cuda.synchronize()
    return out


def run_ours(args):
    import torch
    global USE_GRAPH
    USE_GRAPH = not args.direct
    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2603_00839_gb300 import api
    h = api.Handle(torch.cuda.current_device())
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        peaks = {"hbm_gbs": 6800.0, "fallback": True}
    probs = make_problems(h, api, torch, args.problems, seed0=1000 * rank)
    X = api.empty(probs[0]["p"].dims, torch.float32)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    grid = workloads.mu_grid()
    B = args.batch
    Xb = [api.empty(probs[0]["p"].dims, torch.float32) for _ in range(B)]
    nb = max(1, len(probs) // B)
    only_b = args.only_batched

    def batch_of(k):
        return [dict(C=probs[(k * B + i) % len(probs)]["C"], A=probs[(k * B + i) % len(probs)]["A"],
                     B=probs[(k * B + i) % len(probs)]["B"], m=probs[0]["p"].m,
                     sketch_dims=probs[0]["p"].sketch_dims, seed=probs[(k * B + i) % len(probs)]["p"].seed,
                     lam=probs[0]["p"].lam, tol=probs[(k * B + i) % len(probs)]["tol"], X=Xb[i])
                for i in range(B)]

    slots = args.queue_slots if args.group_max <= 1 else 0

    def batched(bt, bf16=False):
        return h.gmres_solve_batched(bt, mu_grid=grid, use_graph=not args.direct, group_max=args.group_max,
                                     queue_slots=slots, max_restarts=RESTARTS, bf16_basis=bf16)

    # ---- plain FP32 form: one solve per step, every problem of the batch at
    # least once (the forms are compared on the same mix of problems)
    single_steps = max(args.steps, len(probs))
    plain_ms, plain_res = float("nan"), []
    if not only_b:
        for s in range(args.warmup):
            solve(h, probs[s % len(probs)], X)
        plain_ms, plain_res = device_timed(lambda s: solve(h, probs[s % len(probs)], X)[1], single_steps, stream,
                                           flush)
        for r in plain_res:
            if r.device_status != 0:
                raise RuntimeError(f"solve failed: device status {r.device_status}")

    # ---- sketched Golub-Kahan (Algorithm 4) on the same problems (no restarts)
    def gk(pr):
        p = pr["p"]
        return h.gk_solve(pr["C"], p.m, p.sketch_dims, p.seed, p.lam, pr["A"], pr["B"], X=X,
                          tol=pr["tol"], mu_grid=p.mu_grid)[1]
    gk_ms, gk_res = float("nan"), []
    if not only_b:
        for s in range(args.warmup):
            gk(probs[s % len(probs)])
        gk_ms, gk_res = device_timed(lambda s: gk(probs[s % len(probs)]), single_steps, stream, flush)

    # ---- chosen form: batched (B problems per CUDA-graph launch), one batch per step
    for s in range(args.warmup):
        batched(batch_of(s % nb))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        ms, outs = device_timed(lambda s: batched(batch_of(s % nb))[1], args.steps, stream, flush)
    res_b = [r for o in outs for r in o]
    for r in res_b:
        if r.device_status != 0:
            raise RuntimeError(f"batched solve failed: device status {r.device_status}")
    launches = sum(r.launches for r in res_b)
    if world > 1:
        torch.distributed.barrier()
    ms_max, plain_max = job_times([ms, plain_ms], world, "cuda")
    # the metric counts the solves that reach rho*; the others (a cycle ended
    # at j = m above it) cost their time and are reported, not counted
    reach_b = sum(bool(r.converged) for r in res_b) / max(args.steps, 1)
    reach_p = (sum(bool(r.converged) for r in plain_res) / len(plain_res)) if plain_res else 1.0
    value = job_rate(world, reach_b, ms_max / 1e3)
    plain_value = job_rate(world, reach_p, plain_max / 1e3)
    # every kernel group's algorithmic bytes summed over one batch's solves
    # (the last timed batch) against the batch's device time
    nd_n = int(np.prod(probs[0]["p"].dims))
    nd_d = int(np.prod([min(a, b) for a, b in zip(probs[0]["p"].sketch_dims, probs[0]["p"].dims)]))
    step_bytes = sum(phase_bytes(k, nd_n, nd_d, r.iters, 4, probs[0]["p"].m)
                     for r in outs[-1] for k in ("apply", "sketch", "update", "assemble", "init"))
    whole = {"algorithmic_bytes": int(step_bytes), "gbs": round(step_bytes / (ms / 1e3) / 1e9, 1),
             "frac_of_measured_hbm": round(step_bytes / (ms / 1e3) / 1e9 / peaks.get("hbm_gbs", 6800.0), 4),
             "note": "apply, sketch, update, assembly and start groups of every solve of the batch (the byte "
                     "model of the roofline) over the batch's device time"}

    # ---- end to end through the C ABI with pinned host buffers, every step:
    # H2D of the batch's observations, the batched solve, D2H of the
    # solutions.  Two sets of device buffers: the next batch's observations
    # go up on a copy stream while the current batch is solved, and its
    # solutions come back while the next one is solved.  The timed region
    # runs from the first upload to the end of the last download.
    n = int(np.prod(probs[0]["p"].dims))
    dims = probs[0]["p"].dims
    for pr in probs:
        ch = torch.empty(tuple(reversed(pr["p"].dims)), dtype=torch.float32, pin_memory=True)
        ch = ch.permute(2, 1, 0)
        ch.copy_(pr["C"].cpu())
        pr["C_host"] = ch
    Cdev = [[api.empty(dims, torch.float32) for _ in range(B)] for _ in range(2)]
    Xdev = [[api.empty(dims, torch.float32) for _ in range(B)] for _ in range(2)]
    Xh = [[torch.empty(tuple(reversed(dims)), dtype=torch.float32, pin_memory=True).permute(2, 1, 0)
           for _ in range(B)] for _ in range(2)]
    copy_s = torch.cuda.Stream()

    def upload(k, slot):
        with torch.cuda.stream(copy_s):
            for i in range(B):
                Cdev[slot][i].copy_(probs[(k * B + i) % len(probs)]["C_host"], non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(copy_s)
        return ev

    def download(slot):
        copy_s.wait_stream(stream)
        with torch.cuda.stream(copy_s):
            for i in range(B):
                Xh[slot][i].copy_(Xdev[slot][i], non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(copy_s)
        return ev

    def e2e_run(steps):
        got = 0
        ready = upload(0, 0)
        done = [None, None]
        for s in range(steps):
            slot = s % 2
            stream.wait_event(ready)
            if done[slot] is not None:           # the download of this slot's previous solutions
                stream.wait_event(done[slot])
            nxt = upload((s + 1) % nb, 1 - slot) if s + 1 < steps else None
            bt = batch_of(s % nb)
            for i in range(B):
                bt[i]["C"], bt[i]["X"] = Cdev[slot][i], Xdev[slot][i]
            _, res = batched(bt)                 # returns when the solve is done
            got += sum(bool(r.converged) for r in res)
            done[slot] = download(slot)
            ready = nxt
        copy_s.synchronize()
        torch.cuda.synchronize()
        return got

    if not only_b:
        e2e_run(2)
    t0 = time.perf_counter()
    e2e_reached = e2e_run(args.steps) if not only_b else 0
    e2e_s = (time.perf_counter() - t0) / args.steps if not only_b else float("nan")
    e2e_val = job_rate(world, e2e_reached / max(args.steps, 1), job_times([e2e_s], world, "cuda")[0])

    extra = rank == 0 and not only_b and not args.no_extra_forms
    # ---- batched form with the BF16 basis (precision form on the image workload)
    bf_form = None
    if extra:
        for s in range(2):
            batched(batch_of(s % nb), bf16=True)
        ms_bf, outs_bf = device_timed(lambda s: batched(batch_of(s % nb), bf16=True)[1], args.steps, stream, flush)
        rbf = [r for o in outs_bf for r in o]
        bf_form = {"value": round(sum(bool(r.converged) for r in rbf) / args.steps / (ms_bf / 1e3), 2),
                   "ms_per_batch": round(ms_bf, 4), "batch": B,
                   "mean_iters": float(np.mean([r.iters for r in rbf])), "reached_stop_level": reached(rbf),
                   "basis": "BF16 (FP32 arithmetic, FP64 Gram-Schmidt / Givens / Tikhonov)"}
    rs_form = None
    if extra:
        def batched_rs(bt):
            return h.gmres_solve_batched(bt, mu_grid=grid, max_restarts=3, queue_slots=slots)
        for s in range(2):
            batched_rs(batch_of(s % nb))
        ms_rs, outs_rs = device_timed(lambda s: batched_rs(batch_of(s % nb))[1], args.steps, stream, flush)
        rrs = [r for o in outs_rs for r in o]
        rs_form = {"value": round(sum(bool(r.converged) for r in rrs) / args.steps / (ms_rs / 1e3), 2),
                   "ms_per_batch": round(ms_rs, 4), "batch": B, "restarts": 3,
                   "mean_iters": float(np.mean([r.iters for r in rrs])), "reached_stop_level": reached(rrs),
                   "iters_per_problem": [r.iters for r in outs_rs[0]],
                   "note": "every solve runs to rho* (restarted up to 3 times)"}
    vid = video_form(h, api, torch, stream, flush, peaks) if extra else None
    uneven = uneven_form(h, api, torch, stream, flush, args.uneven) if extra else None
    queue = queue_form(api, torch, stream, flush, batch_of(0), grid, (0, 16, 32)) if extra and slots else None

    ws_form = None
    if rank == 0 and not args.no_warm_start and not only_b:
        ws_form = (warm_start_form(h, api, torch, probs[:16], train_n=20000, steps=3000, held_out=512)
                   if args.ws_full else warm_start_form(h, api, torch, probs[:16]))

    # phase timing holds the stream at gates the host opens; a profiler that
    # serialises every launch would wait on them, so --direct (the profiler
    # mode) leaves it out
    phased = rank == 0 and not args.direct and not only_b
    roof_plain, phases = phase_report(h, probs[:16], X, peaks, WORKLOAD) if phased else (None, None)
    roof, phases_b = (batched_phase_report(h, batch_of(0)[:16], grid, peaks, WORKLOAD) if phased
                      else (None, None))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not only_b:
        cpu = cpu_baseline(args.cpu_seconds)
    if rank == 0:
        out = {"metric": METRIC, "value": round(value, 2), "unit": "solves/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max, 4),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": {"workload": WORKLOAD, "dims": [512, 512, 3], "m": 50, "restarts": RESTARTS,
                          "sketch": [128, 128, 3], "blur": "gaussian sigma 2.5 radius 7 + 3x3 mix",
                          "noise": 1e-2, "gcv_grid": 8, "mean_iters": float(np.mean([r.iters for r in res_b])),
                          "stop": "rho <= max(1e-3, 1.01*nu_C), else m steps (then `restarts` restarted "
                                  "cycles); value counts only the solves that reach rho*",
                          "reached_stop_level": reached(res_b), "problems": len(probs),
                          "l2": "flushed (256 MB write) between timed steps",
                          "form": f"batched: {B} problems per CUDA-graph launch (one step = one batch)",
                          "launch": ("direct launches" if args.direct else "cuda graph") +
                                    (f" (lock-step groups of up to {args.group_max} problems)"
                                     if args.group_max > 1 else
                                     f" ({slots} branches taking the problems from a device work queue, "
                                     "device-side WHILE loops)" if slots else
                                     " (one branch per problem, device-side WHILE loops)")},
               "forms": {"batched_fp32": {"value": round(value, 2), "ms_per_batch": round(ms_max, 4),
                                          "batch": B, "queue_slots": slots, "reached_stop_level": reached(res_b),
                                          "whole_step": whole,
                                          "vs_plain_fp32": round(value / plain_value, 3) if plain_value else None},
                         "plain_fp32": {"value": round(plain_value, 2), "ms_per_solve": round(plain_max, 4),
                                        "mean_iters": float(np.mean([r.iters for r in plain_res])) if plain_res else None,
                                        "reached_stop_level": reached(plain_res),
                                        "launch": "direct" if args.direct else "cuda graph"},
                         "batched_bf16_basis": dict(bf_form, vs_plain_fp32=round(bf_form["value"] / plain_value, 3))
                                               if bf_form else None,
                         "batched_fp32_restarted": rs_form,
                         "golub_kahan_fp32": {"value": round((sum(bool(r.converged) for r in gk_res) /
                                                              max(len(gk_res), 1)) * 1e3 / gk_ms, 2),
                                              "ms_per_solve": round(gk_ms, 4),
                                              "mean_iters": float(np.mean([r.iters for r in gk_res])) if gk_res else None,
                                              "reached_stop_level": reached(gk_res),
                                              "vs_plain_fp32": round((sum(bool(r.converged) for r in gk_res) /
                                                                      len(gk_res)) * 1e3 / gk_ms / plain_value, 3)
                                                               if gk_res else None,
                                              "method": "sketched Golub-Kahan (Algorithm 4), no restarts"},
                         "precision_video": vid,
                         "batched_uneven_256": uneven,
                         "batched_layouts": queue,
                         "warm_start_fp32": ws_form},
               "e2e": {"value": round(e2e_val, 2), "unit": "solves/s",
                       # per problem: C and X, plus the 328-byte descriptor and the 2376-byte
                       # info record of the batch call
                       "h2d_bytes_per_step": (4 * n + 328) * B, "d2h_bytes_per_step": (4 * n + 2376) * B,
                       "copies": "every step's observations up and solutions down through pinned host "
                                 "buffers on a copy stream, overlapped with the neighbouring steps' solves "
                                 "(two device buffer sets); host wall clock from the first upload to the "
                                 "last download"},
               "gpu_launches": launches,
               "roofline": roof, "kernels": phases_b, "roofline_plain": roof_plain, "kernels_plain": phases,
               "cpu_baseline": cpu, "clocks": clk.summary()}
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    global RESTARTS
    args = parse()
    RESTARTS = args.restarts
    if args.cpu_leg > 0:
        cpu_leg_main(args.cpu_leg, args.cpu_seconds)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
