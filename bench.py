#!/usr/bin/env python
"""Benchmark of the variance-reduced ProxSkip hot path on one GB300 (or N replicas).

Workload (default ``par2d_512``): 512x512 seeded ellipse phantom, 720 parallel-beam angles
over [0, 180), 768 unit bins, Poisson noise at 1e4 incident photons (log data), 20
staggered subsets, isotropic TV (alpha = 0.01) + nonnegativity, ProxSVRGSkip with p = 0.1,
gamma = 1/L, 100 warm-started FGP inner iterations, FP32 kernels.

Metric: seconds to a 1e-4 relative objective gap (F(x+) - F*)/F*.  F* is the smallest
objective seen by a long FISTA reference run (200 FGP iterations) and by the solver
itself.  Deterministic replay: one run with per-epoch evaluation finds k*, the first
iteration count whose gap is <= 1e-4; every timed step then runs vrps_solve for exactly k*
iterations from x0 = 0 with no evaluation.  A "step" is therefore one whole
reconstruction to the target gap.  The L2 cache is flushed (256 MB write) between steps.

Prints one JSON line (see the key list at the end of main()).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synthetic  # noqa: E402

WORKLOADS = {
    # alpha = 1.0: the TV weight with the smallest reconstruction error against the phantom
    # (sweep 0.002 .. 10 with long FISTA runs); the workload's description leaves it open
    "par2d_512": dict(n=512, n_angles=720, n_bins=768, n_subsets=20, noise="poisson", alpha=1.0,
                      algo="VR_PROXSKIP", estimator="SVRG", p=0.1, fgp_iters=100, seed=20260209,
                      target_gap=1e-4, max_epochs=150),
    "par2d_64": dict(n=64, n_angles=90, n_bins=96, n_subsets=10, noise="gauss", alpha=0.01,
                     algo="VR_PROXSKIP", estimator="SVRG", p=0.1, fgp_iters=50, seed=20260209,
                     target_gap=1e-4, max_epochs=150),
}

# Iteration counts of the replayed trajectory (same seed and draws on any machine), used only
# by the CPU oracle legs to scale a bounded sample up to a whole reconstruction.  Recorded from
# the GPU replay of this workload; the GPU arm recomputes them every run.
TRAJECTORY = {
    "par2d_512": dict(iterations=1920, prox_calls=180, snapshots=96),
    "par2d_64": dict(iterations=None, prox_calls=None, snapshots=None),
}

# dram bytes (read + write) per launch of the dominant kernel from one ncu capture, with the
# profile summary it comes from; None when the kernel changed since the capture.
NCU_TRAFFIC = {}


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def make_problem(wl, rank):
    w = WORKLOADS[wl]
    return synthetic.make_problem_2d(w["n"], w["n_angles"], w["n_bins"], w["n_subsets"], seed=w["seed"] + rank,
                                     noise=w["noise"], alpha=w["alpha"], truth=False)


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- oracle legs
def oracle_sample(wl, P, seconds_cap=30.0):
    """Time the float64 oracle on a bounded sample of one reconstruction's work: one
    ProxSVRG subset iteration (grad f_i at x and at the snapshot), one FGP prox call, and
    one subset gradient (the full gradient of a snapshot costs about N of them)."""
    from oracle import joseph2d, solvers, tv
    w = WORKLOADS[wl]
    op = solvers.Operator(joseph2d.Geometry2D.from_spec(P.spec))
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 0.01, size=op.shape)
    xs = rng.uniform(0, 0.01, size=op.shape)
    t0 = time.perf_counter()
    g = solvers.grad_fi(op, P.b, x, 3)
    t1 = time.perf_counter()
    g2 = solvers.grad_fi(op, P.b, xs, 3)
    v = x - 1e-3 * (w["n_subsets"] * (g - g2))
    t2 = time.perf_counter()
    tv.fgp(v, 1e-4, w["fgp_iters"], True, None, op.D)
    t3 = time.perf_counter()
    return {"t_subset_grad": t1 - t0, "t_svrg_iter": t2 - t0, "t_prox": t3 - t2, "sample_s": t3 - t0}


def oracle_extrapolate(samp, counts, N):
    it, pc, sn = counts["iterations"], counts["prox_calls"], counts["snapshots"]
    return it * samp["t_svrg_iter"] + pc * samp["t_prox"] + sn * N * samp["t_subset_grad"]


# --------------------------------------------------------------------------- roofline
def algorithmic_bytes(kernel, g, rows_subset):
    """Algorithmic DRAM bytes of one launch (float32, each array touched once)."""
    n, nb = g.n, g.desc.get("n_bins", 0)
    if kernel == "fgp2d_iter":       # read v, w_k(2), w_{k-1}(2); write w_{k+1}(2)
        return 28 * n
    if kernel == "fgp2d_out":        # read v, w(2), x, xhat, h; write x, xT, h
        return 36 * n
    if kernel == "adj2d_kernel":     # read dr (m_i), x, h, gbar; write x + xT (skip) or v + xhat
        return 4 * rows_subset * nb + 20 * n
    if kernel == "fwd2d_kernel":     # read x or xT (n), table (m_i); write dr (m_i)
        return 4 * n + 8 * rows_subset * nb
    return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--workload", default="par2d_512", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--alpha", type=float, default=None, help="override the workload's TV weight")
    ap.add_argument("--profile-once", type=int, default=0, metavar="K",
                    help="profiling driver: run K solver iterations of the workload once (no F* search, "
                         "no timing) and exit")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), _env_int("LOCAL_RANK", 0)
    wl = args.workload
    w = WORKLOADS[wl]
    if args.alpha is not None:
        w["alpha"] = args.alpha

    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2602_09527_gb300 as vr

    if args.profile_once:
        P = make_problem(wl, rank)
        g = vr.Geometry.from_spec(P.spec)
        b_dev = torch.tensor(P.b.astype(np.float32).ravel(), device="cuda")
        L = vr.power_iteration(g, 100, seed=w["seed"])
        vr.solve(b_dev, g, w["alpha"], w["algo"], p=w["p"], gamma=1.0 / L, seed=w["seed"], estimator=w["estimator"],
                 fgp_iters=w["fgp_iters"], max_iters=args.profile_once)
        torch.cuda.synchronize()
        g.close()
        return

    P = make_problem(wl, rank)
    g = vr.Geometry.from_spec(P.spec)
    N = w["n_subsets"]
    b_dev = torch.tensor(P.b.astype(np.float32).ravel(), device="cuda")
    b_host = torch.tensor(P.b.astype(np.float32).ravel()).pin_memory()
    L = vr.power_iteration(g, 100, seed=w["seed"])
    gamma = 1.0 / L

    # F*: long FISTA reference (more FGP iterations), then the smallest value ever seen
    _, rep_ref, hist_ref = vr.solve(b_dev, g, w["alpha"], "FISTA", gamma=gamma, seed=w["seed"], fgp_iters=200,
                                    max_iters=4000, eval_every=100, history_cap=64)
    f_ref = min(h[1] for h in hist_ref)
    max_it = w["max_epochs"] * N
    _, rep_tr, hist = vr.solve(b_dev, g, w["alpha"], w["algo"], p=w["p"], gamma=gamma, seed=w["seed"],
                               estimator=w["estimator"], fgp_iters=w["fgp_iters"], max_iters=max_it,
                               eval_every=N, history_cap=max_it // N + 1)
    f_star = min(f_ref, min(h[1] for h in hist))
    k_star = None
    for h in hist:
        if (h[1] - f_star) / abs(f_star) <= w["target_gap"]:
            k_star = int(h[0])
            break
    reached = k_star is not None
    if not reached:
        k_star = max_it

    def run_once(host=False):
        bb = b_host if host else b_dev
        return vr.solve(bb, g, w["alpha"], w["algo"], p=w["p"], gamma=gamma, seed=w["seed"],
                        estimator=w["estimator"], fgp_iters=w["fgp_iters"], max_iters=k_star)

    flush = torch.empty(64 * 1024 * 1024, device="cuda", dtype=torch.float32)
    for _ in range(args.warmup):
        x_last, rep, _ = run_once()
    torch.cuda.synchronize()
    gap_check = vr.objective(g, x_last, b_dev, w["alpha"])[0]

    stream = torch.cuda.current_stream()
    times = []
    launches0 = vr.kernel_launches()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x_last, rep, _ = run_once()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
    launches = (vr.kernel_launches() - launches0) // args.steps
    total = sum(times)
    if dist is not None:
        t = torch.tensor([total], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    sec_per = total / args.steps

    # end to end through the public API with host buffers (H2D of b, D2H of x inside)
    e2e = []
    for _ in range(max(2, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xh, _, _ = run_once(host=True)
        e2e.append(time.perf_counter() - t0)

    # live per-kernel timing of one reconstruction (CUDA events around every launch)
    vr.profile_enable(True)
    run_once()
    prof = vr.profile_read()
    vr.profile_enable(False)
    tot_ms = sum(v[1] for v in prof.values())
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    dom_name, (dom_launch, dom_ms) = dom
    rows_subset = w["n_angles"] // N
    ab = algorithmic_bytes(dom_name, g, rows_subset)
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    avg_s = dom_ms / 1e3 / max(dom_launch, 1)
    roofline = None
    if ab is not None:
        ach = ab / avg_s / 1e9
        roofline = {"kernel": dom_name, "bound": "hbm", "achieved": round(ach, 1), "peak": hbm_peak,
                    "peak_source": peak_src, "unit": "GB/s", "frac": round(ach / hbm_peak, 4),
                    "traffic": NCU_TRAFFIC.get(dom_name), "bytes_per_launch": ab,
                    "avg_launch_us": round(avg_s * 1e6, 3), "share": round(dom_ms / tot_ms, 4)}
    kernels = {k: {"launches": v[0], "ms": round(v[1], 4), "share": round(v[1] / tot_ms, 4)} for k, v in prof.items()}

    # projector throughput (G ray-voxel/s): subset forward and adjoint kernels, each launch
    # timed by CUDA events around it (library profiling), so host call overhead is excluded
    samples_sub = g.samples(0)
    xs = torch.rand(g.n, device="cuda")
    ys = vr.proj_fwd(g, 0, xs)
    for _ in range(3):
        vr.proj_fwd(g, 0, xs, ys)
        vr.proj_adj(g, 0, ys, xs)
    vr.profile_enable(True)
    for _ in range(20):
        vr.proj_fwd(g, 0, xs, ys)
        vr.proj_adj(g, 0, ys, xs)
    pp = vr.profile_read()
    vr.profile_enable(False)
    t_fwd = pp["fwd2d_kernel"][1] / pp["fwd2d_kernel"][0] / 1e3
    t_adj = pp["adj2d_kernel"][1] / pp["adj2d_kernel"][0] / 1e3
    gvox = 2 * samples_sub / (t_fwd + t_adj) / 1e9

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        samp = oracle_sample(wl, P)
        counts = {"iterations": rep["iterations"], "prox_calls": rep["prox_calls"], "snapshots": rep["snapshots"]}
        cpu = {"value": round(oracle_extrapolate(samp, counts, N), 2), "unit": "s", "cores": 1, "kind": "oracle",
               "sample": (f"float64 oracle on this host: one ProxSVRG subset iteration ({samp['t_svrg_iter']:.2f} s), "
                          f"one {w['fgp_iters']}-iteration FGP prox ({samp['t_prox']:.2f} s), one subset gradient "
                          f"({samp['t_subset_grad']:.2f} s; a snapshot = N of them), scaled by this run's counts "
                          f"{counts}")}

    clocks = clk.summary()
    out = {
        "metric": "s to 1e-4 rel. objective gap",
        "value": round(sec_per, 6),
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(sec_per * 1e3, 4),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded ellipse phantom, analytic sinogram, Poisson 1e4 photons)",
        "config": {"workload": wl, "image": f"{w['n']}x{w['n']}", "angles": w["n_angles"], "bins": w["n_bins"],
                   "subsets": N, "algo": "ProxSVRGSkip", "p": w["p"], "fgp_iters": w["fgp_iters"],
                   "alpha": w["alpha"], "gamma": "1/L", "k_star": k_star, "target_reached": reached,
                   "f_star": f_star, "gap_at_k_star": (gap_check - f_star) / abs(f_star),
                   "prox_calls": rep["prox_calls"], "snapshots": rep["snapshots"], "passes": rep["passes"],
                   "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
        "e2e": {"value": round(statistics.mean(e2e), 6), "unit": "s", "h2d_bytes_per_step": 4 * g.m,
                "d2h_bytes_per_step": 4 * g.n},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "kernels": kernels,
        "projector": {"metric": "G ray-voxel/s", "value": round(gvox, 3), "samples_per_subset": samples_sub,
                      "fwd_us": round(t_fwd * 1e6, 3), "adj_us": round(t_adj * 1e6, 3),
                      "what": "subset 0 (36 angles x 768 bins): 2 x Joseph samples / (forward + adjoint kernel time)"},
        "reconstructions_per_s": round(world / sec_per, 4),
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(out))
    g.close()
    if dist is not None:
        dist.destroy_process_group()


def reference_arm(args, rank, world):
    """The oracle, as it stands, on the host cores: each step times a bounded sample of one
    reconstruction's work and scales it to a whole reconstruction with the trajectory's
    recorded iteration counts.  Under torchrun only rank 0 works."""
    if rank != 0:
        return
    wl = args.workload
    w = WORKLOADS[wl]
    counts = TRAJECTORY[wl]
    if counts["iterations"] is None:
        print(json.dumps({"impl": "reference", "unavailable": "trajectory counts for this workload not recorded yet"}))
        return
    P = make_problem(wl, 0)
    for _ in range(args.warmup):
        oracle_sample(wl, P)
    vals, samples = [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s = oracle_sample(wl, P)
        samples.append(s)
        vals.append(oracle_extrapolate(s, counts, w["n_subsets"]))
    wall = time.perf_counter() - t0
    v = statistics.mean(vals)
    out = {
        "impl": "reference",
        "metric": "s to 1e-4 rel. objective gap",
        "value": round(v, 3),
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(v * 1e3, 1),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded ellipse phantom, analytic sinogram, Poisson 1e4 photons)",
        "config": {"workload": wl, "image": f"{w['n']}x{w['n']}", "angles": w["n_angles"], "bins": w["n_bins"],
                   "subsets": w["n_subsets"], "algo": "ProxSVRGSkip", "p": w["p"], "fgp_iters": w["fgp_iters"],
                   "trajectory_counts": counts},
        "cpu_baseline": {"value": round(v, 3), "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": "per step: one ProxSVRG subset iteration, one FGP prox, one subset gradient, "
                                   f"scaled by the recorded counts {counts}; {wall:.1f} s of sampling in total"},
        "e2e": {"value": round(v, 3), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


if __name__ == "__main__":
    main()
