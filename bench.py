#!/usr/bin/env python
"""Benchmark: Sigma_SOX builds/s on one GB300 (or N replicas under torchrun).

A step is one full bare-SOX build through the C ABI: both THC mixed tensors,
projections, the A intermediate, the fused B/C/Hadamard reduction, the
back-projection to orbitals, for every tau point and spin of the workload
(default: n=120, N=600, 80 tau, unrestricted; the mid-size molecule stand-in).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the host cores instead (a bounded tau sample per step, scaled to builds/s).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Σ_SOX builds/s vs plain FP64 GPU at max|ΔΣ|≤1e-8 Ha; tensor-pipe % of peak"
UNIT = "builds/s"


def workload(name: str):
    import synth

    if name == "c1":
        return synth.config(1)
    if name == "c0":
        return synth.config(0)
    if name == "c2":
        return synth.config(2)
    raise SystemExit(f"unknown workload {name}")


def flops_per_build(w) -> dict:
    """Algorithmic real flops of one build (2 per multiply-add)."""
    n, N, T, S = w.n, w.N, w.n_tau, w.n_spin
    bc = 4.0 * N * N * n * n * T * S          # B and C contractions (fused kernel)
    had = 2.0 * N * N * n * T * S             # Hadamard-reduce over v
    a = 2.0 * N * n ** 3 * T * S              # A intermediate
    mixed = 2.0 * N * N * n * n               # one mixed THC tensor
    proj = 4.0 * N * n * n * T * S            # G_Rq and G_wP
    back = 2.0 * (N * N * n + N * n * n) * T * S
    return {"bcd": bc + had, "A": a, "mixed": mixed, "proj": proj, "back": back,
            "total": bc + had + a + mixed + proj + back}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region (median SM clock, throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_tau_points_per_s(w, n_points: int):
    """Time the CPU oracle (complex128 chain) on n_points (spin, tau) pairs."""
    from oracle import sox as osox

    pts = [(s, j) for j in (0, w.n_tau // 2, w.n_tau - 1, w.n_tau // 4) for s in range(w.n_spin)][:n_points]
    t0 = time.perf_counter()
    for s, j in pts:
        osox.sigma_tau(w.X[0], w.V[0], w.V[0], w.G[s, 0], taus=[j])
    dt = time.perf_counter() - t0
    return len(pts) / dt, dt, pts


def cpu_baseline(w, n_points: int) -> dict:
    rate, dt, pts = oracle_tau_points_per_s(w, n_points)
    per_build = w.n_tau * w.n_spin
    return {"value": rate / per_build, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{len(pts)} (spin, tau) points of one build ({per_build} per build), "
                      f"numpy complex128 chain, {dt:.1f} s; builds/s = points/s / {per_build}"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args.workload)
    per_build = w.n_tau * w.n_spin
    for _ in range(args.warmup):
        oracle_tau_points_per_s(w, 1)
    times = []
    for _ in range(args.steps):
        rate, dt, _ = oracle_tau_points_per_s(w, 1)
        times.append(dt)
    value = 1.0 / (np.mean(times) * per_build)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": w.name, "n": w.n, "N": w.N, "n_tau": w.n_tau,
                                            "n_spin": w.n_spin, "step": "one (spin, tau) point of a build"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"1 (spin, tau) point per step of {per_build} per build"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2412_18829_gb300 as pkg

    w = workload(args.workload)
    dev = torch.device("cuda", local)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G = torch.from_numpy(w.G).to(dev)
    X = torch.from_numpy(w.X).to(dev)
    V = torch.from_numpy(w.V).to(dev)
    S = torch.empty_like(G)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    h = pkg.Handle(args.precision, device=local)
    stream = torch.cuda.current_stream(dev)

    def step():
        pkg.sox_sigma(h, p, G, X, V, S, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    pkg.sox_profile_enable(h, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    launches, _ = pkg.sox_profile_read(h, None)
    hot = "sox_bcd_tc" if args.precision == "f16x2" else "sox_bcd"
    hot_n, hot_ms = pkg.sox_profile_read(h, hot)
    pkg.sox_profile_enable(h, False)
    clocks = sampler.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    t_local = float(np.sum(ms)) / 1e3
    t_max = t_local
    if dist:
        t = torch.tensor([t_local], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    builds = args.steps * world
    value = builds / t_max

    # accuracy of this build: against the FP64 GPU path (all points) and the oracle (sampled)
    out = S.cpu().numpy()
    extra = {}
    if rank == 0 and not args.skip_accuracy:
        from oracle import sox as osox

        taus = [0, w.n_tau - 1]
        err = 0.0
        smax = 0.0
        for s in range(w.n_spin):
            ref = osox.sigma_tau(w.X[0], w.V[0], w.V[0], w.G[s, 0], taus=taus, dtype=np.float64)
            err = max(err, float(np.abs(out[s, 0, taus] - ref).max()))
            smax = max(smax, float(np.abs(ref).max()))
        extra["max_abs_err_Ha_vs_oracle"] = err
        extra["max_rel_err_vs_oracle"] = err / smax
        extra["oracle_sample"] = f"tau {taus} x {w.n_spin} spins"
    if rank == 0 and args.precision != "fp64" and not args.skip_fp64:
        with pkg.Handle("fp64", device=local) as h64:
            S64 = torch.empty_like(G)
            pkg.sox_sigma(h64, p, G, X, V, S64, stream)   # warm
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            a.record(stream)
            pkg.sox_sigma(h64, p, G, X, V, S64, stream)
            b.record(stream)
            torch.cuda.synchronize()
            t64 = a.elapsed_time(b) / 1e3
            extra["fp64_gpu_builds_per_s"] = 1.0 / t64
            extra["speedup_vs_fp64_gpu"] = value / world * t64
            extra["max_abs_err_Ha_vs_fp64_gpu_all_points"] = float((S - S64).abs().max().item())

    # end-to-end through the C ABI with host buffers (pinned), copies inside the timed region
    Gh = torch.from_numpy(w.G).pin_memory()
    Xh = torch.from_numpy(w.X).pin_memory()
    Vh = torch.from_numpy(w.V).pin_memory()
    Sh = torch.empty_like(Gh).pin_memory()
    pkg.sox_sigma(h, p, Gh.numpy(), Xh.numpy(), Vh.numpy(), Sh.numpy(), stream)
    e2e_t = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pkg.sox_sigma(h, p, Gh.numpy(), Xh.numpy(), Vh.numpy(), Sh.numpy(), stream)
        e2e_t.append(time.perf_counter() - t0)
    e2e_val = world / float(np.mean(e2e_t))
    h2d = (w.G.nbytes + w.X.nbytes + w.V.nbytes)
    d2h = w.G.nbytes

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    fl = flops_per_build(w)
    pk, pk_src = peaks()
    per_launch_units = (w.n_tau * w.n_spin) / max(1, hot_n / args.steps)
    hot_flops_launch = fl["bcd"] / (w.n_tau * w.n_spin) * per_launch_units
    hot_avg_s = (hot_ms / max(1, hot_n)) / 1e3
    achieved = hot_flops_launch / hot_avg_s / 1e12 if hot_n else None
    if args.precision == "f16x2":
        peak = pk.get("bf16_tflops_sustained", 1700.0)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None, "traffic": None,
                "kernel": hot, "peak_source": f"{pk_src} bf16 sustained (fp16 dense rate = bf16 rate)",
                "mma_issued_tflops": 3 * achieved if achieved else None,
                "tensor_pipe_frac": 3 * achieved / peak if achieved else None,
                "note": "achieved counts algorithmic flops 4N^2n^2 per (tau,spin); the FP16x2 split issues 3 MMAs per product"}
    else:
        peak = 1.20
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None, "traffic": None, "kernel": hot,
                "peak_source": "measured FP64 FMA rate (paper_2412_18829_gb300/probes/fp_rate.cu)"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f16x2+f32acc,f64" if args.precision == "f16x2" else "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "N": w.N, "n_tau": w.n_tau, "n_spin": w.n_spin,
                   "beta": w.beta, "precision": args.precision,
                   "l2": "flushed between steps (256 MiB write outside the events)",
                   "parallelism": f"{world} independent builds (one per GPU)",
                   "algorithmic_tflops_per_s": fl["total"] * value / 1e12, **extra},
        "roofline": roof,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if world == 1 and not args.skip_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_points)
    print(json.dumps(line), flush=True)
    h.close()
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f16x2", choices=["f16x2", "fp64"])
    ap.add_argument("--workload", default="c1")
    ap.add_argument("--cpu-points", type=int, default=16)
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-accuracy", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
