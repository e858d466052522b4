#!/usr/bin/env python
"""Benchmark: Sigma_SOX builds/s on one GB300 (or N GPUs under torchrun).

A step is one full build through the C ABI.  Workloads (``--workload``):

* c4 (default, the largest configuration) the uneven batch of 16 molecules
  (n in [40, 400], N=6n, 120 tau): per instance Phi and Sigma (phi_sox), dPhi/dG
  from the kept Sigma (phi_sox_grad_G) and dPhi/dX, dPhi/dV (phi_sox_backward);
  instances are sharded over ranks.
* c1 bare SOX, mid-size molecule: n=120, N=600, 80 tau, 2 spins.  Both
  THC mixed tensors, projections, A, the fused B/C/Hadamard reduction and the
  back-projection to orbitals for every tau point and spin.
* c0 bare SOX, small molecule (n=20, N=80, 30 tau).
* c2 statically screened SOSEX (n=250, N=2000, 100 tau): Pi(0), W(0) and
  SOX(W(0), v) per step.
* c3 dynamically screened SOSEX of a solid (3x3x3 k-mesh, n=26, N=300, 60 tau),
  W_d from a synthetic single-pole form (or the GPU RPA with --rpa-w).
* c1d dynamically screened SOSEX of the mid-size molecule (c1's shapes, 79
  bosonic frequencies, W_d from the single-pole form).

``--kernel resident|streamed|pair`` forces the split path's fused B/C/D kernel
variant (default: timed per shape); ``--shard tau|v|replicas`` chooses how N > 1
ranks share the work.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the host cores instead (a bounded sample per step, scaled to builds/s).

``--profile-case KIND`` runs one small case for an ncu capture instead (one
process, one GPU, a few GB on the device): KIND is molecule (sox_sigma twice at
n=120, N=600, 2 spins), screened (sox_sigma twice at n=250, N=2000), batch
(phi_sox + phi_sox_grad_G twice at the batch's largest instance, n=298, N=1788),
adjoint (phi_sox_backward twice at that instance; --profile-sizes n,N for others), solid (sosex_dynamic_sigma at
the 3x3x3 solid's shapes; --mesh and --profile-sizes n,N change them), dynmol
(sosex_dynamic_sigma at the mid-size molecule's shapes) or wdyn (sox_w_dynamic at
the solid's shapes); --profile-tau sets the tau points, --kernel the fused variant.
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

    if name in ("c0", "c1", "c2", "c3"):
        return synth.config(int(name[1]))
    if name == "c1d":   # the dynamic molecule's shapes are c1's
        return synth.config(1)
    if name == "c4":   # the oracle baselines of the batch time points of its median instance
        sizes = synth.batch_c4_sizes()
        return synth.c4_instance(int(np.argsort(sizes, kind="stable")[len(sizes) // 2]))
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
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
            return
        t0 = time.perf_counter()   # the timed region starts once nvidia-smi is sampling
        while time.perf_counter() - t0 < 5.0 and self.p.poll() is None and os.path.getsize(self.f.name) == 0:
            time.sleep(0.01)

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


def oracle_tau_points_per_s(w, n_points: int, budget_s: float = 20.0):
    """Time the CPU oracle (complex128 chain) on n_points (spin, tau) pairs of one build.

    Molecules: SOX at one tau point (SOSEX has the same chain and cost with W(0) in
    the first slot).  Solids: the static momentum-resolved chain at one tau point,
    all k (the dynamic part is not timed by this sample)."""
    from oracle import grid as ogrid, kpoints as okp, sox as osox

    taus = sorted({int(round(x)) for x in np.linspace(0, w.n_tau - 1, max(1, -(-n_points // w.n_spin)))})
    pts = [(s, j) for j in taus for s in range(w.n_spin)][:n_points]
    t0 = time.perf_counter()
    done = []
    for s, j in pts:
        if done and time.perf_counter() - t0 > budget_s:
            break
        done.append((s, j))
        if w.nk == (1, 1, 1):
            osox.sigma_tau(w.X[0], w.V[0], w.V[0], w.G[s, 0], taus=[j])
        else:
            Gm = ogrid.g_minus_tau(np.asarray(w.G[s], complex))
            okp.sigma_chain(w.X, w.V, w.V, w.G[s][:, j], Gm[:, j], w.nk)
    dt = time.perf_counter() - t0
    return len(done) / dt, dt, done


def points_per_build(name: str, w) -> float:
    """Oracle sample points (one tau point of one spin of ``w``) that make one build."""
    return float(w.n_tau * w.n_spin)


def batch_oracle_sample(budget_s: float = 20.0):
    """The oracle on the uneven batch: one tau point (complex128 chain) of instances taken
    smallest first over distinct sizes, stopping once `budget_s` is spent (at least three
    sizes).  The time of one tau point of every instance is predicted from a power-law fit
    t = a * cost^b over the sampled (cost, time) pairs, cost = 4 N^2 n^2 (the fit follows
    the oracle's own growth, which is slower than the cost model at large n), and one build
    is the predicted sum over instances times 120 tau points.  Returns
    (builds/s, seconds spent, description)."""
    import synth
    from oracle import sox as osox
    from paper_2412_18829_gb300 import sharding

    sizes = [int(n) for n in synth.batch_c4_sizes()]
    order = sorted(range(len(sizes)), key=lambda i: (sizes[i], i))
    seen, picks = set(), []
    for i in order:
        if sizes[i] not in seen:
            seen.add(sizes[i])
            picks.append(i)
    t0 = time.perf_counter()
    pts = []
    for i in picks:
        if len(pts) >= 3 and time.perf_counter() - t0 > budget_s:
            break
        w = synth.c4_instance(i)
        a = time.perf_counter()
        osox.sigma_tau(w.X[0], w.V[0], w.V[0], w.G[0, 0], taus=[0])
        pts.append((sharding.build_cost(w.n, w.N, 1), time.perf_counter() - a, w.n))
    spent = time.perf_counter() - t0
    c = np.log([p[0] for p in pts])
    t = np.log([p[1] for p in pts])
    b, loga = np.polyfit(c, t, 1)
    per_point = sum(float(np.exp(loga + b * np.log(sharding.build_cost(n, 6 * n, 1)))) for n in sizes)
    value = 1.0 / (per_point * 120)
    desc = (f"1 tau point of each of {len(pts)} instances (n = {[p[2] for p in pts]}), numpy complex128 chain, "
            f"{spent:.1f} s; per-point time of all 16 instances from the fit t = a cost^{b:.3f} "
            f"(cost 4 N^2 n^2) over those points, x 120 tau points per build")
    return value, spent, desc


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload == "c4":
        for _ in range(args.warmup):
            batch_oracle_sample(budget_s=0.0)
        vals, times = [], []
        for _ in range(args.steps):
            v, dt, desc = batch_oracle_sample()
            vals.append(v)
            times.append(dt)
        value = float(np.mean(vals))
        cfg = {"workload": "sox-c4-batch16-N6n-t120", "n": [int(n) for n in __import__("synth").batch_c4_sizes()],
               "N": "6n", "n_tau": 120, "step": "one tau point of several batch instances"}
        sample = desc
    else:
        w = workload(args.workload)
        per_build = points_per_build(args.workload, w)
        for _ in range(args.warmup):
            oracle_tau_points_per_s(w, 1)
        times = []
        for _ in range(args.steps):
            rate, dt, _ = oracle_tau_points_per_s(w, 1)
            times.append(dt)
        value = 1.0 / (np.mean(times) * per_build)
        cfg = {"workload": w.name, "n": w.n, "N": w.N, "n_tau": w.n_tau, "n_spin": w.n_spin,
               "step": "one (spin, tau) point of a build"}
        sample = f"1 (spin, tau) point of {w.name} per step, {per_build:.4g} such points per build"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _apply_v_shard(case, pkg, n):
    """A build split over the orbital index v: this rank keeps the terms of its v range
    (sox_set_v_range), and the step ends with one all-reduce of the orbital-basis Sigma."""
    case.units = 1.0
    if getattr(case, "v_shard", None) is None:
        return
    from paper_2412_18829_gb300 import sharding

    rank, world, _ = case.v_shard
    v0, v1 = sharding.v_shards(n, world)[rank]
    pkg.sox_set_v_range(case.h, v0, v1)
    case.units = 1.0 / world


def _reduce_v_shard_host(case, Sh):
    """The e2e form of the exchange: the rank's partial Sigma from its host buffer to the
    device, the all-reduce, the sum back to the host; returns the extra (h2d, d2h) bytes."""
    if getattr(case, "v_shard", None) is None or case.v_shard[1] == 1 or case.v_shard[2] is None:
        return 0, 0
    t = case.torch.from_numpy(Sh).to(case.dev)
    _reduce_v_shard(case, t)
    Sh[...] = t.cpu().numpy()
    return Sh.nbytes, Sh.nbytes


def _reduce_v_shard(case, S):
    if getattr(case, "v_shard", None) is None:
        return
    _, world, dist = case.v_shard
    if dist is not None and world > 1:
        t = case.torch.view_as_real(S) if S.is_complex() else S
        dist.all_reduce(t)


class Case:
    """One workload on one rank: device-resident step, host-buffer step, accounting."""

    name = ""
    dtype = "f64"
    hot = "sox_bcd"
    units = 1.0                 # builds per step on this rank
    cpu_points_per_build = 1.0  # oracle sample points that make one build
    config: dict = {}

    def step(self):
        raise NotImplementedError

    def e2e_step(self):
        """One step with host buffers through the C ABI; returns (h2d_bytes, d2h_bytes)."""
        raise NotImplementedError

    def hot_flops_per_step(self) -> float:
        raise NotImplementedError

    def accuracy(self) -> dict:
        return {}

    def fp64_compare(self, value: float) -> dict:
        return {}


def _tensor_peak(pk, pk_src, achieved):
    peak = pk.get("bf16_tflops_sustained", 1700.0)
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if achieved else None, "traffic": None,
            "peak_source": f"{pk_src} bf16 sustained (fp16 dense rate = bf16 rate)",
            "mma_issued_tflops": 3 * achieved if achieved else None,
            "tensor_pipe_frac": 3 * achieved / peak if achieved else None,
            "note": "achieved counts algorithmic flops 4N^2n^2 + 2N^2n per (tau, spin); "
                    "the FP16x2 split issues 3 MMAs per product"}


def _alu_peak(achieved, what):
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS if achieved else None, "traffic": None,
            "peak_source": "nominal GB300 FP64 rate (1.25 TFLOP/s dense)", "note": what}


FP64_PEAK_TFLOPS = 1.25
# DRAM bytes (read + write) of one fused-kernel launch over 16 (spin, tau) batches at n=120,
# N=600, from an ncu capture of k_sox_bcd_tc; the U2 operand (36.9 MB) is read once per
# launch, the rest scales with the batches of a launch
BCD_TRAFFIC = {"shape": (120, 600), "batches": 16, "bytes": 726826496 + 20508672, "shared": 36.9e6,
               "source": "ncu dram__bytes_read+write of k_sox_bcd_tc_res (the autotuner's pick at this shape; "
                         "k_sox_bcd_tc reads the same bytes) on 16 batches, scaled to the launch's batches"}
# DRAM bytes (read + write) of the B and C GEMM launches of one static (tau, v) pair of the
# 3x3x3 solid (n=26, N=300), from an ncu capture; compared with the pair's algorithmic bytes
SOLID_BC_TRAFFIC = {"shape": ((3, 3, 3), 26, 300), "bytes": 64837120 + 467264000 + 117595392 + 464676864,
                    "source": "ncu dram__bytes_read+write of the B and C k_gemm_f16x2 launches of one static "
                              "(tau, v) pair (profile_case solid f16x2 4)"}


class MoleculeCase(Case):
    """Bare SOX (c0, c1) or statically screened SOSEX with Pi(0) and W(0) per step (c2)."""

    def __init__(self, torch, pkg, w, prec, dev, stream, screened: bool, variant: str = "sosex",
                 tau_shard=None):
        self.torch, self.pkg, self.w, self.prec, self.dev, self.stream = torch, pkg, w, prec, dev, stream
        self.screened = screened
        self.variant = variant
        self.tau_shard = tau_shard   # (rank, world, dist): this rank's mirror pairs of one build
        self.name = w.name
        self.dtype = "f16x2+f32acc,f64" if prec == "f16x2" else "f64"
        self.hot = "sox_bcd_tc" if prec == "f16x2" else "sox_bcd"
        self.units = 1.0
        self.cpu_points_per_build = w.n_tau * w.n_spin
        self.p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
        self.G = torch.from_numpy(w.G).to(dev)
        self.X = torch.from_numpy(w.X).to(dev)
        self.V = torch.from_numpy(w.V).to(dev)
        self.S = torch.empty_like(self.G)
        _, wts = pkg.sox_tau_grid(w.n_tau, w.beta)
        self.wts_h = np.ascontiguousarray(wts)
        self.wts = torch.from_numpy(self.wts_h).to(dev)
        self.Pi = torch.empty(w.n_spin, w.N, w.N, dtype=torch.float64, device=dev)
        self.W0 = torch.empty(1, w.N, w.N, dtype=torch.float64, device=dev)
        self.h = _kernel_handle(pkg, prec, dev.index or 0)
        if tau_shard is not None:
            from paper_2412_18829_gb300 import sharding

            rank, world, _ = tau_shard
            self.orders = sharding.tau_shards(w.n_tau, world)
            order = self.orders[rank]
            self.kmax = max(len(o) for o in self.orders)
            self.p = pkg.problem(w.n, w.N, len(order), w.n_spin, w.beta)
            self.G = self.G[:, :, order].contiguous()
            self.S = torch.empty_like(self.G)
            self.padded = torch.zeros(w.n_spin, 1, self.kmax, w.n, w.n, dtype=torch.float64, device=dev)
            self.gathered = torch.empty(world, w.n_spin, 1, self.kmax, w.n, w.n, dtype=torch.float64, device=dev)
            self.units = 1.0 / world
        self.config = {"workload": w.name, "n": w.n, "N": w.N, "n_tau": w.n_tau, "n_spin": w.n_spin,
                       "beta": w.beta, "precision": prec,
                       "step": ({"sosex": "Pi(0) + W(0) + SOX(W(0), v)",
                                 "2sosex": "Pi(0) + W(0) + 2SOSEX = SOX(v, W(0)) + SOX(W(0) - v, v)",
                                 "g3w2": "Pi(0) + W(0) + SOX(W(0), W(0))"}[variant] + " through the C ABI"
                                if screened else "bare SOX(v, v) through the C ABI")}

    def _run(self, h, G, X, V, S, Pi, W0, stream):
        pkg = self.pkg
        if not self.screened:
            pkg.sox_sigma(h, self.p, G, X, V, S, stream)
            return
        pkg.sox_pi0(h, self.p, G, X, self.wts if isinstance(G, self.torch.Tensor) else self.wts_h, Pi, stream)
        pkg.sox_w_static(h, self.p, V, Pi[0:1] if self.w.n_spin == 1 else Pi.sum(0, keepdim=True), W0, stream)
        if self.variant == "2sosex":
            pkg.sosex2_static_sigma(h, self.p, G, X, V, W0, S, stream=stream)
        elif self.variant == "g3w2":
            pkg.g3w2_static_sigma(h, self.p, G, X, W0, S, stream=stream)
        else:
            pkg.sosex_static_sigma(h, self.p, G, X, V, W0, S, slot=1, stream=stream)

    def step(self):
        self._run(self.h, self.G, self.X, self.V, self.S, self.Pi, self.W0, self.stream)
        if self.tau_shard is not None:   # the one exchange: every rank receives every rank's slices
            _, world, dist = self.tau_shard
            k = self.S.shape[2]
            self.padded[:, :, :k].copy_(self.S)
            if dist is None:
                self.gathered[0].copy_(self.padded)
            else:
                dist.all_gather_into_tensor(self.gathered, self.padded)

    def e2e_step(self):
        w = self.w
        if not hasattr(self, "Gh"):
            pin = lambda a: self.torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()   # noqa: E731
            Gsrc = w.G if self.tau_shard is None else w.G[:, :, self.orders[self.tau_shard[0]]]
            self.Gh, self.Xh, self.Vh = pin(Gsrc), pin(w.X), pin(w.V)
            self.Sh = pin(np.empty_like(Gsrc))
        self._run(self.h, self.Gh, self.Xh, self.Vh, self.Sh, self.Pi, self.W0, self.stream)
        if self.tau_shard is not None:   # the slices of every rank, back on this rank's host
            _, world, dist = self.tau_shard
            k = self.Sh.shape[2]
            self.padded[:, :, :k].copy_(self.torch.from_numpy(self.Sh), non_blocking=True)
            if dist is None:
                self.gathered[0].copy_(self.padded)
            else:
                dist.all_gather_into_tensor(self.gathered, self.padded)
            gathered_h = self.gathered.cpu()
            return (self.Gh.nbytes + w.X.nbytes + w.V.nbytes + self.Sh.nbytes,
                    self.Sh.nbytes + gathered_h.numel() * 8)
        h2d = w.G.nbytes + w.X.nbytes + w.V.nbytes
        if self.screened:   # Pi(0) reads G, X, w; W(0) reads V; SOSEX reads G, X, V again
            h2d += w.G.nbytes + w.X.nbytes + self.wts_h.nbytes + w.V.nbytes
        return h2d, w.G.nbytes

    def hot_flops_per_step(self):
        w = self.w
        builds = 2 if (self.screened and self.variant == "2sosex") else 1   # 2SOSEX: two SOX builds
        return builds * (4.0 * w.N ** 2 * w.n ** 2 + 2.0 * w.N ** 2 * w.n) * self.p.n_tau * w.n_spin

    def accuracy(self) -> dict:
        from oracle import grid as ogrid, screening as oscr, sox as osox

        w = self.w
        if self.tau_shard is not None:   # Sigma of the whole build from the gathered slices
            from paper_2412_18829_gb300 import sharding

            g = self.gathered.cpu()
            out = sharding.assemble([g[r][:, :, :len(o)] for r, o in enumerate(self.orders)], self.orders,
                                    w.n_tau).numpy()
        else:
            out = self.S.cpu().numpy()
        if not self.screened:
            taus = [0, w.n_tau - 1]
            err = smax = 0.0
            for s in range(w.n_spin):
                ref = osox.sigma_tau(w.X[0], w.V[0], w.V[0], w.G[s, 0], taus=taus, dtype=np.float64)
                err = max(err, float(np.abs(out[s, 0, taus] - ref).max()))
                smax = max(smax, float(np.abs(ref).max()))
            return {"max_abs_err_Ha_vs_oracle": err, "max_rel_err_vs_oracle": err / smax,
                    "oracle_sample": f"tau {taus} x {w.n_spin} spins"}
        wt = ogrid.clenshaw_curtis(w.n_tau, w.beta)
        Pi = oscr.pi0_quadrature(w.X[0], w.G[0, 0], wt).real
        Wr = oscr.w_static(w.V[0], 0.5 * (Pi + Pi.T))
        j = 0   # the largest |Sigma|
        st = lambda U1, U2: osox.sigma_tau(w.X[0], U1, U2, w.G[0, 0], taus=[j], dtype=np.float64)  # noqa: E731
        if self.variant == "2sosex":
            ref = st(w.V[0], Wr) + st(Wr - w.V[0], w.V[0])
        elif self.variant == "g3w2":
            ref = st(Wr, Wr)
        else:
            ref = st(Wr, w.V[0])
        err = float(np.abs(out[0, 0, [j]] - ref).max())
        werr = float((self.W0[0].cpu() - self.torch.from_numpy(Wr)).abs().max()) / float(np.abs(Wr).max())
        return {"max_abs_err_Ha_vs_oracle": err, "max_rel_err_vs_oracle": err / float(np.abs(ref).max()),
                "W0_max_rel_err_vs_oracle": werr,
                "oracle_sample": f"tau index {j}; oracle W(0) from its own Pi(0)"}

    def fp64_compare(self, value: float) -> dict:
        if self.prec == "fp64" or self.tau_shard is not None:
            return {}
        torch = self.torch
        with self.pkg.Handle("fp64", device=self.dev.index or 0) as h64:
            S64 = torch.empty_like(self.G)
            self.pkg.sox_reserve(h64, self.p)
            self._run(h64, self.G, self.X, self.V, S64, self.Pi, self.W0, self.stream)   # warm
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(self.stream)
            self._run(h64, self.G, self.X, self.V, S64, self.Pi, self.W0, self.stream)
            b.record(self.stream)
            torch.cuda.synchronize()
            t64 = a.elapsed_time(b) / 1e3
            return {"fp64_gpu_builds_per_s": 1.0 / t64, "speedup_vs_fp64_gpu": value * t64,
                    "max_abs_err_Ha_vs_fp64_gpu_all_points": float((self.S - S64).abs().max().item())}


def _zflops(*cmacs):
    return 8.0 * float(sum(cmacs))


class SolidCase(Case):
    """Dynamically screened SOSEX of a solid (c3): SOX(v, v) + Sigma_d, split precision on the
    tensor cores (complex FP16 pairs, FP32 accumulation, FP64 ends) or FP64 complex."""

    def __init__(self, torch, pkg, w, prec, dev, stream, rpa_w=False, v_shard=None):
        import synth

        self.torch, self.pkg, self.w, self.dev, self.stream = torch, pkg, w, dev, stream
        self.v_shard = v_shard   # (rank, world, dist): this rank's v range of one build
        self.rpa_w = rpa_w
        self.prec = prec
        self.name = w.name
        self.dtype = "cf16x2+f32acc,c128" if prec == "f16x2" else "c128"
        self.hot = "kpoint_bc" if prec == "f16x2" else "kpoint_dynamic_f64"
        self.units = 1.0
        self.cpu_points_per_build = w.n_tau * w.n_spin
        M = (w.n_tau - 1) // 2
        _, Tf, Ti = synth.bosonic_transforms(w.tau, w.beta, M)
        Wd = synth.pole_screening(w.V, w.beta, M)
        self.nO = 2 * M + 1
        self.p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta, nk=w.nk, dtype=1)
        to = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=complex)).to(dev)   # noqa: E731
        self.G, self.X, self.V, self.Wd, self.Tf, self.Ti = (to(a) for a in (w.G, w.X, w.V, Wd, Tf, Ti))
        self.host = (w.G, w.X, w.V, Wd, Tf, Ti)
        self.S = torch.empty_like(self.G)
        self.h = _kernel_handle(pkg, prec, dev.index or 0)
        _apply_v_shard(self, pkg, w.n)
        self.config = {"workload": w.name, "nk": list(w.nk), "n": w.n, "N": w.N, "n_tau": w.n_tau,
                       "n_omega": self.nO, "beta": w.beta, "precision": prec,
                       "W_d": ("RPA W(i Omega) - v from G on the GPU (sox_w_dynamic) inside every step" if rpa_w
                               else "synthetic single-pole form (synth.pole_screening), input"),
                       "step": "SOX(v, v) + dynamically screened Sigma_d through the C ABI"}

    def step(self):
        if self.rpa_w:   # W_d(i Omega) = RPA W - v from this step's G, on the GPU
            self.pkg.sox_w_dynamic(self.h, self.p, self.G, self.X, self.V, self.Tf, self.nO, self.Wd, self.stream)
        self.pkg.sosex_dynamic_sigma(self.h, self.p, self.G, self.X, self.V, self.Wd, self.Tf, self.Ti,
                                     self.nO, self.S, self.stream)
        _reduce_v_shard(self, self.S)

    def e2e_step(self):
        if not hasattr(self, "hp"):
            self.hp = [self.torch.from_numpy(np.ascontiguousarray(a, dtype=complex)).pin_memory().numpy()
                       for a in self.host]
            self.Sh = self.torch.from_numpy(np.empty_like(self.hp[0])).pin_memory().numpy()
        G, X, V, Wd, Tf, Ti = self.hp
        self.pkg.sosex_dynamic_sigma(self.h, self.p, G, X, V, Wd, Tf, Ti, self.nO, self.Sh, self.stream)
        xh, xd = _reduce_v_shard_host(self, self.Sh)
        return sum(a.nbytes for a in self.hp) + xh, self.Sh.nbytes + xd

    def phase_flops(self):
        w = self.w
        nk = w.nk[0] * w.nk[1] * w.nk[2]
        n, N, T, nO = w.n, w.N, w.n_tau, self.nO
        mixed = nk * nk * N * N * n * n
        static = mixed + T * (nk * nk * N * n ** 3 + 2 * nk * nk * n * N * N * n + nk ** 3 * n * N * N
                              + nk * (N * N * n + N * n * n))
        dyn = mixed + 2 * nk * T * N * n * n + n * nk * (nk * nO * T * N * n + nk * nO * N * N * n
                                                          + nk * T * nO * N * n) \
            + n * T * (2 * nk * nk * N * N * n + nk ** 3 * N * N) + T * nk * (N * N * n + N * n * n)
        return _zflops(static), _zflops(dyn)

    def hot_flops_per_step(self):
        return self.phase_flops()[1]

    def bc_bytes_per_step(self):
        """Algorithmic HBM bytes of the B and C GEMMs, static and dynamic parts: per (tau, v)
        the two n_k^2 x N x N complex FP32 outputs and their FP16-pair operands (K = n)."""
        w = self.w
        nk = w.nk[0] * w.nk[1] * w.nk[2]
        N, n = w.N, w.n
        kp2 = -(-2 * n // 64) * 64                 # halves per split row
        out = 2 * nk * nk * N * N * 8
        ops = (nk * nk * N + nk * 2 * N + nk * N + nk * nk * 2 * N) * kp2 * 4
        return 2 * w.n_tau * n * w.n_spin * (out + ops)

    def d_bytes_per_step(self):
        """Algorithmic HBM bytes of the D step: B and C read once, D (FP64 complex) read and written."""
        w = self.w
        nk = w.nk[0] * w.nk[1] * w.nk[2]
        ldn = w.N + (w.N & 1)
        return 2 * w.n_tau * w.n * w.n_spin * (2 * nk * nk * w.N * w.N * 8 + 2 * nk * w.N * ldn * 16)

    def fp64_compare(self, value: float) -> dict:
        if self.prec == "fp64":
            return {}
        torch = self.torch
        with self.pkg.Handle("fp64", device=self.dev.index or 0) as h64:
            S64 = torch.empty_like(self.S)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(self.stream)
            self.pkg.sosex_dynamic_sigma(h64, self.p, self.G, self.X, self.V, self.Wd, self.Tf, self.Ti, self.nO, S64,
                                         self.stream)
            b.record(self.stream)
            torch.cuda.synchronize()
            t64 = a.elapsed_time(b) / 1e3
            return {"fp64_gpu_builds_per_s": 1.0 / t64, "speedup_vs_fp64_gpu": value * t64,
                    "max_abs_err_Ha_vs_fp64_gpu_all_points": float((self.S - S64).abs().max().item()),
                    "max_abs_sigma_Ha": float(S64.abs().max().item())}


class DynMoleculeCase(Case):
    """Dynamically screened SOSEX of the mid-size molecule (n=120, N=600, 80 tau, 2 spins):
    SOX(v, v) + Sigma_d per step, W_d from the synthetic single-pole form."""

    def __init__(self, torch, pkg, w, prec, dev, stream, v_shard=None):
        import synth

        self.torch, self.pkg, self.w, self.prec, self.dev, self.stream = torch, pkg, w, prec, dev, stream
        self.v_shard = v_shard   # (rank, world, dist): this rank's v range of one build
        self.name = w.name + "-dyn"
        self.dtype = "f16x2+f32acc,f64" if prec == "f16x2" else "f64"
        self.hot = "sox_bcd_dyn_tc" if prec == "f16x2" else "sosex_dynamic_f64"
        self.units = 1.0
        self.cpu_points_per_build = w.n_tau * w.n_spin
        M = (w.n_tau - 1) // 2
        _, Tf, Ti = synth.bosonic_transforms(w.tau, w.beta, M)
        Wd = synth.pole_screening(w.V, w.beta, M)
        self.nO = 2 * M + 1
        self.p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
        to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)   # noqa: E731
        self.G, self.X, self.V, self.Wd = (to(a) for a in (w.G, w.X, w.V, Wd))
        self.Tf, self.Ti = to(Tf), to(Ti)
        self.host = (w.G, w.X, w.V, Wd, Tf, Ti)
        self.S = torch.empty_like(self.G)
        self.h = _kernel_handle(pkg, prec, dev.index or 0)
        _apply_v_shard(self, pkg, w.n)
        self.config = {"workload": self.name, "n": w.n, "N": w.N, "n_tau": w.n_tau, "n_spin": w.n_spin,
                       "n_omega": self.nO, "beta": w.beta, "precision": prec,
                       "W_d": "synthetic single-pole form (synth.pole_screening), input",
                       "step": "SOX(v, v) + dynamically screened Sigma_d through the C ABI"}

    def _run(self, h, S):
        self.pkg.sosex_dynamic_sigma(h, self.p, self.G, self.X, self.V, self.Wd, self.Tf, self.Ti, self.nO, S,
                                     self.stream)

    def step(self):
        self._run(self.h, self.S)
        _reduce_v_shard(self, self.S)

    def e2e_step(self):
        if not hasattr(self, "hp"):
            self.hp = [self.torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in self.host]
            self.Sh = self.torch.from_numpy(np.empty_like(self.hp[0])).pin_memory().numpy()
        G, X, V, Wd, Tf, Ti = self.hp
        self.pkg.sosex_dynamic_sigma(self.h, self.p, G, X, V, Wd, Tf, Ti, self.nO, self.Sh, self.stream)
        xh, xd = _reduce_v_shard_host(self, self.Sh)
        return sum(a.nbytes for a in self.hp) + xh, self.Sh.nbytes + xd

    def phase_flops(self):
        """Algorithmic flops: the static SOX(v, v) and the dynamic part (per v: transform
        2 T N n (x 2 re/im) x n_omega, W_d product 2 n_omega N^2 n x 2, inverse transform
        2 T N n x 2 n_omega, then the fused B/C/D 4 N^2 n per (tau, v) and the Hadamard)."""
        w = self.w
        n, N, T, S, nO = w.n, w.N, w.n_tau, w.n_spin, self.nO
        static = (4.0 * N * N * n * n + 2.0 * N * N * n + 2.0 * N * n ** 3) * T * S + 2.0 * N * N * n * n
        dyn = S * n * (4.0 * nO * T * N * n + 4.0 * nO * N * N * n + 4.0 * T * nO * N * n) \
            + (4.0 * N * N * n * n + 2.0 * N * N * n) * T * S
        return static, dyn

    def hot_flops_per_step(self):
        w = self.w
        return (4.0 * w.N ** 2 * w.n ** 2 + 2.0 * w.N ** 2 * w.n) * w.n_tau * w.n_spin

    def accuracy(self) -> dict:
        """Against the FP64 GPU path (the oracle's dynamic chain at this size takes hours)."""
        return {}

    def fp64_compare(self, value: float) -> dict:
        if self.prec == "fp64":
            return {}
        torch = self.torch
        with self.pkg.Handle("fp64", device=self.dev.index or 0) as h64:
            S64 = torch.empty_like(self.S)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(self.stream)
            self._run(h64, S64)
            b.record(self.stream)
            torch.cuda.synchronize()
            t64 = a.elapsed_time(b) / 1e3
            return {"fp64_gpu_builds_per_s": 1.0 / t64, "speedup_vs_fp64_gpu": value * t64,
                    "max_abs_err_Ha_vs_fp64_gpu_all_points": float((self.S - S64).abs().max().item()),
                    "max_abs_sigma_Ha": float(S64.abs().max().item()),
                    "accuracy_note": "against the FP64 GPU path, itself at 1e-12 of the oracle in the parity tests"}


class BatchCase(Case):
    """The uneven batch (c4): Phi and Sigma of every instance, then dPhi/dG from the kept
    Sigma; the 16 instances are dealt out over the ranks (no data-path collective)."""

    def __init__(self, torch, pkg, prec, dev, stream, rank, world, backward=True):
        import synth
        from paper_2412_18829_gb300 import sharding

        self.torch, self.pkg, self.prec, self.dev, self.stream = torch, pkg, prec, dev, stream
        self.backward = backward
        sizes = [int(n) for n in synth.batch_c4_sizes()]
        costs = [sharding.build_cost(n, 6 * n, 120) for n in sizes]
        self.mine = sharding.shard(costs, world)[rank]
        self.world = world
        self.name = "sox-c4-batch16-N6n-t120"
        self.dtype = "f16x2+f32acc,f64" if prec == "f16x2" else "f64"
        self.hot = "sox_bcd_tc" if prec == "f16x2" else "sox_bcd"
        self.units = 1.0 / world
        self.h = _kernel_handle(pkg, prec, dev.index or 0)
        self.inst = []
        for i in self.mine:
            w = synth.c4_instance(i)
            _, wts = pkg.sox_tau_grid(w.n_tau, w.beta)
            d = {"w": w, "p": pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta),
                 "G": torch.from_numpy(w.G).to(dev), "X": torch.from_numpy(w.X).to(dev),
                 "V": torch.from_numpy(w.V).to(dev), "wt": torch.from_numpy(np.ascontiguousarray(wts)).to(dev),
                 "wt_h": np.ascontiguousarray(wts)}
            d["S"] = torch.empty_like(d["G"])
            d["dG"] = torch.empty_like(d["G"])
            d["dX"] = torch.empty_like(d["X"])
            d["dV"] = torch.empty_like(d["V"])
            d["phi"] = torch.empty(w.n_spin, dtype=torch.float64, device=dev)
            d["dphi"] = torch.ones(w.n_spin, dtype=torch.float64, device=dev)
            self.inst.append(d)
        self.config = {"workload": self.name, "instances": len(sizes), "n": sizes, "N": "6n", "n_tau": 120,
                       "beta": 100.0, "precision": prec, "instances_on_rank0": self.mine if rank == 0 else None,
                       "step": ("phi_sox_batch (Phi and Sigma of every instance, one persistent fused launch "
                                "per tau chunk), then per instance phi_sox_grad_G (dPhi/dG from the kept Sigma) + "
                                "phi_sox_backward (dPhi/dX, dPhi/dV)") if backward else
                               ("phi_sox_batch (Phi and Sigma of every instance), then per instance "
                                "phi_sox_grad_G (dPhi/dG from the kept Sigma)")}

    def _forward(self, h, G, X, V, wt, S, phi):
        """Phi and Sigma of every instance on this rank in one batched call: one persistent
        fused launch per tau chunk over all instances (split precision)."""
        self.pkg.phi_sox_batch(h, [d["p"] for d in self.inst], G, X, V, wt, phi, S, self.stream)

    def _rest(self, h, d, G, X, V, wt, S, dG, dX=None, dV=None):
        self.pkg.phi_sox_grad_G(h, d["p"], S, wt, d["dphi"], dG, self.stream)
        if dX is not None:   # dPhi/dX and dPhi/dV by the adjoint of the THC chain
            self.pkg.phi_sox_backward(h, d["p"], G, X, V, wt, d["dphi"], None, dX, dV, self.stream)

    def step(self):
        if not self.inst:
            return
        ins = self.inst
        self._forward(self.h, [d["G"] for d in ins], [d["X"] for d in ins], [d["V"] for d in ins],
                      [d["wt"] for d in ins], [d["S"] for d in ins], [d["phi"] for d in ins])
        for d in ins:
            self._rest(self.h, d, d["G"], d["X"], d["V"], d["wt"], d["S"], d["dG"],
                       d["dX"] if self.backward else None, d["dV"] if self.backward else None)

    def e2e_step(self):
        h2d = d2h = 0
        if not self.inst:
            return h2d, d2h
        for d in self.inst:
            if "Gh" not in d:
                pin = lambda a: self.torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
                w = d["w"]
                d["Gh"], d["Xh"], d["Vh"] = pin(w.G), pin(w.X), pin(w.V)
                d["Sh"], d["dGh"], d["phih"] = pin(np.empty_like(w.G)), pin(np.empty_like(w.G)), pin(np.zeros(w.n_spin))
            if "dXh" not in d:
                d["dXh"] = self.torch.from_numpy(np.empty_like(d["w"].X)).pin_memory().numpy()
                d["dVh"] = self.torch.from_numpy(np.empty_like(d["w"].V)).pin_memory().numpy()
        ins = self.inst
        self._forward(self.h, [d["Gh"] for d in ins], [d["Xh"] for d in ins], [d["Vh"] for d in ins],
                      [d["wt_h"] for d in ins], [d["Sh"] for d in ins], [d["phih"] for d in ins])
        bw = self.backward
        for d in ins:
            self._rest(self.h, d, d["Gh"], d["Xh"], d["Vh"], d["wt_h"], d["Sh"], d["dGh"],
                       d["dXh"] if bw else None, d["dVh"] if bw else None)
            h2d += d["Gh"].nbytes + d["Xh"].nbytes + d["Vh"].nbytes + 2 * d["wt_h"].nbytes + d["Sh"].nbytes
            d2h += d["Sh"].nbytes + d["phih"].nbytes + d["dGh"].nbytes
            if bw:
                h2d += d["Gh"].nbytes + d["Xh"].nbytes + d["Vh"].nbytes + d["wt_h"].nbytes
                d2h += d["dXh"].nbytes + d["dVh"].nbytes
        return h2d, d2h

    def hot_flops_per_step(self):
        return sum((4.0 * d["w"].N ** 2 * d["w"].n ** 2 + 2.0 * d["w"].N ** 2 * d["w"].n) * d["w"].n_tau
                   for d in self.inst)

    def _smallest(self):
        import synth

        small = synth.c4_smallest(3)
        return [d for i, d in zip(self.mine, self.inst) if i in small]

    def _largest(self):
        return max(self.inst, key=lambda d: d["w"].n) if self.inst else None

    def accuracy(self) -> dict:
        """max|dSigma| against the oracle: two tau points of the three smallest instances and
        tau index 0 (the largest |Sigma|) of the largest instance on this rank."""
        from oracle import sox as osox

        err = rel = 0.0
        picks = [(d, [0, d["w"].n_tau // 2]) for d in self._smallest()]
        big = self._largest()
        if big is not None and all(big is not d for d, _ in picks):
            picks.append((big, [0]))
        for d, taus in picks:
            w = d["w"]
            ref = osox.sigma_tau(w.X[0], w.V[0], w.V[0], w.G[0, 0], taus=taus, dtype=np.float64)
            e = float(np.abs(d["S"].cpu().numpy()[0, 0, taus] - ref).max())
            err, rel = max(err, e), max(rel, e / float(np.abs(ref).max()))
        return {"max_abs_err_Ha_vs_oracle": err, "max_rel_err_vs_oracle": rel,
                "oracle_sample": "tau 0 and n_tau/2 of the three smallest instances, tau 0 of the largest "
                                 f"(n={big['w'].n})" if big is not None else ""}

    def fp64_compare(self, value: float) -> dict:
        """The plain FP64 GPU path on one mirror pair of tau points {j, n_tau-1-j} of EVERY
        instance, scaled by n_tau / 2: static SOX, Phi and the adjoint are local in tau (the
        pair is itself a mirror-symmetric grid), so the per-point cost is the same at every
        tau and the scaled time is the full build's.  Forward (phi_sox + phi_sox_grad_G) and
        the X/V adjoint (phi_sox_backward) are timed separately; the split path is timed on the
        same pairs and compared value by value."""
        torch = self.torch
        if not self.inst:
            return {}
        ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))  # noqa: E731

        def timed(fn):
            fn()
            torch.cuda.synchronize()
            a, b = ev()
            a.record(self.stream)
            fn()
            b.record(self.stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / 1e3

        sub = []
        for d in self.inst:
            w = d["w"]
            j = w.n_tau // 4
            order = [j, w.n_tau - 1 - j]
            e = {"d": d, "p": self.pkg.problem(w.n, w.N, 2, w.n_spin, w.beta), "G": d["G"][:, :, order].contiguous(),
                 "wt": d["wt"][order].contiguous(), "scale": w.n_tau / 2.0}
            for k in ("S", "S64", "dG", "dX", "dV", "dX64", "dV64"):
                src = d["X"] if "X" in k else (d["V"] if "V" in k else e["G"])
                e[k] = torch.empty_like(src)
            e["phi"] = torch.empty(w.n_spin, dtype=torch.float64, device=self.dev)
            sub.append(e)

        def fwd(h, key):
            for e in sub:
                self.pkg.phi_sox(h, e["p"], e["G"], e["d"]["X"], e["d"]["V"], e["wt"], e["phi"], e[key], self.stream)
                self.pkg.phi_sox_grad_G(h, e["p"], e[key], e["wt"], e["d"]["dphi"], e["dG"], self.stream)

        def adj(h, kx, kv):
            for e in sub:
                self.pkg.phi_sox_backward(h, e["p"], e["G"], e["d"]["X"], e["d"]["V"], e["wt"], e["d"]["dphi"], None,
                                          e[kx], e[kv], self.stream)

        scale = sub[0]["scale"] if all(e["scale"] == sub[0]["scale"] for e in sub) else None
        t_fwd = timed(lambda: fwd(self.h, "S")) * scale
        t_adj = timed(lambda: adj(self.h, "dX", "dV")) * scale if self.backward else 0.0
        with self.pkg.Handle("fp64", device=self.dev.index or 0) as h64:
            t64_fwd = timed(lambda: fwd(h64, "S64")) * scale
            t64_adj = timed(lambda: adj(h64, "dX64", "dV64")) * scale if self.backward else 0.0
        rel = lambda a, b: float((a - b).abs().max() / b.abs().max())   # noqa: E731
        out = {"fp64_gpu_sample": "one mirror pair {n_tau/4, 3 n_tau/4 - 1} of tau points of every instance, "
                                  "times scaled by n_tau/2 (static SOX, Phi and the adjoint are local in tau)",
               "fp64_gpu_builds_per_s": self.units / (t64_fwd + t64_adj),
               "fp64_gpu_forward_s": t64_fwd, "fp64_gpu_adjoint_s": t64_adj,
               "split_forward_s_same_sample": t_fwd, "split_adjoint_s_same_sample": t_adj,
               "speedup_vs_fp64_gpu": (t64_fwd + t64_adj) / (t_fwd + t_adj),
               "max_abs_err_Ha_vs_fp64_gpu_sampled_pairs": max(float((e["S"] - e["S64"]).abs().max()) for e in sub)}
        if self.backward:
            out["adjoint_split_vs_fp64_max_rel_dX"] = max(rel(e["dX"], e["dX64"]) for e in sub)
            out["adjoint_split_vs_fp64_max_rel_dV"] = max(rel(e["dV"], e["dV64"]) for e in sub)
        return out


KERNEL = "auto"   # --kernel: the split path's fused-kernel variant on every handle the bench opens


def _kernel_handle(pkg, prec, device):
    h = pkg.Handle(prec, device=device)
    if prec == "f16x2" and KERNEL != "auto":
        pkg.sox_set_kernel_variant(h, KERNEL)
    return h


def make_case(args, torch, pkg, dev, stream, rank, world, dist_mod=None):
    if args.workload == "c4":
        return BatchCase(torch, pkg, args.precision, dev, stream, rank, world, backward=not args.forward_only)
    vsh = (rank, world, dist_mod) if (args.shard in ("v", "auto") and world > 1) else None
    if args.workload == "c1d":
        return DynMoleculeCase(torch, pkg, workload("c1"), args.precision, dev, stream, v_shard=vsh)
    w = workload(args.workload)
    if args.workload == "c3":
        if args.mesh != "3,3,3":   # the same solid recipe on another mesh
            import synth

            nk = tuple(int(x) for x in args.mesh.split(","))
            w = synth.solid(3, nk, w.n, w.N, w.n_tau, w.beta, name=f"sosexdyn-k{''.join(map(str, nk))}-n{w.n}-N{w.N}-t{w.n_tau}")
        return SolidCase(torch, pkg, w, args.precision, dev, stream, rpa_w=args.rpa_w, v_shard=vsh)
    shard = (rank, world, dist_mod) if (args.shard == "tau" and args.workload in ("c0", "c1")) else None
    if args.shard == "v" and args.workload in ("c0", "c1", "c2"):
        raise SystemExit("--shard v is wired for the dynamic workloads (c3, c1d)")
    return MoleculeCase(torch, pkg, w, args.precision, dev, stream, screened=(args.workload == "c2"),
                        variant=args.variant, tau_shard=shard)


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
    from paper_2412_18829_gb300 import sharding

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    case = make_case(args, torch, pkg, dev, stream, rank, world, dist)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    for _ in range(args.warmup):
        case.step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    pkg.sox_profile_enable(case.h, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        case.step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    launches, _ = pkg.sox_profile_read(case.h, None)
    hot_n, hot_ms = pkg.sox_profile_read(case.h, case.hot)
    phases = {}
    if isinstance(case, SolidCase):
        for ph in (("kpoint_tc", "kpoint_dynamic_tc", "kpoint_D") if case.prec == "f16x2"
                   else ("kpoint_f64", "kpoint_dynamic_f64")) + (("w_dynamic",) if case.rpa_w else ()):
            phases[ph] = pkg.sox_profile_read(case.h, ph)
    if isinstance(case, DynMoleculeCase):
        phases["sosex_dynamic_tc"] = pkg.sox_profile_read(case.h, "sosex_dynamic_tc")
    if isinstance(case, BatchCase) and case.backward:
        phases["adjoint"] = pkg.sox_profile_read(case.h, "phi_adjoint_tc" if case.prec == "f16x2" else "phi_adjoint_f64")
    pkg.sox_profile_enable(case.h, False)
    clocks = sampler.stop()
    if dist:
        dist.barrier()
    t_local = float(np.sum([a.elapsed_time(b) for a, b in ev])) / 1e3
    t_max = sharding.max_over_ranks(t_local, dist, dev)
    total_units = case.units * world          # builds of the whole job per step
    value = total_units * args.steps / t_max

    extra = {}
    if rank == 0 and not args.skip_accuracy:
        extra.update(case.accuracy())
    if rank == 0 and not args.skip_fp64:
        extra.update(case.fp64_compare(case.units / (t_local / args.steps)))

    e2e = None
    if not args.skip_e2e:
        h2d, d2h = case.e2e_step()    # warm the pinned buffers and staging workspace
        torch.cuda.synchronize()
        e2e_t = []
        for _ in range(max(1, min(args.steps, 3))):
            flush.zero_()
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            t0 = time.perf_counter()
            case.e2e_step()
            torch.cuda.synchronize()
            e2e_t.append(time.perf_counter() - t0)
        te = sharding.max_over_ranks(float(np.mean(e2e_t)), dist, dev)
        e2e = {"value": total_units / te, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    pk, pk_src = peaks()
    hot_s = hot_ms / 1e3
    achieved = case.hot_flops_per_step() * args.steps / hot_s / 1e12 if hot_n and hot_s > 0 else None
    if isinstance(case, SolidCase) and case.prec == "f16x2":
        gbs = case.bc_bytes_per_step() * args.steps / hot_s / 1e9 if hot_n and hot_s > 0 else None
        roof = {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": gbs / pk["hbm_gbs"] if gbs else None, "traffic": None,
                "kernel": "k_gemm_f16x2 (the B and C GEMMs of the solid chain)", "peak_source": pk_src,
                "note": "algorithmic bytes: per (tau, v) the n_k^2 N x N complex FP32 B and C tiles written "
                        "and their FP16-pair operands read, static and dynamic parts"}
        f_static, f_dyn = case.phase_flops()
        extra["phase_ms_per_step"] = {k: v[1] / args.steps for k, v in phases.items()}
        extra["phase_ms_per_step"]["kpoint_bc"] = hot_ms / args.steps
        w = case.w
        if (tuple(w.nk), w.n, w.N) == SOLID_BC_TRAFFIC["shape"]:
            pair = case.bc_bytes_per_step() / (2 * w.n_tau * w.n * w.n_spin)
            roof["traffic"] = SOLID_BC_TRAFFIC["bytes"]
            roof["traffic_unit"] = "bytes per static (tau, v) pair of B and C launches"
            roof["algorithmic_bytes_per_pair"] = pair
            roof["traffic_source"] = SOLID_BC_TRAFFIC["source"]
        d_n, d_ms = phases.get("kpoint_D", (0, 0.0))
        extra["phase_ms_per_step"]["kpoint_D"] = d_ms / args.steps
        if d_ms:
            extra["d_step_gbs"] = case.d_bytes_per_step() * args.steps / (d_ms / 1e3) / 1e9
        extra["algorithmic_tflops_per_s"] = (f_static + f_dyn) * value / 1e12
    elif isinstance(case, SolidCase):
        f_static, f_dyn = case.phase_flops()
        roof = _alu_peak(achieved, "dominant phase: the dynamic part (GG, transforms, W_d product, B/C, "
                                   "n_k^3 D step) in FP64 complex on CUDA cores; algorithmic flops at 8 per complex MAC")
        roof["kernel"] = case.hot
        n_s, ms_s = phases["kpoint_f64"]
        extra["static_phase_tflops"] = f_static * args.steps / (ms_s / 1e3) / 1e12 if ms_s else None
        extra["phase_ms_per_step"] = {"kpoint_f64": ms_s / args.steps, case.hot: hot_ms / args.steps}
    elif isinstance(case, DynMoleculeCase) and case.prec == "f16x2":
        roof = _tensor_peak(pk, pk_src, achieved)
        roof["kernel"] = "k_sox_bcd_tc with X in the G_Rq slot (the dynamic part's fused B/C/D)"
        f_static, f_dyn = case.phase_flops()
        extra["algorithmic_tflops_per_s"] = (f_static + f_dyn) * value / 1e12
        extra["phase_ms_per_step"] = {k: v[1] / args.steps for k, v in phases.items()}
    elif case.dtype.startswith("f16x2"):
        roof = _tensor_peak(pk, pk_src, achieved)
        roof["kernel"] = case.hot
        if isinstance(case, BatchCase):
            roof["kernel"] = "k_sox_bcd_multi (the fused B/C/D kernel, one persistent launch per tau chunk over all instances)"
        w = getattr(case, "w", None)
        if isinstance(case, MoleculeCase) and (w.n, w.N) == BCD_TRAFFIC["shape"] and hot_n:
            b_launch = case.p.n_tau * w.n_spin / (hot_n / args.steps)
            per_b = (BCD_TRAFFIC["bytes"] - BCD_TRAFFIC["shared"]) / BCD_TRAFFIC["batches"]
            roof["traffic"] = per_b * b_launch + BCD_TRAFFIC["shared"]
            roof["traffic_source"] = BCD_TRAFFIC["source"]
        if "adjoint" in phases and phases["adjoint"][1]:
            adj_fl = sum(12.0 * d["w"].N ** 2 * d["w"].n ** 2 * d["w"].n_tau for d in case.inst)
            extra["adjoint_ms_per_step"] = phases["adjoint"][1] / args.steps
            extra["adjoint_algorithmic_tflops"] = adj_fl * args.steps / (phases["adjoint"][1] / 1e3) / 1e12
            extra["forward_fused_kernel_ms_per_step"] = hot_ms / args.steps
    else:
        roof = _alu_peak(achieved, "fused FP64 B/C/Hadamard kernel")
        roof["kernel"] = case.hot
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
        "scaling": "strong" if (isinstance(case, BatchCase) or getattr(case, "tau_shard", None)
                                or getattr(case, "v_shard", None)) else "weak",
        "vs_baseline": None,
        "dtype": case.dtype, "data": "synthetic",
        "config": {**case.config, "l2": "flushed between steps (256 MiB write outside the events)",
                   "parallelism": (f"batch instances sharded over {world} GPUs" if isinstance(case, BatchCase)
                                   else (f"one build split over {world} GPUs by tau mirror pairs, all-gather of "
                                         f"Sigma in the step" if getattr(case, "tau_shard", None)
                                         else (f"one build split over {world} GPUs by the orbital index v, one "
                                               f"all-reduce of Sigma in the step" if getattr(case, "v_shard", None)
                                               else f"{world} independent builds (one per GPU)"))), **extra},
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if args.precision == "f16x2":
        line["config"]["fused_kernel"] = KERNEL if KERNEL != "auto" else "autotuned per shape"
    if world == 1 and not args.skip_cpu_baseline:
        if isinstance(case, BatchCase):
            v, dt, desc = batch_oracle_sample()
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                    "sample": desc + " (forward Sigma only: the oracle has no adjoint chain)"}
        else:
            w0 = workload(args.workload)
            rate, dt, pts = oracle_tau_points_per_s(w0, args.cpu_points)
            line["cpu_baseline"] = {
                "value": rate / case.cpu_points_per_build, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                "sample": f"{len(pts)} (spin, tau) points of {w0.name} ({case.cpu_points_per_build:.4g} such points "
                          f"per build), numpy complex128 chain, {dt:.1f} s; builds/s = points/s / points per build"
                          + ("; the static SOX(v, v) chain only: the dynamic part is not tau-local and the "
                             "oracle's dynamic chain at this size runs for hours, so this bounds the oracle's "
                             "rate from above" if isinstance(case, DynMoleculeCase) else "")}
    print(json.dumps(line), flush=True)
    case.h.close()
    if dist:
        dist.destroy_process_group()


def profile_case(args):
    """One small case on cuda:0 for an ncu capture (a few GB on the device at most)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_2412_18829_gb300 as pkg
    import synth

    kind, prec = args.profile_case, args.precision
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()   # noqa: E731
    if kind in ("molecule", "screened"):
        T = args.profile_tau or (8 if kind == "molecule" else 4)
        w = (synth.molecule(1, 120, 600, T, 100.0, n_spin=2) if kind == "molecule"
             else synth.molecule(2, 250, 2000, T, 100.0, 1))
        p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
        G, X, V = (dev(a) for a in (w.G, w.X, w.V))
        out = torch.empty_like(G)
        with _kernel_handle(pkg, prec, 0) as h:
            for _ in range(2):
                pkg.sox_sigma(h, p, G, X, V, out)
            pkg.sox_check_device(h)
    elif kind in ("batch", "adjoint"):
        T = args.profile_tau or 8
        n = int(synth.batch_c4_sizes().max())
        n, N = (int(x) for x in args.profile_sizes.split(",")) if args.profile_sizes else (n, 6 * n)
        w = synth.molecule(4, n, N, T, 100.0, 1)
        _, wts = pkg.sox_tau_grid(w.n_tau, w.beta)
        p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
        G, X, V, tw = (dev(a) for a in (w.G, w.X, w.V, wts))
        d = torch.ones(1, dtype=torch.float64, device="cuda")
        phi = torch.empty(1, dtype=torch.float64, device="cuda")
        S, dG, dX, out = torch.empty_like(G), torch.empty_like(G), torch.empty_like(X), torch.empty_like(V)
        with _kernel_handle(pkg, prec, 0) as h:
            for _ in range(2):
                if kind == "batch":
                    pkg.phi_sox(h, p, G, X, V, tw, phi, S)
                    pkg.phi_sox_grad_G(h, p, S, tw, d, dG)
                else:
                    pkg.phi_sox_backward(h, p, G, X, V, tw, d, None, dX, out)
            pkg.sox_check_device(h)
    elif kind in ("solid", "dynmol"):
        T = args.profile_tau or 4
        M = (T - 1) // 2
        if kind == "solid":
            mesh = tuple(int(x) for x in args.mesh.split(","))
            n, N = (int(x) for x in args.profile_sizes.split(",")) if args.profile_sizes else (26, 300)
            w = synth.solid(3, mesh, n, N, T, 300.0)
            p = pkg.problem(w.n, w.N, T, 1, w.beta, nk=w.nk, dtype=1)
            cast = lambda a: dev(np.asarray(a, dtype=complex))   # noqa: E731
        else:
            n, N = (int(x) for x in args.profile_sizes.split(",")) if args.profile_sizes else (120, 600)
            w = synth.molecule(1, n, N, T, 100.0, 1)
            p = pkg.problem(w.n, w.N, T, 1, w.beta)
            cast = dev
        _, Tf, Ti = synth.bosonic_transforms(w.tau, w.beta, M)
        Wd = synth.pole_screening(w.V, w.beta, M)
        G, X, V, W = (cast(a) for a in (w.G, w.X, w.V, Wd))
        F, I = (dev(np.asarray(a, dtype=complex)) for a in (Tf, Ti))
        out = torch.empty_like(G)
        with _kernel_handle(pkg, prec, 0) as h:
            pkg.sosex_dynamic_sigma(h, p, G, X, V, W, F, I, 2 * M + 1, out)
            pkg.sox_check_device(h)
    else:   # wdyn
        T = args.profile_tau or 60
        w = synth.solid(3, (3, 3, 3), 26, 300, T, 300.0)
        M = (T - 1) // 2
        _, Tf, _ = synth.bosonic_transforms(w.tau, w.beta, M)
        G, X, V, F = (dev(np.asarray(a, dtype=complex)) for a in (w.G, w.X, w.V, Tf))
        out = torch.empty(27, 2 * M + 1, w.N, w.N, dtype=torch.complex128, device="cuda")
        p = pkg.problem(w.n, w.N, T, 1, w.beta, nk=w.nk, dtype=1)
        with pkg.Handle("fp64") as h:
            pkg.sox_w_dynamic(h, p, G, X, V, F, 2 * M + 1, out)
    torch.cuda.synchronize()
    print("profile case", kind, "ok", float(out.abs().max()))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default per workload: c0 100, c1 40, c2 10, c3 5, c4 3; "
                         "the reference arm 10, 10, 3, 1, 3)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f16x2", choices=["f16x2", "fp64"])
    ap.add_argument("--workload", default="c4", choices=["c0", "c1", "c2", "c3", "c4", "c1d"])
    ap.add_argument("--cpu-points", type=int, default=16)
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-accuracy", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--forward-only", action="store_true", help="batch workload: no dPhi/dX, dPhi/dV")
    ap.add_argument("--shard", default="auto", choices=["auto", "replicas", "tau", "v"],
                    help="N GPUs: auto = one build split by the orbital index v with one all-reduce of Sigma "
                         "for the dynamic workloads (c3, c1d), N independent builds for bare SOX and SOSEX "
                         "(c0-c2), instances dealt out for the batch (c4); tau = one bare-SOX build split by "
                         "tau mirror pairs with an all-gather; v = the v split; replicas = independent builds")
    ap.add_argument("--mesh", default="3,3,3", help="solid workload: k-mesh (default 3,3,3)")
    ap.add_argument("--rpa-w", action="store_true",
                    help="solid workload: build W_d(i Omega) from G on the GPU inside every step")
    ap.add_argument("--kernel", default="auto", choices=["auto", "resident", "streamed", "pair"],
                    help="fused B/C/D kernel variant of the split path (auto: timed per shape)")
    ap.add_argument("--variant", default="sosex", choices=["sosex", "2sosex", "g3w2"],
                    help="screened workload: SOSEX, 2SOSEX or G3W2 with W(0)")
    ap.add_argument("--profile-case", default=None,
                    choices=["molecule", "screened", "batch", "adjoint", "solid", "wdyn", "dynmol"],
                    help="run one small case for an ncu capture instead of the benchmark")
    ap.add_argument("--profile-tau", type=int, default=None, help="tau points of the profile case")
    ap.add_argument("--profile-sizes", default=None, help="profile case sizes n,N (solid, dynmol)")
    args = ap.parse_args()
    global KERNEL
    KERNEL = args.kernel
    if args.profile_case:
        profile_case(args)
        return
    if args.steps is None:   # about a second of timed GPU work for c1; bounded oracle runs for the reference
        ours = {"c0": 100, "c1": 40, "c2": 10, "c3": 5, "c4": 3, "c1d": 5}
        ref = {"c0": 10, "c1": 10, "c2": 3, "c3": 1, "c4": 3, "c1d": 3}
        args.steps = (ref if args.impl == "reference" else ours)[args.workload]
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
