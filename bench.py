#!/usr/bin/env python3
"""Benchmark: stencil GLUP/s and HBM-roofline fraction of the fused KPM path.

Workload (default): the topological-insulator slab of Eq. TB_H_topi,
256 x 256 x 64 sites, periodic in x and y, open in z, t = 1, m = 2, box
disorder W = 2 (seed 2); a block of R = 8 random-phase vectors; 2048 KPM
moments per vector = 1024 fused Chebyshev sweeps (stencil + recurrence +
fp64 dot products).  One benchmark step = one full KPM run.  complex64
storage / fp32 stencil / fp64 moments is the headline; the same workload in
complex128 / fp64 is measured alongside (fewer moments, same per-sweep
work) together with the moment error of complex64 against it.

LUP = one lattice site updated for one vector; value = sites * R * sweeps / s
summed over ranks.  Vectors (1 GiB each) exceed the 129 MB L2, so no flush
is needed between steps.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank runs its own R vectors (independent seeds; weak
scaling, no collective on the data path) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "stencil GLUP/s & %HBM roofline: FP32/batched vs plain FP64, same accuracy"
UNIT = "GLUP/s"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the
# benchmark's sweep, from an ncu capture of a half-depth slab scaled by the number of
# sites, per (workload, R, kernel); reported only while the kernel sources still hash to
# the captured version
TRAFFIC = {("ti_slab", 8, "ti_sweep"): {"bytes_per_launch": 3.220e9, "source_sha256_16": "df26e831c975b98f"},
           ("ti_slab", 8, "ti_sweep_xmarch"): {"bytes_per_launch": 3.222e9, "source_sha256_16": "df26e831c975b98f"},
           ("ti_slab", 8, "ti_sweep_tma"): {"bytes_per_launch": 3.216e9, "source_sha256_16": "9c34eb70b45ba370"}}
KERNEL_SOURCES = ("paper_1708_09689_gb300/csrc/sweep.cuh", "paper_1708_09689_gb300/csrc/common.cuh",
                  "paper_1708_09689_gb300/csrc/sweep_tma.cuh")


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--R", type=int, default=8)
    ap.add_argument("--M", type=int, default=2048)
    ap.add_argument("--W", type=float, default=2.0)
    ap.add_argument("--dims", type=int, nargs=3, default=list(W.CONFIG_TI_SLAB.dims))
    ap.add_argument("--fp64-moments", type=int, default=0,
                    help="moments of the complex128 comparison run (0: all M moments)")
    ap.add_argument("--no-compare", action="store_true", help="skip the complex128 comparison")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the default launch shape instead of the autotuned one")
    ap.add_argument("--workload", default="ti_slab",
                    choices=["ti_slab", "ti_cube", "graphene_qd", "batched", "adjoint", "ti_akE", "chebfd",
                             "wsm_kpm"],
                    help="ti_slab (default): the benchmark line; the others measure the remaining "
                         "workloads (16^3 cube KPM, graphene QD-array propagation, batched KPM over "
                         "64 lattices, adjoint gradient, A(k,E) of a clean TI, ChebFD interior "
                         "eigenpairs, Weyl-semimetal KPM) and print one JSON line each")
    ap.add_argument("--sweeps-only", type=int, default=0,
                    help="profiling case: one KPM call of this many complex64 sweeps (stencil, "
                         "recurrence, dots) on the lattice (ti_slab, ti_akE, wsm_kpm), this many "
                         "complex64 propagation time steps (graphene_qd), or one complex64 filter of "
                         "this many series terms (chebfd, R from --R), and exit without timing")
    ap.add_argument("--batched-count", type=int, default=8,
                    help="with --workload batched --sweeps-only: number of lattices of the batch")
    ap.add_argument("--q64", action="store_true",
                    help="with --sweeps-only: the fixed-point (PVSC_Q64) KPM sweep instead")
    ap.add_argument("--qd-on-the-fly", action="store_true",
                    help="graphene_qd: regenerate the quantum-dot potential inside the sweeps "
                         "instead of reading it")
    ap.add_argument("--launch", default=None,
                    help="JSON launch shape (threads, blocks_per_sm, zslab, vpt, tile_x, tile_y, kernel) "
                         "to use instead of autotuning, e.g. for profiling runs")
    ap.add_argument("--q64-launch", default=None,
                    help="JSON launch shape of the fixed-point (PVSC_Q64) sweep (its default otherwise)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while active."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# --------------------------------------------------------------------------- CPU baseline
def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_worker(conn, dims, R, Wd, seed_r):
    """One host core: the fp64 CSR oracle on the bounded sample, driven by
    ("run", seconds) messages; replies (spMVM steps, seconds) per run."""
    import oracle as O
    n = dims[0] * dims[1] * dims[2]
    V = W.disorder_potential(n, Wd, 2)
    H = O.ti_hamiltonian(dims, (1, 1, 0), 1.0, 2.0, V)
    a, b = O.cheb_scale(*O.gershgorin(H))
    r = W.random_phase_block(4 * n, R, seed_r)
    O.kpm_moments(H, r, 3, a, b)  # warm
    conn.send("ready")
    M = 8
    while True:
        msg = conn.recv()
        if msg[0] != "run":
            break
        steps, t0 = 0, time.perf_counter()
        while True:
            O.kpm_moments(H, r, M, a, b)
            steps += M - 1
            if time.perf_counter() - t0 > msg[1]:
                break
        conn.send((steps, time.perf_counter() - t0))
    conn.close()


class OracleOnHostCores:
    """The fp64 CSR oracle timed on every host core: one spawned process per
    core runs the oracle's KPM recurrence on its own block of R random-phase
    vectors over a bounded sample of the workload (a 4-plane slab of the lattice,
    the same x/y extent, couplings and disorder).  The processes start together;
    the rate is all processes' lattice updates over the longest of their times."""

    def __init__(self, dims, R, Wd, cores=None):
        import multiprocessing as mp
        self.sdims = (dims[0], dims[1], min(4, dims[2]))
        self.R = R
        self.cores = cores or host_cores()
        ctx = mp.get_context("spawn")
        env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in env_keep:
            os.environ[k] = "1"   # one thread per worker process
        self.conns, self.procs = [], []
        try:
            for i in range(self.cores):
                a, b = ctx.Pipe()
                p = ctx.Process(target=_oracle_worker, args=(b, self.sdims, R, Wd, 3 + i), daemon=True)
                p.start()
                self.conns.append(a)
                self.procs.append(p)
        finally:
            for k, v in env_keep.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        for c in self.conns:
            assert c.recv() == "ready"

    def measure(self, seconds: float) -> dict:
        for c in self.conns:
            c.send(("run", seconds))
        res = [c.recv() for c in self.conns]
        steps = sum(r[0] for r in res)
        dt = max(r[1] for r in res)
        n = self.sdims[0] * self.sdims[1] * self.sdims[2]
        value = n * self.R * steps / dt / 1e9
        return {"value": round(value, 5), "unit": UNIT, "cores": self.cores, "kind": "oracle",
                "cpu_model": cpu_model(),
                "sample": f"fp64 CSR oracle KPM recurrence (scipy), one process per host core "
                          f"({self.cores}), each on its own block of R={self.R} random-phase vectors "
                          f"over a {self.sdims[0]}x{self.sdims[1]}x{self.sdims[2]} slab of the workload "
                          f"(same x/y extent, couplings, disorder): {steps} spMVM block steps in "
                          f"{dt:.1f} s; the per-LUP rate is extrapolated to the full slab"}

    def close(self):
        for c in self.conns:
            try:
                c.send(("stop",))
            except (OSError, BrokenPipeError):
                pass
        for p in self.procs:
            p.join(timeout=10)


def cpu_baseline(dims, R, Wd, budget_s=15.0):
    """The oracle on all host cores, on a bounded sample of the workload."""
    ob = OracleOnHostCores(dims, R, Wd)
    try:
        return ob.measure(budget_s)
    finally:
        ob.close()


def slab_config(args) -> dict:
    """The benchmark workload's description, identical in both arms."""
    return {"workload": "TI slab KPM: 256x256x64 sites (PBC x,y; open z), t=1, m=2, W=2, "
                        "R random-phase vectors, 2048 moments",
            "dims": list(args.dims), "R": args.R, "moments": args.M, "W": args.W,
            "sweeps_per_step": (args.M + 1) // 2,
            "l2": "vectors (1 GiB each) exceed L2; no flush"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    ob = OracleOnHostCores(args.dims, args.R, args.W)
    try:
        for _ in range(args.warmup):
            ob.measure(1.0)
        vals, t0 = [], time.perf_counter()
        for _ in range(args.steps):
            cb = ob.measure(3.0)
            vals.append(cb["value"])
        elapsed = time.perf_counter() - t0
    finally:
        ob.close()
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000 * elapsed / args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic",
            "config": slab_config(args),
            "cpu_baseline": {**cb, "value": value},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- other workloads
def _timed(fn, reps, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _hbm_roof(bytes_per_lup, lups, ms, kernel):
    peak, kind = measured_peaks()
    achieved = bytes_per_lup * lups / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": None, "kernel": kernel,
            "bytes_per_lup": bytes_per_lup, "peak_kind": f"{kind} hbm_gbs"}


TI_KERNEL_NAMES = {0: "ti_sweep (z-march)", 1: "ti_sweep_flat", 2: "ti_sweep (cp.async ring)",
                   3: "ti_sweep (deep cp.async ring)", 4: "ti_kpm2_sweep", 5: "ti_sweep (column tiles)",
                   6: "ti_sweep_xmarch", 7: "ti_sweep_tma (TMA-staged plane tiles)",
                   8: "ti_sweep_tma (TMA-staged tiles marching along x)"}


def ti_kernel_name(tuning: dict, what: str) -> str:
    """The TI sweep a tuning entry selects, for the roofline record."""
    k = int(tuning.get("kernel", 0)) if tuning else 0
    return f"{TI_KERNEL_NAMES.get(k, 'ti_sweep')} {what}"


def series_bytes_per_site(K: int, vb: float = 4.0) -> float:
    """Algorithmic HBM bytes per graphene site of one complex64 propagation time
    step with K series terms (R = 1, fp32 copy of V: vb = 4 bytes per sweep, 0 when
    the potential is regenerated in the sweep): the complex128 -> complex64
    conversion of w_0 (16 + 8), sweep 1 (x 8, w_1 8, psi 16, acc 16, V), sweeps
    j = 2 .. K-2 (x 8, y_in 8, y_out 8, V, and acc 16 + 16 on j = 4, 7, 10, ...,
    the sweeps that add three terms), and the last sweep (x 8, y_in 8, V, acc 16,
    psi 16)."""
    if K < 3:
        raise ValueError("K >= 3")
    total = 24.0 + 2 * (48.0 + vb)
    for j in range(2, K - 1):
        total += 24.0 + vb + (32.0 if j % 3 == 1 else 0.0)
    return total


def run_workload(args, pv, dev, rank, world):
    """The remaining workloads, one JSON line each (single GPU; rank 0 prints)."""
    import torch
    from paper_1708_09689_gb300.sharding import max_over_ranks
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(dev.index or 0)
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": world, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "data": "synthetic"}
    if args.workload == "ti_cube":
        cfg = W.CONFIG_TI_CUBE
        lat = pv.Lattice.ti(cfg.dims, cfg.periodic, t=cfg.t, m=cfg.m, disorder=(cfg.W, cfg.seed_V))
        emin, emax, a, b = lat.spectral_bounds()
        lat.autotune(1, pv.C128)
        v = torch.from_numpy(W.gaussian_block(cfg.D, 1, 1)).to(dev)
        y = torch.empty_like(v)
        work = pv.work_buffer(lat.work_bytes(pv.OP_KPM, 1, pv.C128, cfg.M), dev)
        mu = torch.empty((1, cfg.M), dtype=torch.float64, device=dev)

        def step():
            pv.apply_H(lat, v, y)
            pv.kpm_moments(lat, cfg.M, a, b, R=1, prec=pv.C128, seed=cfg.seed_r, work=work, mu=mu)
        for _ in range(args.warmup):
            step()
        clocks.start()
        ms = max_over_ranks(_timed(step, args.steps, stream), dev)
        clk = clocks.stop()
        lups = cfg.n_sites * (1 + cfg.M // 2)
        line.update({"workload": "ti_cube", "value": round(world * lups / (ms * 1e-3) / 1e9, 3),
                     "ms_per_step": round(ms, 4), "dtype": "c128",
                     "config": {"workload": "TI 16^3 periodic, W=1: one H.v + 256 KPM moments (R=1)",
                                "l2": "whole state L2-resident (< 1 MiB): a latency workload, no % roof"},
                     "roofline": None, "clocks": clk, "gpu_launches": args.steps * (2 + cfg.M // 2),
                     "mu_0": float(mu[0, 0].item())})
    elif args.workload == "graphene_qd":
        cfg = W.CONFIG_GRAPHENE_QD
        if args.qd_on_the_fly:  # Eq. qdotarray regenerated inside every sweep
            lat = pv.Lattice.graphene(cfg.cells, (0, 0), t=cfg.t,
                                      qdots=(cfg.ndots, cfg.R_dot, cfg.V0, cfg.w))
        else:
            lat = pv.Lattice.graphene(cfg.cells, (0, 0), t=cfg.t, V=cfg.potential())
        emin, emax, a, b = lat.spectral_bounds()
        nterms = len(pv.propagation_coeffs(a * cfg.dt, cfg.trunc))
        psi0 = torch.from_numpy(cfg.packet()).to(dev)
        nsteps = args.steps if args.steps > 5 else cfg.nsteps
        if args.sweeps_only:
            # profiling case: this many complex64 propagation time steps, untimed
            if args.launch:
                shape = {k: v for k, v in json.loads(args.launch).items() if k != "time_ms"}
                lat.set_tuning(1, pv.C64, **shape)
            else:
                lat.autotune(1, pv.C64)
            work = pv.work_buffer(lat.work_bytes(pv.OP_SERIES, 1, pv.C64, nterms), dev)
            psi = psi0.clone()
            pv.cheb_propagate(lat, psi, cfg.dt, args.sweeps_only, a, b, cfg.trunc, prec=pv.C64, work=work)
            torch.cuda.synchronize()
            if rank == 0:
                print(json.dumps({"time_steps": args.sweeps_only, "sweeps_per_time_step": nterms - 1,
                                  "launch": lat.get_tuning(1, pv.C64)}))
            return 0
        res = {}
        for prec, name in ((pv.C64, "c64"), (pv.C128, "c128")):
            lat.autotune(1, prec)
            work = pv.work_buffer(lat.work_bytes(pv.OP_SERIES, 1, prec, nterms), dev)
            psi = psi0.clone()
            pv.cheb_propagate(lat, psi, cfg.dt, 1, a, b, cfg.trunc, prec=prec, work=work)  # warm
            psi = psi0.clone()
            n = nsteps if prec == pv.C64 else max(nsteps // 5, 1)
            if prec == pv.C64:
                clocks.start()
            ms = _timed(lambda: pv.cheb_propagate(lat, psi, cfg.dt, n, a, b, cfg.trunc, prec=prec,
                                                  work=work), 1, stream)
            if prec == pv.C64:
                clk = clocks.stop()
            ms = max_over_ranks(ms, dev)
            res[name] = (psi, n, ms)
        psi64, n64, ms64 = res["c64"]
        psi128, n128, ms128 = res["c128"]
        lups = cfg.n_sites * (nterms - 1)
        v64 = lups * n64 / (ms64 * 1e-3) / 1e9
        v128 = lups * n128 / (ms128 * 1e-3) / 1e9
        # same number of steps in both precisions for the state error
        p64 = psi0.clone()
        pv.cheb_propagate(lat, p64, cfg.dt, n128, a, b, cfg.trunc, prec=pv.C64)
        line.update({"workload": "graphene_qd", "value": round(world * v64, 3),
                     "ms_per_step": round(ms64 / n64, 4), "steps": n64, "dtype": "c64",
                     "config": {"workload": "graphene 4096x2048 four-site cells (2^25 sites), open, 8x8 "
                                            "QD array V0=0.1 R=40 w=5, Gaussian packet, dt=1, trunc 1e-14",
                                "sweeps_per_time_step": nterms - 1,
                                "potential": "regenerated in the sweep" if args.qd_on_the_fly
                                             else "stored (fp32 copy read by the sweep)"},
                     "roofline": _hbm_roof(round(series_bytes_per_site(nterms, 0.0 if args.qd_on_the_fly
                                                                        else 4.0) / (nterms - 1), 3), lups,
                                           ms64 / n64,
                                           "gr_sweep<float,1,*> (complex64 w, complex128 accumulator "
                                           "touched on every third sweep), time-step average"),
                     "compare_fp64": {"c128_glups": round(v128, 3), "c64_over_c128": round(v64 / v128, 2),
                                      "c128_steps": n128,
                                      "norm_drift_c64": abs(torch.linalg.vector_norm(psi64).item() - 1),
                                      "norm_drift_c128": abs(torch.linalg.vector_norm(psi128).item() - 1),
                                      "c64_vs_c128_state_err": torch.linalg.vector_norm(p64 - psi128).item()},
                     "clocks": clk, "gpu_launches": (nterms) * n64})
    elif args.workload == "ti_akE":
        # A(k, E) along k_x of a clean TI cuboid (the dispersion figure's 512 x 64 x 8 sites,
        # periodic): 64 k-points, 16 per KPM call (R = 64: four Bloch states each), complex64
        dims, M, nk_call, NE = (512, 64, 8), 1024, 16, 1024
        lat = pv.Lattice.ti(dims, (1, 1, 1), t=1.0, m=2.0)
        emin, emax, a, b = lat.spectral_bounds()
        R = 4 * nk_call
        if args.sweeps_only:  # profiling case: one KPM call of this many sweeps on 16 k-points, untimed
            if args.launch:
                lat.set_tuning(R, pv.C64, **{k: v for k, v in json.loads(args.launch).items() if k != "time_ms"})
            psi = pv.bloch_vectors(lat, [(2 * math.pi * (j - 8) / 64, 0.0, 0.0) for j in range(nk_call)], pv.C64)
            mu = pv.kpm_moments(lat, 2 * args.sweeps_only, a, b, r0=psi)
            torch.cuda.synchronize()
            if rank == 0:
                print(json.dumps({"sweeps": args.sweeps_only, "mu_0": float(mu[0, 0].item())}))
            return 0
        if not args.no_autotune:
            lat.autotune(R, pv.C64)
        kx = [2 * math.pi * (j - 32) / 64 for j in range(64)]
        calls = [[(k, 0.0, 0.0) for k in kx[c * nk_call:(c + 1) * nk_call]] for c in range(64 // nk_call)]
        E = torch.linspace(b - a * 0.999, b + a * 0.999, NE, dtype=torch.float64, device=dev)
        A = torch.empty((64, NE), dtype=torch.float64, device=dev)
        psis = [pv.bloch_vectors(lat, ks, pv.C64) for ks in calls]
        # the KPM calls are independent: each on its own stream with its own work
        # buffer and moments, so that their sweeps overlap one another's tails
        works = [pv.work_buffer(lat.work_bytes(pv.OP_KPM, R, pv.C64, M), dev) for _ in calls]
        mus = [torch.empty((R, M), dtype=torch.float64, device=dev) for _ in calls]
        side = [torch.cuda.Stream(device=dev) for _ in calls]
        mu = mus[0]

        def step():
            main = torch.cuda.current_stream(dev)
            for c, psi in enumerate(psis):
                side[c].wait_stream(main)
                with torch.cuda.stream(side[c]):
                    pv.kpm_moments(lat, M, a, b, r0=psi, work=works[c], mu=mus[c])
                    for q in range(nk_call):
                        pv.kpm_density(mus[c][4 * q:4 * q + 4], E, a, b, out=A[c * nk_call + q])
            for sc in side:
                main.wait_stream(sc)
        for _ in range(args.warmup):
            step()
        clocks.start()
        ms = max_over_ranks(_timed(step, args.steps, stream), dev)
        clk = clocks.stop()
        # density alone (all 64 k-points), for the record
        t_d = _timed(lambda: [pv.kpm_density(mu[4 * q:4 * q + 4], E, a, b, out=A[q]) for q in range(64 // 4)],
                     3, stream)
        lups = lat.n_sites * R * ((M + 1) // 2) * len(calls)
        Ah = A.cpu().numpy()
        En = E.cpu().numpy()
        # upper-band peak at k = 0, where the closed form gives E = |m - 3t| = 1
        peak = lambda q, lo, hi: float(En[(En > lo) & (En < hi)][np.argmax(Ah[q][(En > lo) & (En < hi)])])
        line.update({"workload": "ti_akE", "value": round(world * lups / (ms * 1e-3) / 1e9, 3),
                     "ms_per_step": round(ms, 3), "steps": args.steps, "dtype": "c64",
                     "config": {"workload": "A(k,E) of a clean TI, 512x64x8 sites periodic, m=2, t=1: "
                                            "64 k-points along k_x, 4 Bloch states each, 1024 moments, "
                                            "Jackson kernel, 1024 energies",
                                "kpm_calls_per_step": len(calls), "R_per_call": R,
                                "kpm_calls_concurrent": len(calls),
                                "launch": lat.get_tuning(R, pv.C64)},
                     "density_ms_64k": round(t_d, 4),
                     "peak_at_k0": peak(32, 0.5, 1.5), "closed_form_k0": 1.0,
                     "roofline": _hbm_roof(96.0, lups, ms, ti_kernel_name(lat.get_tuning(R, pv.C64),
                                                                         "KPM sweeps (R = 64, V = 0)")),
                     "clocks": clk, "gpu_launches": args.steps * len(calls) * ((M + 1) // 2 + 1 + nk_call)})
    elif args.workload == "chebfd":
        # interior eigenpairs of a disordered TI slab, the filter-diagonalization test case of
        # 240 x 240 x 6 sites, 40 states around E = 0 (window from the KPM DOS), complex64 filter
        dims = (240, 240, 6)
        lat = pv.Lattice.ti(dims, (1, 1, 0), t=1.0, m=2.0, disorder=(1.0, 5))
        emin, emax, a, b = lat.spectral_bounds()
        if args.sweeps_only:  # profiling case: one complex64 filter of this many series terms, untimed
            Rf = args.R
            if args.launch:
                lat.set_tuning(Rf, pv.C64, **{k: v for k, v in json.loads(args.launch).items() if k != "time_ms"})
            x = pv.random_vectors(lat, Rf, pv.C128, 3)
            y = pv.cheb_filter(lat, x, [1.0 / (k + 1) for k in range(args.sweeps_only)], a, b, prec=pv.C64)
            torch.cuda.synchronize()
            if rank == 0:
                print(json.dumps({"series_terms": args.sweeps_only, "R": Rf, "y_max": float(y.abs().max().item())}))
            return 0
        t0 = time.perf_counter()
        mu = pv.kpm_moments(lat, 8192, a, b, R=32, prec=pv.C64, seed=9)
        Eg = np.linspace(-0.5, 0.5, 20001)
        cum = np.cumsum(pv.dos(lat, mu, Eg, a, b).cpu().numpy()) * (Eg[1] - Eg[0])
        lam = next(l for l in np.linspace(0.001, 0.5, 5000)
                   if np.interp(l, Eg, cum) - np.interp(-l, Eg, cum) >= 40)
        torch.cuda.synchronize()
        t_dos = time.perf_counter() - t0
        deg, ns = 4000, 64
        # the filter runs series sweeps (accumulating + plain): tune the launch shape on those
        if not args.no_autotune:
            lat.autotune(ns, pv.C64, op=pv.OP_SERIES)
        clocks.start()
        t0 = time.perf_counter()
        theta, res, X, n_in, iters = pv.chebfd(lat, -lam, lam, a, b, n_search=ns, degree=deg, max_iter=30,
                                               tol=1e-6, prec=pv.C64)
        torch.cuda.synchronize()
        secs = max_over_ranks(time.perf_counter() - t0, dev)
        clk = clocks.stop()
        inside = (theta >= -lam) & (theta <= lam)
        lups = lat.n_sites * ns * deg * iters  # filter sweeps dominate
        line.update({"workload": "chebfd", "value": round(world * lups / secs / 1e9, 3),
                     "ms_per_step": round(1000 * secs, 1), "steps": 1, "dtype": "c64 filter, c128 Ritz",
                     "config": {"workload": "ChebFD: TI slab 240x240x6 (PBC x,y; open z), m=2, W=1, eigenpairs "
                                            "in [-lambda, lambda] holding ~40 states (lambda from the KPM DOS), "
                                            "64 search vectors, degree 4000, tol 1e-6",
                                "lambda": lam, "dos_seconds": round(t_dos, 3),
                                "launch": lat.get_tuning(ns, pv.C64)},
                     "iterations": iters, "eigenpairs_found": int(n_in),
                     "max_residual": float(res[inside].max()) if n_in else None,
                     "kramers_pairs": bool(n_in % 2 == 0),
                     "roofline": _hbm_roof(96.0 + 8.0 / ns + 128.0 / 3, lups, 1000 * secs,
                                           ti_kernel_name(lat.get_tuning(ns, pv.C64),
                                                          "series sweeps (R = 64; accumulator on every "
                                                          "third sweep), solver average")),
                     "clocks": clk, "gpu_launches": None})
    elif args.workload == "wsm_kpm":
        # KPM DOS of the Weyl semimetal on the dispersion figure's 256 x 32 x 32 cuboid (periodic
        # x, y; open z), box disorder W = 1, 16 random-phase vectors, 2048 moments, complex64
        dims, R, M = (256, 32, 32), 16, 2048
        lat = pv.Lattice.wsm(dims, (1, 1, 0), disorder=(1.0, 11))
        emin, emax, a, b = lat.spectral_bounds()
        if args.sweeps_only:  # profiling case: one KPM call of this many sweeps, untimed
            if args.launch:
                lat.set_tuning(R, pv.C64, **{k: v for k, v in json.loads(args.launch).items() if k != "time_ms"})
            r0 = pv.random_vectors(lat, R, pv.C64, 13)
            mu = pv.kpm_moments(lat, 2 * args.sweeps_only, a, b, r0=r0)
            torch.cuda.synchronize()
            if rank == 0:
                print(json.dumps({"sweeps": args.sweeps_only, "mu_0": float(mu[0, 0].item())}))
            return 0
        if not args.no_autotune:
            lat.autotune(R, pv.C64)
        r0 = pv.random_vectors(lat, R, pv.C64, 13)
        work = pv.work_buffer(lat.work_bytes(pv.OP_KPM, R, pv.C64, M), dev)
        mu = torch.empty((R, M), dtype=torch.float64, device=dev)
        run = lambda: pv.kpm_moments(lat, M, a, b, r0=r0, work=work, mu=mu)
        for _ in range(args.warmup):
            run()
        clocks.start()
        ms = max_over_ranks(_timed(run, args.steps, stream), dev)
        clk = clocks.stop()
        lups = lat.n_sites * R * (M // 2)
        E0 = torch.tensor([0.0], dtype=torch.float64, device=dev)
        line.update({"workload": "wsm_kpm", "value": round(world * lups / (ms * 1e-3) / 1e9, 3),
                     "ms_per_step": round(ms, 3), "steps": args.steps, "dtype": "c64",
                     "config": {"workload": "Weyl semimetal KPM: 256x32x32 sites (PBC x,y; open z), k0=pi/2, "
                                            "W=1, 16 random-phase vectors, 2048 moments", "launch": lat.get_tuning(R, pv.C64)},
                     "dos_at_E0_per_site": float(pv.dos(lat, mu, E0, a, b)[0].item()) / lat.n_sites,
                     "roofline": _hbm_roof(48.0 + 4.0 / R, lups, ms,
                                           {7: "ti_sweep_tma<*,*,8,F_DOTS,3> (TMA-staged Weyl cells)",
                                            0: "wsm_march_sweep<float,2,F_DOTS> (z-marching cells)"}.get(
                                               int(lat.get_tuning(R, pv.C64).get("kernel", 1)),
                                               "wsm_sweep<float,2,F_DOTS> (flat two-site cells)")),
                     "clocks": clk, "gpu_launches": args.steps * (M // 2)})
    elif args.workload == "batched":
        specs = W.batched_lattices()
        if args.sweeps_only:  # profiling case: the first --batched-count lattices, untimed
            specs = specs[:args.batched_count]
        lats = [pv.Lattice.ti((L, L, L), (1, 1, 1), disorder=(Wd, s)) for L, Wd, s in specs]
        ab = [lat.spectral_bounds()[2:] for lat in lats]
        R, M = 16, 1024
        if args.sweeps_only:
            M = 2 * args.sweeps_only
            work = pv.work_buffer(pv.batched_work_bytes(lats, R, pv.C64, M), dev)
            mu = pv.kpm_moments_batched(lats, M, [x[0] for x in ab], [x[1] for x in ab], R=R,
                                        prec=pv.C64, seeds=[vector_seed_for(i, rank) for i in range(len(lats))],
                                        work=work)
            torch.cuda.synchronize()
            if rank == 0:
                print(json.dumps({"lattices": [L for L, _, _ in specs], "R": R, "moments": M,
                                  "mu0_min": float(mu[:, :, 0].min().item())}))
            return 0
        seeds = [vector_seed_for(i, rank) for i in range(len(lats))]
        tuning = None
        if not args.no_autotune:  # the launch shape timed on the batch itself, 32 moments
            tuning = pv.autotune_batched(lats, 32, [x[0] for x in ab], [x[1] for x in ab], R=R, prec=pv.C64,
                                         seeds=seeds)
        work = pv.work_buffer(pv.batched_work_bytes(lats, R, pv.C64, M), dev)
        mu = torch.empty((len(lats), R, M), dtype=torch.float64, device=dev)
        run = lambda: pv.kpm_moments_batched(lats, M, [x[0] for x in ab], [x[1] for x in ab], R=R,
                                             prec=pv.C64, seeds=seeds, work=work, mu=mu)
        for _ in range(args.warmup):
            run()
        clocks.start()
        ms = max_over_ranks(_timed(run, args.steps, stream), dev)
        clk = clocks.stop()
        sites = sum(L ** 3 for L, _, _ in specs)
        lups = sites * R * (M // 2)
        per_lattice = bool(tuning) and int(tuning.get("kernel", 0)) == 7
        persistent = None
        if per_lattice:
            # the batch as the one persistent cooperative launch too (its measured best shape:
            # 256 threads, one block per SM, whole columns), for the record
            lats[0].set_tuning(R, pv.C64, threads=256, blocks_per_sm=1, zslab=0, kernel=0)
            work_p = pv.work_buffer(pv.batched_work_bytes(lats, R, pv.C64, M), dev)
            run_p = lambda: pv.kpm_moments_batched(lats, M, [x[0] for x in ab], [x[1] for x in ab], R=R,
                                                   prec=pv.C64, seeds=seeds, work=work_p, mu=mu)
            for _ in range(args.warmup):
                run_p()
            ms_p = max_over_ranks(_timed(run_p, args.steps, stream), dev)
            roof_p = _hbm_roof(96.0 + 8.0 / R, lups, ms_p, "kpm_batched_kernel<float,2>")
            persistent = {"value": round(world * lups / (ms_p * 1e-3) / 1e9, 3), "ms_per_step": round(ms_p, 3),
                          "frac": roof_p["frac"], "launch": lats[0].get_tuning(R, pv.C64)}
            lats[0].set_tuning(R, pv.C64, **{k: v for k, v in tuning.items() if k != "time_ms"})
            del work_p
        mode = ("every lattice's KPM as a chain of TMA-staged sweeps, the chains on 4 forked streams "
                "in one CUDA graph" if per_lattice else "one persistent cooperative launch in a CUDA graph")
        line.update({"workload": "batched", "value": round(world * lups / (ms * 1e-3) / 1e9, 3),
                     "ms_per_step": round(ms, 3), "steps": args.steps, "dtype": "c64",
                     "config": {"workload": "64 periodic TI cubes, L from {24,32,48,64,96}, W~U[0,5), R=16, "
                                            "1024 moments, " + mode,
                                "sites": sites, "mu0_min": float(mu[:, :, 0].min().item()), "launch": tuning},
                     "roofline": _hbm_roof(96.0 + 8.0 / R, lups, ms,
                                           "ti_sweep_tma<16,F_DOTS> (per-lattice chains)" if per_lattice
                                           else "kpm_batched_kernel<float,2>"),
                     "clocks": clk, "persistent_launch": persistent,
                     "gpu_launches": args.steps * (len(specs) * (2 + M // 2) if per_lattice else 1)})
    elif args.workload == "adjoint":
        cfg = W.CONFIG_GRAPHENE_ADJ
        V = cfg.potential()
        lat = pv.Lattice.graphene(cfg.cells, (0, 0), V=V)
        emin, emax, a, b = lat.spectral_bounds()
        lat.autotune(1, pv.C128)
        psi0 = torch.from_numpy(cfg.packet()).to(dev)
        mask = torch.from_numpy(cfg.detector()).to(dev)
        Vt = torch.tensor(V, dtype=torch.float64, device=dev, requires_grad=True)

        def fwd_bwd():
            Vt.grad = None
            psi = pv.propagate_with_grad(Vt, psi0, lat, cfg.dt, cfg.nsteps, a, b,
                                         every=W.ADJ_CHECKPOINT_EVERY)
            loss = (psi.abs() ** 2 * mask).sum()
            loss.backward()
            return loss
        loss = fwd_bwd()
        clocks.start()
        t0 = time.perf_counter()
        loss = fwd_bwd()
        torch.cuda.synchronize()
        secs = max_over_ranks(time.perf_counter() - t0, dev)
        clk = clocks.stop()
        g = Vt.grad.cpu().numpy()
        # central differences at 32 seeded sites, h = 1e-6
        rng = np.random.default_rng(W.ADJ_FD_SEED)
        sites = rng.choice(len(V), W.ADJ_FD_SITES, replace=False)
        work = pv.work_buffer(lat.work_bytes(pv.OP_SERIES, 1, pv.C128, 32), dev)

        def L(Vv):
            lat.set_potential(torch.from_numpy(Vv).to(dev))
            p = psi0.clone()
            pv.cheb_propagate(lat, p, cfg.dt, cfg.nsteps, a, b, prec=pv.C128, work=work)
            return float((p.abs() ** 2 * mask).sum().item())
        errs = []
        for s in sites:
            Vp, Vm = V.copy(), V.copy()
            Vp[s] += W.ADJ_FD_H
            Vm[s] -= W.ADJ_FD_H
            fd = (L(Vp) - L(Vm)) / (2 * W.ADJ_FD_H)
            errs.append(abs(fd - g[s]) / max(abs(g).max(), 1e-300))
        nterms = len(pv.propagation_coeffs(a * cfg.dt, cfg.trunc))
        lups = cfg.n_sites * (nterms - 1) * cfg.nsteps * 4  # forward, recompute, reverse (~2 sweeps)
        line.update({"workload": "adjoint", "value": round(lups / secs / 1e9, 3),
                     "ms_per_step": round(1000 * secs, 1), "dtype": "c128",
                     "config": {"workload": "graphene 1024x512 cells (2^21 sites), 4x4 QD R=30 V0=0.1, 200 steps, "
                                            "checkpoints every 20, loss = detector probability"},
                     "loss": float(loss.item()), "fd_sites": len(sites),
                     "fd_max_err_rel_to_max_grad": float(max(errs)),
                     "seconds_fwd_bwd": round(secs, 3), "roofline": None, "clocks": clk})
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def vector_seed_for(unit, rank):
    from paper_1708_09689_gb300.sharding import vector_seed
    return vector_seed(100 + 1000 * rank, unit)


# --------------------------------------------------------------------------- native
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    rank, world, local = dist_env()
    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1708_09689_gb300 as pv
    from paper_1708_09689_gb300.sharding import max_over_ranks, vector_seed

    if args.workload != "ti_slab":
        return run_workload(args, pv, dev, rank, world)

    dims, R, M, Wd = tuple(args.dims), args.R, args.M, args.W
    n_sites = dims[0] * dims[1] * dims[2]
    D = 4 * n_sites
    lat = pv.Lattice.ti(dims, (1, 1, 0), t=1.0, m=2.0, disorder=(Wd, 2))
    emin, emax, a, b = lat.spectral_bounds(0.01)
    seed = vector_seed(3, rank)  # each rank owns its own block of random vectors
    sweeps = (M + 1) // 2
    lups_per_step = n_sites * R * sweeps

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident run (headline)
    stream = torch.cuda.current_stream()
    # launch shape: autotuned once, outside the timed region (or given)
    if args.launch:
        shape = {k: v for k, v in json.loads(args.launch).items() if k != "time_ms"}
        lat.set_tuning(R, pv.C64, **shape)
        tuning = lat.get_tuning(R, pv.C64)
    else:
        tuning = None if args.no_autotune else lat.autotune(R, pv.C64)
    if args.q64_launch:
        lat.set_tuning(R, pv.Q64, **{k: v for k, v in json.loads(args.q64_launch).items() if k != "time_ms"})
    if args.sweeps_only:
        # one KPM call of this many sweeps (2 x sweeps moments) in the benchmark's kernel,
        # or in the fixed-point kernel with --q64
        prec = pv.Q64 if args.q64 else pv.C64
        r0 = pv.random_vectors(lat, R, pv.C128 if args.q64 else pv.C64, seed)
        Ms = 2 * args.sweeps_only
        w = pv.work_buffer(lat.work_bytes(pv.OP_KPM, R, prec, Ms), dev)
        mu = pv.kpm_moments(lat, Ms, a, b, r0=r0, prec=prec, work=w)
        torch.cuda.synchronize()
        print(json.dumps({"sweeps": args.sweeps_only, "dims": list(dims), "R": R, "q64": args.q64,
                          "launch": tuning, "mu_0": float(mu[0, 0].item())}))
        return 0
    # start block: random-phase vectors from the counter hash, generated on the device
    r0 = pv.random_vectors(lat, R, pv.C64, seed)
    work = pv.work_buffer(lat.work_bytes(pv.OP_KPM, R, pv.C64, M), dev)
    mu = torch.empty((R, M), dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        pv.kpm_moments(lat, M, a, b, r0=r0, work=work, mu=mu)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        pv.kpm_moments(lat, M, a, b, r0=r0, work=work, mu=mu)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    ms = max_over_ranks(ms, dev)
    value = world * lups_per_step / (ms * 1e-3) / 1e9
    mu64 = mu.clone()

    # ---- roofline of the dominant kernel (the complex64 TI KPM sweep)
    two_step = bool(tuning) and tuning.get("kernel") == 4
    if two_step:
        # two recurrence steps per launch: w_{k-1}, w_k read and w_{k+1}, w_{k+2} written
        # once (4 x 32 B per site and vector over two steps), the fp32 potential once
        bytes_per_lup = 64.0 + 2.0 / R
        launches = 1 + (sweeps - 1) // 2 + (sweeps - 1) % 2
        kname = "ti_kpm2_sweep (complex64, two KPM steps per sweep)"
    elif bool(tuning) and tuning.get("kernel") == 7:
        bytes_per_lup = 96.0 + 4.0 / R
        launches = sweeps
        kname = f"ti_sweep_tma<{R},F_DOTS> (complex64 KPM sweep, TMA-staged plane tiles)"
    elif bool(tuning) and tuning.get("kernel") == 8:
        bytes_per_lup = 96.0 + 4.0 / R
        launches = sweeps
        kname = f"ti_sweep_tma_xm<{R},F_DOTS> (complex64 KPM sweep, TMA-staged tiles marching along x)"
    elif bool(tuning) and tuning.get("kernel") == 6:
        bytes_per_lup = 96.0 + 4.0 / R
        launches = sweeps
        kname = f"ti_sweep_xmarch<float,{tuning.get('vpt') or 2},F_DOTS> (complex64 KPM sweep marching along x)"
    else:
        bytes_per_lup = 96.0 + 4.0 / R      # x 32 + y_in 32 + y_out 32 (B), fp32 V 4 per site
        launches = sweeps
        kname = "ti_sweep<float,2,F_DOTS> (complex64 KPM sweep)"
    launch_ms = ms / launches                # upper bound: includes launch gaps of the graph
    achieved = bytes_per_lup * lups_per_step / (ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None, "kernel": kname,
                "bytes_per_lup": bytes_per_lup, "peak_kind": f"{peak_kind} hbm_gbs",
                "launch_ms": round(launch_ms, 4)}
    kkey = kname.split("<")[0]
    tr = TRAFFIC.get(("ti_slab", R, kkey)) if tuple(dims) == tuple(W.CONFIG_TI_SLAB.dims) else None
    if tr and not two_step and tr["source_sha256_16"] == kernel_source_hash():
        roofline["traffic"] = tr["bytes_per_launch"]
        roofline["traffic_over_algorithmic"] = round(tr["bytes_per_launch"] / (bytes_per_lup * n_sites * R), 3)

    # ---- complex128 / fp64 comparison (same lattice, same start block, fewer moments)
    compare = None
    if not args.no_compare:
        Mc = min(args.fp64_moments or M, M)
        if not args.no_autotune:
            lat.autotune(R, pv.C128)
        r0d = r0.to(torch.complex128)
        w128 = pv.work_buffer(lat.work_bytes(pv.OP_KPM, R, pv.C128, Mc), dev)
        mu128 = torch.empty((R, Mc), dtype=torch.float64, device=dev)
        pv.kpm_moments(lat, Mc, a, b, r0=r0d, work=w128, mu=mu128)
        barrier()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        pv.kpm_moments(lat, Mc, a, b, r0=r0d, work=w128, mu=mu128)
        c1.record(stream)
        barrier()
        ms128 = c0.elapsed_time(c1)
        v128 = n_sites * R * ((Mc + 1) // 2) / (ms128 * 1e-3) / 1e9
        # complex64 moment error against complex128 on the same start block, per moment
        # (max over the R vectors, relative to mu_0), reported in bands of 128 moments
        dmu = ((mu64[:, :Mc] - mu128).abs() / mu128[:, :1].abs()).amax(dim=0).cpu().numpy()
        band = 128
        compare = {"c128_glups": round(v128, 3), "c64_over_c128": round(value / world / v128, 2),
                   "c128_moments": Mc, "c64_vs_c128_max_dmu": float(dmu.max()),
                   "c64_vs_c128_argmax_moment": int(dmu.argmax()),
                   "c64_vs_c128_dmu_by_band": {f"{lo}-{min(lo + band, Mc) - 1}": float(dmu[lo:lo + band].max())
                                               for lo in range(0, Mc, band)},
                   "c128_bound": "fp64 pipe (0.50 T instr/s measured on GB300)"}
        del w128
        # fixed-point vectors of the same size (exact integer stencil): same start block
        wq = pv.work_buffer(lat.work_bytes(pv.OP_KPM, R, pv.Q64, Mc), dev)
        muq = torch.empty((R, Mc), dtype=torch.float64, device=dev)
        pv.kpm_moments(lat, Mc, a, b, r0=r0d, prec=pv.Q64, work=wq, mu=muq)
        barrier()
        c0.record(stream)
        pv.kpm_moments(lat, Mc, a, b, r0=r0d, prec=pv.Q64, work=wq, mu=muq)
        c1.record(stream)
        barrier()
        msq = c0.elapsed_time(c1)
        vq = n_sites * R * ((Mc + 1) // 2) / (msq * 1e-3) / 1e9
        bq = 192.0 + 16.0 / R  # x, y_in, y_out 64 B each; per-site (d+, d-) 16 B
        compare.update({"q64_glups": round(vq, 3), "q64_over_c128": round(vq / v128, 2),
                        "q64_vs_c128_max_dmu": float(((muq - mu128).abs() / mu128[:, :1].abs()).max().item()),
                        "q64_bytes_per_lup": bq,
                        "q64_hbm_frac": round(bq * vq / peak, 4),
                        "q64_launch": lat.get_tuning(R, pv.Q64) if args.q64_launch else "default",
                        "q64_note": "complex128-sized Q4.59 fixed-point vectors, exact integer stencil; "
                                    "call time includes the per-call Gershgorin check and conversion"})
        del wq

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        r0_host = r0.cpu().pin_memory()
        mu_host = torch.empty((R, M), dtype=torch.float64).pin_memory()
        # two device copies of the start block: step i+1's host-to-device copy runs on a
        # second stream while step i sweeps (each copy waits until the step that read
        # its buffer is done); every step's copy and its moments' read-back stay inside
        # the timed region
        r0_dev = [torch.empty_like(r0), torch.empty_like(r0)]
        copy_stream = torch.cuda.Stream()
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        used = [torch.cuda.Event(), torch.cuda.Event()]

        def e2e_steps(n):
            with torch.cuda.stream(copy_stream):
                r0_dev[0].copy_(r0_host, non_blocking=True)
                copied[0].record(copy_stream)
            for i in range(n):
                cur, nxt = i % 2, 1 - i % 2
                if i + 1 < n:
                    with torch.cuda.stream(copy_stream):
                        if i >= 1:
                            copy_stream.wait_event(used[nxt])
                        r0_dev[nxt].copy_(r0_host, non_blocking=True)
                        copied[nxt].record(copy_stream)
                stream.wait_event(copied[cur])
                pv.kpm_moments(lat, M, a, b, r0=r0_dev[cur], work=work, mu=mu)
                used[cur].record(stream)
                mu_host.copy_(mu, non_blocking=True)
            torch.cuda.synchronize()
        e2e_steps(max(args.warmup, 2))  # untimed: each start-block buffer captures its graph once
        barrier()
        t0 = time.perf_counter()
        e2e_steps(args.steps)
        barrier()
        te = max_over_ranks((time.perf_counter() - t0) / args.steps, dev)
        e2e = {"value": round(world * lups_per_step / te / 1e9, 3), "unit": UNIT,
               "h2d_bytes_per_step": r0.numel() * 8, "d2h_bytes_per_step": R * M * 8,
               "overlap": "each step's start block copied from pinned host memory on a second stream "
                          "during the previous step's sweeps (two device buffers)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(dims, R, Wd)

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64",
                "data": "synthetic",
                "config": {**slab_config(args), "launch": tuning},
                "roofline": roofline, "compare_fp64": compare, "e2e": e2e,
                "gpu_launches": launches * args.steps, "clocks": clk, "cpu_baseline": cpu,
                "spectral": {"emin": emin, "emax": emax, "a": a, "b": b}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
