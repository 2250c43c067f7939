#!/usr/bin/env python
"""Throughput of the particle stochastic-Galerkin time step (arXiv:2404.19602) on GB300.

A bench "step" advances the whole ensemble by --time-steps time steps (default 500 of 1 fs);
K = 10 timed steps are one full run of the workload (5000 time steps) from the Fermi-Dirac
state.  Metric: particle-gPC-steps/s = particles x time steps / device time.  The default
workload is the largest single-GPU one: 4e6 particles, band gap and field random, total degree
5 (21 coefficients) on 6 x 6 nodes, FP32 state (its 672 MB state exceeds L2; L2 is also flushed
by a 256 MiB write between timed steps).  The line also carries the error of the moments against
the FP64 oracle on a reduced ensemble of the same workload (key "parity"), measured outside the
timed region on the same oracle run that gives the CPU baseline.

  python bench.py [--gpus N --steps K --warmup W] [--workload gap_field|gap_uq|det|...]
  python bench.py --impl reference      # the FP64 CPU oracle on a bounded sample

Under torchrun (N > 1) each rank advances its own independent ensemble (stream_id = rank):
the particle ensembles of a batch of cases need no exchange (weak scaling), and the timing is
the maximum over ranks.  One JSON line is printed by rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2404_19602_gb300 import workloads as W  # noqa: E402

WORKLOADS = {"gap_uq": W.GAP_UQ_1E6, "det": W.DET_FP64_1E4, "gap_field": W.GAP_FIELD_UQ_4E6, "sweep": None,
             "adjoint": W.ADJOINT_1E6,
             "gap_uq_fp64": W.scaled(W.GAP_UQ_1E6, precision="fp64", name="gapU[0.1,0.3]eV_M5_Q6_N1e6_fp64"),
             "sg_error": W.TEST3_WIDTH_1E4, "mc_compare": W.TEST3_WIDTH_1E4,
             "gap_uq_strang": W.scaled(W.GAP_UQ_1E6, splitting=1, name="gapU[0.1,0.3]eV_M5_Q6_N1e6_fp32_strang"),
             "gap_field_tc": W.scaled(W.GAP_FIELD_UQ_4E6, tc_proj=1,
                                      name="gapU[0.1,0.3]eV_fieldU[1,10]kVcm_M5_Q36_N4e6_fp32_tcgen05_f16x3")}
METRIC = "particle-gPC-steps/s"
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pgc", choices=["pgc", "reference"])
    ap.add_argument("--workload", default="gap_field", choices=sorted(WORKLOADS),
                    help="gap_field (default: 4e6 particles, 2 random inputs, 21 x 36), gap_uq (1e6 particles, "
                         "1 random input), det (1e4, FP64), sweep (64 cases in one batched CUDA-graph sequence), adjoint (forward + "
                         "reverse sweep of the steady-current sensitivities, 1e6 particles), gap_uq_fp64 "
                         "(the gap_uq ensemble in the FP64 mode), sg_error (the stochastic-Galerkin error "
                         "study of Test 3: degrees 0..25 against 30, two scenarios, 1e4 particles), mc_compare "
                         "(Test 4: MC-sG against Algorithm 1 at sampled inputs, 5e4 particles, reference 5e6 "
                         "particles at degree 30), gap_uq_strang (the gap_uq ensemble with the Strang splitting), "
                         "gap_field_tc (the gap_field ensemble with the reconstruction of the streaming kernel on "
                         "the tensor cores, FP16 hi/lo split)")
    ap.add_argument("--fd-check", action="store_true",
                    help="adjoint workload: also central differences (h = 1e-3 relative, common random numbers)")
    ap.add_argument("--time-steps", type=int, default=500, help="time steps per bench step")
    ap.add_argument("--moments-every", type=int, default=10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + SMI_FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for name, v in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"], f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
            os.unlink(self.path)
        except Exception:
            return None
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _src_sha():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2404_19602_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def _traffic(kernel: str, workload: str, key: str = "dram_bytes_per_launch"):
    """A per-launch figure of `kernel` (DRAM bytes, or warp instructions with key
    "warp_inst_per_launch") from the committed ncu summary, if it was taken on the current kernel
    sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
        e = d[workload][kernel]
        if e.get("src_sha") != _src_sha():
            return None
        return e[key]
    except Exception:
        return None


def max_over_ranks(x: float, device) -> float:
    """Maximum of a per-rank number over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_workload(p: dict, rank: int) -> dict:
    """The ensemble a rank advances: the same workload on its own Philox stream."""
    return W.scaled(p, stream_id=p.get("stream_id", 0) + rank)


def throughput(n_particles: int, world: int, time_steps: int, steps: int, ms: float) -> float:
    """Whole-job particle-steps/s: every rank advances n_particles for time_steps x steps."""
    return n_particles * world * time_steps * steps / (ms / 1e3)


def cpu_sample(p):
    """(particles, time steps) of the bounded oracle sample of a workload: ~2-5 s on 16 cores."""
    if p["eps0_lo"] == p["eps0_hi"] and p["Ex_lo"] == p["Ex_hi"]:
        return 10000, 400
    if p["Q1"] <= 6 and (p["eps0_lo"] == p["eps0_hi"] or p["Ex_lo"] == p["Ex_hi"]):
        return 20000, 300
    return 2000, 500


def cpu_baseline(p, every):
    """The oracle as it stands, on the host cores, on a bounded sample of the workload.  Returns
    the baseline record and the oracle's moment series of that sample (for the parity key)."""
    import oracle as O

    O.build()
    n, steps = cpu_sample(p)
    q = W.scaled(p, N=n)
    o = O.Oracle(q)
    t0 = time.perf_counter()
    o.step(steps, every)
    dt = time.perf_counter() - t0
    moments = o.moments()
    cores = O.num_threads()
    # the same oracle on one core, on a tenth of the sample
    n1, s1 = max(n // 10, 200), max(steps // 3, 10)
    O.set_threads(1)
    try:
        o1 = O.Oracle(W.scaled(p, N=n1))
        t1 = time.perf_counter()
        o1.step(s1, every)
        dt1 = time.perf_counter() - t1
    finally:
        O.set_threads(0)
    return {"value": n * steps / dt, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": "%d particles x %d time steps of the same workload (FP64, OpenMP)" % (n, steps),
            "seconds": round(dt, 3),
            "single_core": {"value": n1 * s1 / dt1, "sample": "%d particles x %d time steps, 1 thread" % (n1, s1),
                            "seconds": round(dt1, 3)}}, (q, steps, moments)


def _moment_errors(g, r, n):
    """Normwise relative errors |a(t) - b(t)| / max_t |b| over the first n output times of the
    z-mean and z-variance of J_x, V_x and the energy."""
    import numpy as np

    out = {}
    for name, comp in (("Jx", 3), ("Vx", 0), ("energy", 2)):
        for kind in ("mean", "var"):
            a, b = g[kind][:n, comp], r[kind][:n, comp]
            scale = float(np.abs(b).max())
            out["%s_%s" % (kind, name)] = float(np.abs(a - b).max() / scale) if scale > 0 else 0.0
    return out


def parity(pgc, p, q, qsteps, every, ref, timed, S):
    """Errors of the moment series, outside the timed region.

    fp64_vs_oracle: the library's FP64 mode on the oracle's sample (same workload, particles, seed
    and time steps) against the FP64 oracle: the same discrete decisions, rounding-level errors.
    fp32_vs_fp64: the timed run itself (its first S time steps, the whole ensemble) against the
    FP64 mode on the same ensemble; since the FP64 mode equals the oracle, this is the error of
    the production path against the FP64 oracle at the full size."""
    t_samp = q["N"] * qsteps
    sim = pgc.Simulation(W.scaled(q, precision="fp64"), max_outputs=qsteps // max(every, 1) + 2)
    sim.step(qsteps, every)
    g = sim.moments()
    sim.close()
    n = min(len(g["t_fs"]), len(ref["t_fs"]))
    a = _moment_errors(g, ref, n)
    out = {"fp64_vs_oracle": dict(a, sample="%d particles x %d time steps (%d particle-steps), every %d-th step"
                                  % (q["N"], qsteps, t_samp, every)), "tolerance": 1e-3}
    if p.get("precision", "fp32") != "fp64":
        s64 = pgc.Simulation(W.scaled(p, precision="fp64"), max_outputs=S // max(every, 1) + 2)
        s64.step(S, every)
        m64 = s64.moments()
        s64.close()
        n = min(len(m64["t_fs"]), len(timed["t_fs"]))
        b = _moment_errors(timed, m64, n)
        out["fp32_vs_fp64"] = dict(b, sample="the timed FP32 run, all %d particles, first %d time steps" % (p["N"], S))
        out.update(b)   # the headline errors: the production path against FP64 at full size
        out["note"] = ("FP32 rounding now and then flips a cell or threshold decision and the Pauli histogram "
                       "spreads it: over thousands of steps the FP32 and FP64 trajectories decorrelate and the "
                       "difference becomes Monte Carlo noise of two equivalent ensembles")
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O

    O.build()
    p = WORKLOADS[args.workload] or W.sweep64()[0]
    n = 20000 if p["N"] >= 100_000 and p["Q1"] <= 6 else (10000 if p["N"] <= 10000 else 2000)
    S = 20 if p["Q1"] <= 6 else 4
    q = W.scaled(p, N=n)
    o = O.Oracle(q)
    for _ in range(args.warmup):
        o.step(S, args.moments_every)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(S, args.moments_every)
    dt = time.perf_counter() - t0
    value = n * S * args.steps / dt
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": p["name"], "sample_particles": n, "time_steps_per_step": S,
                   "note": "FP64 CPU oracle (C, OpenMP) on a bounded sample of the workload"},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": O.num_threads(), "kind": "oracle",
                         "sample": "%d particles x %d time steps per step" % (n, S)},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_sweep(args, pgc, torch, dev, rank, world):
    """64 cases (field x band-gap width, uneven particle counts) advanced together by one
    persistent launch sequence per time step, replayed from a CUDA graph, tile autotuned."""
    import torch.distributed as dist

    cases = [W.scaled(c, stream_id=c["stream_id"] + 64 * rank) for c in W.sweep64()]
    S, K, every = args.time_steps, args.steps, args.moments_every
    ntot = sum(c["N"] for c in cases)
    cap = (K + args.warmup) * S // max(every, 1) + 8
    b = pgc.BatchSimulation(cases, max_outputs=cap)
    tile, _ = b.autotune(2)
    for _ in range(args.warmup):
        b.step(S, every)
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    launches0 = pgc.pgc_launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(K):
        flush.fill_(float(k))
        ev[k][0].record(b.stream)
        b.step(S, every)
        ev[k][1].record(b.stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = pgc.pgc_launch_count() - launches0
    clk = clocks.stop()
    gpu_ms = max_over_ranks(sum(x.elapsed_time(y) for x, y in ev), dev)
    value = throughput(ntot, world, S, K, gpu_ms)
    peak, peak_kind = _peaks()
    by = ntot * (2 * 6 * 4 + 4)
    achieved = by / (gpu_ms / K / S / 1e3) / 1e9
    b.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": gpu_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "sweep64_field1-20kVcm_x_gapwidth0.02-0.2eV_M5_Q6_fp32", "cases": len(cases),
                       "particles_per_gpu": ntot, "time_steps_per_step": S, "tile": tile, "graph": True,
                       "l2": "flushed between timed steps; the 3.4 GB ensemble exceeds L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "kernel": "whole time step (3 launches)", "peak_source": peak_kind,
                         "bytes_per_launch": by},
            "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clk,
        }
        print(json.dumps(line), flush=True)


def run_adjoint(args, pgc, torch, dev, rank, world):
    """One step = a full adjoint evaluation: forward --time-steps steps with checkpoints every 250,
    then the reverse sweep (segment replay + backward kernels) of the window-averaged mean and
    variance of J_x over the last 250 steps; the metric counts forward particle-steps."""
    p = rank_workload(WORKLOADS["adjoint"], rank)
    S, K = args.time_steps, args.steps
    every, window, ckpt = args.moments_every, min(p["steady_window"], S), p["ckpt_every"]
    sims = []

    def one():
        sim = pgc.Simulation(p, max_outputs=S // every + 2)
        nbytes = pgc.pgc_adjoint_query_sizes(sim.ctx, S, ckpt)
        work = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        val, grad = pgc.pgc_adjoint(sim.ctx, S, ckpt, every, window, [1.0, 0.0], work.data_ptr())
        e1.record(sim.stream)
        torch.cuda.synchronize()
        sim.close()
        return e0.elapsed_time(e1), val, grad, nbytes

    for _ in range(args.warmup):
        one()
    launches0 = pgc.pgc_launch_count()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    res = [one() for _ in range(K)]
    clk = clocks.stop()
    launches = pgc.pgc_launch_count() - launches0
    ms = sum(r[0] for r in res)
    val, grad, nbytes = res[-1][1], res[-1][2], res[-1][3]
    fd = None
    if args.fd_check:
        keys = ["Ex_lo", "Ex_hi", "eps0_lo", "eps0_hi"]
        fd = []
        for t, key in enumerate(keys):
            pair = ("Ex_lo", "Ex_hi") if t < 2 else ("eps0_lo", "eps0_hi")
            h = 1e-3 * abs(p[key])
            vals = []
            for sgn in (1, -1):
                q = dict(p)
                if p[pair[0]] == p[pair[1]]:
                    q[pair[0]] += sgn * h
                    q[pair[1]] += sgn * h
                else:
                    q[key] += sgn * h
                vals.append(pgc.window_objective(q, S, every, window)[0])
            f = 2.0 if p[pair[0]] == p[pair[1]] else 1.0
            fd.append((vals[0] - vals[1]) / (2 * h) / f)
    if rank == 0:
        line = {
            "metric": METRIC, "value": p["N"] * world * S * K / (ms / 1e3), "unit": METRIC, "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": p["name"], "particles_per_gpu": p["N"], "time_steps": S, "ckpt_every": ckpt,
                       "window_steps": window, "moments_every": every, "work_bytes": nbytes,
                       "note": "one step = forward with checkpoints + reverse sweep; metric counts forward particle-steps"},
            "adjoint": {"Jbar_A_per_m": val[0], "VarJ": val[1],
                        "dJbar_d(E_lo,E_hi,eps0_lo,eps0_hi)": list(grad),
                        "central_fd_h1e-3_crn": fd},
            "gpu_launches": launches, "clocks": clk, "cpu_baseline": None, "e2e": None, "roofline": None,
        }
        print(json.dumps(line), flush=True)


def run_sg_error(args, pgc, torch, dev, rank, world):
    """Test 3 (Sec. 5): one step = the stochastic-Galerkin error study of both scenarios
    (uncertain width, uncertain field): degrees 0..25 and the reference 30 on M + 1 nodes, 1e4
    particles, dt 2.5 fs, errors of the energy in L2(I_z) at 0.1, 0.5 and 1 ps.  The metric
    counts the particle-steps of all runs over the device time of their pgc_step calls."""
    from paper_2404_19602_gb300 import sg_error as SG

    degrees = [M for M in SG.DEGREES if M != 30]
    scen = {"width": W.TEST3_WIDTH_1E4, "field": W.TEST3_FIELD_1E4}
    steps = W.TEST3_TIMES_STEPS

    def one():
        rec = []
        t0 = time.perf_counter()
        errs = {k: SG.sg_error(rank_workload(p, rank), degrees, 30, steps, record=rec) for k, p in scen.items()}
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        return sum(a.elapsed_time(b) for a, b, _ in rec), sum(n for _, _, n in rec), wall, errs

    for _ in range(args.warmup):
        one()
    launches0 = pgc.pgc_launch_count()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    res = [one() for _ in range(args.steps)]
    clk = clocks.stop()
    launches = pgc.pgc_launch_count() - launches0
    ms = max_over_ranks(sum(r[0] for r in res), dev)
    wall = max_over_ranks(sum(r[2] for r in res), dev)
    ps = res[0][1]
    errs = res[-1][3]
    if rank == 0:
        dt = W.TEST3_WIDTH_1E4["dt_fs"]
        line = {
            "metric": METRIC, "value": ps * world * args.steps / (ms / 1e3), "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "test3_sg_error_width+field_M0-25_ref30_N1e4_dt2.5fs_fp32",
                       "particles_per_run": W.TEST3_WIDTH_1E4["N"], "runs_per_step": 2 * (len(degrees) + 1),
                       "particle_steps_per_step": ps, "degrees": degrees, "M_ref": 30,
                       "l2": "not flushed: each run's 1e4-particle state (<= 2.5 MB) is L2-resident, as in any run of "
                             "that size"},
            "roofline": None,
            "roofline_note": "1e4 particles per run: launch- and latency-bound, as the 1e4-particle deterministic "
                             "workload; the HBM fraction is not meaningful",
            "e2e": {"value": ps * world * args.steps / wall, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 2 * (len(degrees) + 1) * len(steps) * 64 * 4 * 8,
                    "note": "wall clock of the whole study through the public API: context creation, the initial "
                            "sampling on the device (no state upload), the steps and the observations at 64 points"},
            "sg_error": {k: {"t_ps": [n * dt / 1000.0 for n in steps], "M": degrees,
                             "err_eV": [[float(x) for x in v[M]] for M in degrees]} for k, v in errs.items()},
            "gpu_launches": launches, "clocks": clk, "cpu_baseline": None,
        }
        print(json.dumps(line), flush=True)


def run_mc_compare(args, pgc, torch, dev, rank, world):
    """Test 4 (Sec. 5): one step = the error of E_z[V_x] at 0.5 ps (200 steps of 2.5 fs) against an
    sG reference (5e6 particles, degree 30) of MC-sG with 5e4 particles at degrees 0..10 and of
    MC-MC with 5e4 particles per sample at 1..256 samples (the samples in one batch), uncertain
    width.  The metric counts the particle-steps of all runs over the wall time of the step
    (context creation and initial sampling included)."""
    from paper_2404_19602_gb300 import sg_error as SG

    p = rank_workload(W.TEST3_WIDTH_1E4, rank)
    steps, N, N_ref, M_ref = 200, 50_000, 5_000_000, 30
    degrees, samples = (0, 1, 2, 3, 4, 5, 6, 8, 10), (1, 2, 4, 8, 16, 32, 64, 128, 256)
    ps = steps * (N_ref + N * len(degrees) + N * sum(samples))

    def one():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = SG.mc_comparison(p, degrees, samples, N, N_ref, M_ref, steps)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, r

    for _ in range(args.warmup):
        one()
    launches0 = pgc.pgc_launch_count()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    res = [one() for _ in range(args.steps)]
    clk = clocks.stop()
    launches = pgc.pgc_launch_count() - launches0
    wall = max_over_ranks(sum(r[0] for r in res), dev)
    r = res[-1][1]
    if rank == 0:
        value = ps * world * args.steps / wall
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": wall * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "test4_mcsg_vs_mcmc_W6.5-7.5nm_E5kVcm_t0.5ps_N5e4_ref5e6_M30_fp32",
                       "particle_steps_per_step": ps, "timing": "wall clock of the whole step",
                       "l2": "not flushed: the runs follow one another; the 1.2 GB reference state exceeds L2"},
            "roofline": None,
            "roofline_note": "a mix of 20 runs of different shapes; the per-kernel rooflines are those of the "
                             "gap_uq and gap_field lines",
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                    "note": "the value is already wall clock through the public API; initial states are sampled "
                            "on the device"},
            "mc_compare": {"t_ps": steps * p["dt_fs"] / 1000.0, "ref_vx_ms": r["ref_vx"],
                           "mc_sg": {"M": list(degrees), "cost_per_particle": [(M + 1) ** 2 for M in degrees],
                                     "err_vx_ms": [r["sg"][M] for M in degrees]},
                           "mc_mc": {"M2": list(samples), "cost_per_particle": list(samples),
                                     "err_vx_ms": [r["mc"][M2] for M2 in samples]}},
            "gpu_launches": launches, "clocks": clk, "cpu_baseline": None,
        }
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    from paper_2404_19602_gb300 import pgc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2404_19602_gb300 import build as B

    B.build()
    if args.workload in ("sweep", "adjoint", "sg_error", "mc_compare"):
        {"sweep": run_sweep, "adjoint": run_adjoint, "sg_error": run_sg_error, "mc_compare": run_mc_compare}[args.workload](
            args, pgc, torch, dev, rank, world)
        if world > 1:
            dist.destroy_process_group()
        return
    p = rank_workload(WORKLOADS[args.workload], rank)
    S, K = args.time_steps, args.steps
    every = args.moments_every
    cap = (K + args.warmup) * S // max(every, 1) + 8

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up on a separate instance (module load, first launches, clocks)
    warm = pgc.Simulation(p, max_outputs=cap)
    for _ in range(args.warmup):
        warm.step(S, every)
    torch.cuda.synchronize()
    warm.close()
    del warm

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sim = pgc.Simulation(p, max_outputs=cap)
    fused = sim.P * sim.Q <= 64           # pipelined form (the library default): one fused launch per time step
    sim.set_pipeline(fused)
    pgc.pgc_profile(sim.ctx, 50)                # kernel timing samples: every 50th time step
    stream = torch.cuda.current_stream(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = pgc.pgc_launch_count()
    barrier()
    w0 = time.perf_counter()
    for k in range(K):
        flush.fill_(float(k))                    # evict L2 between timed steps (not timed)
        ev[k][0].record(stream)
        sim.step(S, every)
        ev[k][1].record(stream)
    barrier()
    wall = time.perf_counter() - w0
    launches = pgc.pgc_launch_count() - launches0
    clk = clocks.stop()
    gpu_ms = sum(a.elapsed_time(b) for a, b in ev)
    prof = pgc.pgc_profile_read(sim.ctx)
    cnt = sim.counters()
    timed_moments = sim.moments()
    gpu_ms_max = max_over_ranks(gpu_ms, dev)
    N = p["N"]
    value = throughput(N, world, S, K, gpu_ms_max)

    # roofline of the dominant kernel: algorithmic bytes per launch / mean launch time.  The
    # algorithmic bytes of a particle-step are a read and a write of its whole state, 2 x (2 P
    # esz): 32 B (1 x 1, FP64), 96 B (P = 6), 336 B (P = 21).  The kernels write back only the
    # coefficients that change (the drifted ones, and the colliders' states), so the bytes they
    # touch are fewer; both counts are given.
    P, Q = sim.P, sim.Q
    esz = 8 if p.get("precision") == "fp64" else 4
    n_drift = 1 if p["Ex_lo"] == p["Ex_hi"] else 2
    queued = cnt["queued"] / max(cnt["steps"], 1)
    unit_bytes = 2 * (2 * P * esz)                       # read + write of one particle's state
    bytes1 = N * (2 * P * esz + n_drift * esz)          # touched: read the state, write the drifted coefficients
    bytes2 = queued * (2 * (2 * P * esz) + 4)           # colliders: read + write the state, queue index
    peak, peak_kind = _peaks()
    if fused:
        # the fused launch is a whole time step: streaming work of step n + collider work of n - 1
        dominant, ms_dom, by, units = "k_step", prof["phase1_ms"], bytes1 + bytes2, N
    else:
        k1 = "k_phase1_tc" if p.get("tc_proj") else "k_phase1"
        dominant = k1 if prof["phase1_ms"] >= prof["phase2_ms"] else "k_phase2"
        ms_dom = max(prof["phase1_ms"], prof["phase2_ms"])
        by, units = (bytes1, N) if dominant == k1 else (bytes2, queued)
    alg = units * unit_bytes
    achieved = alg / (ms_dom / 1e3) / 1e9 if ms_dom > 0 else 0.0
    touched = by / (ms_dom / 1e3) / 1e9 if ms_dom > 0 else 0.0
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": _traffic(dominant, args.workload),
                "kernel": dominant, "peak_source": peak_kind,
                "bytes_per_unit": unit_bytes, "units_per_launch": units, "bytes_per_launch": alg,
                "touched_bytes_per_launch": by, "touched_achieved": touched, "touched_frac": touched / peak,
                "touched_note": "the kernel reads the whole state and writes back only the coefficients the drift "
                                "changes (and the colliders' states)",
                "phase1_ms": prof["phase1_ms"], "phase2_ms": prof["phase2_ms"],
                "samples": prof["samples"], "pipelined": fused}

    # the issue roofline of the same kernel: its ncu instruction count per launch over the event
    # time, against one warp instruction per clock per SM sub-partition at the maximum SM clock
    issue = None
    inst = _traffic(dominant, args.workload, "warp_inst_per_launch")
    if inst and ms_dom > 0:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = (clk or {}).get("sm_max_mhz") or 2070.0
        ach_i, peak_i = inst / (ms_dom / 1e3), sms * 4 * mhz * 1e6
        issue = {"bound": "issue", "achieved": ach_i, "peak": peak_i, "unit": "warp-inst/s", "frac": ach_i / peak_i,
                 "kernel": dominant, "warp_inst_per_launch": inst,
                 "peak_source": "%d SMs x 4 schedulers x 1 warp instruction per clock x %.0f MHz" % (sms, mhz)}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        host_state = sim.state_native()              # the ensemble in page-locked host memory (device layout)
        sim.close()
        sim2 = pgc.Simulation(p, max_outputs=cap)
        barrier()
        e0 = time.perf_counter()
        for k in range(K):
            sim2.set_state_native(host_state)        # H2D of the step's input state
            sim2.step(S, every)
            m = sim2.moments()                       # D2H of the moment series (synchronizes)
        barrier()
        e_dt = max_over_ranks(time.perf_counter() - e0, dev)
        state_bytes = pgc.pgc_query_sizes(sim2.cfg)["state_bytes"]
        e2e = {"value": throughput(N, world, S, K, e_dt * 1e3), "unit": METRIC,
               "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": int(m["t_fs"].size * (1 + 4 * Q + 8) * 8)}
        sim2.close()
    else:
        sim.close()

    base, par = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base, (q, qsteps, ref) = cpu_baseline(p, every)
        par = parity(pgc, p, q, qsteps, every, ref, timed_moments, S)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": gpu_ms_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if p.get("precision") == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": p["name"], "particles_per_gpu": N, "P": P, "Q": Q,
                       "time_steps_per_step": S, "dt_fs": p["dt_fs"], "moments_every": every,
                       "l2": "flushed (256 MiB write) between timed steps; the state stays L2-resident "
                             "across the time steps of one step when it fits (1e6 x P = 6: 48 MB), and "
                             "exceeds L2 otherwise (4e6 x P = 21: 672 MB)",
                       "parallelism": "independent ensembles per GPU" if world > 1 else "1 GPU"},
            "roofline": roofline,
            "roofline_issue": issue,
            "cpu_baseline": base,
            "parity": par,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "wall_s": wall,
            "collisions_per_step": cnt["attempts"] / max(cnt["steps"], 1),
            "queued_per_step": queued,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
