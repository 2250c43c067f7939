"""The stochastic-Galerkin error study of Test 3 (Sec. 5) and the comparison with Monte Carlo
sampling of the random input of Test 4, over the public API.

For one random input (the ribbon width, or the field), runs of increasing gPC degree M are
compared with a reference degree M_ref at fixed times t through the energy E(t, z):

    sG error(M, t) = || E_ref(t, .) - E_M(t, .) ||_{L2(I_z)},   z uniform on I_z,

evaluated with a Gauss-Legendre rule in z, the energies of the particles reconstructed at each
point by pgc_observe_at.  Every run starts from the same initial data (the per-particle uniforms
of the Fermi-Dirac sampling are common to all degrees) and draws the same random numbers (the
Philox counters (particle, step, attempt) do not depend on M): the common-random-number form of
the comparison.  Degree M runs on M + 1 Gauss nodes, so the compiled one-dimensional shapes set
the degrees available: 0..6, 8, 10, 12, 15, 20, 25, 30.
"""
from __future__ import annotations

import numpy as np

from . import pgc
from . import workloads as W

DEGREES = (0, 1, 2, 3, 4, 5, 6, 8, 10, 12, 15, 20, 25, 30)


def l2_rule(n: int = 64):
    """Gauss-Legendre points on [-1, 1] and weights of the uniform law (summing to 1)."""
    z, w = np.polynomial.legendre.leggauss(n)
    return z, w / 2.0


def energy_at_times(p: dict, M: int, steps, z, record=None) -> np.ndarray:
    """Energy E(t, z) [len(steps)][len(z)] of the degree-M run of workload p after each
    cumulative number of time steps in `steps` (increasing).  If `record` is a list, a pair of
    CUDA events around each pgc_step call and its particle-steps are appended to it."""
    q = W.scaled(p, M=M, Q1=M + 1)
    s = pgc.Simulation(q, max_outputs=4)
    zz = np.asarray(z, dtype=np.float64).reshape(-1, 1)
    out, done = [], 0
    for n in steps:
        if record is not None:
            import torch

            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            ev[0].record(s.stream)
        s.step(int(n) - done, 0)
        if record is not None:
            ev[1].record(s.stream)
            record.append((ev[0], ev[1], q["N"] * (int(n) - done)))
        done = int(n)
        out.append(s.observe_at(zz)[:, 2])
    s.close()
    return np.array(out)


def sg_error(p: dict, degrees, M_ref: int, steps, nz: int = 64, record=None) -> dict:
    """{M: sG error at each entry of `steps`} for the degrees given, against degree M_ref."""
    z, w = l2_rule(nz)
    ref = energy_at_times(p, M_ref, steps, z, record)
    return {M: np.sqrt((((energy_at_times(p, M, steps, z, record) - ref) ** 2) * w).sum(axis=1))
            for M in degrees}


# ------------------------------------------------------------------------------------------
# Test 4 (Sec. 5): the particle stochastic-Galerkin method (MC-sG) against Algorithm 1 run at
# sampled values of the random input (MC-MC), by the error of E_z[V_x] at a fixed time against a
# large-ensemble, high-degree sG reference.  Cost per particle and time step: (M + 1)^2 for MC-sG
# (reconstruction and projection over M + 1 coefficients and nodes), M_2 for MC-MC (one
# deterministic run per sample).
# ------------------------------------------------------------------------------------------
def mean_vx_sg(p: dict, M: int, N: int, steps: int) -> float:
    """E_z[V_x] (m/s) after `steps` time steps of the degree-M particle sG run of N particles
    (the quadrature mean over the M + 1 nodes, Sec. 4.2)."""
    s = pgc.Simulation(W.scaled(p, M=M, Q1=M + 1, N=N), max_outputs=4)
    s.step(steps, steps)
    v = float(s.moments()["mean"][-1, 0])
    s.close()
    return v


def deterministic_at(p: dict, z: float) -> dict:
    """Workload p with its random input fixed at the point z of [-1, 1] (the affine maps of the
    library: the width for the width law, else the band minimum, else the field)."""
    t = 0.5 * (z + 1.0)
    if (p.get("W_lo") or 0.0) > 0.0:
        if p["W_lo"] != p["W_hi"]:
            w = p["W_lo"] + (p["W_hi"] - p["W_lo"]) * t
            return W.scaled(p, W_lo=w, W_hi=w, M=0, Q1=1)
    elif p["eps0_lo"] != p["eps0_hi"]:
        e = p["eps0_lo"] + (p["eps0_hi"] - p["eps0_lo"]) * t
        return W.scaled(p, eps0_lo=e, eps0_hi=e, M=0, Q1=1)
    if p["Ex_lo"] != p["Ex_hi"]:
        f = p["Ex_lo"] + (p["Ex_hi"] - p["Ex_lo"]) * t
        return W.scaled(p, Ex_lo=f, Ex_hi=f, M=0, Q1=1)
    return W.scaled(p, M=0, Q1=1)


def mc_mc_samples(p: dict, M2: int, N: int, steps: int, seed: int = 1) -> np.ndarray:
    """MC-MC: V_x (m/s) after `steps` time steps of Algorithm 1 at M2 points z_j drawn uniformly
    (numpy generator `seed`), one independent ensemble of N particles per sample (stream_id j),
    the samples advanced together by the batched kernels (at most 256 per batch)."""
    z = np.random.default_rng(seed).uniform(-1.0, 1.0, M2)
    cases = [W.scaled(deterministic_at(p, float(zj)), N=N, stream_id=j) for j, zj in enumerate(z)]
    vals = []
    for c0 in range(0, M2, 256):
        b = pgc.BatchSimulation(cases[c0:c0 + 256], max_outputs=4)
        b.step(steps, steps)
        vals += [float(s.moments()["mean"][-1, 0]) for s in b.sims]
        b.close()
    return np.array(vals)


def mc_comparison(p: dict, degrees, samples, N: int, N_ref: int, M_ref: int, steps: int, seed: int = 1) -> dict:
    """Errors |E_z[V_x] - E_z[V_x^ref]| of MC-sG (per degree) and MC-MC (per sample count) with N
    particles, the reference an sG run of N_ref particles and degree M_ref."""
    ref = mean_vx_sg(p, M_ref, N_ref, steps)
    sg = {M: abs(mean_vx_sg(p, M, N, steps) - ref) for M in degrees}
    mc = {M2: abs(float(mc_mc_samples(p, M2, N, steps, seed).mean()) - ref) for M2 in samples}
    return {"ref_vx": ref, "sg": sg, "mc": mc}
