"""The stochastic-Galerkin error study of Test 3 (Sec. 5) over the public API.

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
