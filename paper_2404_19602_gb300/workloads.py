"""Seeded synthetic workloads shaped like the paper's runs (arXiv:2404.19602, Sec. 5).

This module holds parameter dictionaries and seeded case lists only -- none of the method's
arithmetic.  Both the CUDA library (through :mod:`paper_2404_19602_gb300`) and the FP64 CPU oracle
read these dictionaries, so that the two sides are fed identical inputs.

Keys (units): T_K (K), eps_F (eV), eps0_lo/eps0_hi (conduction-band minimum hbar vF pi/W, eV; equal
ends = deterministic), Ex_lo/Ex_hi (V/cm), mech_mask (bit set of the rate vector of Eq. (20);
63 = all), alpha (Eq. (19)), Nk and Lk_hvF (grid of Sec. 3), M (gPC degree), Q1 (Gauss nodes per
random dimension), N (particles), dt_fs, seed (Philox key), stream_id, pauli_norm
(0 = maximum of the initial histogram, 1 = current maximum, 2 = off), final_state (0 = the
paper's |k| -+ omega/vF, 1 = exact energy), n_theta (trapezoid points of the edge integral),
splitting (0 = the paper's Lie splitting, 1 = Strang).

A band gap E_g maps to eps0 = E_g / 2 (the conduction-band minimum of the gapped Dirac cone).
With W_lo/W_hi (nm) present the ribbon width is the input instead: W(z) spreads affinely over
[W_lo, W_hi] and eps0(z) = pi hbar vF / W(z) (eps0_lo/eps0_hi are then unused).
"""
from __future__ import annotations

import numpy as np

#: Sec. 5 simulation parameters (grid, self-scattering) and the physical defaults of the runs.
COMMON = dict(T_K=300.0, eps_F=0.4, mech_mask=63, alpha=0.1, Nk=240, Lk_hvF=5.0, n_theta=64,
              pauli_norm=0, final_state=0, max_coll=32, seed=1, stream_id=0, splitting=0)


def _w(**kw):
    d = dict(COMMON)
    d.update(kw)
    return d


#: Deterministic inputs: gap 0.2 eV, 5 kV/cm, 1e4 particles, 2000 steps of 1 fs, FP64.
DET_FP64_1E4 = _w(name="det_gap0.2eV_5kVcm_N1e4_fp64", eps0_lo=0.1, eps0_hi=0.1, Ex_lo=5000.0,
                  Ex_hi=5000.0, M=0, Q1=1, N=10_000, dt_fs=1.0, steps=2000, precision="fp64")

#: One random input: gap ~ U[0.1,0.3] eV, Legendre degree 5, 6 Gauss nodes, 1e6 particles.
GAP_UQ_1E6 = _w(name="gapU[0.1,0.3]eV_M5_Q6_N1e6_fp32", eps0_lo=0.05, eps0_hi=0.15, Ex_lo=5000.0,
                Ex_hi=5000.0, M=5, Q1=6, N=1_000_000, dt_fs=1.0, steps=5000, precision="fp32")

#: Two random inputs: gap ~ U[0.1,0.3] eV and field ~ U[1,10] kV/cm, total degree 5 (21
#: coefficients), 6x6 tensor Gauss nodes, 4e6 particles.
GAP_FIELD_UQ_4E6 = _w(name="gapU[0.1,0.3]eV_fieldU[1,10]kVcm_M5_Q36_N4e6_fp32", eps0_lo=0.05,
                      eps0_hi=0.15, Ex_lo=1000.0, Ex_hi=10000.0, M=5, Q1=6, N=4_000_000, dt_fs=1.0,
                      steps=5000, precision="fp32")

#: Sensitivities of the steady current: gap random, field deterministic, 1e6 particles.
ADJOINT_1E6 = _w(name="adjoint_gapU[0.1,0.3]eV_5kVcm_M5_N1e6", eps0_lo=0.05, eps0_hi=0.15,
                 Ex_lo=5000.0, Ex_hi=5000.0, M=5, Q1=6, N=1_000_000, dt_fs=1.0, steps=5000,
                 ckpt_every=250, steady_window=250, precision="fp32")


#: Test 2 (Sec. 5), first scenario: uncertain ribbon width W = (6.5 + z) nm, z ~ U[0,1] (the band
#: minimum pi hbar vF / W(z) is not a polynomial in z), deterministic field 0.5 V/um, eps_F 0.4 eV,
#: dt 2.5 fs, 3 ps, 1e6 particles, M = 5.
TEST2_WIDTH_1E6 = _w(name="test2_W6.5-7.5nm_E5kVcm_epsF0.4_M5_N1e6_fp32", W_lo=6.5, W_hi=7.5,
                     Ex_lo=5000.0, Ex_hi=5000.0, M=5, Q1=6, N=1_000_000, dt_fs=2.5, steps=1200,
                     precision="fp32")

#: Test 2, second scenario: uncertain field E = (0.4 + 0.2 z) V/um, width 7 nm.
TEST2_FIELD_1E6 = _w(name="test2_W7nm_E4-6kVcm_epsF0.4_M5_N1e6_fp32", W_lo=7.0, W_hi=7.0,
                     Ex_lo=4000.0, Ex_hi=6000.0, M=5, Q1=6, N=1_000_000, dt_fs=2.5, steps=1200,
                     precision="fp32")

#: Test 3 (Sec. 5), the stochastic-Galerkin error study: the two Test 2 scenarios with 1e4
#: particles and eps_F 0.4 eV, dt 2.5 fs, errors at 0.1, 0.5 and 1 ps (40, 200, 400 steps) for
#: degrees M = 0..25 against M_ref = 30 (the degree is set per run).
TEST3_WIDTH_1E4 = _w(name="test3_W6.5-7.5nm_E5kVcm_epsF0.4_N1e4_fp32", W_lo=6.5, W_hi=7.5,
                     Ex_lo=5000.0, Ex_hi=5000.0, M=5, Q1=6, N=10_000, dt_fs=2.5, steps=400,
                     precision="fp32")
TEST3_FIELD_1E4 = _w(name="test3_W7nm_E4-6kVcm_epsF0.4_N1e4_fp32", W_lo=7.0, W_hi=7.0,
                     Ex_lo=4000.0, Ex_hi=6000.0, M=5, Q1=6, N=10_000, dt_fs=2.5, steps=400,
                     precision="fp32")
TEST3_TIMES_STEPS = (40, 200, 400)


def sweep64(seed: int = 1, n_lo: float = 1e5, n_hi: float = 4e6, steps: int = 3000):
    """64 cases: field 1..20 kV/cm (8 values) x width 0.02..0.2 eV (8 values) of a band-gap
    interval centred on 0.2 eV; particle counts log-uniform in [n_lo, n_hi]."""
    rng = np.random.default_rng(seed)
    fields = np.linspace(1000.0, 20000.0, 8)
    widths = np.linspace(0.02, 0.2, 8)
    cases = []
    for E in fields:
        for w in widths:
            n = int(round(float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))))
            cases.append(_w(name="sweep", eps0_lo=0.1 - w / 4.0, eps0_hi=0.1 + w / 4.0,
                            Ex_lo=float(E), Ex_hi=float(E), M=5, Q1=6, N=n, dt_fs=1.0,
                            steps=steps, precision="fp32", stream_id=len(cases)))
    return cases


def scaled(w: dict, **kw) -> dict:
    """A copy of a workload with some entries replaced (reduced sizes for parity tests)."""
    d = dict(w)
    d.update(kw)
    return d
