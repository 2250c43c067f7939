"""Oracle pins of the width law of the band minimum (Test 2 of Sec. 5: the ribbon width is the
uncertain input, W = (6.5 + z) nm, and the band minimum is the lowest transverse subband
eps0 = pi hbar vF / W of Sec. 2, a non-polynomial function of z).  No GPU."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2404_19602_gb300 import workloads as W

HVF = 6.582119569e-16 * 1.0e6 * 1.0e9   # hbar vF in eV nm (CODATA hbar, vF = 1e8 cm/s of Table 1)


def test_node_band_minima_and_their_mean():
    """eps0 at the Gauss nodes of the width law, and its z-mean against the closed form
    E_z[pi hbar vF / W] = pi hbar vF ln(W_hi / W_lo) / (W_hi - W_lo) for W ~ U[W_lo, W_hi]
    (6 Gauss-Legendre nodes integrate 1/W on [6.5, 7.5] to ~1e-11).  The largest band minimum
    sits at the narrowest ribbon, z = -1."""
    p = W.scaled(W.TEST2_WIDTH_1E6, N=10)
    o = O.Oracle(p)
    t = o.tables()
    assert o.d == 1 and o.P == 6
    z, wq = np.polynomial.legendre.leggauss(6)
    Wq = 6.5 + 0.5 * (7.5 - 6.5) * (z + 1.0)
    assert np.allclose(t["eps0"], math.pi * HVF / Wq, rtol=1e-12, atol=0)
    assert np.all(np.diff(t["eps0"]) < 0)
    mean = float(np.dot(t["w"], t["eps0"]))
    closed = math.pi * HVF * math.log(7.5 / 6.5) / (7.5 - 6.5)
    assert abs(mean - closed) <= 1e-10 * closed


def test_deterministic_width_equals_the_band_minimum_run():
    """A deterministic width is the deterministic run with eps0 = pi hbar vF / W: the width enters
    the scheme only through the band minimum (dispersion, Fermi-Dirac sampling, the 1/W of the edge
    rate, the density)."""
    base = dict(N=1500, seed=5, Ex_lo=5000.0, Ex_hi=5000.0, M=0, Q1=1)
    w = O.Oracle(dict(base, W_lo=7.0, W_hi=7.0))
    e0 = float(w.tables()["eps0"][0])
    assert abs(e0 - math.pi * HVF / 7.0) <= 1e-14
    a = O.Oracle(dict(base, eps0_lo=e0, eps0_hi=e0))
    assert w.P == a.P == 1
    w.step(120, 40)
    a.step(120, 40)
    assert np.array_equal(w.state(), a.state())
    assert np.array_equal(w.moments()["mean"], a.moments()["mean"])


def test_width_law_galerkin_moments_against_brute_force_z_sampling():
    """E_z and Var_z by Gauss quadrature over the nodes against plain Monte Carlo over z of the
    same reconstructed particles (tiny ensemble), with the non-polynomial band minimum."""
    p = W.scaled(W.TEST2_WIDTH_1E6, N=100, seed=3, Q1=24)
    o = O.Oracle(p)
    o.step(40, 40)
    m = o.moments()
    rng = np.random.default_rng(4)
    nz = 20000
    zs = rng.uniform(-1, 1, size=(nz, 1))
    obs = np.array([o.observe_at(z) for z in zs])
    for comp in (0, 2, 3):
        mc_mean = obs[:, comp].mean()
        se = obs[:, comp].std() / math.sqrt(nz)
        assert abs(m["mean"][-1, comp] - mc_mean) < 4.5 * se + 1e-6 * abs(mc_mean)
        mc_var = obs[:, comp].var()
        se_var = ((obs[:, comp] - mc_mean) ** 2).std() / math.sqrt(nz)
        assert abs(m["var"][-1, comp] - mc_var) < 4.5 * se_var + 1e-6 * mc_var


def test_degenerate_width_interval_reduces_to_deterministic_run():
    """A width interval of one ulp runs the Galerkin machinery and gives the deterministic run."""
    base = dict(N=1200, seed=6, M=3, Q1=4)
    det = O.Oracle(dict(base, W_lo=7.0, W_hi=7.0))
    gpc = O.Oracle(dict(base, W_lo=7.0, W_hi=float(np.nextafter(7.0, 8.0))))
    assert det.P == 1 and gpc.P == 4
    det.step(100, 50)
    gpc.step(100, 50)
    a, b = det.moments(), gpc.moments()
    for comp in range(4):
        scale = np.abs(a["mean"][:, comp]).max()
        assert np.abs(a["mean"][:, comp] - b["mean"][:, comp]).max() < 1e-9 * scale
