"""Pins of the oracle's full time step (Algorithm 1 / Algorithm 2 of arXiv:2404.19602) against
properties the paper and the mathematics fix: the closed-form ballistic drift, conservation of
particles, non-negative reconstructed distributions, zero mean velocity and a stationary
Maxwellian energy distribution at zero field, Poisson collision counts, the Galerkin mean and
variance against brute-force sampling over z, and the degenerate interval.  No GPU.
"""
import math

import numpy as np
import pytest
import scipy.stats as st

import oracle as O
from paper_2404_19602_gb300 import workloads as W

HBAR_EVFS = 6.582119569e-16 * 1e15


def _eps(k, e0, hvF=0.6582119569):
    return np.sqrt(hvF ** 2 * (k[0] ** 2 + k[1] ** 2) + e0 ** 2)


def _velocity_fd(kx, ky, e0):
    """group velocity (Sec. 2, v = grad_k eps / hbar) by a central finite difference, m/s"""
    h = 1e-6
    vx = (_eps((kx + h, ky), e0) - _eps((kx - h, ky), e0)) / (2 * h) / HBAR_EVFS * 1e6
    vy = (_eps((kx, ky + h), e0) - _eps((kx, ky - h), e0)) / (2 * h) / HBAR_EVFS * 1e6
    return vx, vy


@pytest.mark.parametrize("random_field", [False, True])
def test_ballistic_drift_closed_form(random_field):
    """Mechanisms off: k(t) = k(0) - (e/hbar) E t for every particle and node (Eq. (17) and the
    sG forcing term of Sec. 4.1), and the velocity follows from the dispersion."""
    p = dict(N=300, mech_mask=0, eps0_lo=0.1, eps0_hi=0.1, Ex_lo=5000.0, Ex_hi=5000.0)
    if random_field:
        p.update(Ex_lo=1000.0, Ex_hi=10000.0, M=4, Q1=5)
    o = O.Oracle(p)
    k0 = o.state()
    nsteps = 250
    o.step(nsteps, 50)
    k1 = o.state()
    xg, _ = np.polynomial.legendre.leggauss(o.Q)
    E_nodes = p["Ex_lo"] + 0.5 * (p["Ex_hi"] - p["Ex_lo"]) * (xg + 1) if random_field else np.array([p["Ex_lo"]])
    psi = o.tables()["psi"]  # [Q, P]
    kx0 = psi @ k0[0]
    kx1 = psi @ k1[0]
    shift = E_nodes * 1e-7 * nsteps * p.get("dt_fs", 1.0) / HBAR_EVFS
    assert np.allclose(kx1, kx0 - shift[:, None], atol=1e-12, rtol=0)
    assert np.array_equal(k1[1], k0[1])
    # velocities of the last output against finite differences of the dispersion
    m = o.moments()
    assert np.isclose(m["t_fs"][-1], nsteps * 1.0)
    ky1 = psi @ k1[1]
    vx, vy = _velocity_fd(kx1, ky1, 0.1)
    assert np.allclose(m["nodes"][-1, :, 0], vx.mean(axis=1), rtol=1e-7, atol=1e-3)
    assert np.allclose(m["nodes"][-1, :, 1], vy.mean(axis=1), rtol=1e-7, atol=1e-3)


def test_conservation_and_positivity():
    p = W.scaled(W.GAP_UQ_1E6, N=3000)
    o = O.Oracle(p)
    for _ in range(3):
        o.step(20, 10)
        H, _ = o.hist()
        cnt = o.counters()
        assert H.min() >= 0
        assert int(H.sum()) + cnt["out_of_grid"] == p["N"] * o.Q
    # distribution reconstructed at arbitrary z (Eq. (24)) is a non-negative count of N particles
    z = np.linspace(-1, 1, 7)
    Hz, mx = o.reconstruct_f(z)
    assert Hz.min() >= 0
    assert np.all(Hz.reshape(7, -1).sum(axis=1) <= p["N"])
    assert np.all(mx == Hz.reshape(7, -1).max(axis=1))


def test_zero_field_zero_mean_velocity():
    p = W.scaled(W.DET_FP64_1E4, N=20000, Ex_lo=0.0, Ex_hi=0.0)
    o = O.Oracle(p)
    o.step(200, 100)
    k = o.state()
    vx, vy = _velocity_fd(k[0, 0], k[1, 0], 0.1)
    m = o.moments()
    for comp, v in ((0, vx), (1, vy)):
        sigma = v.std() / math.sqrt(p["N"])
        assert abs(m["mean"][-1, comp]) < 4.5 * sigma


def _mb_cdf(eps, e0, kT):
    # density proportional to eps * exp(-eps/kT) on [e0, inf)
    return 1.0 - np.exp(-(eps - e0) / kT) * (eps + kT) / (e0 + kT)


def test_maxwellian_is_stationary_at_zero_field():
    """Without Pauli blocking and with energy-conserving final states, the jump process of Sec. 3
    satisfies detailed balance for eps*exp(-eps/kT); the scheme is an exact simulation of it at
    zero field, so the energy distribution must stay Maxwellian (KS test after many phonon
    events; a hot lattice is used so that absorption is frequent)."""
    T = 1500.0
    kT = 8.617333262e-5 * T
    e0 = 0.1
    p = dict(N=20000, T_K=T, eps_F=e0 - 30 * kT, eps0_lo=e0, eps0_hi=e0, Ex_lo=0.0, Ex_hi=0.0,
             pauli_norm=O.PAULI_OFF, final_state=O.FS_EXACT_ENERGY, dt_fs=2.0, seed=11)
    o = O.Oracle(p)
    k = o.state()
    eps = _eps((k[0, 0], k[1, 0]), e0)
    assert st.kstest(eps, lambda x: _mb_cdf(x, e0, kT)).pvalue > 1e-3
    o.step(1000, 1000)
    cnt = o.counters()
    assert cnt["real"] > 3 * p["N"]  # several real collisions per particle
    k = o.state()
    eps = _eps((k[0, 0], k[1, 0]), e0)
    assert st.kstest(eps, lambda x: _mb_cdf(x, e0, kT)).pvalue > 1e-3
    # and the angle stays isotropic
    th = np.arctan2(k[1, 0], k[0, 0])
    assert st.kstest(th, st.uniform(loc=-math.pi, scale=2 * math.pi).cdf).pvalue > 1e-3


def test_paper_final_states_drift_from_maxwellian():
    """Control for the previous test: with the paper's |k| -+ omega/vF final states energy is not
    conserved exactly for eps0 > 0, and the same KS statistic detects the drift."""
    T = 1500.0
    kT = 8.617333262e-5 * T
    e0 = 0.3
    p = dict(N=20000, T_K=T, eps_F=e0 - 30 * kT, eps0_lo=e0, eps0_hi=e0, Ex_lo=0.0, Ex_hi=0.0,
             pauli_norm=O.PAULI_OFF, final_state=O.FS_PAPER, dt_fs=2.0, seed=11)
    o = O.Oracle(p)
    o.step(1000, 1000)
    k = o.state()
    eps = _eps((k[0, 0], k[1, 0]), e0)
    assert st.kstest(eps, lambda x: _mb_cdf(x, e0, kT)).pvalue < 1e-6


def test_collision_count_is_poisson_in_the_majorant():
    """Free flights dt = -ln(xi)/Gamma_tot (Eq. (18)) redrawn after every collision: the number of
    collision attempts in one step is Poisson with mean Gamma_tot dt (Pauli off)."""
    p = dict(N=20000, pauli_norm=O.PAULI_OFF, dt_fs=5.0, Ex_lo=0.0, Ex_hi=0.0, seed=5)
    o = O.Oracle(p)
    k = o.state()
    alpha = 0.1
    lam = 0.0
    for i in range(p["N"]):
        lam += (1 + alpha) * o.rates(k[0, 0, i], k[1, 0, i], 0.1).sum() * p["dt_fs"]
    o.step(1, 0)
    att = o.counters()["attempts"]
    assert abs(att - lam) < 5 * math.sqrt(lam) + 0.01 * lam


@pytest.mark.parametrize("two_d", [False, True])
def test_galerkin_mean_and_variance_against_brute_force_z_sampling(two_d):
    """QoI of Sec. 4.2: E_z and Var_z of the observables by Gauss quadrature over the nodes
    against plain Monte Carlo over z of the same reconstructed particles (tiny ensemble).
    With N = 100 the observables are rough functions of z (a few particles whose collisions were
    accepted at some nodes only), so the quadrature uses more nodes than the M + 1 of the default
    (the quadrature order is a free parameter of the scheme); with M + 1 nodes the mean still
    agrees to a few 1e-3 but the variance carries a quadrature error of order 10 %."""
    base = W.GAP_FIELD_UQ_4E6 if two_d else W.GAP_UQ_1E6
    p = W.scaled(base, N=100, seed=3, Q1=12 if two_d else 24)
    o = O.Oracle(p)
    o.step(60, 60)
    m = o.moments()
    rng = np.random.default_rng(2)
    nz = 20000
    zs = rng.uniform(-1, 1, size=(nz, o.d))
    obs = np.array([o.observe_at(z) for z in zs])  # [nz, 4]
    for comp in (0, 2, 3):
        mc_mean = obs[:, comp].mean()
        se = obs[:, comp].std() / math.sqrt(nz)
        assert abs(m["mean"][-1, comp] - mc_mean) < 4.5 * se + 1e-6 * abs(mc_mean)
        mc_var = obs[:, comp].var()
        dev = (obs[:, comp] - mc_mean) ** 2
        se_var = dev.std() / math.sqrt(nz)
        assert abs(m["var"][-1, comp] - mc_var) < 4.5 * se_var + 1e-6 * mc_var


def test_degenerate_interval_reduces_to_deterministic_run():
    """A random band minimum whose interval has zero width (one ulp) gives the deterministic
    run (P = Q = 1, Algorithm 1) through the Galerkin machinery of Algorithm 2."""
    e0 = 0.1
    base = dict(N=2000, seed=4, eps0_lo=e0, eps0_hi=e0)
    det = O.Oracle(base)
    gpc = O.Oracle(dict(base, eps0_hi=np.nextafter(e0, 1.0), M=3, Q1=4))
    assert det.P == 1 and gpc.P == 4
    det.step(150, 50)
    gpc.step(150, 50)
    a, b = det.moments(), gpc.moments()
    for comp in range(4):
        scale = np.abs(a["mean"][:, comp]).max()
        assert np.abs(a["mean"][:, comp] - b["mean"][:, comp]).max() < 1e-9 * scale
    ka, kb = det.state(), gpc.state()
    assert np.allclose(ka[:, 0, :], kb[:, 0, :], atol=1e-12)
    assert np.abs(kb[:, 1:, :]).max() < 1e-12


def test_initial_state_is_fermi_dirac():
    """Sampled energies follow eps*FD(eps) (KS) and the angle is uniform."""
    p = dict(N=20000, eps0_lo=0.1, eps0_hi=0.1, seed=9)
    o = O.Oracle(p)
    k = o.state()
    eps = _eps((k[0, 0], k[1, 0]), 0.1)
    kT = 8.617333262e-5 * 300
    tot = O.fd_total(0.1, 0.4, kT)
    grid = np.linspace(0.1, 0.4 + 40 * kT, 4000)
    dens = grid / (1 + np.exp((grid - 0.4) / kT))
    cdf = np.concatenate([[0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(grid))]) / tot
    assert st.kstest(eps, lambda x: np.interp(x, grid, cdf)).pvalue > 1e-3
    th = np.arctan2(k[1, 0], k[0, 0])
    assert st.kstest(th, st.uniform(loc=-math.pi, scale=2 * math.pi).cdf).pvalue > 1e-3
