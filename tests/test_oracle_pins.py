"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix (no GPU).

Every check here compares the oracle with something other than itself: published known-answer
vectors, library routines (scipy, numpy), closed forms, brute-force quadrature of the
definitions in Sec. 2 of arXiv:2404.19602, or statistical properties of the exact process.
"""
import math
import os

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    vals = {}
    with open(os.path.join(GOLDEN, "table1_parameters.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, val, _unit = line.split()
            vals[name] = float(val)
    return vals


# ------------------------------------------------------------------------------------------
# Philox4x32-10 and the uniform map
# ------------------------------------------------------------------------------------------
def test_philox_known_answers():
    n = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            out = O.philox(w[0:4], w[4:6])
            assert list(out) == w[6:10]
            n += 1
    assert n == 3


def test_uniform_map_exact_in_fp32():
    xs = [0, 1, 255, 256, 0x7FFFFFFF, 0xFFFFFF00, 0xFFFFFFFF, 123456789]
    for x in xs:
        u = O.u01(x)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u  # exactly representable in FP32
        assert u == (((x >> 8) | 1) / 2.0 ** 24)
    assert O.u01(0) == 2.0 ** -24
    assert O.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24


# ------------------------------------------------------------------------------------------
# special functions and quadrature
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("x", [-1e-8, -0.1, -0.5, -0.999, -1.0, -1.5, -7.0, -300.0, -1e6])
def test_li2_against_scipy(x):
    # scipy's spence(z) = Li2(1 - z)
    ref = sp.spence(1.0 - x)
    assert abs(O.li2_neg(x) - ref) <= 2e-15 * max(1.0, abs(ref))


def test_li2_closed_values():
    assert abs(O.li2_neg(-1.0) + math.pi ** 2 / 12) < 1e-15
    # inversion identity Li2(-x) + Li2(-1/x) = -pi^2/6 - ln(x)^2/2
    for x in [2.0, 10.0, 1e4]:
        lhs = O.li2_neg(-x) + O.li2_neg(-1.0 / x)
        assert abs(lhs + math.pi ** 2 / 6 + 0.5 * math.log(x) ** 2) < 1e-12


@pytest.mark.parametrize("n", [1, 2, 3, 6, 11, 16, 31])
def test_gauss_legendre_against_numpy(n):
    x, w = O.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x, xr, atol=2e-15, rtol=0)
    assert np.allclose(w, wr / 2.0, atol=2e-15, rtol=0)
    # exact for monomials up to degree 2n-1 against the uniform density on [-1,1]
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 1.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14


def _onb(h, z):
    c = np.zeros(h + 1)
    c[h] = 1.0
    return math.sqrt(2 * h + 1) * np.polynomial.legendre.legval(z, c)


@pytest.mark.parametrize("two_d", [False, True])
def test_basis_is_orthonormal_legendre(two_d):
    M = 5
    p = dict(eps0_lo=0.05, eps0_hi=0.15, M=M, Q1=M + 1, N=4)
    if two_d:
        p.update(Ex_lo=1000.0, Ex_hi=10000.0)
    o = O.Oracle(p)
    xg, wg = np.polynomial.legendre.leggauss(24)
    wg = wg / 2.0
    if not two_d:
        V = np.array([o.psi_at([z]) for z in xg])           # [nq, P]
        for h in range(o.P):
            assert np.allclose(V[:, h], _onb(h, xg), atol=1e-13)
        G = (V * wg[:, None]).T @ V
    else:
        pts = [(a, b) for a in xg for b in xg]
        ww = np.array([wa * wb for wa in wg for wb in wg])
        V = np.array([o.psi_at([a, b]) for a, b in pts])
        # graded order: (t-j, j)
        idx = [(t - j, j) for t in range(M + 1) for j in range(t + 1)]
        assert o.P == len(idx) == 21
        for h, (i1, i2) in enumerate(idx):
            ref = np.array([_onb(i1, a) * _onb(i2, b) for a, b in pts])
            assert np.allclose(V[:, h], ref, atol=1e-12)
        G = (V * ww[:, None]).T @ V
    assert np.allclose(G, np.eye(o.P), atol=1e-12)


@pytest.mark.parametrize("two_d", [False, True])
def test_projection_exact_for_degree_le_M(two_d):
    """The gPC projection (Eq. (23) coefficients by Gauss quadrature) of a polynomial of
    degree <= M returns its coefficients exactly; reconstruction returns its node values."""
    M = 5
    p = dict(eps0_lo=0.05, eps0_hi=0.15, M=M, Q1=M + 1, N=4)
    if two_d:
        p.update(Ex_lo=1000.0, Ex_hi=10000.0)
    o = O.Oracle(p)
    rng = np.random.default_rng(7)
    coef = rng.normal(size=o.P)
    xg, _ = np.polynomial.legendre.leggauss(M + 1)
    if not two_d:
        vals = sum(coef[h] * _onb(h, xg) for h in range(o.P))
    else:
        idx = [(t - j, j) for t in range(M + 1) for j in range(t + 1)]
        vals = np.array([sum(coef[h] * _onb(i1, a) * _onb(i2, b) for h, (i1, i2) in enumerate(idx))
                         for a in xg for b in xg])
    got = o.project_nodes(vals)
    assert np.allclose(got, coef, atol=1e-13)
    assert np.allclose(o.recon_nodes(coef), vals, atol=1e-13)


# ------------------------------------------------------------------------------------------
# scattering rates: closed forms of Appendix A against quadrature of the definitions (Sec. 2)
# ------------------------------------------------------------------------------------------
def _rates_by_quadrature(kx, ky, eps0, T=300.0):
    """Gamma_nu(k) = int S_nu(k, k') dk' over a Cartesian k' grid, the Dirac delta replaced by a
    narrow Gaussian, with the matrix elements of Eqs. (6)-(9) and Table 1 (SI units).  Reading:
    the prefactor of Eq. (7) is 2/(2 pi)^2 as in Appendix A."""
    t1 = _table1()
    e = 1.602176634e-19
    hbar = 6.582119569e-16 * e
    kT = 8.617333262e-5 * T * e
    vF = t1["vF"] * 1e-2
    sig = t1["sigma_m"] * 1e-3 / 1e-4
    vp = t1["v_p"] * 1e-2
    Dac = t1["D_ac"] * e
    DO = t1["D_O"] * e * 1e2
    DK = t1["D_K"] * e * 1e2
    hwO = t1["hw_O"] * e
    hwK = t1["hw_K"] * e
    wO, wK = hwO / hbar, hwK / hbar
    Ni = t1["N_i"] * 1e2
    V0 = t1["V_0"] * e * 1e-4
    a = t1["a"] * 1e-2
    nO = 1.0 / math.expm1(hwO / kT)
    nK = 1.0 / math.expm1(hwK / kT)
    e0 = eps0 * e
    W = math.pi * hbar * vF / e0
    # grid in 1/m
    L, h = 1.6e9, 1.5e6
    g = np.arange(-L, L + h / 2, h)
    KX, KY = np.meshgrid(g, g, indexing="ij")
    k = np.array([kx, ky]) * 1e9
    eps = math.sqrt((hbar * vF) ** 2 * (k @ k) + e0 ** 2)
    epsp = np.sqrt((hbar * vF) ** 2 * (KX ** 2 + KY ** 2) + e0 ** 2)
    kmod = math.hypot(*k)
    cosang = (KX * k[0] + KY * k[1]) / (np.sqrt(KX ** 2 + KY ** 2) * kmod + 1e-300)
    sE = 0.003 * e

    def delta(x):
        return np.exp(-0.5 * (x / sE) ** 2) / (math.sqrt(2 * math.pi) * sE)

    pref = 2.0 / (2 * math.pi) ** 2
    M_ac = pref * math.pi * Dac ** 2 * kT / (4 * hbar * sig * vp ** 2) * (1 + cosang)
    M_O = pref * math.pi * DO ** 2 / (sig * wO)
    M_K = pref * math.pi * DK ** 2 / (sig * wK) * (1 - cosang)
    S = {
        "ac": M_ac * delta(epsp - eps),
        "Om": M_O * (nO + 1) * delta(epsp - eps + hwO),
        "Op": M_O * nO * delta(epsp - eps - hwO),
        "Km": M_K * (nK + 1) * delta(epsp - eps + hwK),
        "Kp": M_K * nK * delta(epsp - eps - hwK),
        "edg": pref * math.pi * Ni * V0 ** 2 / (hbar * W) * np.exp(-2 * (k[0] - KX) ** 2 * a ** 2)
        * delta(epsp - eps),
    }
    return np.array([S[n].sum() * h * h * 1e-15 for n in ["ac", "Om", "Op", "Km", "Kp", "edg"]])


@pytest.mark.parametrize("kx,ky,eps0", [(0.45, 0.2, 0.1), (-0.3, 0.75, 0.15), (0.9, -0.1, 0.05),
                                        (0.12, 0.05, 0.1)])
def test_rates_match_quadrature_of_transition_rates(kx, ky, eps0):
    o = O.Oracle(dict(N=4, eps0_lo=eps0, eps0_hi=eps0))
    got = o.rates(kx, ky, eps0)
    ref = _rates_by_quadrature(kx, ky, eps0)
    for m in range(6):
        if ref[m] < 1e-9 * ref.max():
            assert got[m] == 0.0
        else:
            assert abs(got[m] - ref[m]) <= 3e-3 * ref[m], (m, got[m], ref[m])


def test_rates_detailed_balance():
    """(n+1) * DOS(final) at eps vs n * DOS at eps - hw: Gamma^-(eps) eps e^{-eps/kT} equals
    Gamma^+(eps - hw) (eps - hw) e^{-(eps-hw)/kT} (microscopic reversibility, Sec. 2)."""
    o = O.Oracle(dict(N=4))
    c = o.constants()
    hvF, kT = c["hvF"], c["kT"]
    e0 = 0.1
    for eps in [0.35, 0.5, 0.8]:
        for m_em, m_ab, hw in [(1, 2, c["hwO"]), (3, 4, c["hwK"])]:
            k1 = math.sqrt(eps ** 2 - e0 ** 2) / hvF
            eps2 = eps - hw
            k2 = math.sqrt(eps2 ** 2 - e0 ** 2) / hvF
            g1 = o.rates(k1, 0.0, e0)[m_em]
            g2 = o.rates(k2, 0.0, e0)[m_ab]
            lhs = g1 * eps * math.exp(-eps / kT)
            rhs = g2 * eps2 * math.exp(-eps2 / kT)
            assert abs(lhs - rhs) <= 1e-12 * lhs


@pytest.mark.parametrize("beta", [0.0, 0.01, 0.5, 2.3])
@pytest.mark.parametrize("c", [-1.0, -0.3, 0.0, 0.7, 1.0])
def test_edge_integral(beta, c):
    ref, _ = si.quad(lambda t: math.exp(-beta * (math.cos(t) - c) ** 2), 0, 2 * math.pi,
                     epsabs=1e-14, epsrel=1e-13, limit=200)
    assert abs(O.edge_T(beta, c) - ref) <= 1e-12 * ref
    if beta == 0.0:
        assert O.edge_T(beta, c) == pytest.approx(2 * math.pi, abs=1e-14)


# ------------------------------------------------------------------------------------------
# angle samplers (final states h^1..h^6 of Sec. 3)
# ------------------------------------------------------------------------------------------
def test_ac_and_k_angles_invert_their_cdfs():
    us = (np.arange(2000) + 0.5) / 2000
    for u in us:
        t = O.angle_ac(u)
        assert abs((t + math.sin(t)) / (2 * math.pi) - u) < 1e-14
        t = O.angle_k(u)
        assert abs((t - math.sin(t)) / (2 * math.pi) - u) < 1e-14


@pytest.mark.parametrize("beta,c", [(2.0, 0.6), (0.5, -0.2), (0.005, 0.9)])
def test_edge_angle_follows_its_density(beta, c):
    dens = lambda t: math.exp(-beta * (c - math.cos(t)) ** 2)
    Z, _ = si.quad(dens, 0, 2 * math.pi, limit=200)
    us = (np.arange(400) + 0.5) / 400
    for u in us:
        t = O.angle_edge(beta, c, u)
        cdf, _ = si.quad(dens, 0, t, limit=200)
        # the CDF is interpolated linearly between the 64 trapezoid points
        assert abs(cdf / Z - u) < 2e-3 * max(beta, 0.05)


# ------------------------------------------------------------------------------------------
# Fermi-Dirac initial state and density (Sec. 2, Eq. (13))
# ------------------------------------------------------------------------------------------
def _fd_int(eps0, mu, kT, hi=None):
    f = lambda x: x / (1.0 + math.exp(min((x - mu) / kT, 700.0)))
    top = hi if hi is not None else max(mu, eps0) + 80 * kT
    pts = [mu] if eps0 < mu < top else None
    v, _ = si.quad(f, eps0, top, points=pts, epsabs=0, epsrel=1e-13, limit=400)
    return v


@pytest.mark.parametrize("eps0,mu", [(0.05, 0.4), (0.15, 0.4), (0.1, 0.2), (0.3, 0.2), (0.1, -0.4)])
def test_fd_integral_and_inverse_cdf(eps0, mu):
    kT = 8.617333262e-5 * 300
    tot = O.fd_total(eps0, mu, kT)
    ref = _fd_int(eps0, mu, kT)
    assert abs(tot - ref) <= 1e-10 * ref
    for u in [2.0 ** -24, 0.01, 0.3, 0.5, 0.77, 0.999, 1 - 2.0 ** -24]:
        e = O.fd_sample(eps0, mu, kT, u)
        part = _fd_int(eps0, mu, kT, hi=e)
        assert abs(part / ref - u) < 1e-9


def test_fd_zero_temperature_limit():
    # int_{eps0}^{mu} x dx = (mu^2 - eps0^2)/2 when kT -> 0
    assert abs(O.fd_total(0.1, 0.4, 1e-7) - (0.16 - 0.01) / 2) < 1e-9


def test_density_table():
    o = O.Oracle(dict(N=4, eps0_lo=0.05, eps0_hi=0.15, M=3, Q1=4))
    t = o.tables()
    c = o.constants()
    for q in range(o.Q):
        ref = 2.0 / (math.pi * c["hvF"] ** 2) * _fd_int(t["eps0"][q], 0.4, c["kT"]) * 1e18
        assert abs(t["n"][q] - ref) <= 1e-10 * ref


def test_gauss_nodes_map_parameters_affinely():
    o = O.Oracle(dict(N=4, eps0_lo=0.05, eps0_hi=0.15, Ex_lo=1000.0, Ex_hi=10000.0, M=5, Q1=6))
    t = o.tables()
    xg, wg = np.polynomial.legendre.leggauss(6)
    q = 0
    for a, wa in zip(xg, wg):
        for b, wb in zip(xg, wg):
            assert abs(t["eps0"][q] - (0.05 + 0.05 * (a + 1))) < 1e-15
            assert abs(t["Ex"][q] - (1000.0 + 4500.0 * (b + 1))) < 1e-11
            assert abs(t["w"][q] - wa * wb / 4) < 1e-15
            q += 1
