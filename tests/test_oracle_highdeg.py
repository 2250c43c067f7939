"""Oracle pins at the degrees of the stochastic-Galerkin error study (Test 3, Sec. 5, degrees up
to M_ref = 30 on M + 1 Gauss nodes): the quadrature rule and the orthonormal Legendre basis
against library routines, exact projection at degree 30, and the degree-0 run (one node, the
centre of I_z) against the deterministic run at that input."""
import numpy as np
import pytest

import oracle as O
from paper_2404_19602_gb300 import workloads as W


def _onb(h, z):
    """sqrt(2h+1) P_h(z) by the library Legendre series."""
    return np.sqrt(2 * h + 1) * np.polynomial.legendre.legval(z, [0.0] * h + [1.0])


def _oracle(M, **kw):
    return O.Oracle(W.scaled(W.TEST3_WIDTH_1E4, N=kw.pop("N", 1), M=M, Q1=M + 1, **kw))


@pytest.mark.parametrize("M", [1, 10, 25, 30])
def test_rule_matches_library_gauss_legendre(M):
    t = _oracle(M).tables()
    x, w = np.polynomial.legendre.leggauss(M + 1)
    assert np.allclose(t["z"][:, 0], x, atol=2e-15)
    assert np.allclose(t["w"], w / 2.0, atol=1e-15)


def test_basis_matches_library_legendre_to_degree_30():
    o = _oracle(30)
    for z in (-1.0, -0.73, 0.0, 0.377, 0.999, 1.0):
        ref = np.array([_onb(h, z) for h in range(31)])
        assert np.allclose(o.psi_at([z]), ref, rtol=1e-12, atol=1e-12)


def test_orthonormal_under_its_own_rule_at_degree_30():
    t = _oracle(30).tables()
    G = (t["psi"] * t["w"][:, None]).T @ t["psi"]
    assert np.abs(G - np.eye(31)).max() < 1e-12


def test_projection_exact_at_degree_30():
    o = _oracle(30)
    rng = np.random.default_rng(11)
    coef = rng.normal(size=31) / np.arange(1, 32)
    x, _ = np.polynomial.legendre.leggauss(31)
    vals = sum(coef[h] * _onb(h, x) for h in range(31))
    assert np.allclose(o.project_nodes(vals), coef, atol=1e-12)
    assert np.allclose(o.recon_nodes(coef), vals, atol=1e-12)


def test_degree_zero_is_the_deterministic_run_at_the_centre():
    """M = 0: one Gauss node z = 0, W = 7 nm for W = (6.5 + z') nm, z' = (z + 1)/2 on [0, 1]."""
    g = _oracle(0, N=1500)
    d = O.Oracle(W.scaled(W.TEST3_WIDTH_1E4, N=1500, W_lo=7.0, W_hi=7.0))
    assert g.P == d.P == 1 and g.d == 1 and d.d == 0
    g.step(60, 20)
    d.step(60, 20)
    assert np.array_equal(g.state(), d.state())
    assert np.array_equal(g.moments()["mean"], d.moments()["mean"])


def _energy_curve(base, M, steps=40):
    z, w = np.polynomial.legendre.leggauss(64)
    o = O.Oracle(W.scaled(base, N=300, M=M, Q1=M + 1, mech_mask=0))
    o.step(steps, steps)
    return np.array([o.observe_at([zz])[2] for zz in z]), w / 2.0


def test_ballistic_sg_error_is_exact_for_an_affine_field():
    """Scattering off, uncertain field: every particle's k(z) = k0 - (e/hbar) E(z) t is affine in z,
    so any degree M >= 1 represents it exactly and the Test 3 error vanishes to rounding."""
    ref, w = _energy_curve(W.TEST3_FIELD_1E4, 30)
    for M in (1, 2, 5):
        e, _ = _energy_curve(W.TEST3_FIELD_1E4, M)
        assert np.sqrt(((e - ref) ** 2 * w).sum()) < 1e-13


def test_ballistic_sg_error_converges_spectrally_for_the_width():
    """Scattering off, uncertain width: k(z) depends analytically on z through the initial sampling
    at eps0(z) = pi hbar vF / W(z), so the L2(I_z) error of the energy against degree 30 falls
    geometrically with M (measured ~50x per two degrees)."""
    ref, w = _energy_curve(W.TEST3_WIDTH_1E4, 30)
    err = []
    for M in (2, 4, 6, 8):
        e, _ = _energy_curve(W.TEST3_WIDTH_1E4, M)
        err.append(np.sqrt(((e - ref) ** 2 * w).sum()))
    assert err[0] > 1e-7
    for a, b in zip(err, err[1:]):
        assert b < a / 10.0, err


@pytest.mark.parametrize("base", ["width", "gap_field"])
def test_observe_at_the_nodes_gives_the_moment_record(base):
    """The oracle's two observation routines agree: observables of the particles reconstructed at
    a quadrature node (Eq. (23) at z_q) are the node values of its moment record."""
    p = {"width": W.scaled(W.TEST3_WIDTH_1E4, N=700), "gap_field": W.scaled(W.GAP_FIELD_UQ_4E6, N=300)}[base]
    o = O.Oracle(p)
    o.step(20, 20)
    rec = o.moments()["nodes"][-1]
    for q, zq in enumerate(o.tables()["z"]):
        assert np.allclose(o.observe_at(zq), rec[q], rtol=1e-12, atol=1e-9)
