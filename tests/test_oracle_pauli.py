"""Pins of the oracle's Pauli test and of the histogram it reads (arXiv:2404.19602, Sec. 3,
Eq. (22) for the deterministic scheme and Eq. (27) for the stochastic-Galerkin scheme: a candidate
k' is accepted iff f^n < eta in the cell of k', with f^n = N_rl / max N_rl of Eq. (24)).

The histogram f^n is planted with a test hook, so the expected outcome of every collision is
known without re-deriving the candidates:

* every cell saturated (f = 1): every in-grid candidate is rejected, so each particle only
  drifts (the ballistic closed form of Eq. (17));
* every cell empty (f = 0): every candidate is accepted, so the run equals the one with the
  Pauli test switched off, bit for bit (same Philox numbers);
* f = 1/4 or 3/4 everywhere: the rejected share of the real-mechanism selections is f
  (binomial error);
* the current-maximum normaliser divides by the largest count of the current histogram;
* a half-plane histogram (f = 1 for k_x >= 0, f = 0 below) with a strong field: the grid moves
  with the drift (Sec. 3), so a candidate is looked up at cell(k' + (e/hbar) E dt) (Lie) or
  cell(k' + (e/hbar) E dt / 2) (Strang); in both forms every accepted final state then lies
  left of -(e/hbar) E dt, and the accepted states reach that boundary;
* outside [-Lk, Lk]^2 the distribution is zero (f = 0): with every in-grid cell saturated,
  only candidates that leave the grid are accepted.

A flipped inequality, a wrong sign or size of the shift, a wrong normaliser or a lost boundary
rule fails one of these.  No GPU.
"""
import math

import numpy as np
import pytest

import oracle as O

HBAR_EVFS = 6.582119569e-16 * 1e15   # hbar in eV fs
HVF = 0.6582119569                   # hbar vF in eV nm (vF = 1e6 m/s)


def _drift(E_Vcm, dt_fs):
    """(e/hbar) E dt in nm^-1 (E in V/cm, dt in fs)."""
    return E_Vcm * 1e-7 * dt_fs / HBAR_EVFS


def _ring_states(n, e_lo, e_hi, eps0, seed):
    """n wave-vectors with energies uniform in [e_lo, e_hi] eV and uniform angles."""
    rng = np.random.default_rng(seed)
    eps = rng.uniform(e_lo, e_hi, n)
    th = rng.uniform(0.0, 2.0 * math.pi, n)
    km = np.sqrt(eps ** 2 - eps0 ** 2) / HVF
    return km * np.cos(th), km * np.sin(th)


def _oracle(kx, ky, **p):
    """Oracle whose particles have node values k(z_q) = (kx, ky) at every node (only the
    coefficient of Psi_0 = 1 is set)."""
    base = dict(N=kx.size, eps0_lo=0.1, eps0_hi=0.1, Ex_lo=5000.0, Ex_hi=5000.0, M=0, Q1=1,
                pauli_norm=O.PAULI_INITIAL_MAX)
    base.update(p)
    o0 = O.Oracle(dict(base, N=1))
    P = o0.P
    k = np.zeros((2, P, kx.size))
    k[0, 0] = kx
    k[1, 0] = ky
    return O.Oracle(base, init_khat=k)


def _nodes(o):
    """Node values [2][Q][N] of the oracle's state (reconstruction with the oracle's tables)."""
    psi = o.tables()["psi"]
    k = o.state()
    return np.stack([psi @ k[0], psi @ k[1]])


def _passes(o, npass):
    idx = np.arange(o.N)
    for n in range(npass):
        o.set_step(n)
        o.step_particles(idx)


CASES = {
    # deterministic scheme (Algorithm 1)
    "det": dict(M=0, Q1=1),
    # stochastic Galerkin with a random field (every node has its own drift)
    "field": dict(M=5, Q1=6, Ex_lo=2000.0, Ex_hi=8000.0),
}


def _cells(k, Lk, dk, Nk):
    r = np.floor((k[0] + Lk) / dk)
    l = np.floor((k[1] + Lk) / dk)
    ok = (r >= 0) & (l >= 0) & (r < Nk) & (l < Nk)
    return r.astype(np.int64), l.astype(np.int64), ok


def test_grid_constants():
    o = O.Oracle(dict(N=10))
    c = o.constants()
    Lk = 5.0 / HVF                     # Lk hbar vF = 5 eV
    assert math.isclose(c["Lk"], Lk, rel_tol=1e-9)
    assert math.isclose(c["dk"], 2 * Lk / 240, rel_tol=1e-9)


@pytest.mark.parametrize("case", ["det", "gap_field_2d"])
def test_histogram_and_initial_maximum(case):
    """f^0 of Eq. (24): per node, the count of particles in each half-open cell
    floor((k + Lk) / dk), recomputed with numpy from the node values reconstructed by numpy's
    own Legendre basis; the normaliser of the initial-maximum reading is its maximum."""
    rng = np.random.default_rng(5)
    if case == "det":
        p = dict(N=5000, M=0, Q1=1)
    else:
        p = dict(N=3000, M=5, Q1=6, eps0_lo=0.05, eps0_hi=0.15, Ex_lo=1000.0, Ex_hi=10000.0)
    o0 = O.Oracle(dict(p, N=1))
    P, Q = o0.P, o0.Q
    k = np.zeros((2, P, p["N"]))
    # concentrated states (several particles per cell) plus small higher coefficients
    k[:, 0] = rng.normal(0.0, 0.25, (2, p["N"]))
    if P > 1:
        k[:, 1:] = rng.normal(0.0, 0.02, (2, P - 1, p["N"]))
    o = O.Oracle(p, init_khat=k)
    c = o.constants()
    Lk, dk, Nk = c["Lk"], c["dk"], 240
    # independent basis: orthonormal Legendre at Gauss-Legendre nodes, total degree, graded order
    x, _ = np.polynomial.legendre.leggauss(6)
    if case == "det":
        psi = np.ones((1, 1))
    else:
        def leg(h, z):
            return math.sqrt(2 * h + 1) * np.polynomial.legendre.legval(z, [0] * h + [1])
        psi = np.zeros((Q, P))
        for q1 in range(6):
            for q2 in range(6):
                j = 0
                for t in range(6):
                    for h2 in range(t + 1):
                        psi[q1 * 6 + q2, j] = leg(t - h2, x[q1]) * leg(h2, x[q2])
                        j += 1
    H, nmax = o.hist()
    for q in range(Q):
        kq = np.stack([psi[q] @ k[0], psi[q] @ k[1]])
        r, l, ok = _cells(kq, Lk, dk, Nk)
        ref = np.zeros((Nk, Nk), dtype=np.int64)
        np.add.at(ref, (r[ok], l[ok]), 1)
        assert np.array_equal(H[q].astype(np.int64), ref), q
        assert nmax[q] == ref.max() > 1
    assert o.counters()["out_of_grid"] == 0


@pytest.mark.parametrize("case", list(CASES))
def test_saturated_histogram_rejects_every_candidate(case):
    """f = 1 in every cell: eta < 1 always, so every real collision is rejected and the
    particles only drift (Eq. (17)): k = k0 - npass (e/hbar) E dt at every node."""
    dt = 20.0
    kx, ky = _ring_states(3000, 0.2, 0.6, 0.1, seed=1)
    o = _oracle(kx, ky, dt_fs=dt, **CASES[case])
    Q = o.Q
    o.set_hist(np.ones((Q, 240, 240), dtype=np.uint32))
    o.set_nmax(np.ones(Q, dtype=np.uint32))
    npass = 4
    _passes(o, npass)
    cnt = o.counters()
    assert cnt["real"] == 0
    assert cnt["rejected"] > 500
    Ex = o.tables()["Ex"]
    shift = _drift(Ex, dt)
    assert np.allclose(o.tables()["d"], shift, rtol=1e-12, atol=0)
    k = _nodes(o)
    if case == "det":   # P = Q = 1: the recon/projection of the collision loop are exact
        ref = kx.copy()
        for _ in range(npass):
            ref = ref - o.tables()["dhat"][0]
        assert o.tables()["dhat"][0] == shift[0]
        assert np.array_equal(k[0, 0], ref)
        assert np.array_equal(k[1, 0], ky)
    else:
        assert np.allclose(k[0], kx[None, :] - npass * shift[:, None], rtol=0, atol=1e-12)
        assert np.allclose(k[1], ky[None, :], rtol=0, atol=1e-12)


@pytest.mark.parametrize("case", list(CASES))
def test_empty_histogram_accepts_every_candidate(case):
    """f = 0 in every cell: eta > 0 always, so every candidate is accepted and the run equals
    the run without the Pauli test (same Philox numbers), bit for bit."""
    dt = 20.0
    kx, ky = _ring_states(3000, 0.2, 0.6, 0.1, seed=2)
    o = _oracle(kx, ky, dt_fs=dt, **CASES[case])
    off = _oracle(kx, ky, dt_fs=dt, pauli_norm=O.PAULI_OFF, **CASES[case])
    o.set_hist(np.zeros((o.Q, 240, 240), dtype=np.uint32))
    o.set_nmax(np.ones(o.Q, dtype=np.uint32))
    _passes(o, 4)
    _passes(off, 4)
    a, b = o.counters(), off.counters()
    assert a["rejected"] == 0 and b["rejected"] == 0
    assert a["real"] == b["real"] > 300
    assert a["attempts"] == b["attempts"]
    assert np.array_equal(o.state(), off.state())


@pytest.mark.parametrize("H,nmax", [(1, 4), (3, 4), (1, 2)])
def test_rejected_share_equals_f(H, nmax):
    """f = H / Nmax in every cell: a real-mechanism candidate is rejected iff eta <= f, so the
    rejected share of the real selections is f (deterministic scheme, one node)."""
    kx, ky = _ring_states(4000, 0.2, 0.6, 0.1, seed=3)
    o = _oracle(kx, ky, dt_fs=20.0)
    o.set_hist(np.full((1, 240, 240), H, dtype=np.uint32))
    o.set_nmax(np.array([nmax], dtype=np.uint32))
    _passes(o, 16)
    c = o.counters()
    n = c["real"] + c["rejected"]
    f = H / nmax
    assert n > 4000
    share = c["rejected"] / n
    assert abs(share - f) < 4.5 * math.sqrt(f * (1 - f) / n)


def test_current_maximum_normaliser():
    """CURRENT_MAX: f = N_rl / max_rl N_rl of the histogram being read (Eq. (24) at step n),
    whatever the stored initial maximum; INITIAL_MAX divides by the stored one."""
    kx, ky = _ring_states(4000, 0.2, 0.6, 0.1, seed=4)
    H = np.ones((1, 240, 240), dtype=np.uint32)
    H[0, 2, 3] = 4          # far from every candidate: only sets the current maximum
    cur = _oracle(kx, ky, dt_fs=20.0, pauli_norm=O.PAULI_CURRENT_MAX)
    cur.set_hist(H)
    cur.set_nmax(np.array([1], dtype=np.uint32))
    _passes(cur, 8)
    c = cur.counters()
    n = c["real"] + c["rejected"]
    assert abs(c["rejected"] / n - 0.25) < 4.5 * math.sqrt(0.25 * 0.75 / n)
    ini = _oracle(kx, ky, dt_fs=20.0, pauli_norm=O.PAULI_INITIAL_MAX)
    ini.set_hist(H)
    ini.set_nmax(np.array([1], dtype=np.uint32))
    _passes(ini, 8)
    c = ini.counters()
    assert c["real"] == 0 and c["rejected"] > 1000


@pytest.mark.parametrize("splitting", [0, 1])
@pytest.mark.parametrize("case", list(CASES))
def test_lookup_cell_moves_with_the_drift(case, splitting):
    """f = 1 in the cells with k_x >= 0, f = 0 below, and a field whose drift per step spans
    several cells.  The grid moves with the drift (Sec. 3): a candidate k' is looked up at
    cell(k' + s) with s = (e/hbar) E dt (Lie) or s / 2 (Strang, whose second half drift then
    follows), so every node value changed by an accepted collision ends the step with
    k_x + (e/hbar) E dt < 0, and the accepted values reach that boundary."""
    dt = 20.0
    p = dict(CASES[case])
    scale = 25.0   # field strength: drift per step ~0.3 nm^-1 (about 5 cells)
    p["Ex_lo"] = p.get("Ex_lo", 5000.0) * scale
    p["Ex_hi"] = p.get("Ex_hi", 5000.0) * scale
    kx, ky = _ring_states(12000, 0.3, 0.6, 0.1, seed=6)
    # centre the drifted states on k_x = 0 so that the candidates fall on both sides
    s_mean = _drift(0.5 * (p["Ex_lo"] + p["Ex_hi"]), dt)
    kx = kx + s_mean
    o = _oracle(kx, ky, dt_fs=dt, splitting=splitting, **p)
    Q = o.Q
    # (Strang: the oracle's step drifts by half, collides, drifts by half; an unchanged node
    # value ends at k0 - s as in the Lie form)
    H = np.zeros((Q, 240, 240), dtype=np.uint32)
    H[:, 120:, :] = 1
    o.set_hist(H)
    o.set_nmax(np.ones(Q, dtype=np.uint32))
    o.set_step(0)
    o.step_particles(np.arange(o.N))
    c = o.counters()
    assert c["real"] > 200 and c["rejected"] > 200
    s = _drift(o.tables()["Ex"], dt)                      # per node
    k = _nodes(o)
    drifted = kx[None, :] - s[:, None]
    changed = (np.abs(k[0] - drifted) > 1e-9) | (np.abs(k[1] - ky[None, :]) > 1e-9)
    assert changed.sum() > 200
    edge = (k[0] + s[:, None])[changed]
    assert edge.max() < 1e-9
    dk = o.constants()["dk"]
    assert s.min() > 2 * dk
    # the boundary is at -s, not further left: accepted values come within a tenth of s of it
    assert edge.max() > -0.1 * s.min()


def test_outside_the_grid_is_empty():
    """Zero boundary (Sec. 3): outside [-Lk, Lk]^2 the distribution is zero, so with every
    in-grid cell saturated only the candidates that leave the grid are accepted.  Optical
    absorption only (|k'| = |k| + omega/vF, uniform direction) from states just inside the
    right edge of the grid, on a hot lattice so that absorption is frequent."""
    Lk = 5.0 / HVF
    rng = np.random.default_rng(7)
    n = 3000
    kx = Lk - rng.uniform(0.02, 0.12, n)
    ky = rng.uniform(-0.5, 0.5, n)
    o = _oracle(kx, ky, dt_fs=20.0, Ex_lo=0.0, Ex_hi=0.0, mech_mask=O.OPP, T_K=3000.0)
    o.set_hist(np.ones((1, 240, 240), dtype=np.uint32))
    o.set_nmax(np.array([1], dtype=np.uint32))
    _passes(o, 1)
    c = o.counters()
    assert c["real"] > 200 and c["rejected"] > 200
    k = _nodes(o)[:, 0]
    changed = (np.abs(k[0] - kx) > 1e-12) | (np.abs(k[1] - ky) > 1e-12)
    assert changed.sum() > 200
    r, l, ok = _cells(k, o.constants()["Lk"], o.constants()["dk"], 240)
    assert not ok[changed].any()
    assert ok[~changed].all()
