"""Oracle pins of the Strang splitting T_{dt/2} C_dt T_{dt/2} (Sec. 3 names higher-order
splittings as possible; the paper's scheme is the Lie splitting C_dt T_dt).

Strang over n steps is T_{dt/2} (C_dt T_dt)^{n-1} C_dt T_{dt/2}: the Lie recursion run from the
initial state moved by half a drift, and moved back by half a drift at the end.  Without the
Pauli test the collision step does not look at the histogram, so the two runs must agree to
rounding with the same random numbers, whatever the collisions do.  With the Pauli test, the
Strang run looks the histogram up at half the drift offset, and the two differ."""
import numpy as np

import oracle as O
from paper_2404_19602_gb300 import workloads as W

HALF = lambda o: 0.5 * o.tables()["dhat"]


def _shift(khat, dx):
    k = khat.copy()
    k[0] += dx[:, None]
    return k


def _pair(p, steps):
    s = O.Oracle(dict(p, splitting=1))
    k0 = s.state()
    lie = O.Oracle(p, init_khat=_shift(k0, HALF(s)))
    s.step(steps, steps)
    lie.step(steps, steps)
    return s, lie


def test_strang_is_the_half_drift_conjugate_of_lie_without_pauli():
    for base in (W.GAP_UQ_1E6, W.GAP_FIELD_UQ_4E6, W.DET_FP64_1E4):
        p = W.scaled(base, N=400 if base is W.GAP_FIELD_UQ_4E6 else 2000, pauli_norm=2)
        s, lie = _pair(p, 60)
        want = _shift(lie.state(), -HALF(s))
        got = s.state()
        assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max()
        c_s, c_l = s.counters(), lie.counters()
        assert c_s["attempts"] == c_l["attempts"] > 0 and c_s["real"] == c_l["real"]


def test_strang_differs_from_the_conjugate_with_pauli():
    p = W.scaled(W.GAP_UQ_1E6, N=4000)
    s, lie = _pair(p, 80)
    want = _shift(lie.state(), -HALF(s))
    assert np.abs(s.state() - want).max() > 1e-6        # the lookups moved by half a drift
    assert s.counters()["rejected"] > 0


def test_ballistic_strang_equals_the_closed_form():
    p = W.scaled(W.GAP_UQ_1E6, N=500, mech_mask=0, splitting=1)
    o = O.Oracle(p)
    k0 = o.state()
    o.step(100, 100)
    want = _shift(k0, -100 * o.tables()["dhat"])
    assert np.abs(o.state() - want).max() <= 1e-12 * np.abs(want).max()


def test_strang_moments_at_t0_and_counts_unchanged():
    """The initial record is the same for both splittings, and N is conserved."""
    p = W.scaled(W.GAP_UQ_1E6, N=1500)
    a, b = O.Oracle(p), O.Oracle(dict(p, splitting=1))
    a.step(20, 10)
    b.step(20, 10)
    ma, mb = a.moments(), b.moments()
    assert np.array_equal(ma["mean"][0], mb["mean"][0])
    H, _ = b.hist()
    assert (H.reshape(b.Q, -1).sum(axis=1) + 0 <= p["N"]).all()
    assert np.abs(ma["mean"][-1] - mb["mean"][-1]).max() > 0
