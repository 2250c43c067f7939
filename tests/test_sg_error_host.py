"""Host logic of the Test 3 / Test 4 studies (no GPU): the L2(I_z) rule, and the map from a point
z of the random input to the deterministic workload that Algorithm 1 runs at that point (MC-MC),
checked against the oracle's band minimum and field at its quadrature nodes."""
import numpy as np
import pytest

import oracle as O
from paper_2404_19602_gb300 import sg_error as SG
from paper_2404_19602_gb300 import workloads as W


def test_l2_rule_is_the_uniform_law_and_exact_for_polynomials():
    z, w = SG.l2_rule(64)
    assert abs(w.sum() - 1.0) < 1e-14
    for deg in (0, 2, 10, 127):
        exact = 1.0 / (deg + 1) if deg % 2 == 0 else 0.0     # mean of z^deg under U[-1, 1]
        assert abs((w * z ** deg).sum() - exact) < 1e-13


@pytest.mark.parametrize("base", ["width", "field", "gap"])
def test_deterministic_point_matches_the_oracle_nodes(base):
    p = {"width": W.TEST3_WIDTH_1E4, "field": W.TEST3_FIELD_1E4, "gap": W.GAP_UQ_1E6}[base]
    t = O.Oracle(W.scaled(p, N=1)).tables()
    for q, zq in enumerate(t["z"][:, 0]):
        d = SG.deterministic_at(p, float(zq))
        td = O.Oracle(W.scaled(d, N=1)).tables()
        assert td["z"].shape[1] == 0                       # no random input left
        assert td["eps0"][0] == pytest.approx(t["eps0"][q], rel=1e-15)
        assert td["Ex"][0] == pytest.approx(t["Ex"][q], rel=1e-15)


def test_degrees_are_the_compiled_ones():
    assert SG.DEGREES[0] == 0 and SG.DEGREES[-1] == 30 and list(SG.DEGREES) == sorted(SG.DEGREES)
