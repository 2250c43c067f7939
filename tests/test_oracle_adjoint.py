"""Pin of the oracle's pathwise tangents (the reference gradient of the adjoint): central finite
differences with common random numbers, at a step small enough that no discrete event changes
(checked with the event counters), reproduce the tangents."""
import numpy as np
import pytest

import oracle as O
from paper_2404_19602_gb300 import workloads as W

KEYS = ["Ex_lo", "Ex_hi", "eps0_lo", "eps0_hi"]


def _perturbed(base, t, dv):
    p = dict(base)
    key = KEYS[t]
    pair = ("Ex_lo", "Ex_hi") if t < 2 else ("eps0_lo", "eps0_hi")
    if base[pair[0]] == base[pair[1]]:  # deterministic input: move the common value
        p[pair[0]] += dv
        p[pair[1]] += dv
        return p, 2.0  # each endpoint carries half of the derivative of the common value
    p[key] += dv
    return p, 1.0


@pytest.mark.parametrize("base", [W.scaled(W.DET_FP64_1E4, N=300), W.scaled(W.GAP_UQ_1E6, N=200),
                                  W.scaled(W.GAP_FIELD_UQ_4E6, N=60)], ids=["det", "gap", "gap_field"])
def test_tangents_equal_event_preserving_central_differences(base):
    steps, every, window = 40, 5, 20
    _, grad = O.Oracle(base).tangent_run(steps, every, window)
    for t in range(4):
        h = 1e-7 * abs(base[KEYS[t]])
        pp, f = _perturbed(base, t, +h)
        pm, _ = _perturbed(base, t, -h)
        op, om = O.Oracle(pp), O.Oracle(pm)
        vp = op.window_objective(steps, every, window)
        vm = om.window_objective(steps, every, window)
        cp, cm = op.counters(), om.counters()
        assert all(cp[k] == cm[k] for k in ("attempts", "real", "rejected")), "an event changed; use a smaller h"
        fd = (vp - vm) / (2 * h) / f
        for o in range(2):
            if grad[o, t] == 0.0 and fd[o] == 0.0:
                continue
            assert abs(fd[o] - grad[o, t]) <= 2e-5 * max(abs(grad[o, t]), 1e-30) + 1e-9, (t, o, fd[o], grad[o, t])
