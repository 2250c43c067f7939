"""Pipelined step (one fused launch per step: the collider work of step n - 1, carrying its
particles on into step n, beside the streaming work of step n) against the two-launch form of
the same steps: the trajectories, histograms and event counters are identical, the moments agree
to the summation order of the FP32 warp sums (in the FP64 mode up to FP64 rounding)."""
import numpy as np
import pytest

from paper_2404_19602_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19602_gb300 import build

    build.build()


def _run(p, calls, every, pipeline):
    """calls: list of step counts of consecutive pgc_step calls."""
    from paper_2404_19602_gb300 import pgc

    total = sum(calls)
    s = pgc.Simulation(p, max_outputs=total // max(every, 1) + 2)
    s.set_pipeline(pipeline)
    for n in calls:
        s.step(n, every)
    out = dict(state=s.state(), hist=s.hist()[0], moments=s.moments(), counters=s.counters())
    s.close()
    return out


def _compare(a, b, rtol):
    assert np.array_equal(a["state"], b["state"])
    assert np.array_equal(a["hist"], b["hist"])
    for k in ("attempts", "changed", "rejected", "capped", "out_of_grid", "queued", "steps"):
        assert a["counters"][k] == b["counters"][k], (k, a["counters"][k], b["counters"][k])
    ma, mb = a["moments"], b["moments"]
    assert np.array_equal(ma["t_fs"], mb["t_fs"])
    assert np.allclose(ma["nodes"], mb["nodes"], rtol=rtol, atol=1e-12 * np.abs(mb["nodes"]).max())
    assert np.allclose(ma["mean"], mb["mean"], rtol=rtol, atol=1e-12 * np.abs(mb["mean"]).max())


CASES = [
    ("det_fp64", W.scaled(W.DET_FP64_1E4, N=7001), [40, 1, 23], 5, 1e-12),
    ("gap_fp32", W.scaled(W.GAP_UQ_1E6, N=50001), [2, 37, 1, 20], 10, 2e-5),
    ("gap_fp64", W.scaled(W.GAP_UQ_1E6, N=20000, precision="fp64"), [30], 1, 1e-12),
    ("gap_current_max_fp32", W.scaled(W.GAP_UQ_1E6, N=40000, pauli_norm=1), [31], 10, 2e-5),
    ("gap_field_fp32", W.scaled(W.GAP_FIELD_UQ_4E6, N=30001), [25, 3], 7, 2e-5),
]


@pytest.mark.parametrize("name,p,calls,every,rtol", CASES, ids=[c[0] for c in CASES])
def test_pipelined_equals_two_launch_form(name, p, calls, every, rtol):
    a = _run(p, calls, every, pipeline=True)
    b = _run(p, calls, every, pipeline=False)
    assert b["counters"]["queued"] > 0 and b["counters"]["changed"] > 0
    _compare(a, b, rtol)


def test_pipeline_switch_between_calls():
    """Calls with the pipeline on and off may alternate on one context."""
    from paper_2404_19602_gb300 import pgc

    p = W.scaled(W.GAP_UQ_1E6, N=30000)
    ref = _run(p, [12, 12, 12], 4, pipeline=False)
    s = pgc.Simulation(p, max_outputs=20)
    for k, on in enumerate([True, False, True]):
        s.set_pipeline(on)
        s.step(12, 4)
    got = dict(state=s.state(), hist=s.hist()[0], moments=s.moments(), counters=s.counters())
    s.close()
    _compare(got, ref, 2e-5)


def test_pipeline_unavailable_for_36_nodes_fp64():
    """The fused kernel's two argument blocks exceed the parameter space for P = 21, Q = 36 in FP64."""
    from paper_2404_19602_gb300 import pgc

    s = pgc.Simulation(W.scaled(W.GAP_FIELD_UQ_4E6, N=1000, precision="fp64"), max_outputs=4)
    with pytest.raises(pgc.PgcError):
        s.set_pipeline(True)
    s.set_pipeline(False)
    s.step(3, 0)
    s.close()


@pytest.mark.parametrize("N", [1, 33, 1023, 1025, 4 * 1024 * 3 + 7])
def test_pipelined_ragged_sizes(N):
    """Ensembles smaller than one phase-1 tile, around a tile edge and ragged: same results as the
    two-launch form, moments on every step."""
    p = W.scaled(W.GAP_UQ_1E6, N=N, precision="fp64")
    a = _run(p, [9, 2], 1, pipeline=True)
    b = _run(p, [9, 2], 1, pipeline=False)
    _compare(a, b, 1e-12)
