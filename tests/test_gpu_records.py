"""Moment records are reduced beside the following step launches (a second stream, partial-sum
slots rotating mod 3): a record depends only on the state of its step, so runs that record every
1, 2 or 3 steps, pipelined or as two launches per step, split into several step calls, give the
same records at the steps they share (up to the summation order of the partial sums)."""
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


def _records(p, every, pipeline, calls):
    from paper_2404_19602_gb300 import pgc

    s = pgc.Simulation(p, max_outputs=64)
    if pipeline is not None:
        s.set_pipeline(pipeline)
    for n in calls:
        s.step(n, every)
    m = s.moments()
    s.close()
    return m


def _at(m, steps_fs):
    idx = [int(np.flatnonzero(np.isclose(m["t_fs"], t))[0]) for t in steps_fs]
    return {k: m[k][idx] for k in ("nodes", "mean", "var")}


# FP32: the two forms group the particles of the FP32 pass sums differently (as in the
# pipelined-vs-two-launch test); FP64 sums agree to rounding.  A record reduced from the partials
# of another step (a slot three steps off) differs by far more than either tolerance.
@pytest.mark.parametrize("name,p,pipes,rtol", [
    ("gap_fp32", W.scaled(W.GAP_UQ_1E6, N=20011), (True, False), 2e-5),
    ("gap_fp64", W.scaled(W.GAP_UQ_1E6, N=8000, precision="fp64"), (True, False), 1e-11),
    ("gap_field_fp32", W.scaled(W.GAP_FIELD_UQ_4E6, N=6001), (None,), 2e-5),
])
def test_records_independent_of_recording_pattern(name, p, pipes, rtol):
    calls = [5, 1, 6, 6]                      # 18 steps in four calls (joins, short calls)
    shared = [6.0 * k * p["dt_fs"] for k in (1, 2, 3)]
    ref = None
    for pipe in pipes:
        for every in (1, 2, 3):
            got = _at(_records(p, every, pipe, calls), shared)
            if ref is None:
                ref = got
                continue
            for k in ("nodes", "mean", "var"):
                scale = np.abs(ref[k]).max()
                np.testing.assert_allclose(got[k], ref[k], rtol=rtol, atol=1e-12 * scale,
                                           err_msg="%s every=%d pipeline=%s %s" % (name, every, pipe, k))
