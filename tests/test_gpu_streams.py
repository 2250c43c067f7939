"""Contexts on different CUDA streams: concurrent stepping, and contexts created while a dropped
context's work is still queued, give exactly the trajectories of solo runs (the binding allocates a
context's buffers on the context's own stream, so the caching allocator orders block reuse behind
the work queued there)."""
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


def _solo(p, steps):
    from paper_2404_19602_gb300 import pgc

    s = pgc.Simulation(p, max_outputs=4)
    s.step(steps, 0)
    k = s.state()
    s.close()
    return k


def test_concurrent_contexts_on_two_streams():
    from paper_2404_19602_gb300 import pgc

    pa = W.scaled(W.GAP_UQ_1E6, N=40000, stream_id=0)
    pb = W.scaled(W.GAP_UQ_1E6, N=25000, stream_id=1, Ex_lo=9000.0, Ex_hi=9000.0)
    ka, kb = _solo(pa, 24), _solo(pb, 24)
    a = pgc.Simulation(pa, max_outputs=4, stream=torch.cuda.Stream())
    b = pgc.Simulation(pb, max_outputs=4, stream=torch.cuda.Stream())
    for _ in range(4):                     # interleaved, asynchronous on two streams
        a.step(6, 0)
        b.step(6, 0)
    assert np.array_equal(a.state(), ka)
    assert np.array_equal(b.state(), kb)
    a.close()
    b.close()


def test_context_created_while_dropped_work_is_queued():
    """A context dropped with its work still queued on the default stream, then a new context on
    another stream: the new one must not receive memory the old work still writes."""
    from paper_2404_19602_gb300 import pgc

    p = W.scaled(W.GAP_UQ_1E6, N=30000, seed=9)
    ref = _solo(p, 15)
    for _ in range(3):
        old = pgc.Simulation(W.scaled(p, N=200000), max_outputs=4)
        old.step(20, 0)                    # queued, not synchronised
        del old
        new = pgc.Simulation(p, max_outputs=4, stream=torch.cuda.Stream())
        new.step(15, 0)
        assert np.array_equal(new.state(), ref)
        new.close()
