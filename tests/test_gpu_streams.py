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


@pytest.mark.parametrize("prec,split", [("fp32", 0), ("fp64", 0), ("fp32", 1)])
def test_native_state_transfer_round_trips(prec, split):
    """pgc_get_state_native / pgc_set_state_native: a checkpoint of context a at step 15,
    uploaded into context b at the same step (same key, different history), makes b continue
    bit-identically to a.  The Pauli normaliser is the current maximum here, so that it does
    not depend on the history either."""
    from paper_2404_19602_gb300 import pgc

    p = W.scaled(W.GAP_UQ_1E6, N=20001, precision=prec, splitting=split, pauli_norm=1)
    a = pgc.Simulation(p, max_outputs=4)
    b = pgc.Simulation(p, init_khat=0.9 * a.state(), max_outputs=4)
    a.step(15, 0)
    b.step(15, 0)
    assert not np.array_equal(a.state(), b.state())
    ck = a.state_native()
    assert ck.is_pinned() and ck.numel() == pgc.pgc_query_sizes(a.cfg)["state_bytes"]
    b.set_state_native(ck)
    assert np.array_equal(b.state_native().numpy(), ck.numpy())
    assert np.array_equal(b.hist()[0], a.hist()[0])
    a.step(15, 0)
    b.step(15, 0)
    assert np.array_equal(a.state(), b.state())
    assert a.counters()["changed"] > 0
    a.close()
    b.close()
