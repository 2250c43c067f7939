"""Batched sweep (pgc_batch_*): every case of a batch follows exactly the trajectory of its
standalone run (same Philox streams, same arithmetic), with and without CUDA-graph replay and
for any tile size the autotuner picks."""
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


def _cases(prec, base=W.GAP_UQ_1E6, ns=(3000, 5000, 1000, 7001)):
    out = []
    for c, n in enumerate(ns):
        E = 1000.0 + 6000.0 * c
        w = 0.02 + 0.05 * c
        out.append(W.scaled(base, N=n, Ex_lo=E, Ex_hi=E, eps0_lo=0.1 - w / 4, eps0_hi=0.1 + w / 4,
                            precision=prec, stream_id=c, seed=7))
    return out


def _single(p, steps, every):
    from paper_2404_19602_gb300 import pgc

    s = pgc.Simulation(p, max_outputs=steps // max(every, 1) + 2)
    s.step(steps, every)
    return s.state(), s.moments(), s.hist()[0], s.counters()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_cases_equal_standalone_runs(prec, use_graph):
    from paper_2404_19602_gb300 import pgc

    cases = _cases(prec)
    steps, every = 40, 10
    b = pgc.BatchSimulation(cases, max_outputs=steps // every + 2, tile=2048)
    b.step(steps, every, use_graph=use_graph)
    torch.cuda.synchronize()
    rtol = 1e-9 if prec == "fp64" else 1e-5
    for p, sim in zip(cases, b.sims):
        ks, ms, hs, cs = _single(p, steps, every)
        assert np.array_equal(sim.state(), ks), p["stream_id"]
        assert np.array_equal(sim.hist()[0], hs), p["stream_id"]
        mb = sim.moments()
        assert np.array_equal(mb["t_fs"], ms["t_fs"])
        # FP32 warp sums grouped differently (batch tiles vs the pipelined standalone step):
        # rounding ~1e-7 of the column's magnitude, which a near-zero column (V_y) shows as a
        # large relative error
        scale = np.abs(ms["nodes"]).max(axis=(0, 1), keepdims=True)
        assert np.allclose(mb["nodes"], ms["nodes"], rtol=rtol, atol=(1e-13 if prec == "fp64" else 1e-6) * scale)
        cb = sim.counters()
        for k in ("attempts", "changed", "rejected", "capped", "steps"):
            assert cb[k] == cs[k], (k, cb[k], cs[k])
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_cases_against_oracle(prec):
    """Each case of an uneven batch (different fields and band-minimum intervals, ragged sizes)
    against the FP64 CPU oracle run of that case alone (Algorithm 2 of Sec. 4.1 per case): in
    FP64 the same decisions and states to rounding, in FP32 the moments within 1e-3."""
    import oracle as O
    from paper_2404_19602_gb300 import pgc

    O.build()
    cases = _cases(prec, ns=(2000, 3001, 777))
    steps, every = 60, 10
    b = pgc.BatchSimulation(cases, max_outputs=steps // every + 2, tile=1024)
    b.step(steps, every)
    torch.cuda.synchronize()
    for p, sim in zip(cases, b.sims):
        o = O.Oracle(p)
        o.step(steps, every)
        mb, mo = sim.moments(), o.moments()
        assert np.allclose(mb["t_fs"], mo["t_fs"])
        tol = 1e-9 if prec == "fp64" else 1e-3
        for comp in (0, 2, 3):
            for kind in ("mean", "var"):
                a, r = mb[kind][:, comp], mo[kind][:, comp]
                err = np.abs(a - r).max() / max(np.abs(r).max(), 1e-300)
                assert err <= tol, (p["stream_id"], kind, comp, err)
        g, r = sim.state(), o.state()
        diverged = (np.abs(g - r).max(axis=(0, 1)) > (1e-9 if prec == "fp64" else 1e-4) * np.abs(r).max()).sum()
        assert diverged <= (0 if prec == "fp64" else 2), diverged
        if prec == "fp64":
            cb, co = sim.counters(), o.counters()
            assert cb["attempts"] == co["attempts"] and cb["rejected"] == co["rejected"]
    b.close()


@pytest.mark.parametrize("base", ["gap", "gap_field"])
def test_batch_autotune_keeps_trajectories(base):
    """The autotuner's candidates (tile, block size, particles per thread, both grids) advance the
    cases; afterwards every case still equals its standalone run, the chosen configuration is a
    valid one, and a later batch of the same kind starts from it."""
    from paper_2404_19602_gb300 import pgc

    if base == "gap":
        cases = _cases("fp32")
    else:   # two random inputs (21 coefficients on 6 x 6 nodes), uneven sizes
        cases = [W.scaled(W.GAP_FIELD_UQ_4E6, N=n, Ex_lo=1000.0 + 1500.0 * c, Ex_hi=6000.0 + 1500.0 * c,
                          stream_id=c, seed=7) for c, n in enumerate((3000, 5000, 1000, 7001))]
    b = pgc.BatchSimulation(cases, max_outputs=8)
    tile, ms = b.autotune(2)
    lc = b.launch_config()
    assert lc["tile"] == tile and ms > 0
    assert lc["block"] in (128, 256) and lc["tile"] % (lc["block"] * lc["ppt"]) == 0
    assert lc["ppt"] in ((4, 2, 1) if base == "gap" else (1,))
    assert lc["g1_per_sm"] >= 1 and lc["g2_per_sm"] >= 2
    b.step(10, 0)
    torch.cuda.synchronize()
    steps = b.sims[0].counters()["steps"]
    for p, sim in zip(cases, b.sims):
        assert sim.counters()["steps"] == steps
        ks, _, hs, _ = _single(p, steps, 0)
        assert np.array_equal(sim.state(), ks)
        assert np.array_equal(sim.hist()[0], hs)
    b.close()
    b2 = pgc.BatchSimulation(cases, max_outputs=8)       # tile 0: the cached choice
    assert b2.launch_config() == lc
    b2.close()


def test_batch_two_random_inputs_fp64():
    from paper_2404_19602_gb300 import pgc

    cases = [W.scaled(W.GAP_FIELD_UQ_4E6, N=n, precision="fp64", stream_id=c) for c, n in enumerate((600, 257))]
    b = pgc.BatchSimulation(cases, max_outputs=4, tile=512)
    b.step(12, 6)
    torch.cuda.synchronize()
    for p, sim in zip(cases, b.sims):
        ks, ms, hs, _ = _single(p, 12, 6)
        assert np.array_equal(sim.state(), ks)
        assert np.allclose(sim.moments()["nodes"], ms["nodes"], rtol=1e-9, atol=0)
    b.close()


def test_batch_rejects_mismatched_cases():
    from paper_2404_19602_gb300 import pgc

    a = pgc.Simulation(W.scaled(W.GAP_UQ_1E6, N=100))
    c = pgc.Simulation(W.scaled(W.GAP_UQ_1E6, N=100, precision="fp64"))
    with pytest.raises(pgc.PgcError):
        pgc.pgc_batch_query_sizes([a.ctx, c.ctx])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_then_pipelined_single_steps(prec):
    """Contexts advanced by the batch and then alone (pipelined form, which keeps its own collider
    bitmaps and queue counters) follow the standalone trajectory."""
    from paper_2404_19602_gb300 import pgc

    cases = _cases(prec, ns=(3000, 1700))
    b = pgc.BatchSimulation(cases, max_outputs=8, tile=1024)
    b.step(10, 5, use_graph=True)
    torch.cuda.synchronize()
    for p, sim in zip(cases, b.sims):
        sim.set_pipeline(True)
        sim.step(12, 0)
        ks, _, hs, cs = _single(p, 22, 5)
        assert np.array_equal(sim.state(), ks), p["stream_id"]
        assert np.array_equal(sim.hist()[0], hs)
        for k in ("attempts", "changed", "rejected", "steps"):
            assert sim.counters()[k] == cs[k], k
    b.close()
