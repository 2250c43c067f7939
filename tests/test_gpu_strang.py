"""The Strang splitting T_{dt/2} C_dt T_{dt/2} on the GPU against the oracle's Strang form.

The library keeps the state half a drift ahead of the step boundary (every step is then the Lie
recursion) and moves the grid of the histograms and the observables back by half a drift; the
oracle takes the two half drifts literally.  FP64 trajectories, histograms, observables and
counters agree to rounding; the pipelined and two-launch forms are bit-identical; the state
transfer converts; the batch and adjoint entry points refuse the Strang form."""
import numpy as np
import pytest

import oracle as O
from paper_2404_19602_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19602_gb300 import build

    build.build()
    O.build()


def _pgc():
    from paper_2404_19602_gb300 import pgc

    return pgc


def _normwise(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


def _run_pair(p, steps, every):
    s = _pgc().Simulation(p, max_outputs=steps // every + 2)
    s.step(steps, every)
    o = O.Oracle(p)
    o.step(steps, every)
    return s, o


FP64 = [("det", W.scaled(W.DET_FP64_1E4, N=5000, splitting=1), 120),
        ("gap", W.scaled(W.GAP_UQ_1E6, N=3000, precision="fp64", splitting=1), 60),
        ("width", W.scaled(W.TEST2_WIDTH_1E6, N=2000, precision="fp64", splitting=1), 40),
        ("gap_field", W.scaled(W.GAP_FIELD_UQ_4E6, N=500, precision="fp64", splitting=1), 20),
        ("gap_current_max", W.scaled(W.GAP_UQ_1E6, N=2000, precision="fp64", splitting=1, pauli_norm=1), 40),
        ("field_M10", W.scaled(W.TEST3_FIELD_1E4, N=1000, M=10, Q1=11, precision="fp64", splitting=1), 40)]


@pytest.mark.parametrize("name,p,steps", FP64, ids=[c[0] for c in FP64])
def test_fp64_strang_matches_oracle(name, p, steps):
    s, o = _run_pair(p, steps, 10)
    g, r = s.state(), o.state()
    assert np.abs(g - r).max() <= 1e-9 * max(np.abs(r).max(), 1.0)
    mg, mr = s.moments(), o.moments()
    for comp in (0, 2, 3):
        assert _normwise(mg["mean"][:, comp], mr["mean"][:, comp]) <= 1e-9
    Hg, _ = s.hist()
    Hr, _ = o.hist()
    assert np.abs(Hg.astype(np.int64) - Hr.astype(np.int64)).sum() <= 2 * s.Q
    cg, cr = s.counters(), o.counters()
    assert cg["attempts"] == cr["attempts"] and cg["rejected"] == cr["rejected"] > 0
    z = np.linspace(-1.0, 1.0, 7).reshape(-1, 1) if s.d == 1 else np.array([[-0.5, 0.3], [0.9, -1.0]])
    if s.d > 0:
        obs_g = s.observe_at(z)
        obs_r = np.array([o.observe_at(zz) for zz in z])
        for comp in (0, 2, 3):
            assert _normwise(obs_g[:, comp], obs_r[:, comp]) <= 1e-9
        Zg, _ = s.reconstruct_f(z)
        Zr, _ = o.reconstruct_f(z)
        assert np.abs(Zg.astype(np.int64) - Zr.astype(np.int64)).sum() <= 2 * len(z)
    s.close()


@pytest.mark.parametrize("steps", [30, 120])
def test_fp32_strang_moments_match_oracle(steps):
    """Means within 1e-3 at any horizon; the z-variance (a few % of the mean squared, moved by
    ~1 % by one particle of 2e4 whose FP32 rounding decided a cell or a threshold differently)
    only on the short horizon; diverged particles a tiny fraction."""
    p = W.scaled(W.GAP_UQ_1E6, N=20000, splitting=1)
    s, o = _run_pair(p, steps, 10)
    mg, mr = s.moments(), o.moments()
    for comp in (0, 2, 3):
        assert _normwise(mg["mean"][:, comp], mr["mean"][:, comp]) <= 1e-3
        if steps <= 30:
            assert _normwise(mg["var"][:, comp], mr["var"][:, comp]) <= 1e-3
    g, r = s.state(), o.state()
    assert (np.abs(g - r).max(axis=(0, 1)) > 1e-4).sum() <= 0.001 * p["N"]
    s.close()


def test_strang_is_the_half_drift_conjugate_of_lie_without_pauli():
    """GPU Strang run = GPU Lie run from the state moved by half a drift, moved back (FP64)."""
    pgc = _pgc()
    p = W.scaled(W.GAP_UQ_1E6, N=4000, precision="fp64", pauli_norm=2)
    a = pgc.Simulation(dict(p, splitting=1), max_outputs=4)
    half = 0.5 * O.Oracle(W.scaled(p, N=1)).tables()["dhat"]
    k0 = a.state()
    k1 = k0.copy()
    k1[0] += half[:, None]
    b = pgc.Simulation(p, init_khat=k1, max_outputs=4)
    a.step(50, 50)
    b.step(50, 50)
    want = b.state()
    want[0] -= half[:, None]
    assert np.abs(a.state() - want).max() <= 1e-11 * np.abs(want).max()
    assert a.counters()["attempts"] == b.counters()["attempts"] > 0
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_strang_pipelined_equals_two_launch_form(prec):
    pgc = _pgc()
    out = []
    for on in (True, False):
        s = pgc.Simulation(W.scaled(W.GAP_UQ_1E6, N=30001, precision=prec, splitting=1), max_outputs=8)
        s.set_pipeline(on)
        s.step(25, 5)
        out.append((s.state(), s.hist()[0], s.counters(), s.moments()["mean"]))
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert out[0][2]["changed"] == out[1][2]["changed"] > 0
    assert np.allclose(out[0][3], out[1][3], rtol=2e-5, atol=1e-12 * np.abs(out[1][3]).max())


def test_strang_state_transfer_continues_the_run():
    """pgc_get_state returns the state at the step boundary; uploading it and continuing gives
    the uninterrupted run (FP64, to rounding of the half-drift conversion)."""
    pgc = _pgc()
    p = W.scaled(W.GAP_UQ_1E6, N=3000, precision="fp64", splitting=1)
    ref = pgc.Simulation(p, max_outputs=4)
    ref.step(40, 0)
    a = pgc.Simulation(p, max_outputs=4)
    a.step(20, 0)
    k = a.state()
    o = O.Oracle(p)
    o.step(20, 0)
    assert np.abs(k - o.state()).max() <= 1e-9 * np.abs(k).max()
    a.set_state(k)
    a.step(20, 0)
    assert np.abs(a.state() - ref.state()).max() <= 1e-9 * np.abs(ref.state()).max()
    a.close()
    ref.close()


def test_batch_and_adjoint_refuse_strang():
    pgc = _pgc()
    with pytest.raises(pgc.PgcError):
        pgc.BatchSimulation([W.scaled(W.GAP_UQ_1E6, N=1000, splitting=1)])
    s = pgc.Simulation(W.scaled(W.GAP_UQ_1E6, N=1000, splitting=1), max_outputs=4)
    with pytest.raises(pgc.PgcError):
        n = pgc.pgc_adjoint_query_sizes(s.ctx, 10, 5)
        work = torch.empty(max(n, 256), dtype=torch.uint8, device="cuda")
        pgc.pgc_adjoint(s.ctx, 10, 5, 5, 5, [1.0, 0.0], work.data_ptr())
    s.close()
