"""One-dimensional shapes of high degree (the degrees M = 0..30 of the stochastic-Galerkin error
study, Test 3 of Sec. 5) on the GPU: trajectories against the oracle in the FP64 mode, moments in
the FP32 mode, the degree-0 run against the deterministic run, the pipelined form, the study
itself against the oracle's, and its statement (the error falls as M grows)."""
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


def _deg(base, M, **kw):
    return W.scaled(base, M=M, Q1=M + 1, **kw)


def _normwise(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


def _run_pair(p, steps, every):
    s = _pgc().Simulation(p, max_outputs=steps // every + 2)
    s.step(steps, every)
    o = O.Oracle(p)
    o.step(steps, every)
    return s, o


FP64 = [("width_M1", _deg(W.TEST3_WIDTH_1E4, 1, N=1500)),
        ("width_M10", _deg(W.TEST3_WIDTH_1E4, 10, N=1500)),
        ("width_M30", _deg(W.TEST3_WIDTH_1E4, 30, N=601)),
        ("field_M4", _deg(W.TEST3_FIELD_1E4, 4, N=1500)),
        ("field_M20", _deg(W.TEST3_FIELD_1E4, 20, N=777)),
        ("gap_M12", _deg(W.GAP_UQ_1E6, 12, N=1000, dt_fs=2.5))]


@pytest.mark.parametrize("name,p", FP64, ids=[c[0] for c in FP64])
def test_fp64_trajectories_match_oracle(name, p):
    p = dict(p, precision="fp64")
    s, o = _run_pair(p, 40, 10)
    g, r = s.state(), o.state()
    assert g.shape == r.shape == (2, p["M"] + 1, p["N"])
    assert np.abs(g - r).max() <= 1e-9 * max(np.abs(r).max(), 1.0)
    mg, mr = s.moments(), o.moments()
    for comp in (0, 2, 3):
        assert _normwise(mg["mean"][:, comp], mr["mean"][:, comp]) <= 1e-9
        assert _normwise(mg["var"][:, comp], mr["var"][:, comp]) <= 1e-8
    assert s.counters()["changed"] > 0
    s.close()


def test_observations_at_degree_30_match_oracle():
    """FP64 degree-30 run: observables and the reconstructed distribution at points off the
    nodes, in passes of exactly 32 and 64 points, equal the oracle's on the same state."""
    pgc = _pgc()
    p = _deg(W.TEST3_WIDTH_1E4, 30, N=900, precision="fp64")
    s = pgc.Simulation(p, max_outputs=4)
    s.step(30, 30)
    o = O.Oracle(p, init_khat=s.state())
    for nz in (32, 64):
        z = np.random.default_rng(nz).uniform(-1.0, 1.0, size=(nz, 1))
        g = s.observe_at(z)
        r = np.array([o.observe_at(zz) for zz in z])
        for comp in (0, 2, 3):
            assert _normwise(g[:, comp], r[:, comp]) <= 1e-12
    z = np.array([[-0.95], [0.1], [0.77]])
    Hg, mg = s.reconstruct_f(z)
    Hr, mr = o.reconstruct_f(z)
    assert np.abs(Hg.astype(np.int64) - Hr.astype(np.int64)).sum() <= 2 * len(z)
    s.close()


@pytest.mark.parametrize("M", [8, 25])
def test_fp32_moments_match_oracle(M):
    """Means within 1e-3 normwise.  The variance over z is the small difference of node values
    whose decisions (Pauli, selection) FP32 rounding occasionally flips at one node and not at
    its neighbours; with 26 nodes that moves the variance of V_x by ~0.4 % (measured), so the
    variances are held to 1e-2."""
    p = _deg(W.TEST3_WIDTH_1E4, M, N=20000)
    s, o = _run_pair(p, 40, 10)
    mg, mr = s.moments(), o.moments()
    for comp in (0, 2, 3):
        assert _normwise(mg["mean"][:, comp], mr["mean"][:, comp]) <= 1e-3, comp
        assert _normwise(mg["var"][:, comp], mr["var"][:, comp]) <= 1e-2, comp
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_degree_zero_equals_deterministic_run(prec):
    pgc = _pgc()
    a = pgc.Simulation(_deg(W.TEST3_WIDTH_1E4, 0, N=3000, precision=prec), max_outputs=8)
    b = pgc.Simulation(W.scaled(W.TEST3_WIDTH_1E4, N=3000, W_lo=7.0, W_hi=7.0, M=0, Q1=1, precision=prec),
                       max_outputs=8)
    assert a.d == 1 and b.d == 0
    for s in (a, b):
        s.step(50, 25)
    assert np.array_equal(a.state(), b.state())
    # the block partial sums of the moments follow the dynamic tile assignment of the streaming
    # kernel, so two runs agree to the FP64 accumulation order only
    ma, mb = a.moments()["mean"], b.moments()["mean"]
    assert np.allclose(ma, mb, rtol=1e-12, atol=1e-12 * np.abs(mb).max())
    a.close()
    b.close()


@pytest.mark.parametrize("M", [3, 6])
def test_pipelined_equals_two_launch_form(M):
    pgc = _pgc()
    out = []
    for on in (True, False):
        s = pgc.Simulation(_deg(W.TEST3_FIELD_1E4, M, N=20001), max_outputs=8)
        s.set_pipeline(on)
        s.step(30, 10)
        out.append((s.state(), s.hist()[0], s.counters()))
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert out[0][2]["changed"] == out[1][2]["changed"] > 0


def test_uncompiled_degree_and_other_entry_points_are_rejected():
    pgc = _pgc()
    with pytest.raises(pgc.PgcError):
        pgc.Simulation(_deg(W.TEST3_WIDTH_1E4, 7, N=100))           # P = Q = 8 is not compiled
    with pytest.raises(pgc.PgcError):
        pgc.BatchSimulation([_deg(W.GAP_UQ_1E6, 10, N=1000)])
    s = pgc.Simulation(_deg(W.GAP_UQ_1E6, 10, N=1000), max_outputs=4)
    with pytest.raises(pgc.PgcError):
        n = pgc.pgc_adjoint_query_sizes(s.ctx, 10, 5)
        work = torch.empty(max(n, 256), dtype=torch.uint8, device="cuda")
        pgc.pgc_adjoint(s.ctx, 10, 5, 5, 5, [1.0, 0.0], work.data_ptr())
    s.step(3, 0)                                                       # still usable
    s.close()


def _oracle_sg_error(p, degrees, M_ref, steps, nz=64):
    z, w = np.polynomial.legendre.leggauss(nz)
    w = w / 2.0

    def energy(M):
        o = O.Oracle(_deg(p, M))
        out, done = [], 0
        for n in steps:
            o.step(n - done, n - done)
            done = n
            out.append([o.observe_at([zz])[2] for zz in z])
        return np.array(out)

    ref = energy(M_ref)
    return {M: np.sqrt((((energy(M) - ref) ** 2) * w).sum(axis=1)) for M in degrees}


def test_sg_error_study_matches_oracle_fp64():
    from paper_2404_19602_gb300 import sg_error

    p = W.scaled(W.TEST3_WIDTH_1E4, N=800, precision="fp64")
    steps = (40, 100)
    g = sg_error.sg_error(p, (0, 2, 5, 15), 30, steps)
    r = _oracle_sg_error(p, (0, 2, 5, 15), 30, steps)
    for M in r:
        assert np.all(r[M] > 0)
        assert np.allclose(g[M], r[M], rtol=1e-5, atol=1e-10), (M, g[M], r[M])


@pytest.mark.parametrize("base", ["width", "field"])
def test_sg_error_falls_with_the_degree(base):
    """Test 3 at the paper's settings (1e4 particles, dt 2.5 fs, t = 0.1, 0.5, 1 ps, M_ref = 30):
    the error at M = 25 is well below the error at M = 1 at every time."""
    from paper_2404_19602_gb300 import sg_error

    p = W.TEST3_WIDTH_1E4 if base == "width" else W.TEST3_FIELD_1E4
    e = sg_error.sg_error(p, (1, 5, 25), 30, W.TEST3_TIMES_STEPS)
    assert np.all(e[25] < e[1] / 4.0), e
    assert np.all(e[5] < e[1]), e


def test_mc_mc_batched_samples_equal_standalone_runs():
    """Test 4's MC-MC samples (Algorithm 1 at sampled inputs, advanced together by the batched
    kernels) are the standalone deterministic runs at those inputs."""
    from paper_2404_19602_gb300 import sg_error

    pgc = _pgc()
    p = W.scaled(W.TEST3_WIDTH_1E4, N=3000)
    got = sg_error.mc_mc_samples(p, 3, 3000, 30, seed=5)
    z = np.random.default_rng(5).uniform(-1.0, 1.0, 3)
    for j, zj in enumerate(z):
        q = W.scaled(sg_error.deterministic_at(p, float(zj)), stream_id=j)
        assert q["W_lo"] == q["W_hi"] == pytest.approx(6.5 + 0.5 * (zj + 1.0))
        s = pgc.Simulation(q, max_outputs=4)
        s.step(30, 30)
        # same trajectories; the moment sums group the particles differently in the batch
        assert s.moments()["mean"][-1, 0] == pytest.approx(got[j], rel=1e-5)
        s.close()


def test_mc_sg_and_mc_mc_estimates_agree():
    """E_z[V_x] at 0.25 ps by MC-sG (degree 5, 2e5 particles) and by MC-MC (64 samples of 2e4
    particles) agree within four standard errors (sample spread of MC-MC; particle noise of the
    sG ensemble bounded by v_F / sqrt(N) since |v_x| <= v_F)."""
    from paper_2404_19602_gb300 import sg_error

    p = W.TEST3_WIDTH_1E4
    sg = sg_error.mean_vx_sg(p, 5, 200_000, 100)
    v = sg_error.mc_mc_samples(p, 64, 20_000, 100, seed=2)
    se = v.std(ddof=1) / np.sqrt(v.size)
    tol = 4.0 * np.sqrt(se ** 2 + 1e12 / 200_000)
    assert abs(sg - v.mean()) <= tol, (sg, v.mean(), tol)
    assert abs(sg) > 10 * tol / 4.0          # a drift well resolved at this time


def test_ballistic_sg_error_converges_spectrally_fp64():
    """Scattering off (FP64): the Test 3 error of the energy against degree 30 falls geometrically
    with M for the uncertain width and vanishes to rounding for the affine field."""
    from paper_2404_19602_gb300 import sg_error

    w = W.scaled(W.TEST3_WIDTH_1E4, N=2000, mech_mask=0, precision="fp64")
    e = sg_error.sg_error(w, (2, 4, 6, 8), 30, (40,))
    errs = [float(e[M][0]) for M in (2, 4, 6, 8)]
    assert errs[0] > 1e-7
    for a, b in zip(errs, errs[1:]):
        assert b < a / 10.0, errs
    f = W.scaled(W.TEST3_FIELD_1E4, N=2000, mech_mask=0, precision="fp64")
    e = sg_error.sg_error(f, (1, 3), 30, (40,))
    assert max(float(e[1][0]), float(e[3][0])) < 1e-12, e
