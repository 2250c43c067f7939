"""Observables at arbitrary points z (pgc_observe_at) against the oracle's observe_at on the same
state.  The state is stepped on the GPU and handed to the oracle; both then evaluate V_x, V_y,
energy and J_x of the particles reconstructed at the same points (Eq. (23) off the nodes,
Eqs. (35)-(37)).  Covered: points off the nodes in passes of 32 with a ragged tail, the nodes
themselves (which give the node values of the moment record), the width law, two random inputs,
the deterministic shape, the full 1e6-particle ensemble on sampled points, and the error cases."""
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


def _pgc():
    from paper_2404_19602_gb300 import pgc

    return pgc


def _stepped(p, steps):
    s = _pgc().Simulation(p, max_outputs=4)
    s.step(steps, steps)
    return s


def _points(d, n, seed):
    rng = np.random.default_rng(seed)
    z = rng.uniform(-1.0, 1.0, size=(n, max(d, 1)))
    z[0], z[-1] = -1.0, 1.0            # the interval ends
    return z


def _compare(g, r, rtol):
    """Normwise per observable; the two velocity components share the V_x scale (V_y averages to
    about zero).  An FP32 state gives about 1e-7 relative per particle on either component."""
    vscale = max(np.abs(r[:, 0]).max(), 1.0)
    scales = [vscale, vscale, np.abs(r[:, 2]).max(), np.abs(r[:, 3]).max()]
    for c in range(4):
        err = np.abs(g[:, c] - r[:, c]).max()
        assert err <= rtol * scales[c], (c, err, scales[c])


CASES = [
    ("gap_fp64", W.scaled(W.GAP_UQ_1E6, N=3001, precision="fp64"), 40, 1e-12),
    ("gap_fp32", W.scaled(W.GAP_UQ_1E6, N=30001), 40, 2e-5),
    ("width_fp64", W.scaled(W.TEST2_WIDTH_1E6, N=2999, precision="fp64"), 30, 1e-12),
    ("width_fp32", W.scaled(W.TEST2_WIDTH_1E6, N=20000), 30, 2e-5),
    ("field2d_fp64", W.scaled(W.GAP_FIELD_UQ_4E6, N=777, precision="fp64"), 10, 1e-12),
    ("field2d_fp32", W.scaled(W.GAP_FIELD_UQ_4E6, N=5003), 10, 2e-5),
    ("det_fp64", W.scaled(W.DET_FP64_1E4, N=4097), 50, 1e-12),
]


@pytest.mark.parametrize("name,p,steps,rtol", CASES, ids=[c[0] for c in CASES])
def test_observe_at_matches_oracle(name, p, steps, rtol):
    s = _stepped(p, steps)
    o = O.Oracle(p, init_khat=s.state())
    z = _points(s.d, 45, 1)               # two passes: 32 points and a tail of 13
    g = s.observe_at(z)
    r = np.array([o.observe_at(zj) for zj in z])
    s.close()
    assert g.shape == (45, 4) and np.isfinite(g).all()
    _compare(g, r, rtol)


@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("base", ["gap", "field2d", "width"])
def test_nodes_give_the_node_values_of_the_moment_record(base, prec, rtol):
    b = {"gap": W.GAP_UQ_1E6, "field2d": W.GAP_FIELD_UQ_4E6, "width": W.TEST2_WIDTH_1E6}[base]
    p = W.scaled(b, N=4001, precision=prec)
    s = _stepped(p, 20)
    zq = O.Oracle(W.scaled(p, N=1)).tables()["z"]     # node q = q1 * Q1 + q2
    g = s.observe_at(zq)
    rec = s.moments()["nodes"][-1]                    # [Q][4] at the last step = current state
    s.close()
    _compare(g, rec, rtol)


def test_deterministic_shape_every_point_is_the_record():
    s = _stepped(W.scaled(W.DET_FP64_1E4, N=1000), 10)
    g = s.observe_at(np.zeros(40))
    rec = s.moments()["nodes"][-1][0]
    s.close()
    assert np.all(g == g[0])
    _compare(g[:1], rec[None, :], 1e-12)


def test_repeated_calls_are_bit_identical():
    s = _stepped(W.scaled(W.GAP_UQ_1E6, N=100_000), 10)
    z = _points(1, 70, 3)
    a, b = s.observe_at(z), s.observe_at(z)
    s.close()
    assert np.array_equal(a, b)


def test_full_size_ensemble_sampled_points():
    """The 1e6-particle default ensemble (FP32 state) after 50 steps, at 5 points."""
    p = W.GAP_UQ_1E6
    s = _stepped(p, 50)
    z = np.array([[-1.0], [-0.37], [0.0], [0.61], [1.0]])
    g = s.observe_at(z)
    o = O.Oracle(p, init_khat=s.state())
    r = np.array([o.observe_at(zj) for zj in z])
    s.close()
    _compare(g, r, 2e-5)


def test_empty_and_invalid_points():
    pgc = _pgc()
    s = _stepped(W.scaled(W.GAP_UQ_1E6, N=500), 2)
    assert s.observe_at(np.zeros((0, 1))).shape == (0, 4)
    for bad in ([[1.5]], [[-1.0000001]], [[np.nan]]):
        with pytest.raises(pgc.PgcError):
            s.observe_at(np.array(bad))
    # the context stays usable after a rejected call
    s.step(2, 0)
    assert np.isfinite(s.observe_at([[0.25]])).all()
    s.close()


@pytest.mark.parametrize("prec,rtol_mean,rtol_var", [("fp64", 1e-7, 1e-4), ("fp32", 1e-5, 2e-3)])
def test_quadrature_moments_against_fine_grid_ballistic(prec, rtol_mean, rtol_var):
    """Sec. 4.2: the Galerkin mean and variance over z (Gauss quadrature of the node values)
    against the plain mean and variance of the observables at 512 equally spaced points of the
    uniform law (midpoint rule).  With the scattering off every particle's node values are a smooth
    function of z and the degree-5 reconstruction resolves it, so the two agree closely.  (With
    scattering, Pauli and selection decisions taken node by node make k(z) rough between the
    nodes and the two differ by about 1 % in the mean: a property of the scheme, which the
    oracle shows too.)"""
    s = _stepped(W.scaled(W.GAP_UQ_1E6, N=100_000, mech_mask=0, precision=prec), 300)
    z = ((np.arange(512) + 0.5) / 256.0 - 1.0)[:, None]
    obs = s.observe_at(z)
    m = s.moments()
    s.close()
    for comp in (0, 2, 3):
        q, v = m["mean"][-1, comp], m["var"][-1, comp]
        assert abs(obs[:, comp].mean() - q) <= rtol_mean * abs(q), (comp, obs[:, comp].mean(), q)
        assert abs(obs[:, comp].var() - v) <= rtol_var * v, (comp, obs[:, comp].var(), v)
