"""Adjoint (pgc_adjoint): the hand-written reverse-mode kernels against the oracle's forward-mode
pathwise tangents (which are themselves pinned to central differences with unchanged events in
tests/test_oracle_adjoint.py), on the same seeded inputs, and through torch.autograd."""
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


CASES = {
    "det": W.scaled(W.DET_FP64_1E4, N=3000),
    "gap": W.scaled(W.GAP_UQ_1E6, N=2000, precision="fp64"),
    "gap_field": W.scaled(W.GAP_FIELD_UQ_4E6, N=300, precision="fp64"),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_adjoint_matches_oracle_tangents_fp64(name):
    from paper_2404_19602_gb300 import pgc

    p = CASES[name]
    steps, every, window, ckpt = 60, 5, 30, 16
    o = O.Oracle(p)
    val_o, grad_o = o.tangent_run(steps, every, window)
    for w in ([1.0, 0.0], [0.0, 1.0]):
        val, grad = pgc.adjoint(p, steps, ckpt, every, window, weights=w)
        # (the z-variance of a deterministic run is 0 up to rounding: compare on the mean's scale)
        assert np.allclose(val, val_o, rtol=1e-9, atol=1e-9 * abs(val_o[0])), (val, val_o)
        ref = w[0] * grad_o[0] + w[1] * grad_o[1]
        if name == "det" and w[1] == 1.0:
            ref_scale = np.abs(grad_o[0]).max() * abs(val_o[0])  # d Var / d theta ~ 0
        else:
            ref_scale = np.abs(ref).max()
        assert np.abs(grad - ref).max() <= 1e-6 * ref_scale, (name, w, grad, ref)


def test_adjoint_fp32_close_to_oracle():
    from paper_2404_19602_gb300 import pgc

    p = W.scaled(W.GAP_UQ_1E6, N=4000)
    steps, every, window, ckpt = 30, 5, 15, 8
    o = O.Oracle(p)
    _, grad_o = o.tangent_run(steps, every, window)
    _, grad = pgc.adjoint(p, steps, ckpt, every, window, weights=[1.0, 0.0])
    assert np.abs(grad - grad_o[0]).max() <= 1e-3 * np.abs(grad_o[0]).max(), (grad, grad_o[0])


def test_adjoint_checkpoint_interval_does_not_matter():
    from paper_2404_19602_gb300 import pgc

    p = CASES["gap"]
    _, g1 = pgc.adjoint(p, 40, 40, 5, 20, weights=[1.0, 0.5])
    _, g2 = pgc.adjoint(p, 40, 7, 5, 20, weights=[1.0, 0.5])
    assert np.allclose(g1, g2, rtol=1e-12, atol=0)


def test_autograd_function():
    from paper_2404_19602_gb300 import pgc

    p = CASES["gap"]
    theta = torch.tensor([p["Ex_lo"], p["Ex_hi"], p["eps0_lo"], p["eps0_hi"]], dtype=torch.float64, requires_grad=True)
    out = pgc.steady_current(theta, p, 40, 5, 20, ckpt_every=10)
    (out[0] + 0.25 * out[1]).backward()
    _, g = pgc.adjoint(p, 40, 10, 5, 20, weights=[1.0, 0.25])
    assert np.allclose(theta.grad.numpy(), g, rtol=1e-12, atol=0)


@pytest.mark.parametrize("name", ["det", "gap"])
def test_window_objective_equals_adjoint_value_and_oracle(name):
    """pgc_window_objective (the objective without the gradient) equals the value pgc_adjoint
    returns and the oracle's window average of the same run (FP64)."""
    from paper_2404_19602_gb300 import pgc

    p = CASES[name]
    steps, every, window, ckpt = 60, 5, 30, 16
    J, V = pgc.window_objective(p, steps, every, window)
    val, _ = pgc.adjoint(p, steps, ckpt, every, window, weights=[1.0, 0.0])
    # (the two runs group the FP64 moment partials differently; var_z of a deterministic input is
    # rounding noise of ~1e-11 J^2)
    assert abs(J - val[0]) <= 1e-12 * abs(val[0]) and abs(V - val[1]) <= 1e-9 * abs(val[1]) + 1e-9 * J ** 2
    o = O.Oracle(p)
    ref = o.window_objective(steps, every, window)
    assert abs(J - ref[0]) <= 1e-9 * abs(ref[0])
    # (a deterministic input has var_z = 0: the FP64 difference of squares leaves ~1e-11 J^2)
    assert abs(V - ref[1]) <= 1e-7 * abs(ref[1]) + 1e-9 * ref[0] ** 2
