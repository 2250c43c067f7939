"""The block-private histogram window of the streaming step (16-bit cells in shared memory,
flushed to the global histogram f^{n+1} of Eq. (24)) at an ensemble large enough that every
streaming block counts more than 2^16 particles: all particles sit in one cell, so that cell's
count must come out exact, in the pipelined (fused, dynamic tiles) and the two-launch form."""
import numpy as np
import pytest

from paper_2404_19602_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HVF = 0.6582119569


@pytest.mark.parametrize("pipelined", [True, False])
def test_window_counts_past_16_bits(pipelined):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19602_gb300 import build, pgc

    build.build()
    N = 1 << 25          # ~74k particles per streaming block at 456 blocks
    p = W.scaled(W.DET_FP64_1E4, N=N, precision="fp32", mech_mask=0, Ex_lo=0.0, Ex_hi=0.0)
    k = np.zeros((2, 1, N))
    k[0, 0] = 0.3
    k[1, 0] = -0.2
    sim = pgc.Simulation(p, init_khat=k, max_outputs=8)
    sim.set_pipeline(pipelined)
    Lk = 5.0 / HVF
    dk = 2 * Lk / 240
    r, l = int(np.floor((0.3 + Lk) / dk)), int(np.floor((-0.2 + Lk) / dk))
    for _ in range(2):
        sim.step(3, 0)
        H, _ = sim.hist()
        ref = np.zeros_like(H)
        ref[0, r, l] = N
        assert np.array_equal(H, ref)
    assert sim.counters()["out_of_grid"] == 0
    sim.close()
