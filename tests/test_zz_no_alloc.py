"""pgc_observe_static, the observation entry point that allocates nothing, against the regular
entry points (pgc_moments record and pgc_get_hist) on two calls in a row.

Callers that may not allocate device memory while they run (a framework pool owns it, or an
allocation could synchronize the device under queued work) use it to sample the ensemble; its
scratch is a fixed device array inside the library.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2404_19602_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_static_observation_matches_regular_entry_points():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19602_gb300 import build, pgc

    build.build()
    p = W.scaled(W.GAP_UQ_1E6, N=20000)
    sim = pgc.Simulation(p, max_outputs=16)
    Q, Nk = sim.Q, sim.Nk
    stream = torch.cuda.current_stream()
    for call in range(2):
        sim.step(10, 10)                       # records the moments of the post-step state
        m = sim.moments()
        H, _ = sim.hist()
        hist = torch.full((Q, Nk, Nk), 7, dtype=torch.int32, device="cuda")
        rec = torch.full((1 + 4 * Q + 8,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        pgc.pgc_observe_static(sim.ctx, hist.data_ptr(), rec.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        if call == 1:
            # after the first call's one-time set-up, a call takes no device memory
            assert torch.cuda.mem_get_info()[0] == free0
        h = hist.cpu().numpy().view(np.uint32)
        r = rec.cpu().numpy()
        assert np.array_equal(h, H), call
        assert r[0] == m["t_fs"][-1]
        nodes = r[1:1 + 4 * Q].reshape(Q, 4)
        # same FP64 accumulation of FP32 warp sums, grouped differently: FP32 rounding level
        assert np.allclose(nodes, m["nodes"][-1], rtol=1e-5, atol=0), call
        mean, var = r[1 + 4 * Q:1 + 4 * Q + 4], r[1 + 4 * Q + 4:]
        assert np.allclose(mean, m["mean"][-1], rtol=1e-5, atol=0), call
        scale = np.abs(m["var"][-1])
        assert np.all(np.abs(var - m["var"][-1]) <= 1e-3 * scale + 1e-30), call
    sim.close()
