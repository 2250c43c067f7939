"""The reference arm of bench.py on the host (no GPU): one JSON line with the contract's keys,
the oracle timed on a bounded sample of the workload; under torchrun only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, *args):
    env = dict(os.environ, **(extra_env or {}))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", *args], capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [l for l in r.stdout.splitlines() if l.strip()]


def test_reference_line_has_the_contract_keys():
    lines = _run()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == d["unit"] == "particle-gPC-steps/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    assert d["config"]["workload"] and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_prints_on_rank_zero_only():
    assert _run({"RANK": "1", "WORLD_SIZE": "2"}) == []


def test_reference_line_for_another_workload():
    d = json.loads(_run(None, "--workload", "det")[0])
    assert d["config"]["workload"].startswith("det_") and d["value"] > 0


def test_traffic_figures_follow_the_kernel_sources(tmp_path, monkeypatch):
    """The DRAM bytes and instruction counts of profiles/traffic.json are used only while the
    kernel sources hash to the value they were captured on."""
    sys.path.insert(0, ROOT)
    import bench

    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    e = t["gap_uq"]["k_step"]
    if e["src_sha"] == bench._src_sha():
        assert bench._traffic("k_step", "gap_uq") == e["dram_bytes_per_launch"]
        assert bench._traffic("k_step", "gap_uq", "warp_inst_per_launch") == e["warp_inst_per_launch"]
    monkeypatch.setattr(bench, "_src_sha", lambda: "0" * 16)
    assert bench._traffic("k_step", "gap_uq") is None
    assert bench._traffic("no_such_kernel", "gap_uq") is None
    assert bench.throughput(1000, 2, 10, 5, 11.0) == 1000 * 2 * 10 * 5 / 11e-3


def test_parity_errors_are_normwise_over_the_shared_output_times():
    """The `parity` key's errors: max over the first n output times of |a - b|, divided by the
    largest |b| over those times, per quantity (J_x, V_x, energy) and moment (mean, var)."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench

    T = 6
    b = {"mean": np.zeros((T, 4)), "var": np.zeros((T, 4))}
    b["mean"][:, 3] = np.linspace(1.0, 2.0, T)          # J_x: 1.0 ... 2.0, largest |b| of the first 5 is 1.8
    b["mean"][:, 0] = -np.linspace(3.0, 4.0, T)         # V_x
    b["mean"][:, 2] = 5.0
    b["var"][:, 3] = 0.5
    a = {k: v.copy() for k, v in b.items()}
    a["mean"][2, 3] += 0.018                            # J_x off by 0.018 at one time: 0.01 of 1.8
    a["mean"][T - 1, 0] += 0.4                          # V_x off beyond the compared times
    a["var"][:, 3] *= 1.1                               # var J_x 10 % off everywhere
    e = bench._moment_errors(a, b, T - 1)
    assert abs(e["mean_Jx"] - 0.01) < 1e-12
    assert e["mean_Vx"] == 0.0                          # only the first n = T - 1 times count
    assert abs(e["var_Jx"] - 0.1) < 1e-12
    assert e["mean_energy"] == 0.0 and e["var_Vx"] == 0.0 and e["var_energy"] == 0.0   # zero reference: 0
    assert set(e) == {"%s_%s" % (k, q) for k in ("mean", "var") for q in ("Jx", "Vx", "energy")}
