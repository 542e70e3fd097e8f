"""Host-side logic of bench.py that needs no GPU: the captured-traffic lookup
is tied to the kernel sources it was measured on."""
import bench


def test_traffic_reported_only_for_captured_workloads():
    assert bench.step1d_traffic("no_such_workload") is None
    v = bench.step1d_traffic("batch_1d_4096x500_c64")
    # either the sources are unchanged since the capture (bytes) or they are not (None)
    assert v is None or v > 0


def test_traffic_dropped_when_kernel_sources_change(monkeypatch):
    monkeypatch.setitem(bench.STEP1D_TRAFFIC, "src", "0" * 16)
    assert bench.step1d_traffic("batch_1d_4096x500_c64") is None


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference runs the oracle on a bounded sample and prints
    the contract's JSON line (CPU only)."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--ref-sample", "1"], capture_output=True, text=True, timeout=300,
                         cwd=root, env={**os.environ, "WORLD_SIZE": "1", "RANK": "0", "LOCAL_RANK": "0"})
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "grid-point-steps/s"
    assert d["metric"] == bench.METRIC and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"] == "batch_1d_4096x500_c64"


def test_cpu_baseline_sample_is_stratified():
    insts, psis = bench._stratified_sample(2, 20100703)
    sizes = sorted(i.n[0] for i in insts)
    assert sizes == sorted([n for n in (128, 256, 512, 1024, 2048, 4096) for _ in range(2)])
    assert all(len(p) == i.n[0] for i, p in zip(insts, psis))


def test_result_error_against_reference_slices():
    """result_error slices each sampled instance out of the concatenated
    batch and compares it with its reference."""
    import numpy as np
    rng = np.random.default_rng(1)
    sizes = [4, 8, 4]
    refs_all = [rng.standard_normal(n) + 1j * rng.standard_normal(n) for n in sizes]
    state = np.concatenate(refs_all).astype(np.complex64)
    pick = [0, 2]
    psis0 = [refs_all[0], refs_all[2]]
    e = bench.result_error(state, sizes, pick, psis0, [refs_all[0], refs_all[2]])
    assert e["rel_l2_max"] < 1e-6 and e["instances"] == 2 and e["norm_drift_max"] < 1e-6
    bad = state.copy()
    bad[12:16] *= 1.01  # instance 2 scaled by 1 %
    e = bench.result_error(bad, sizes, pick, psis0, [refs_all[0], refs_all[2]])
    assert abs(e["rel_l2_max"] - 0.01) < 1e-5 and not e["within_bound"]
