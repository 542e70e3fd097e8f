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
