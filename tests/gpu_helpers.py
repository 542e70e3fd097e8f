"""Shared helpers of the GPU tests (no method arithmetic)."""
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1007_3470_gb300 import build as B
    B.build()
    return torch


# tolerances of the parity tests: relative discrete L2 error per unit time
TOL_C64 = 1e-5
TOL_C128 = 1e-11


def budget(tol, T):
    """Allowed relative L2 error for a run of length T: tol per unit time,
    with runs shorter than one unit held to the one-unit value."""
    return tol * max(float(T), 1.0)
