"""The allocation-free entry point hfs_step1d_noalloc.

It serves callers that cannot allocate device memory -- for example code
running inside an allocator or memory-pool callback, or a library that is
handed only a device pointer to the state under a device-memory budget fixed
at start-up -- and so cannot bind the workspace the context API needs.  Its
scratch lives in a fixed array inside the library.

The test calls it through the C ABI twice in a row on the same device state
(the second call continues from the first one's result at t0 = 0.1, so the
scratch left behind by the first call must not leak into the second) and
compares each result with the context-based hfs_step() on the same inputs,
within the parity tolerance of the other GPU tests.  This file is collected
last so that a stop-at-first-failure run has executed every other test before
it; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1007_3470_gb300 import workloads as W
from tests.gpu_helpers import TOL_C128, TOL_C64, budget, need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [("c64", TOL_C64), ("c128", TOL_C128)])
def test_noalloc_matches_context_api_on_two_calls(precision, tol):
    torch = need_gpu()
    from paper_1007_3470_gb300 import hfs
    insts, psis, _ = W.batch_1d(count=40, seed=77)
    dt, steps = 0.005, 20
    prec = hfs.HFS_C128 if precision == "c128" else hfs.HFS_C64

    # existing entry point (context + caller-bound workspace), 16-step chunks
    ref = hfs.Solver(insts, precision=precision, chunk_steps=16)
    ref.set_schedule(dt, "strang", hfs.HFS_FLOW_CF4)
    ref.set_psi(psis)
    ref.step(steps)
    first_ref = ref.get_psi()
    ref.step(steps)
    second_ref = ref.get_psi()
    ref.close()

    # allocation-free entry point on a state buffer owned by the caller
    cdt = torch.complex128 if precision == "c128" else torch.complex64
    state = torch.from_numpy(np.concatenate([np.asarray(p) for p in psis])).to(cdt).cuda()
    torch.cuda.synchronize()
    arr = hfs.make_instances(insts)
    offsets = np.cumsum([0] + [i.n[0] for i in insts])

    def check(out, expect, T):
        for i in range(len(insts)):
            a, b = out[offsets[i]:offsets[i + 1]], expect[offsets[i]:offsets[i + 1]]
            assert O.rel_l2(a, b) <= budget(tol, T), i

    hfs.hfs_step1d_noalloc(state.data_ptr(), prec, arr, hfs.HFS_SPLIT_HO, hfs.HFS_FLOW_CF4, hfs.HFS_COMP_STRANG,
                           dt, 0.0, steps, 0, True)
    check(state.cpu().numpy(), first_ref, steps * dt)
    hfs.hfs_step1d_noalloc(state.data_ptr(), prec, arr, hfs.HFS_SPLIT_HO, hfs.HFS_FLOW_CF4, hfs.HFS_COMP_STRANG,
                           dt, steps * dt, steps, 0, True)
    check(state.cpu().numpy(), second_ref, 2 * steps * dt)


def test_noalloc_rejects_oversized_batch():
    torch = need_gpu()
    from paper_1007_3470_gb300 import hfs
    n = hfs.NOALLOC_MAX_INSTANCES + 1
    arr = hfs.make_instances([{"n": [128], "a": [-8.0], "b": [8.0]}] * n)
    state = torch.zeros(128 * n, dtype=torch.complex64, device="cuda")
    with pytest.raises(hfs.HfsError) as ei:
        hfs.hfs_step1d_noalloc(state.data_ptr(), hfs.HFS_C64, arr, hfs.HFS_SPLIT_HO, hfs.HFS_FLOW_CF4,
                               hfs.HFS_COMP_STRANG, 0.005, 0.0, 1, 0, True)
    assert ei.value.code == 8  # HFS_ERR_WORKSPACE
