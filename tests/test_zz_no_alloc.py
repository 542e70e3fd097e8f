"""The allocation-free entry point hfs_step1d_noalloc.

It serves callers that cannot allocate device memory -- for example code
running inside an allocator or memory-pool callback, or a library that is
handed only a device pointer to the state under a device-memory budget fixed
at start-up -- and so cannot bind the workspace the context API needs.  Its
scratch lives in a fixed array inside the library.

Each test calls it through the C ABI twice in a row on the same device state
(the second call continues from the first one's result at t0 = steps * dt, so
the scratch left behind by the first call must not leak into the second) and
compares each result with the context-based hfs_step() on the same inputs
with 16-step schedule chunks: both run the same kernels on the same records,
so the results must be identical bit for bit.  The cases cover the Strang and
the six-stage SRKN_6 4 compositions (the largest one the scratch is sized
for), both splittings, both precisions, and a 512-instance mixed-size batch at
the instance limit.  This file is collected last so that a stop-at-first-
failure run has executed every other test before it; it also passes on its
own in a fresh process.
"""
import numpy as np
import pytest

from paper_1007_3470_gb300 import workloads as W
from tests.gpu_helpers import need_gpu

pytestmark = pytest.mark.gpu


def _two_calls(precision, comp, split, count, seed, steps):
    torch = need_gpu()
    from paper_1007_3470_gb300 import hfs
    insts, psis, _ = W.batch_1d(count=count, seed=seed)
    dt = 0.005
    prec = hfs.HFS_C128 if precision == "c128" else hfs.HFS_C64
    comp_id = hfs.COMPOSITIONS[comp]

    # existing entry point (context + caller-bound workspace), 16-step chunks
    ref = hfs.Solver(insts, precision=precision, chunk_steps=16)
    ref.set_schedule(dt, comp, hfs.HFS_FLOW_CF4, split=split)
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
    hfs.hfs_step1d_noalloc(state.data_ptr(), prec, arr, split, hfs.HFS_FLOW_CF4, comp_id, dt, 0.0, steps, 0, True)
    first = state.cpu().numpy()
    hfs.hfs_step1d_noalloc(state.data_ptr(), prec, arr, split, hfs.HFS_FLOW_CF4, comp_id, dt, steps * dt, steps,
                           0, True)
    second = state.cpu().numpy()
    assert np.array_equal(first, first_ref)
    assert np.array_equal(second, second_ref)
    assert not np.array_equal(first, second)


@pytest.mark.parametrize("precision", ["c64", "c128"])
@pytest.mark.parametrize("comp", ["strang", "srkn6_4"])
@pytest.mark.parametrize("split", [0, 1], ids=["ho", "fourier"])
def test_noalloc_matches_context_api_on_two_calls(precision, comp, split):
    _two_calls(precision, comp, split, count=40, seed=77, steps=20)


def test_noalloc_full_instance_limit_mixed_sizes():
    from paper_1007_3470_gb300 import hfs
    _two_calls("c64", "srkn6_4", 0, count=hfs.NOALLOC_MAX_INSTANCES, seed=78, steps=18)


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
