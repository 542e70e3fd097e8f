"""Schedule reuse of the 1D path (hfs_set_schedule_reuse).

A call's phase records are a function of its start time, its step count and
the schedule alone (the FP64 stage flows of Lemma 2 / Theorem 2 merged as in
Eq. prod-genHarmOsc), so records kept from an earlier call, or computed for
the next call in a branch parallel to the step kernel, must give the same
bits as records computed in line.  Every case below compares a context with
reuse on against one with reuse off, bit for bit, after every call: calls
that follow each other in time (each consumes the records its predecessor
prefetched), calls that restart from t = 0 (the kept records of t = 0),
graph replay on and off, streaming launches, the Fourier split, a changed
schedule, calls longer than a chunk (no reuse), and the workspace growth."""
import ctypes

import numpy as np
import pytest

from paper_1007_3470_gb300 import workloads as W
from tests.gpu_helpers import need_gpu

pytestmark = pytest.mark.gpu


def _pair(insts, psis, steps, chunk, graphs=True, mode=None, split=None):
    from paper_1007_3470_gb300 import hfs
    out = []
    for reuse in (False, True):
        s = hfs.Solver(insts, precision="c64", chunk_steps=chunk)
        if split is None:
            s.set_schedule(0.005, "strang", hfs.HFS_FLOW_CF4)
        else:
            s.set_schedule(0.005, "strang", hfs.HFS_FLOW_CF4, split=split)
        s.set_norm_projection(True)
        if mode is not None:
            s.set_mode(*mode)
        s.set_graphs(graphs)
        s.set_schedule_reuse(reuse)
        s.set_psi(psis)
        out.append(s)
    return out


def _same(a, b):
    from paper_1007_3470_gb300 import hfs
    ua, ub = np.asarray(a.get_psi()), np.asarray(b.get_psi())
    assert a.status() == hfs.HFS_OK and b.status() == hfs.HFS_OK
    assert a.time == b.time
    return np.array_equal(ua.view(np.uint32), ub.view(np.uint32))


@pytest.mark.parametrize("graphs", [True, False])
def test_consecutive_and_restarted_calls_bitwise(graphs):
    need_gpu()
    insts, psis, _ = W.batch_1d(count=96, seed=11)
    steps = 24
    a, b = _pair(insts, psis, steps, chunk=steps, graphs=graphs)
    try:
        for _ in range(4):  # each call after the first uses prefetched records
            a.step(steps)
            b.step(steps)
            assert _same(a, b)
        for _ in range(3):  # restarts at t = 0: the records of the first call are kept
            for s in (a, b):
                s.set_time(0.0)
                s.set_psi(psis)
                s.step(steps)
            assert _same(a, b)
        # shorter calls than the chunk, alternating with full ones
        for n in (10, 10, steps, 7):
            a.step(n)
            b.step(n)
            assert _same(a, b)
    finally:
        a.close()
        b.close()


def test_streaming_fourier_split_and_changed_schedule():
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    insts, psis, _ = W.batch_1d(count=64, seed=12)
    steps = 16
    a, b = _pair(insts, psis, steps, chunk=steps, mode=(hfs.HFS_MODE_STREAMING, 1))
    try:
        for _ in range(3):
            a.step(steps)
            b.step(steps)
            assert _same(a, b)
        for s in (a, b):  # a new schedule drops the kept records
            s.set_schedule(0.004, "strang", hfs.HFS_FLOW_M6)
        for _ in range(2):
            a.step(steps)
            b.step(steps)
            assert _same(a, b)
    finally:
        a.close()
        b.close()
    a, b = _pair(insts, psis, steps, chunk=steps, split=hfs.HFS_SPLIT_FOURIER)
    try:
        for _ in range(3):
            a.step(steps)
            b.step(steps)
            assert _same(a, b)
    finally:
        a.close()
        b.close()


def test_calls_longer_than_a_chunk():
    need_gpu()
    insts, psis, _ = W.batch_1d(count=48, seed=13)
    a, b = _pair(insts, psis, 40, chunk=16)
    try:
        for n in (40, 16, 40):  # 40 > chunk: computed in line, 16: reused / prefetched
            a.step(n)
            b.step(n)
            assert _same(a, b)
    finally:
        a.close()
        b.close()


def test_workspace_growth_and_unbound_context():
    """Reuse needs a second record buffer: with the bound workspace too small
    the setter leaves the context unbound (HFS_ERR_WORKSPACE, then
    HFS_ERR_NOT_READY from hfs_step) until it is bound again with the size
    hfs_workspace_size now reports."""
    need_gpu()
    import torch
    from paper_1007_3470_gb300 import hfs
    L = hfs.lib()
    insts, psis, _ = W.batch_1d(count=8, seed=14)
    arr = hfs.make_instances(insts)
    h = ctypes.c_void_p()
    assert L.hfs_create(ctypes.byref(h), 1, hfs.HFS_C64, arr, len(insts)) == 0
    try:
        chunk = 12
        w0 = hfs.hfs_workspace_size(h, chunk)
        elems, _ = hfs.hfs_state_size(h)
        psi = torch.zeros(elems, dtype=torch.complex64, device="cuda")
        work = torch.empty(w0, dtype=torch.uint8, device="cuda")
        hfs.hfs_bind(h, psi.data_ptr(), work.data_ptr(), w0, chunk)
        hfs.hfs_set_schedule(h, hfs.HFS_SPLIT_HO, hfs.HFS_FLOW_CF4, hfs.HFS_COMP_STRANG, 0.005)
        assert L.hfs_set_schedule_reuse(h, 1) == hfs.HFS_ERR_WORKSPACE
        assert L.hfs_step(h, ctypes.c_int64(3)) == 6  # unbound
        w1 = hfs.hfs_workspace_size(h, chunk)
        assert w1 > w0
        work = torch.empty(w1, dtype=torch.uint8, device="cuda")
        hfs.hfs_bind(h, psi.data_ptr(), work.data_ptr(), w1, chunk)
        assert L.hfs_step(h, ctypes.c_int64(3)) == 0
        assert L.hfs_step(h, ctypes.c_int64(3)) == 0
        assert L.hfs_sync_status(h) == 0
        # switching off keeps the larger workspace valid
        assert L.hfs_set_schedule_reuse(h, 0) == 0
        assert L.hfs_step(h, ctypes.c_int64(3)) == 0
        assert L.hfs_sync_status(h) == 0
    finally:
        L.hfs_destroy(h)
    # the Solver re-binds by itself
    s = hfs.Solver(insts, precision="c64", chunk_steps=12)
    try:
        before = s.work_bytes
        s.set_schedule(0.005, "strang", hfs.HFS_FLOW_CF4)
        s.set_schedule_reuse(True)
        assert s.work_bytes > before
        s.set_psi(psis)
        s.step(12)
        assert s.status() == hfs.HFS_OK
    finally:
        s.close()


def test_3d_is_unsupported():
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    inst, psi0, _ = W.gpe_3d(n=32, h=0.005, steps=2)
    s = hfs.Solver([inst], dim=3, precision="c64", chunk_steps=2)
    try:
        assert hfs.lib().hfs_set_schedule_reuse(s.h, 1) == 2  # HFS_ERR_UNSUPPORTED
        assert hfs.lib().hfs_set_schedule_reuse(s.h, 0) == 0
    finally:
        s.close()
