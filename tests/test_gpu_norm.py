"""The norm projection of the 1D complex64 step (hfs_set_norm_projection).

The exact scheme conserves the discrete norm (Lemma 1; the kicks and drifts
are pure phases), so the FP64 oracle's norm is constant to round-off.  FP32
rounding makes the GPU norm random-walk; with the projection on, every
instance of the benchmark's batch (4096 instances x 500 steps, one resident
graph-replayed call) keeps its norm within 1e-6 of the start, its result stays
within the parity bound of the oracle on a stratified sample, and the
projection does not raise the error.  Streaming launches give the same bits
as the resident call (the target norm is recorded by the first launch of a
call and read by the others), and chunked calls keep the same bound."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1007_3470_gb300 import workloads as W
from tests.gpu_helpers import TOL_C64, budget, need_gpu

pytestmark = pytest.mark.gpu

DRIFT = 1e-6


def _solve(insts, psis, steps, project, mode=None, chunk=None, graphs=True):
    from paper_1007_3470_gb300 import hfs
    s = hfs.Solver(insts, precision="c64", chunk_steps=chunk or steps)
    s.set_schedule(0.005, "strang", hfs.HFS_FLOW_CF4)
    s.set_norm_projection(project)
    if mode is not None:
        s.set_mode(*mode)
    s.set_graphs(graphs)
    s.set_psi(psis)
    n0 = s.norm()
    s.step(steps)
    n1 = s.norm()
    out = s.get_psi()
    assert s.status() == hfs.HFS_OK
    parts = [np.asarray(p) for p in s.split(out)]
    s.close()
    return out, parts, np.abs(n1 / n0 - 1.0)


def test_full_batch_drift_and_parity_with_projection():
    need_gpu()
    insts, psis, steps = W.batch_1d(count=4096)
    _, proj, drift_p = _solve(insts, psis, steps, True)
    _, plain, drift_0 = _solve(insts, psis, steps, False)
    assert drift_p.max() <= DRIFT, drift_p.max()
    # the unprojected FP32 drift is a zero-mean random walk well above it
    assert drift_0.max() > 2 * DRIFT
    pick, seen = [], {}
    for i, inst in enumerate(insts):
        if seen.get(inst.n[0], 0) < 3 and i % 5 == 1:
            seen[inst.n[0]] = seen.get(inst.n[0], 0) + 1
            pick.append(i)
    refs = O.run_batch([O.Problem(**insts[i].as_dict()) for i in pick], [psis[i] for i in pick], steps)
    T = steps * 0.005
    ep = np.array([O.rel_l2(proj[i], r) for i, r in zip(pick, refs)])
    e0 = np.array([O.rel_l2(plain[i], r) for i, r in zip(pick, refs)])
    assert ep.max() <= budget(TOL_C64, T), ep.max()
    assert np.median(ep) <= 1.05 * np.median(e0), (np.median(ep), np.median(e0))
    for i, r in zip(pick, refs):
        assert abs(O.norm(O.Problem(**insts[i].as_dict()), proj[i]) /
                   O.norm(O.Problem(**insts[i].as_dict()), r) - 1.0) <= DRIFT


def test_projection_streaming_and_chunks_match_resident_bitwise():
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    insts, psis, _ = W.batch_1d(count=300, seed=5)
    steps = 40
    res, _, d_res = _solve(insts, psis, steps, True)
    stream, _, _ = _solve(insts, psis, steps, True, mode=(hfs.HFS_MODE_STREAMING, 3), graphs=False)
    assert np.array_equal(res, stream)
    assert d_res.max() <= DRIFT
    # schedule chunks split the merged phase at their boundaries (not bitwise
    # the single-chunk call); the later chunks project onto the first one's target
    chunked, _, d_chunk = _solve(insts, psis, steps, True, chunk=16)
    assert d_chunk.max() <= DRIFT
    assert O.rel_l2(chunked, res) <= 1e-5


def test_projection_off_is_the_default_and_unsupported_elsewhere():
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    insts, psis, _ = W.batch_1d(count=64, seed=9)
    a, _, _ = _solve(insts, psis, 30, False)
    s = hfs.Solver(insts, precision="c64", chunk_steps=30)
    s.set_schedule(0.005, "strang", hfs.HFS_FLOW_CF4)
    s.set_psi(psis)
    s.step(30)
    assert np.array_equal(a, s.get_psi())
    s.close()
    for dim, prec, inst in ((1, "c128", insts[:1]), (3, "c64", [W.gpe_3d(n=32)[0]])):
        s = hfs.Solver(inst, dim=dim, precision=prec, chunk_steps=4)
        with pytest.raises(hfs.HfsError) as ei:
            s.set_norm_projection(True)
        assert ei.value.code == 2  # HFS_ERR_UNSUPPORTED
        s.close()


@pytest.mark.parametrize("scheme,h", [("ni5_84", 0.01), ("srkn6_4", 0.01), ("strang", 0.005)])
def test_time_dependent_gpe_full_length_with_projection(scheme, h):
    """The time-dependent GPE (N = 1024, omega = 1 + 0.5 sin 2t, sigma = 10,
    T = 10) with the projection: within the parity bound of the oracle and
    within 1e-6 of the initial norm after 1000-2000 steps."""
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    inst, psi0, steps = W.gpe_tdep_1d(h=h, scheme=scheme)
    ref = O.run(O.Problem(**inst.as_dict()), psi0, steps)
    s = hfs.Solver([inst], precision="c64", chunk_steps=steps)
    s.set_schedule(h, scheme, hfs.HFS_FLOW_CF4)
    s.set_norm_projection(True)
    s.set_psi([psi0])
    n0 = s.norm()[0]
    s.step(steps)
    out = s.get_psi()
    n1 = s.norm()[0]
    s.close()
    assert O.rel_l2(out, ref) <= budget(TOL_C64, steps * h)
    assert abs(n1 / n0 - 1.0) <= DRIFT


def _solve3(steps, project, chunk=None, precision="c64", engine=0):
    from paper_1007_3470_gb300 import hfs
    inst, psi0, _ = W.gpe_3d(n=128, h=0.005)
    s = hfs.Solver([inst], dim=3, precision=precision, chunk_steps=chunk or steps)
    s.set_schedule(inst.h, "strang", hfs.HFS_FLOW_CF4)
    if project:
        s.set_norm_projection(True)
    if engine:
        s.set_dft_engine(engine)
    s.set_psi(psi0.ravel())
    n0 = s.norm()[0]
    s.step(steps)
    out = s.get_psi()
    n1 = s.norm()[0]
    assert s.status() == hfs.HFS_OK
    s.close()
    return out, n1 / n0 - 1.0


@pytest.mark.parametrize("steps", [6, 200])
def test_3d_projection_against_fp64_device(steps):
    """128^3 complex64 with the projection (plain twiddles, per-sub-stage
    rescaling from the plane passes' sums): within the parity bound of the
    FP64 device solve, and within 1e-6 of the initial norm."""
    need_gpu()
    proj, d = _solve3(steps, True)
    ref, _ = _solve3(steps, False, precision="c128")
    assert O.rel_l2(proj, ref) <= budget(TOL_C64, steps * 0.005), O.rel_l2(proj, ref)
    assert abs(d) <= DRIFT


def test_3d_projection_chunks_and_tensor_engine():
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    one, _ = _solve3(40, True)
    chunked, d = _solve3(40, True, chunk=16)
    assert abs(d) <= DRIFT
    assert O.rel_l2(chunked, one) <= 1e-5
    tc, d_tc = _solve3(6, True, engine=hfs.HFS_DFT_TENSOR_3XTF32)
    ref, _ = _solve3(6, False, precision="c128")
    assert O.rel_l2(tc, ref) <= budget(TOL_C64, 6 * 0.005)
    assert abs(d_tc) <= DRIFT
