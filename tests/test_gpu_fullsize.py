"""Parity at the full sizes, in the launch configuration the benchmark times
(4096 mixed-size instances, 500 steps in one resident, graph-replayed call),
on a stratified sample of instances the oracle recomputes one by one; the 3D
workload at its full length (128^3, 200 steps) against the FP64 GPU run; and
the edge cases of the batched entry point."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1007_3470_gb300 import workloads as W
from tests.gpu_helpers import TOL_C64, budget, need_gpu

pytestmark = pytest.mark.gpu


def test_batched_full_size_sampled_against_oracle():
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    insts, psis, steps = W.batch_1d(count=4096)  # 500 steps of 0.005, complex64
    s = hfs.Solver(insts, precision="c64", chunk_steps=steps)
    s.set_schedule(0.005, "strang", hfs.HFS_FLOW_CF4)
    s.autotune(20)
    s.set_graphs(True)
    s.set_psi(psis)
    s.step(steps)
    out = s.split(s.get_psi())
    assert s.status() == hfs.HFS_OK
    s.close()
    # two instances of every grid size, spread over the batch
    pick, seen = [], {}
    for i, inst in enumerate(insts):
        if seen.get(inst.n[0], 0) < 2 and i % 7 == 3:
            seen[inst.n[0]] = seen.get(inst.n[0], 0) + 1
            pick.append(i)
    assert len(pick) == 12
    refs = O.run_batch([O.Problem(**insts[i].as_dict()) for i in pick], [psis[i] for i in pick], steps)
    T = steps * 0.005
    for i, ref in zip(pick, refs):
        assert O.rel_l2(np.asarray(out[i]), ref) <= budget(TOL_C64, T), (i, insts[i].n[0])


def test_3d_full_length_fp32_vs_fp64_gpu():
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    inst, psi0, steps = W.gpe_3d(n=128, h=0.005, steps=200)
    res = {}
    for prec in ("c64", "c128"):
        s = hfs.Solver([inst], dim=3, precision=prec, chunk_steps=steps)
        s.set_schedule(inst.h, "strang", hfs.HFS_FLOW_CF4)
        s.set_psi(psi0.ravel())
        s.step(steps)
        res[prec] = (s.get_psi(), s.norm()[0])
        assert s.status() == hfs.HFS_OK
        s.close()
    T = steps * inst.h
    assert O.rel_l2(res["c64"][0], res["c128"][0]) <= budget(TOL_C64, T)
    assert abs(res["c128"][1] - 1.0) < 1e-12 and abs(res["c64"][1] - 1.0) < 1e-5


def test_single_instance_of_each_size_and_zero_steps():
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    for n in W.BATCH_SIZES:
        insts, psis, _ = W.batch_1d(count=1, sizes=(n,), seed=n)
        s = hfs.Solver(insts, precision="c64")
        s.set_schedule(0.005, "strang", hfs.HFS_FLOW_CF4)
        s.set_psi(psis)
        s.step(0)  # no-op
        assert np.array_equal(s.get_psi(), psis[0].astype(np.complex64))
        s.step(30)
        ref = O.run(O.Problem(**insts[0].as_dict()), psis[0], 30)
        assert O.rel_l2(s.get_psi(), ref) <= budget(TOL_C64, 0.15), n
        s.close()


def test_all_largest_instances_and_partial_work_items():
    """4096-point instances only, and counts that leave every work item
    partially filled (ragged batch of 3 small instances)."""
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    for sizes, count in (((4096,), 9), ((128,), 3), ((128, 512), 5)):
        insts, psis, _ = W.batch_1d(count=count, sizes=sizes, seed=count)
        s = hfs.Solver(insts, precision="c64")
        s.set_schedule(0.005, "strang", hfs.HFS_FLOW_CF4)
        s.set_psi(psis)
        s.step(25)
        out = s.split(s.get_psi())
        refs = O.run_batch([O.Problem(**i.as_dict()) for i in insts], psis, 25)
        assert max(O.rel_l2(o, r) for o, r in zip(out, refs)) <= budget(TOL_C64, 0.125)
        s.close()


def test_degenerate_linear_constant_trap_is_exact():
    """sigma = eps = 0 with constant omega: the scheme is the exact harmonic
    flow for any step, so a coherent state follows its closed form (FP64)."""
    need_gpu()
    import math
    from paper_1007_3470_gb300 import hfs
    inst = W.Instance(n=[512], a=[-16.0], b=[16.0], w0=1.0, ho_flow=W.FLOW_LEMMA2, h=0.7)
    x = inst.x()
    psi0 = math.pi ** -0.25 * np.exp(-(x - 1.5) ** 2 / 2)
    s = hfs.Solver([inst], precision="c128")
    s.set_schedule(0.7, "strang", hfs.HFS_FLOW_LEMMA2)
    s.set_psi([psi0.astype(complex)])
    s.step(10)
    t = 7.0
    q, p = 1.5 * math.cos(t), -1.5 * math.sin(t)
    exact = math.pi ** -0.25 * np.exp(-(x - q) ** 2 / 2 + 1j * p * (x - q / 2) - 0.5j * t)
    assert O.rel_l2(s.get_psi(), exact) < 1e-12
    s.close()
