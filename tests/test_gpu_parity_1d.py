"""GPU parity of the 1D split step (through the C ABI) against the FP64
oracle on the same seeded inputs.  Bar: relative L2 error <= 1e-5 per unit
time for the FP32 path, <= 1e-11 per unit time for the FP64 path."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1007_3470_gb300 import workloads as W
from tests.gpu_helpers import TOL_C128, TOL_C64, budget, need_gpu

pytestmark = pytest.mark.gpu


def _run_gpu(insts, psis, steps, precision, dt, comp="strang", flow=None, split=0, mode=None, chunk=512,
             graphs=False, t0=0.0):
    from paper_1007_3470_gb300 import hfs
    s = hfs.Solver(insts, precision=precision, chunk_steps=chunk)
    s.set_schedule(dt, comp, insts[0].ho_flow if flow is None else flow, split)
    if mode is not None:
        s.set_mode(*mode)
    if graphs:
        s.set_graphs(True)
    if t0:
        s.set_time(t0)
    s.set_psi(psis)
    s.step(steps)
    out = [np.array(v) for v in s.split(s.get_psi())]
    assert s.status() == hfs.HFS_OK
    s.close()
    return out


@pytest.mark.parametrize("precision,tol", [("c128", TOL_C128), ("c64", TOL_C64)])
def test_coherent_quartic_1d(precision, tol):
    """N=256, [-16,16), omega=1, eps x^4, coherent state x0=1, Strang + exact
    harmonic flow (Lemma 2), dt=0.01, 1000 steps (T=10)."""
    need_gpu()
    inst, psi0, steps = W.coherent_1d()
    ref = O.run(O.Problem(**inst.as_dict()), psi0, steps)
    (out,) = _run_gpu([inst], [psi0], steps, precision, inst.h)
    T = steps * inst.h
    assert O.rel_l2(out, ref) <= budget(tol, T)


@pytest.mark.parametrize("h", [0.04, 0.01])
@pytest.mark.parametrize("precision,tol", [("c128", TOL_C128), ("c64", TOL_C64)])
def test_gpe_timedependent_magnus4_ni5(precision, tol, h):
    """N=1024, [-20,20), omega(t)=1+0.5 sin 2t, sigma=10, eps cos 2x, CF4 +
    Theorem 2 inside NI_5(8,4); T=10."""
    need_gpu()
    inst, psi0, steps = W.gpe_tdep_1d(h=h)
    ref = O.run(O.Problem(**inst.as_dict()), psi0, steps)
    (out,) = _run_gpu([inst], [psi0], steps, precision, h, comp="ni5_84")
    assert O.rel_l2(out, ref) <= budget(tol, steps * h)


@pytest.mark.parametrize("comp,flow,split", [("srkn6_4", 1, 0), ("ni4_82", 1, 0), ("strang", 2, 0),
                                             ("ni5_84", 2, 0), ("strang", 1, 1), ("srkn6_4", 1, 1)])
@pytest.mark.parametrize("precision,tol", [("c128", TOL_C128), ("c64", TOL_C64)])
def test_schedule_variants(precision, tol, comp, flow, split):
    need_gpu()
    inst, psi0, _ = W.gpe_tdep_1d(h=0.02, n=512, scheme=comp, ho_flow=flow)
    inst.a, inst.b = [-16.0], [16.0]
    inst.split = split
    psi0 = W.gaussian_1d(inst, x0=0.4)
    steps = 100
    ref = O.run(O.Problem(**inst.as_dict()), psi0, steps)
    (out,) = _run_gpu([inst], [psi0], steps, precision, inst.h, comp=comp, flow=flow, split=split)
    assert O.rel_l2(out, ref) <= budget(tol, steps * inst.h)


@pytest.mark.parametrize("precision,tol", [("c128", TOL_C128), ("c64", TOL_C64)])
def test_custom_composition(precision, tol):
    """A user-supplied, non-symmetric composition (a = (0.3, 0.7),
    b = (0.15, 0.5, 0.35): consistent, second order) on the time-dependent GPE
    against the oracle applying the same coefficients stage by stage; and
    Strang's coefficients passed as a custom set reproduce the built-in
    Strang bitwise."""
    need_gpu()
    import dataclasses
    from paper_1007_3470_gb300 import hfs
    inst, psi0, _ = W.gpe_tdep_1d(h=0.01)
    steps = 120
    a, b = [0.3, 0.7], [0.15, 0.5, 0.35]
    prob = dataclasses.replace(O.Problem(**inst.as_dict()), coeffs=(a, b))
    ref = O.run(prob, psi0, steps)
    s = hfs.Solver([inst], precision=precision)
    s.set_schedule(inst.h, "custom", hfs.HFS_FLOW_CF4, a=a, b=b)
    s.set_psi(psi0)
    s.step(steps)
    out = s.get_psi()
    assert s.status() == hfs.HFS_OK
    s.close()
    assert O.rel_l2(out, ref) <= budget(tol, steps * inst.h)
    # and the coefficients matter: the oracle's NI5(8,4) result of the same instance differs
    assert O.rel_l2(ref, O.run(O.Problem(**inst.as_dict()), psi0, steps)) > 1e-6
    (strang,) = _run_gpu([inst], [psi0], steps, precision, inst.h, comp="strang", flow=hfs.HFS_FLOW_CF4)
    s = hfs.Solver([inst], precision=precision)
    s.set_schedule(inst.h, "custom", hfs.HFS_FLOW_CF4, a=[1.0], b=[0.5, 0.5])
    s.set_psi(psi0)
    s.step(steps)
    assert np.array_equal(s.get_psi(), strang)
    s.close()


@pytest.mark.parametrize("law,lawp", [(W.OMEGA_COS_SQ, [0.3, 2.0, 0.0]),   # small node offset: series path
                                      (W.OMEGA_COS_SQ, [0.3, 40.0, 0.0]),  # law[1] s r3 > 1/32: sincos path
                                      (W.OMEGA_SIN, [0.4, 30.0, 0.7]),
                                      (W.OMEGA_PULSE, [0.5, 2.0, 1.0])])
@pytest.mark.parametrize("flow", [1, 2])  # Magnus-4 + Theorem 2, Magnus-6 + Theorem 1
@pytest.mark.parametrize("precision,tol", [("c128", TOL_C128), ("c64", TOL_C64)])
def test_trap_laws_and_magnus_flows(precision, tol, law, lawp, flow):
    """Every time-dependent trap law of Sec. 4.2 under both Magnus flows,
    including fast laws whose Gauss-node offsets leave the small-angle range."""
    need_gpu()
    inst = W.Instance(n=[512], a=[-14.0], b=[14.0], omega_law=law, w0=1.1, law=lawp, eps=0.05,
                      vi_kind=W.VI_COS, vi_k=1.5, sigma=5.0, ho_flow=flow, h=0.01)
    x = inst.x()
    psi0 = (1.1 / math.pi) ** 0.25 * np.exp(-1.1 * (x - 0.5) ** 2 / 2).astype(complex)
    steps = 200
    ref = O.run(O.Problem(**inst.as_dict()), psi0, steps)
    (out,) = _run_gpu([inst], [psi0], steps, precision, inst.h, flow=flow)
    assert O.rel_l2(out, ref) <= budget(tol, steps * inst.h)


@pytest.mark.parametrize("flow", [0, 1, 2])
@pytest.mark.parametrize("precision,tol", [("c128", TOL_C128), ("c64", TOL_C64)])
def test_mixed_trap_laws_in_one_batch(precision, tol, flow):
    """A batch whose instances follow different trap laws takes the schedule
    path that reads the law per instance."""
    need_gpu()
    laws = [(W.OMEGA_CONST, [0.0, 0.0, 0.0]), (W.OMEGA_SIN, [0.3, 1.0, 0.2]), (W.OMEGA_COS_SQ, [0.4, 2.0, 0.0]),
            (W.OMEGA_PULSE, [0.5, 2.0, 1.0])]
    insts, psis = [], []
    for k, (law, lawp) in enumerate(laws):
        if flow == 0 and law != W.OMEGA_CONST:
            lawp = [0.0, lawp[1], lawp[2]]  # the exact flow needs a constant trap
        inst = W.Instance(n=[256 << (k % 2)], a=[-12.0], b=[12.0], omega_law=law, w0=0.9 + 0.2 * k, law=lawp,
                          eps=0.05, vi_kind=W.VI_COS, vi_k=1.5, sigma=4.0, ho_flow=flow, h=0.01)
        x = inst.x()
        insts.append(inst)
        psis.append((inst.w0 / math.pi) ** 0.25 * np.exp(-inst.w0 * (x - 0.3) ** 2 / 2).astype(complex))
    steps = 100
    refs = O.run_batch([O.Problem(**i.as_dict()) for i in insts], psis, steps)
    outs = _run_gpu(insts, psis, steps, precision, 0.01, flow=flow)
    assert max(O.rel_l2(o, r) for o, r in zip(outs, refs)) <= budget(tol, steps * 0.01)


@pytest.mark.parametrize("flow", [1, 2])
@pytest.mark.parametrize("precision,tol", [("c128", TOL_C128), ("c64", TOL_C64)])
def test_one_law_with_per_instance_parameters(precision, tol, flow):
    """Instances that share the law kind but not its parameters: the schedule
    is specialised on the law yet evaluates the trap per instance (no shared
    node table)."""
    need_gpu()
    insts, psis = [], []
    for k, lawp in enumerate([[0.3, 1.0, 0.0], [0.2, 2.5, 0.4], [0.45, 0.7, -1.0]]):
        inst = W.Instance(n=[256 << k], a=[-12.0], b=[12.0], omega_law=W.OMEGA_SIN, w0=0.8 + 0.3 * k, law=lawp,
                          eps=0.05, vi_kind=W.VI_COS, vi_k=1.5, sigma=4.0, ho_flow=flow, h=0.01)
        x = inst.x()
        insts.append(inst)
        psis.append((inst.w0 / math.pi) ** 0.25 * np.exp(-inst.w0 * (x - 0.2) ** 2 / 2).astype(complex))
    steps = 100
    refs = O.run_batch([O.Problem(**i.as_dict()) for i in insts], psis, steps)
    outs = _run_gpu(insts, psis, steps, precision, 0.01, flow=flow)
    assert max(O.rel_l2(o, r) for o, r in zip(outs, refs)) <= budget(tol, steps * 0.01)


@pytest.mark.parametrize("precision,tol", [("c128", TOL_C128), ("c64", TOL_C64)])
def test_mixed_perturbations_and_boxes_in_one_batch(precision, tol):
    """Instances with different perturbation kinds (cos, x^4, none) and a
    shifted box in one batch run the generic step kernel; batches uniform in
    both run a specialised one.  Both agree with the oracle."""
    need_gpu()
    specs = [dict(vi_kind=W.VI_COS, eps=0.05, a=[-12.0], b=[12.0]), dict(vi_kind=W.VI_X4, eps=0.002, a=[-12.0], b=[12.0]),
             dict(vi_kind=W.VI_COS, eps=0.0, a=[-12.0], b=[12.0]), dict(vi_kind=W.VI_COS, eps=0.05, a=[-10.0], b=[14.0])]
    insts, psis = [], []
    for k, sp in enumerate(specs):
        inst = W.Instance(n=[256 << (k % 3)], omega_law=W.OMEGA_SIN, w0=1.0 + 0.1 * k, law=[0.3, 1.0, 0.0], vi_k=1.5,
                          sigma=4.0, ho_flow=1, h=0.01, **sp)
        x = inst.x()
        insts.append(inst)
        psis.append((inst.w0 / math.pi) ** 0.25 * np.exp(-inst.w0 * (x - 0.4) ** 2 / 2).astype(complex))
    steps = 100
    refs = O.run_batch([O.Problem(**i.as_dict()) for i in insts], psis, steps)
    for sub in (slice(0, 4), slice(0, 1), slice(1, 2), slice(2, 3)):  # generic, then uniform batches
        outs = _run_gpu(insts[sub], psis[sub], steps, precision, 0.01)
        assert max(O.rel_l2(o, r) for o, r in zip(outs, refs[sub])) <= budget(tol, steps * 0.01)


@pytest.mark.parametrize("precision,tol", [("c128", TOL_C128), ("c64", TOL_C64)])
def test_cos_perturbation_far_from_the_centre(precision, tol):
    """eps cos(k x) where |k x| reaches a few hundred radians under the state:
    a packet at x0 = 55 in a weak trap, k = 4, on a symmetric box (the
    kernel specialised for cos) and on a box centred at 40 (the generic
    kernel, whose table adds k x_c / 2 pi mod 1).  A large eps makes the
    perturbation's phase dominate the error budget."""
    need_gpu()
    insts, psis = [], []
    for lo, hi in ((-72.0, 72.0), (-32.0, 112.0)):
        inst = W.Instance(n=[4096], a=[lo], b=[hi], omega_law=W.OMEGA_SIN, w0=0.05, law=[0.3, 1.0, 0.0],
                          eps=0.8, vi_kind=W.VI_COS, vi_k=4.0, sigma=2.0, ho_flow=W.FLOW_CF4, h=0.005)
        insts.append(inst)
        psis.append(W.gaussian_1d(inst, x0=55.0, width2=4.0, p0=0.3))
    steps = 300
    outs = _run_gpu(insts, psis, steps, precision, insts[0].h)
    for inst, p0, out in zip(insts, psis, outs):
        ref = O.run(O.Problem(**inst.as_dict()), p0, steps)
        assert O.rel_l2(out, ref) <= budget(tol, steps * inst.h)


@pytest.mark.parametrize("precision,tol", [("c128", TOL_C128), ("c64", TOL_C64)])
def test_asymmetric_box_and_mass(precision, tol):
    """A box not centred at 0 (K1, K0 terms of the chirp) and mu != 1."""
    need_gpu()
    inst = W.Instance(n=[512], a=[-9.0], b=[15.0], mu=1.7, omega_law=W.OMEGA_SIN, w0=1.2, law=[0.2, 1.3, 0.4],
                      eps=0.05, vi_kind=W.VI_X4, sigma=3.0, ho_flow=W.FLOW_CF4, h=0.01)
    psi0 = W.gaussian_1d(inst, x0=2.0, width2=0.7, p0=0.5)
    steps = 200
    ref = O.run(O.Problem(**inst.as_dict()), psi0, steps)
    (out,) = _run_gpu([inst], [psi0], steps, precision, inst.h)
    assert O.rel_l2(out, ref) <= budget(tol, steps * inst.h)


@pytest.mark.parametrize("precision,tol", [("c128", TOL_C128), ("c64", TOL_C64)])
def test_batched_mixed_sizes(precision, tol):
    """A seeded sample of the batched workload (every size 128..4096, ragged
    concatenation) vs the oracle instance by instance."""
    need_gpu()
    insts, psis, _ = W.batch_1d(count=48, seed=11)
    steps = 60
    refs = O.run_batch([O.Problem(**i.as_dict()) for i in insts], psis, steps)
    outs = _run_gpu(insts, psis, steps, precision, 0.005)
    T = steps * 0.005
    errs = [O.rel_l2(o, r) for o, r in zip(outs, refs)]
    assert max(errs) <= budget(tol, T), max(errs)
    assert sorted({i.n[0] for i in insts}) == [128, 256, 512, 1024, 2048, 4096]


@pytest.mark.parametrize("flow,split", [(W.FLOW_M6, W.SPLIT_HO), (W.FLOW_CF4, W.SPLIT_FOURIER)])
@pytest.mark.parametrize("precision,tol", [("c128", TOL_C128), ("c64", TOL_C64)])
def test_batched_mixed_sizes_flows_and_splits(precision, tol, flow, split):
    """The batched workload (every size, the per-perturbation kernel) under
    the sixth-order Magnus flow and under the Fourier split, instance by
    instance against the oracle."""
    need_gpu()
    import dataclasses
    insts, psis, _ = W.batch_1d(count=24, seed=17)
    insts = [dataclasses.replace(i, ho_flow=flow, split=split) for i in insts]
    steps = 40
    refs = O.run_batch([O.Problem(**i.as_dict()) for i in insts], psis, steps)
    outs = _run_gpu(insts, psis, steps, precision, 0.005, flow=flow, split=split)
    errs = [O.rel_l2(o, r) for o, r in zip(outs, refs)]
    assert max(errs) <= budget(tol, steps * 0.005), max(errs)
    assert sorted({i.n[0] for i in insts}) == [128, 256, 512, 1024, 2048, 4096]


def test_streaming_fp64_matches_resident():
    """The FP64 (complex128) step kernel in streaming launches of one and
    three steps gives bitwise the resident result."""
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    insts, psis, _ = W.batch_1d(count=30, seed=23)
    steps = 7
    base = _run_gpu(insts, psis, steps, "c128", 0.005)
    for mode in ((hfs.HFS_MODE_STREAMING, 1), (hfs.HFS_MODE_STREAMING, 3)):
        out = _run_gpu(insts, psis, steps, "c128", 0.005, mode=mode)
        assert all(np.array_equal(a, b) for a, b in zip(base, out))


def test_streaming_many_items_per_cta():
    """With far more work items than CTAs (every CTA takes several items per
    launch, every plan size present), streaming launches of one and two
    steps give bitwise the resident result."""
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    insts, psis, _ = W.batch_1d(count=3000, seed=9)
    steps = 3
    base = _run_gpu(insts, psis, steps, "c64", 0.005)
    for mode in ((hfs.HFS_MODE_STREAMING, 1), (hfs.HFS_MODE_STREAMING, 2)):
        out = _run_gpu(insts, psis, steps, "c64", 0.005, mode=mode)
        assert all(np.array_equal(a, b) for a, b in zip(base, out))


def test_modes_graphs_and_plans_agree():
    """Streaming (one step per launch), resident, graph replay and both plan
    variants give the same FP32 result (bitwise for the launch modes)."""
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    insts, psis, _ = W.batch_1d(count=40, seed=5)
    steps = 30
    base = _run_gpu(insts, psis, steps, "c64", 0.005)
    stream = _run_gpu(insts, psis, steps, "c64", 0.005, mode=(hfs.HFS_MODE_STREAMING, 1))
    stream4 = _run_gpu(insts, psis, steps, "c64", 0.005, mode=(hfs.HFS_MODE_STREAMING, 4))
    graph = _run_gpu(insts, psis, steps, "c64", 0.005, graphs=True)
    for a, b, c, d in zip(base, stream, stream4, graph):
        assert np.array_equal(a, b) and np.array_equal(a, c) and np.array_equal(a, d)
    s = hfs.Solver(insts, precision="c64", chunk_steps=64)
    s.set_schedule(0.005, "strang", hfs.HFS_FLOW_CF4)
    for n in (128, 256, 512, 1024, 2048):
        s.set_plan(n, 8)
    s.set_psi(psis)
    s.step(steps)
    alt = s.split(s.get_psi())
    for a, b in zip(base, alt):
        assert O.rel_l2(b, a) < 5e-6
    s.close()
    refs = O.run_batch([O.Problem(**i.as_dict()) for i in insts], psis, steps)
    assert max(O.rel_l2(b, r) for b, r in zip(alt, refs)) <= budget(TOL_C64, steps * 0.005)
    # a 4096-point instance with 8 values per thread would need a 512-thread team
    d = hfs.Solver(insts[:2], precision="c64")
    with pytest.raises(RuntimeError):
        d.set_plan(4096, 8)
    d.close()


def test_graph_replay_advances_time():
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    insts, psis, _ = W.batch_1d(count=8, seed=9)
    refs = O.run_batch([O.Problem(**i.as_dict()) for i in insts], psis, 40)
    s = hfs.Solver(insts, precision="c64", chunk_steps=64)
    s.set_schedule(0.005, "strang", hfs.HFS_FLOW_CF4)
    s.set_graphs(True)
    s.set_psi(psis)
    for _ in range(4):
        s.step(10)  # same graph replayed; the device-side time advances
    assert abs(s.time - 0.2) < 1e-15
    outs = s.split(s.get_psi())
    assert max(O.rel_l2(o, r) for o, r in zip(outs, refs)) < TOL_C64


def test_checkpoint_resume_bitwise():
    """2n steps in one call equal n steps, a checkpoint (get/set psi + time)
    and n more steps, bitwise, when the schedule chunks coincide."""
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    insts, psis, _ = W.batch_1d(count=16, seed=3)
    n = 25
    a = hfs.Solver(insts, precision="c64", chunk_steps=n)
    a.set_schedule(0.005, "strang", hfs.HFS_FLOW_CF4)
    a.set_psi(psis)
    a.step(2 * n)
    full = a.get_psi()
    b = hfs.Solver(insts, precision="c64", chunk_steps=n)
    b.set_schedule(0.005, "strang", hfs.HFS_FLOW_CF4)
    b.set_psi(psis)
    b.step(n)
    ck, t = b.get_psi(), b.time
    c = hfs.Solver(insts, precision="c64", chunk_steps=n)
    c.set_schedule(0.005, "strang", hfs.HFS_FLOW_CF4)
    c.set_psi(ck)
    c.set_time(t)
    c.step(n)
    assert np.array_equal(full, c.get_psi())


@pytest.mark.parametrize("precision,tol", [("c128", 1e-12), ("c64", 2e-5)])
def test_time_reversibility(precision, tol):
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    inst, psi0, _ = W.gpe_tdep_1d(h=0.01, n=1024)
    s = hfs.Solver([inst], precision=precision)
    s.set_schedule(0.01, "ni5_84", hfs.HFS_FLOW_CF4)
    s.set_psi([psi0])
    s.step(100)
    mid = s.get_psi()
    s.set_schedule(-0.01, "ni5_84", hfs.HFS_FLOW_CF4)
    s.step(100)
    back = s.get_psi()
    assert O.rel_l2(back, psi0) < tol
    assert O.rel_l2(mid, psi0) > 1e-2


@pytest.mark.parametrize("precision", ["c128", "c64"])
def test_norm_and_energy_match_oracle(precision):
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    insts, psis, _ = W.batch_1d(count=24, seed=21)
    s = hfs.Solver(insts, precision=precision)
    s.set_schedule(0.005, "strang", hfs.HFS_FLOW_CF4)
    s.set_psi(psis)
    s.step(40)
    outs = [np.asarray(v, dtype=np.complex128) for v in s.split(s.get_psi())]
    nrm, en = s.norm(), s.energy()
    t = s.time
    tol = 1e-12 if precision == "c128" else 1e-6
    for i, inst in enumerate(insts):
        p = O.Problem(**inst.as_dict())
        assert abs(nrm[i] - O.norm(p, outs[i])) <= tol * abs(nrm[i])
        assert abs(en[i] - O.energy(p, outs[i], t)) <= tol * 10 * max(1.0, abs(en[i]))
        assert abs(nrm[i] - 1.0) < (1e-12 if precision == "c128" else 1e-6)  # norm conservation


def test_eigenstate_phase_gpu():
    """Hermite eigenstate h_4 of omega = 1.3 gains exp(-i 4.5 omega t)."""
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    omega = 1.3
    inst = W.Instance(n=[256], a=[-12.0], b=[12.0], w0=omega, ho_flow=W.FLOW_LEMMA2, h=0.05)
    x = inst.x()
    xs = math.sqrt(omega) * x
    H = [np.ones_like(xs), 2 * xs]
    for k in range(1, 4):
        H.append(2 * xs * H[k] - 2 * k * H[k - 1])
    psi0 = omega ** 0.25 * H[4] * np.exp(-xs ** 2 / 2) / (math.pi ** 0.25 * math.sqrt(2.0 ** 4 * 24))
    for precision, tol in (("c128", 1e-11), ("c64", 2e-5)):
        s = hfs.Solver([inst], precision=precision)
        s.set_schedule(0.05, "strang", hfs.HFS_FLOW_LEMMA2)
        s.set_psi([psi0.astype(complex)])
        s.step(400)
        out = s.get_psi()
        assert O.rel_l2(out, psi0 * np.exp(-1j * 4.5 * omega * 20.0)) < tol


def test_errors_reported():
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    inst = W.Instance(n=[256], a=[-12.0], b=[12.0], w0=2.0, ho_flow=W.FLOW_LEMMA2, h=0.05)
    s = hfs.Solver([inst], precision="c64")
    s.set_schedule(2.0, "strang", hfs.HFS_FLOW_LEMMA2)  # |h| omega = 4 > pi
    with pytest.raises(hfs.HfsError) as ei:
        s.step(1)
    assert ei.value.code == 3
    s.set_schedule(0.05, "strang", hfs.HFS_FLOW_LEMMA2)
    bad = np.zeros(256, complex)
    bad[10] = np.nan
    s.set_psi(bad)
    s.step(2)
    assert s.status() == 5  # HFS_ERR_NONFINITE
    assert s.status() == 0  # cleared


def test_bind_and_step_preconditions():
    """Buffers must be 256-byte aligned and the workspace large enough for the
    chunk; stepping needs bound buffers and a schedule.  Each refusal leaves
    the context usable."""
    need_gpu()
    import ctypes
    import torch
    from paper_1007_3470_gb300 import hfs
    L = hfs.lib()
    insts, psis, _ = W.batch_1d(count=6, seed=3)
    arr = hfs.make_instances(insts)
    h = ctypes.c_void_p()
    assert L.hfs_create(ctypes.byref(h), 1, hfs.HFS_C64, arr, len(insts)) == 0
    try:
        assert L.hfs_step(h, ctypes.c_int64(1)) == 6                    # nothing bound
        elems, _ = hfs.hfs_state_size(h)
        chunk = 16
        wbytes = hfs.hfs_workspace_size(h, chunk)
        psi = torch.zeros(elems + 64, dtype=torch.complex64, device="cuda")
        work = torch.empty(wbytes + 512, dtype=torch.uint8, device="cuda")
        p0, w0 = psi.data_ptr(), work.data_ptr()
        assert p0 % 256 == 0 and w0 % 256 == 0
        bind = lambda p, w, nb: L.hfs_bind(h, ctypes.c_void_p(p), ctypes.c_void_p(w), ctypes.c_size_t(nb),
                                           ctypes.c_int64(chunk))
        assert bind(p0 + 8, w0, wbytes) == 7                             # psi misaligned
        assert bind(p0, w0 + 128, wbytes) == 7                           # workspace misaligned
        assert bind(p0, w0, wbytes - 1) == 8                             # workspace too small
        assert bind(p0, w0, wbytes) == 0
        assert L.hfs_step(h, ctypes.c_int64(1)) == 6                     # no schedule yet
        hfs.hfs_set_schedule(h, hfs.HFS_SPLIT_HO, hfs.HFS_FLOW_CF4, hfs.HFS_COMP_STRANG, 0.005)
        assert L.hfs_step(h, ctypes.c_int64(-1)) == 1
        assert L.hfs_step(h, ctypes.c_int64(3)) == 0
        assert L.hfs_sync_status(h) == 0
    finally:
        L.hfs_destroy(h)


@pytest.mark.parametrize("graphs", [False, True])
def test_profiling_events(graphs):
    """The step-kernel timing hook works with and without graph replay."""
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    insts, psis, _ = W.batch_1d(count=16, seed=4)
    s = hfs.Solver(insts, precision="c64", chunk_steps=32)
    s.set_schedule(0.005, "strang", hfs.HFS_FLOW_CF4)
    with pytest.raises(hfs.HfsError):
        hfs.hfs_last_step_kernel_ms(s.h)
    hfs.hfs_set_profiling(s.h, True)
    s.set_graphs(graphs)
    s.set_psi(psis)
    for _ in range(3):
        s.step(20)
        ms = hfs.hfs_last_step_kernel_ms(s.h)
        assert 0.0 < ms < 1e4
    assert s.status() == hfs.HFS_OK
