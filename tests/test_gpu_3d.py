"""GPU parity of the 3D split step (diagonal trap (1, 1.5^2, 2^2)(1 + 0.3 sin t)^2,
sigma=100, eps sum_d cos 2x_d) against the FP64 oracle, and FP32 vs FP64 on
the device at 128^3."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1007_3470_gb300 import workloads as W
from tests.gpu_helpers import TOL_C128, TOL_C64, budget, need_gpu

pytestmark = pytest.mark.gpu


def _gpu3d(inst, psi0, steps, precision, chunk=512):
    from paper_1007_3470_gb300 import hfs
    s = hfs.Solver([inst], dim=3, precision=precision, chunk_steps=chunk)
    s.set_schedule(inst.h, inst.scheme, inst.ho_flow, inst.split)
    s.set_psi(psi0.ravel())
    s.step(steps)
    out = s.split(s.get_psi())[0]
    assert s.status() == hfs.HFS_OK
    nrm, en = s.norm()[0], s.energy()[0]
    s.close()
    return np.asarray(out), nrm, en


@pytest.mark.parametrize("n", [32, 64])
@pytest.mark.parametrize("precision,tol", [("c128", TOL_C128), ("c64", TOL_C64)])
def test_3d_vs_oracle(n, precision, tol):
    need_gpu()
    inst, psi0, _ = W.gpe_3d(n=n, h=0.005)
    steps = 20
    ref = O.run(O.Problem(**inst.as_dict()), psi0, steps)
    out, nrm, en = _gpu3d(inst, psi0, steps, precision)
    assert O.rel_l2(out, ref) <= budget(tol, steps * inst.h)
    p = O.Problem(**inst.as_dict())
    rtol = 1e-12 if precision == "c128" else 1e-6
    assert abs(nrm - O.norm(p, ref)) <= rtol
    assert abs(en - O.energy(p, ref, steps * inst.h)) <= (1e-11 if precision == "c128" else 3e-5) * abs(en)


def test_3d_128_fp32_vs_fp64_and_oracle():
    need_gpu()
    inst, psi0, _ = W.gpe_3d(n=128, h=0.005)
    steps = 6
    o32, n32, e32 = _gpu3d(inst, psi0, steps, "c64")
    o64, n64, e64 = _gpu3d(inst, psi0, steps, "c128")
    T = steps * inst.h
    assert O.rel_l2(o32, o64) <= TOL_C64 * max(T, 1.0) * 0.1
    assert abs(n32 - 1.0) < 1e-6 and abs(n64 - 1.0) < 1e-12
    ref = O.run(O.Problem(**inst.as_dict()), psi0, steps)
    assert O.rel_l2(o64, ref) <= TOL_C128 * max(T, 1.0)


def test_3d_chunked_equals_oracle():
    """Several schedule chunks (chunk boundaries re-split the merged phases)."""
    need_gpu()
    inst, psi0, _ = W.gpe_3d(n=32, h=0.01)
    steps = 13
    ref = O.run(O.Problem(**inst.as_dict()), psi0, steps)
    out, _, _ = _gpu3d(inst, psi0, steps, "c128", chunk=4)
    assert O.rel_l2(out, ref) <= budget(TOL_C128, steps * inst.h)


@pytest.mark.parametrize("vi_kind,eps", [(W.VI_X4, 2e-5), (W.VI_NONE, 0.05), (W.VI_COS, 0.0)])
def test_3d_128_plane_kernels_per_perturbation(vi_kind, eps):
    """The 128^3 complex64 plane kernel is compiled per perturbation kind in
    effect (x^4; none; cos with eps = 0 is none); each agrees with the FP64
    line-pass path and with the oracle."""
    need_gpu()
    import dataclasses
    inst, psi0, _ = W.gpe_3d(n=128, h=0.005)
    inst = dataclasses.replace(inst, vi_kind=vi_kind, eps=eps)
    steps = 4
    o32, n32, _ = _gpu3d(inst, psi0, steps, "c64")
    o64, _, _ = _gpu3d(inst, psi0, steps, "c128")
    T = steps * inst.h
    assert O.rel_l2(o32, o64) <= TOL_C64 * max(T, 1.0) * 0.1
    assert abs(n32 - 1.0) < 1e-6
    ref = O.run(O.Problem(**inst.as_dict()), psi0, steps)
    assert O.rel_l2(o64, ref) <= TOL_C128 * max(T, 1.0)


@pytest.mark.parametrize("flow,split,law", [(W.FLOW_M6, W.SPLIT_HO, None), (W.FLOW_CF4, W.SPLIT_FOURIER, None),
                                            (W.FLOW_LEMMA2, W.SPLIT_HO, W.OMEGA_CONST)])
@pytest.mark.parametrize("precision,tol", [("c128", TOL_C128), ("c64", TOL_C64)])
def test_3d_schedule_variants_vs_oracle(precision, tol, flow, split, law):
    """3D with the sixth-order Magnus + Theorem 1 flow, the Fourier split, and
    the exact flow (Lemma 2) of a constant trap, against the oracle."""
    need_gpu()
    import dataclasses
    inst, psi0, _ = W.gpe_3d(n=32, h=0.005)
    inst = dataclasses.replace(inst, ho_flow=flow, split=split)
    if law is not None:
        inst = dataclasses.replace(inst, omega_law=law)
    steps = 16
    ref = O.run(O.Problem(**inst.as_dict()), psi0, steps)
    out, nrm, _ = _gpu3d(inst, psi0, steps, precision)
    assert O.rel_l2(out, ref) <= budget(tol, steps * inst.h)
    assert abs(nrm - 1.0) < (1e-12 if precision == "c128" else 1e-6)


def test_3d_128_fourier_split_plane_vs_fp64():
    """The 128^3 complex64 plane kernels under the Fourier split (trap in the
    x-phase) agree with the FP64 line passes."""
    need_gpu()
    import dataclasses
    inst, psi0, _ = W.gpe_3d(n=128, h=0.005)
    inst = dataclasses.replace(inst, split=W.SPLIT_FOURIER)
    steps = 4
    o32, n32, _ = _gpu3d(inst, psi0, steps, "c64")
    o64, _, _ = _gpu3d(inst, psi0, steps, "c128")
    assert O.rel_l2(o32, o64) <= TOL_C64 * max(steps * inst.h, 1.0) * 0.1
    assert abs(n32 - 1.0) < 1e-6
