"""The tensor-core DFT stages of the 3D z-pass (hfs_set_dft_engine with
HFS_DFT_TENSOR_3XTF32): the radix-16 pass of every forward and inverse
z-transform (Eq. GP1ODE_T along z) as a 3xTF32 matrix product on tcgen05.
Parity against the FP64 oracle at 64^3 and against the FP64 device path at
128^3 over a few steps; over the full 200-step 128^3 workload the measured
systematic norm loss of the tensor-core stages (why the FP32 butterflies stay
the default); the engine's preconditions."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1007_3470_gb300 import workloads as W
from tests.gpu_helpers import TOL_C128, TOL_C64, budget, need_gpu

pytestmark = pytest.mark.gpu


def _run(inst, psi0, steps, precision="c64", engine=0):
    from paper_1007_3470_gb300 import hfs
    s = hfs.Solver([inst], dim=3, precision=precision, chunk_steps=steps)
    s.set_schedule(inst.h, inst.scheme, inst.ho_flow, inst.split)
    if engine:
        s.set_dft_engine(engine)
    s.set_psi(psi0.ravel())
    n0 = s.norm()[0]
    s.step(steps)
    out = np.asarray(s.split(s.get_psi())[0])
    assert s.status() == hfs.HFS_OK
    n1 = s.norm()[0]
    s.close()
    return out, n1 / n0 - 1.0


def test_tc_64_vs_oracle_and_simt():
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    inst, psi0, _ = W.gpe_3d(n=64, h=0.005)
    steps = 20
    ref = O.run(O.Problem(**inst.as_dict()), psi0, steps)
    tc, drift = _run(inst, psi0, steps, engine=hfs.HFS_DFT_TENSOR_3XTF32)
    simt, _ = _run(inst, psi0, steps)
    e_tc, e_simt = O.rel_l2(tc, ref), O.rel_l2(simt, ref)
    print(f"64^3 x {steps}: rel-L2 vs oracle tensor {e_tc:.3e} simt {e_simt:.3e}, drift {drift:.2e}")
    assert e_tc <= budget(TOL_C64, steps * inst.h), e_tc
    assert e_simt <= budget(TOL_C64, steps * inst.h), e_simt


def test_tc_128_short_run_vs_fp64_device():
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    inst, psi0, _ = W.gpe_3d(n=128, h=0.005)
    steps = 6
    tc, _ = _run(inst, psi0, steps, engine=hfs.HFS_DFT_TENSOR_3XTF32)
    f64, _ = _run(inst, psi0, steps, precision="c128")
    assert O.rel_l2(tc, f64) <= budget(TOL_C64, steps * inst.h), O.rel_l2(tc, f64)


def test_tc_128_full_length_norm_loss():
    """Over the full 200-step workload the tensor-core stages lose norm
    systematically (the FP32 accumulation inside the tensor core shrinks
    magnitudes), which sigma |psi|^2 turns into a phase error above the
    parity bound, while the FP32 butterflies stay unbiased: the measured
    reason the engine is not the default."""
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    inst, psi0, _ = W.gpe_3d(n=128, h=0.005)
    steps = 200
    tc, d_tc = _run(inst, psi0, steps, engine=hfs.HFS_DFT_TENSOR_3XTF32)
    simt, d_simt = _run(inst, psi0, steps)
    f64, _ = _run(inst, psi0, steps, precision="c128")
    e_tc, e_simt = O.rel_l2(tc, f64), O.rel_l2(simt, f64)
    print(f"128^3 x 200 vs FP64 device: tensor {e_tc:.3e} (drift {d_tc:.2e}), simt {e_simt:.3e} (drift {d_simt:.2e})")
    assert e_simt <= budget(TOL_C64, steps * inst.h)
    assert d_tc < -1e-5 and abs(d_simt) < 1e-7
    assert e_tc > 5 * e_simt


def test_tc_engine_preconditions():
    need_gpu()
    from paper_1007_3470_gb300 import hfs
    cases = ((3, "c64", W.gpe_3d(n=32)[0]), (3, "c128", W.gpe_3d(n=64)[0]),
             (1, "c64", W.batch_1d(count=1)[0][0]))
    for dim, prec, inst in cases:
        s = hfs.Solver([inst], dim=dim, precision=prec, chunk_steps=4)
        with pytest.raises(hfs.HfsError) as ei:
            s.set_dft_engine(hfs.HFS_DFT_TENSOR_3XTF32)
        assert ei.value.code == 2  # HFS_ERR_UNSUPPORTED
        with pytest.raises(hfs.HfsError) as ei:
            s.set_dft_engine(7)
        assert ei.value.code == 1  # HFS_ERR_INVALID_ARG
        s.set_dft_engine(hfs.HFS_DFT_SIMT)
        s.close()
