"""Pin P8: convergence order under dt halving on the time-dependent GPE of
the Magnus-4 workload (omega(t)=1+0.5 sin 2t, sigma=10, eps cos 2x) -- Strang
order 2, NI_5(8,4) and SRKN_6 4 order 4, NI_4(8,2) order 2 (Table 1) -- and
the pure Magnus orders (Eq. CommutatorFree: 4; sixth-order Magnus of Sec. 4.2:
6) on the linear time-dependent oscillator."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1007_3470_gb300 import workloads as W

T = 2.0


@pytest.fixture(scope="module")
def reference():
    inst, psi0, _ = W.gpe_tdep_1d(h=0.00125, T=T, scheme="ni5_84")
    return O.run(O.Problem(**inst.as_dict()), psi0, int(round(T / inst.h)))


@pytest.mark.parametrize("scheme,flow,order", [("strang", O.FLOW_CF4, 2), ("ni5_84", O.FLOW_CF4, 4),
                                               ("ni5_84", O.FLOW_M6, 4), ("ni4_82", O.FLOW_CF4, 2),
                                               ("srkn6_4", O.FLOW_CF4, 4)])
def test_p8_composition_order(reference, scheme, flow, order):
    hs = (0.04, 0.02, 0.01)
    errs = []
    for h in hs:
        inst, psi0, steps = W.gpe_tdep_1d(h=h, T=T, scheme=scheme, ho_flow=flow)
        errs.append(O.rel_l2(O.run(O.Problem(**inst.as_dict()), psi0, steps), reference))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(abs(r - order) < 0.3 for r in rates), (errs, rates)


@pytest.mark.parametrize("flow,order", [(O.FLOW_CF4, 4), (O.FLOW_M6, 6)])
def test_p8_magnus_order_linear(flow, order):
    def make(h):
        return O.Problem(n=[256], a=[-12.0], b=[12.0], omega_law=O.OMEGA_SIN, w0=1.0, law=[0.5, 2.0, 0.0],
                         ho_flow=flow, scheme="strang", h=h)
    x = make(0.1).x()
    psi0 = math.pi ** -0.25 * np.exp(-(x - 1.0) ** 2 / 2)
    ref = O.run(make(0.00625), psi0, int(round(T / 0.00625)))
    errs = [O.rel_l2(O.run(make(h), psi0, int(round(T / h))), ref) for h in (0.2, 0.1, 0.05)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(abs(r - order) < 0.35 for r in rates), (errs, rates)


def test_p8_exact_flow_constant_omega_any_h():
    """With constant omega and no perturbation the HO split is exact for any
    |h| < pi/omega: results for h and h/2 agree to round-off."""
    def make(h):
        return O.Problem(n=[256], a=[-12.0], b=[12.0], w0=1.0, ho_flow=O.FLOW_LEMMA2, h=h)
    x = make(0.1).x()
    psi0 = math.pi ** -0.25 * np.exp(-(x - 1.0) ** 2 / 2)
    u1 = O.run(make(0.8), psi0, 5)
    u2 = O.run(make(0.4), psi0, 10)
    assert O.rel_l2(u1, u2) < 1e-13


@pytest.mark.parametrize("sigma,factor", [(0.01, 100.0), (1.0, 2.0)])
def test_ho_split_beats_f_split_at_equal_fft_count(sigma, factor):
    """Sec. 4 (HO-split versus F-split): with the same leap-frog composition,
    hence the same number of FFTs per step, the HO split is the more accurate
    one for a weakly perturbed oscillator (sigma = 0.01, 1); the reference is
    the fourth-order NI_5(8,4) HO split at a much smaller step."""
    T = 2.0
    ref_inst, psi0 = W.split_comparison_1d(sigma, n=512, h=0.002)
    ref_inst.scheme = "ni5_84"
    ref = O.run(O.Problem(**ref_inst.as_dict()), psi0, int(round(T / 0.002)))
    for h in (0.04, 0.02):
        errs = {}
        for split in (O.SPLIT_HO, O.SPLIT_FOURIER):
            inst, _ = W.split_comparison_1d(sigma, n=512, h=h, split=split)
            errs[split] = O.rel_l2(O.run(O.Problem(**inst.as_dict()), psi0, int(round(T / h))), ref)
        assert errs[O.SPLIT_HO] * factor < errs[O.SPLIT_FOURIER], (h, errs)
