"""Pins of the oracle's 3D step (diagonal trap x^T M(t) x, Sec. 1): for a
separable linear problem the 3D solution is the product of three 1D
solutions; the anisotropic ground state gains exp(-i t sum_d omega_d/2);
the norm is conserved and the symmetric scheme is reversible with the
nonlinearity switched on."""
import math

import numpy as np

from oracle import oracle as O
from paper_1007_3470_gb300 import workloads as W


def _prob3(n=16, sigma=0.0, eps=0.0, law=O.OMEGA_SIN, h=0.05, t0=0.0, hw=6.0):
    return O.Problem(n=[n, n, n], a=[-hw] * 3, b=[hw] * 3, omega_law=law, w0=1.0, law=[0.3, 1.0, 0.0],
                     axis_scale=[1.0, 1.5, 2.0], eps=eps, vi_kind=O.VI_COS, vi_k=2.0, sigma=sigma,
                     ho_flow=O.FLOW_CF4, h=h, t0=t0)


def test_3d_separable_equals_product_of_1d():
    p3 = _prob3(n=16, eps=0.05)
    x = p3.x(0)
    cs = (1.0, 1.5, 2.0)
    g1 = [np.exp(-c * (x - 0.3 * d) ** 2 / 2 + 0.2j * d * x) for d, c in enumerate(cs)]
    psi3 = g1[2][:, None, None] * g1[1][None, :, None] * g1[0][None, None, :]
    u3 = O.run(p3, psi3, 20)
    outs = []
    for d, c in enumerate(cs):
        p1 = O.Problem(n=[16], a=[-6.0], b=[6.0], omega_law=O.OMEGA_SIN, w0=c, law=[0.3, 1.0, 0.0],
                       eps=0.05, vi_kind=O.VI_COS, vi_k=2.0, ho_flow=O.FLOW_CF4, h=0.05)
        outs.append(O.run(p1, g1[d], 20))
    prod = outs[2][:, None, None] * outs[1][None, :, None] * outs[0][None, None, :]
    assert O.rel_l2(u3, prod) < 1e-12


def test_3d_anisotropic_ground_state_phase():
    p3 = _prob3(n=64, law=O.OMEGA_CONST, h=0.1, hw=9.0)
    x = p3.x(0)
    cs = (1.0, 1.5, 2.0)
    psi = np.exp(-(cs[2] * x[:, None, None] ** 2 + cs[1] * x[None, :, None] ** 2
                   + cs[0] * x[None, None, :] ** 2) / 2).astype(complex)
    u = O.run(p3, psi, 30)
    t = 3.0
    assert O.rel_l2(u, psi * np.exp(-0.5j * t * sum(cs))) < 1e-12


def test_3d_norm_and_reversibility_nonlinear():
    inst, psi0, _ = W.gpe_3d(n=16, h=0.01)
    p = O.Problem(**inst.as_dict())
    u = O.run(p, psi0, 10)
    assert abs(O.norm(p, u) - 1.0) < 1e-13
    d = inst.as_dict()
    d.update(h=-inst.h, t0=10 * inst.h)
    v = O.run(O.Problem(**d), u, 10)
    assert O.rel_l2(v, psi0) < 1e-12
    assert O.rel_l2(u, psi0) > 1e-3


def test_3d_energy_ground_state():
    p3 = _prob3(n=64, law=O.OMEGA_CONST, hw=9.0)
    x = p3.x(0)
    cs = (1.0, 1.5, 2.0)
    psi = np.exp(-(cs[2] * x[:, None, None] ** 2 + cs[1] * x[None, :, None] ** 2
                   + cs[0] * x[None, None, :] ** 2) / 2).astype(complex)
    psi /= math.sqrt(p3.dv() * np.sum(np.abs(psi) ** 2))
    # E = sum_d omega_d / 2 for the product ground state
    assert abs(O.energy(p3, psi, 0.0) - sum(cs) / 2) < 1e-10
