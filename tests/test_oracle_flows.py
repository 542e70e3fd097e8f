"""Pins of the oracle's full split step against what the paper and the
mathematics fix:

* P3  one exact HO step of the ground state over T in (-pi, pi) reproduces
      exp(-iT/2) psi_0 to round-off (Sec. 4, Fig. 1 experiment).
* P4  Hermite eigenstates (Eq. Hermite / EigenHarm) gain exp(-i(n+1/2) omega t).
* P5  a coherent state matches its closed form; its centre follows x0 cos t.
* P6  the norm is conserved (Lemma 1; unitary drift and kicks).
* P7  the symmetric schemes are time reversible.
* P9  one linear step equals scipy.linalg.expm of the discretised Hamiltonian.
* P10 the HO split and the F split converge to the same solution.
* P11 the energy of an autonomous problem stays bounded.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import oracle as O
from paper_1007_3470_gb300 import workloads as W


def hermite_function(n, x):
    """h_n(x) of Eq. EigenHarm from the three-term recursion of H_n."""
    H = [np.ones_like(x), 2 * x]
    for k in range(1, n):
        H.append(2 * x * H[k] - 2 * k * H[k - 1])
    return H[n] * np.exp(-x * x / 2) / (math.pi ** 0.25 * math.sqrt(2.0 ** n * math.factorial(n)))


@pytest.mark.parametrize("T", [-3.0, -2.0, -1.0, -0.3, 0.3, 1.0, 2.0, 3.0])
def test_p3_one_step_ground_state(T):
    prob = O.Problem(n=[1024], a=[-10.0], b=[10.0], h=T, ho_flow=O.FLOW_LEMMA2)
    x = prob.x()
    psi0 = math.pi ** -0.25 * np.exp(-x ** 2 / 2)
    u = O.run(prob, psi0, 1)
    exact = psi0 * np.exp(-0.5j * T)
    assert O.rel_l2(u, exact) < 5e-14


def test_p3_chirp_aliasing_near_pi():
    """Near |T| = pi the chirp f = tan(T/2) is not resolved on a coarse grid
    (|f| max|x| > pi/dx); the fine grid of the paper's experiment still is."""
    T = -3.0
    coarse = O.Problem(n=[256], a=[-12.0], b=[12.0], h=T)
    x = coarse.x()
    psi0 = math.pi ** -0.25 * np.exp(-x ** 2 / 2)
    err = O.rel_l2(O.run(coarse, psi0, 1), psi0 * np.exp(-0.5j * T))
    assert err > 1e-3


@pytest.mark.parametrize("flow", [O.FLOW_LEMMA2, O.FLOW_CF4, O.FLOW_M6])
@pytest.mark.parametrize("n_state", [0, 1, 4, 10])
def test_p4_eigenstate_phase(flow, n_state):
    omega = 1.3
    prob = O.Problem(n=[256], a=[-12.0], b=[12.0], w0=omega, ho_flow=flow, h=0.05, scheme="strang")
    x = prob.x()
    psi0 = omega ** 0.25 * hermite_function(n_state, math.sqrt(omega) * x)
    steps = 400
    u = O.run(prob, psi0, steps)
    t = steps * prob.h
    exact = psi0 * np.exp(-1j * (n_state + 0.5) * omega * t)
    assert O.rel_l2(u, exact) < 1e-11


def test_p5_coherent_state_closed_form():
    x0 = 1.0
    prob = O.Problem(n=[256], a=[-16.0], b=[16.0], w0=1.0, h=0.1, ho_flow=O.FLOW_LEMMA2)
    x = prob.x()

    def coherent(t):
        q, p = x0 * math.cos(t), -x0 * math.sin(t)
        return math.pi ** -0.25 * np.exp(-(x - q) ** 2 / 2 + 1j * p * (x - q / 2) - 0.5j * t)

    u = coherent(0.0)
    for k in range(1, 11):
        u = O.run(O.Problem(n=[256], a=[-16.0], b=[16.0], w0=1.0, h=0.1, t0=(k - 1) * 1.0), u, 10)
        t = k * 1.0
        assert O.rel_l2(u, coherent(t)) < 1e-12
        centre = prob.dv() * np.sum(x * np.abs(u) ** 2)
        assert abs(centre - x0 * math.cos(t)) < 1e-12


@pytest.mark.parametrize("scheme", ["strang", "ni5_84", "srkn6_4", "ni4_82"])
def test_p6_norm_conservation(scheme):
    inst, psi0, _ = W.gpe_tdep_1d(h=0.02, scheme=scheme, n=512)
    prob = O.Problem(**inst.as_dict())
    u = O.run(prob, psi0, 100)
    assert abs(O.norm(prob, u) - O.norm(prob, psi0)) < 1e-13


@pytest.mark.parametrize("scheme,flow", [("strang", O.FLOW_CF4), ("ni5_84", O.FLOW_CF4), ("srkn6_4", O.FLOW_M6)])
def test_p7_time_reversibility(scheme, flow):
    inst, psi0, _ = W.gpe_tdep_1d(h=0.02, scheme=scheme, n=512, ho_flow=flow)
    fwd = O.Problem(**inst.as_dict())
    n = 50
    u = O.run(fwd, psi0, n)
    d = inst.as_dict()
    d.update(h=-inst.h, t0=n * inst.h)
    back = O.Problem(**d)
    v = O.run(back, u, n)
    assert O.rel_l2(v, psi0) < 1e-12
    assert O.rel_l2(u, psi0) > 1e-2


def _dense_ops(prob):
    n = prob.n[0]
    x = prob.x()
    L = prob.b[0] - prob.a[0]
    m = np.where(np.arange(n) < n // 2, np.arange(n), np.arange(n) - n)
    k = 2 * np.pi / L * m
    Fm = np.fft.fft(np.eye(n), axis=0)
    Fi = np.fft.ifft(np.eye(n), axis=0)
    T = Fi @ np.diag(k ** 2 / 2) @ Fm
    P = Fi @ np.diag(k) @ Fm
    X = np.diag(x)
    return X, T, P


@pytest.mark.parametrize("flow", [O.FLOW_LEMMA2, O.FLOW_CF4, O.FLOW_M6])
def test_p9_dense_expm(flow):
    """One linear step (eps = sigma = 0) equals the matrix exponential of the
    discretised harmonic Hamiltonian (Magnus-approximated for omega(t))."""
    law = O.OMEGA_CONST if flow == O.FLOW_LEMMA2 else O.OMEGA_SIN
    prob = O.Problem(n=[64], a=[-8.0], b=[8.0], omega_law=law, w0=1.1, law=[0.4, 1.5, 0.2],
                     ho_flow=flow, h=0.5, t0=0.3)
    X, T, P = _dense_ops(prob)
    x = prob.x()
    psi0 = np.exp(-(x - 0.5) ** 2 / 2 + 0.3j * x)
    u = O.run(prob, psi0, 1)
    s, t0 = prob.h, prob.t0
    if flow == O.FLOW_LEMMA2:
        U = sl.expm(-1j * s * (T + 1.1 ** 2 * X @ X / 2))
    elif flow == O.FLOW_CF4:
        c1, c2 = 0.5 - math.sqrt(3) / 6, 0.5 + math.sqrt(3) / 6
        al = 0.5 - 1 / math.sqrt(3)
        be = 1 - al
        w1, w2 = O.omega2(prob, t0 + c1 * s), O.omega2(prob, t0 + c2 * s)
        wl, wr = al * w1 + be * w2, be * w1 + al * w2
        U = sl.expm(-0.5j * s * (T + wl * X @ X / 2)) @ sl.expm(-0.5j * s * (T + wr * X @ X / 2))
    else:
        r = math.sqrt(15) / 10
        w1, w2, w3 = (O.omega2(prob, t0 + c * s) for c in (0.5 - r, 0.5, 0.5 + r))
        al = (5 * w1 + 8 * w2 + 5 * w3) / 18 + s * s / 486 * (
            17 / 4 * (w1 ** 2 + w3 ** 2) + 8 * w2 ** 2 + w1 * w2 + w2 * w3 - 37 / 2 * w1 * w3)
        be = s * math.sqrt(5 / 3) * (w3 - w1) * (1 / 12 + s * s / 3240 * (5 * w1 + 8 * w2 + 5 * w3))
        ga = 1 + s * s / 54 * (w1 - 2 * w2 + w3)
        U = sl.expm(-0.5j * s * (al * X @ X + be * (X @ P + P @ X) + ga * 2 * T))
    assert O.rel_l2(u, U @ psi0) < 1e-11


def test_p10_cross_split_convergence():
    """The HO split (Eq. HermiteSplit) and the F split (Eq. FourierSplit) are
    independent discretisations in time; both converge at order 2 (Strang)
    to the same limit, computed here by the fourth-order NI_5 HO split."""
    base, _, _ = W.gpe_tdep_1d(h=0.001, n=512, scheme="ni5_84")
    base.a, base.b = [-16.0], [16.0]
    psi0 = W.gaussian_1d(base)
    T = 1.0
    ref = O.run(O.Problem(**base.as_dict()), psi0, int(round(T / base.h)))
    for split in (O.SPLIT_HO, O.SPLIT_FOURIER):
        errs = []
        for h in (0.01, 0.005):
            d = base.as_dict()
            d.update(split=split, scheme="strang", h=h)
            errs.append(O.rel_l2(O.run(O.Problem(**d), psi0, int(round(T / h))), ref))
        assert errs[0] < 1e-2
        assert abs(math.log2(errs[0] / errs[1]) - 2.0) < 0.3, (split, errs)


def test_p11_energy_bounded_autonomous():
    inst = W.Instance(n=[512], a=[-16.0], b=[16.0], w0=1.0, eps=0.1, vi_kind=W.VI_COS, vi_k=2.0,
                      sigma=10.0, ho_flow=W.FLOW_LEMMA2, scheme="strang", h=0.01)
    psi0 = W.gaussian_1d(inst, x0=0.5)
    prob = O.Problem(**inst.as_dict())
    E0 = O.energy(prob, psi0, 0.0)
    u = psi0
    Es = []
    for k in range(20):
        u = O.run(prob, u, 50)
        Es.append(O.energy(prob, u, 0.0))
    dev = np.abs(np.array(Es) - E0) / abs(E0)
    assert dev.max() < 2e-3
    # energy of the ground state of the pure HO is 1/2 (closed form)
    g = O.Problem(n=[256], a=[-12.0], b=[12.0])
    xg = g.x()
    assert abs(O.energy(g, math.pi ** -0.25 * np.exp(-xg ** 2 / 2), 0.0) - 0.5) < 1e-13


def test_energy_kinetic_closed_form():
    # plane-wave Gaussian: <p^2>/2 = 1/4 + p0^2/2 for exp(-x^2/2 + i p0 x)
    g = O.Problem(n=[512], a=[-16.0], b=[16.0], w0=0.0)
    inst = W.Instance(n=[512], a=[-16.0], b=[16.0])
    psi = W.gaussian_1d(inst, p0=1.5)
    assert abs(O.energy(g, psi, 0.0) - (0.25 + 1.5 ** 2 / 2)) < 1e-12
