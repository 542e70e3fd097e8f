"""Pins of the oracle's trap laws, perturbation and mass scaling against what
the paper and the mathematics fix (each law's omega^2(t) is written below from
Sec. 4.2, and the reference flows come from an independent ODE integrator or
from the exact solution of Lemma 1):

* The cos^2 law omega^2(t) = A (1 + eps cos(w t)) (Sec. 4.2, A = 4, eps = 0.1,
  w = 1/2) and the pulse omega(t) = w0 (1 + A t / cosh^2(B (t - 2))) (Sec. 4.2,
  w0 = 4, A = 0.25, B = 2): the oracle's commutator-free Magnus-4 (Eq.
  CommutatorFree + Theorem 2) and sixth-order Magnus (Sec. 4.2 + Theorem 1)
  stage flows have local orders 5 and 7 against the classical flow of
  q' = p / mu, p' = -mu omega^2(t) q integrated by scipy's DOP853.  A misread
  law (omega for omega^2, a missing square of cosh) leaves an O(s) error and
  fails the order.
* The same for mass mu != 1 (Eq. GP1: p^2 / (2 mu) + mu omega^2 x^2 / 2).
* The quartic perturbation V_I = x^4 and the nonlinearity: a step with a zero
  A stage is two B flows of Lemma 1, whose exact solution is
  u exp(-i h (eps x^4 + sigma |u|^2)) (|u| is invariant under B); in 3D the
  perturbation is the separable sum of x_d^4.  Under the Fourier split the B
  flow also carries mu omega^2(t) x^2 / 2 at the frozen stage time
  (Eq. FourierSplit).
* Hermite eigenstates at mu != 1: h_n(sqrt(mu omega) x) gains
  exp(-i (n + 1/2) omega t) under every harmonic flow (the Magnus flows are
  exact for constant omega).
"""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import oracle as O


def K(c):
    return np.array([[1.0, 0.0], [-c, 1.0]])


def D(g):
    return np.array([[1.0, g], [0.0, 1.0]])


def classical_flow(w2, t0, s, mu):
    """Flow matrix of q' = p / mu, p' = -mu w2(t) q over [t0, t0 + s] (DOP853)."""
    def rhs(t, y):
        m = y.reshape(2, 2)
        J = np.array([[0.0, 1.0 / mu], [-mu * w2(t), 0.0]])
        return (J @ m).ravel()
    sol = solve_ivp(rhs, (t0, t0 + s), np.eye(2).ravel(), method="DOP853", rtol=1e-13, atol=1e-15)
    return sol.y[:, -1].reshape(2, 2)


def cos_sq_paper(t):
    """Sec. 4.2: omega^2(t) = A (1 + eps cos(w t)), A = 4, eps = 0.1, w = 1/2."""
    return 4.0 * (1.0 + 0.1 * math.cos(0.5 * t))


def pulse_paper(t):
    """Sec. 4.2: omega(t) = w0 (1 + A t / cosh^2(B (t - 2))), w0 = 4, A = 0.25, B = 2."""
    w = 4.0 * (1.0 + 0.25 * t / math.cosh(2.0 * (t - 2.0)) ** 2)
    return w * w


# (law, w0, law parameters) in the library's parameterisation:
# COS_SQ: omega^2 = w0^2 (1 + law[0] cos(law[1] t)); PULSE: omega = w0 (1 + law[0] t / cosh^2(law[1] (t - law[2])))
LAWS = {
    "cos_sq": (O.OMEGA_COS_SQ, 2.0, [0.1, 0.5, 0.0], cos_sq_paper),
    "pulse": (O.OMEGA_PULSE, 4.0, [0.25, 2.0, 2.0], pulse_paper),
}
STEPS = {  # step sizes in the asymptotic range of each (law, flow)
    ("cos_sq", O.FLOW_CF4): [0.2, 0.1, 0.05],
    ("cos_sq", O.FLOW_M6): [0.4, 0.2, 0.1],
    ("pulse", O.FLOW_CF4): [0.05, 0.025, 0.0125],
    ("pulse", O.FLOW_M6): [0.1, 0.05, 0.025],
}


@pytest.mark.parametrize("law", ["cos_sq", "pulse"])
def test_law_values(law):
    kind, w0, lp, w2 = LAWS[law]
    prob = O.Problem(n=[8], a=[-1.0], b=[1.0], omega_law=kind, w0=w0, law=lp)
    for t in (0.0, 0.4, 1.7, 2.0, 3.3, 9.0):
        assert abs(O.omega2(prob, t) - w2(t)) <= 1e-14 * w2(t)


@pytest.mark.parametrize("mu", [1.0, 0.6])
@pytest.mark.parametrize("flow,order", [(O.FLOW_CF4, 5), (O.FLOW_M6, 7)])
@pytest.mark.parametrize("law", ["cos_sq", "pulse"])
def test_magnus_local_order_paper_laws(law, flow, order, mu):
    kind, w0, lp, w2 = LAWS[law]
    prob = O.Problem(n=[8], a=[-1.0], b=[1.0], omega_law=kind, w0=w0, law=lp, ho_flow=flow, mu=mu)
    t0 = 1.7  # just before the pulse maximum at t = 2
    errs = []
    for s in STEPS[(law, flow)]:
        f, g, e = O.stage_coeffs(prob, t0, s)
        errs.append(np.abs(K(f) @ D(g) @ K(e) - classical_flow(w2, t0, s, mu)).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(abs(r - order) < 0.4 for r in rates), (errs, rates)


@pytest.mark.parametrize("mu", [0.6, 2.5])
def test_mass_scaling_of_the_m6_flow(mu):
    """Theorem 1 at mu != 1 is the mu = 1 flow conjugated by diag(1, mu); one
    stage of the sixth-order Magnus at a fixed s matches the classical flow of
    the mass-mu oscillator to its local error, with a time-dependent law."""
    prob = O.Problem(n=[8], a=[-1.0], b=[1.0], omega_law=O.OMEGA_SIN, w0=1.2, law=[0.4, 1.5, 0.2],
                     ho_flow=O.FLOW_M6, mu=mu)

    def w2(t):
        return (1.2 * (1.0 + 0.4 * math.sin(1.5 * t + 0.2))) ** 2
    s, t0 = 0.1, 0.3
    f, g, e = O.stage_coeffs(prob, t0, s)
    exact = classical_flow(w2, t0, s, mu)
    assert np.abs(K(f) @ D(g) @ K(e) - exact).max() < 1e-9 * max(1.0, mu, 1.0 / mu)
    # the unscaled (mu = 1) coefficients do not give the mass-mu flow
    f1, g1, e1 = O.stage_coeffs(O.Problem(n=[8], a=[-1.0], b=[1.0], omega_law=O.OMEGA_SIN, w0=1.2,
                                          law=[0.4, 1.5, 0.2], ho_flow=O.FLOW_M6), t0, s)
    assert np.abs(K(f1) @ D(g1) @ K(e1) - exact).max() > 1e-3


def _b_only(**kw):
    """A step whose A stage has zero length: B(b_1 h) then B(b_2 h) (Lemma 1)."""
    return O.Problem(coeffs=([0.0], [0.3, 0.7]), **kw)


@pytest.mark.parametrize("sigma", [0.0, 7.0])
def test_quartic_perturbation_b_flow_closed_form(sigma):
    h, eps = 0.37, 0.05
    prob = _b_only(n=[256], a=[-6.0], b=[7.0], eps=eps, vi_kind=O.VI_X4, sigma=sigma, h=h)
    x = prob.x()
    u0 = np.exp(-(x - 0.4) ** 2 / 2 + 0.8j * x) * (1.0 + 0.2 * np.cos(3 * x))
    exact = u0 * np.exp(-1j * h * (eps * x ** 4 + sigma * np.abs(u0) ** 2))
    assert O.rel_l2(O.run(prob, u0, 1), exact) < 1e-13


def test_quartic_perturbation_3d_is_separable_sum():
    h, eps = 0.21, 0.03
    n = 8
    prob = _b_only(n=[n, n, n], a=[-3.0, -2.0, -4.0], b=[3.0, 2.5, 4.0], eps=eps, vi_kind=O.VI_X4, h=h)
    xs = [prob.x(d) for d in range(3)]
    X, Y, Z = xs[0][None, None, :], xs[1][None, :, None], xs[2][:, None, None]
    u0 = np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / 4).astype(np.complex128)
    exact = u0 * np.exp(-1j * h * eps * (X ** 4 + Y ** 4 + Z ** 4))
    assert O.rel_l2(O.run(prob, u0, 1), exact) < 1e-13


@pytest.mark.parametrize("mu", [1.0, 0.7])
def test_fourier_split_b_flow_carries_the_trap(mu):
    h, t0 = 0.23, 0.9
    prob = _b_only(n=[128], a=[-8.0], b=[8.0], mu=mu, omega_law=O.OMEGA_PULSE, w0=4.0, law=[0.25, 2.0, 2.0],
                   split=O.SPLIT_FOURIER, h=h, t0=t0)
    x = prob.x()
    u0 = np.exp(-x ** 2 / 2).astype(np.complex128)
    exact = u0 * np.exp(-1j * h * 0.5 * mu * pulse_paper(t0) * x ** 2)
    assert O.rel_l2(O.run(prob, u0, 1), exact) < 1e-13


def hermite_function(n, x):
    H = [np.ones_like(x), 2 * x]
    for k in range(1, n):
        H.append(2 * x * H[k] - 2 * k * H[k - 1])
    return H[n] * np.exp(-x * x / 2) / (math.pi ** 0.25 * math.sqrt(2.0 ** n * math.factorial(n)))


@pytest.mark.parametrize("flow", [O.FLOW_LEMMA2, O.FLOW_CF4, O.FLOW_M6])
@pytest.mark.parametrize("n_state", [0, 3])
def test_eigenstate_phase_with_mass(flow, n_state):
    """Eigenstates of p^2/(2 mu) + mu omega^2 x^2 / 2 are h_n(sqrt(mu omega) x)
    with energy (n + 1/2) omega, independent of mu."""
    mu, omega = 0.7, 1.3
    prob = O.Problem(n=[256], a=[-14.0], b=[14.0], mu=mu, w0=omega, ho_flow=flow, h=0.05)
    x = prob.x()
    psi0 = hermite_function(n_state, math.sqrt(mu * omega) * x)
    steps = 200
    exact = psi0 * np.exp(-1j * (n_state + 0.5) * omega * steps * prob.h)
    assert O.rel_l2(O.run(prob, psi0, steps), exact) < 1e-11
