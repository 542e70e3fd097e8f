"""Pins on the coefficient layer of the oracle:

* P2: Lemma 2, Theorem 1 and Theorem 2 as identities of 2x2 symplectic
  matrices -- the classical flow of the quadratic Hamiltonian (computed here
  by scipy.linalg.expm, a library routine) equals kick(f) . drift(g) . kick(e)
  with the e-kick applied first.
* The Magnus integrators (Eq. CommutatorFree; the sixth-order Magnus of
  Sec. 4.2) have local order 5 and 7 against the classical flow of
  q'' = -omega^2(t) q integrated to 1e-13 by scipy's DOP853.
* The Table 1 coefficient sets satisfy their order / quadrature conditions.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sl
from scipy.integrate import solve_ivp

from oracle import oracle as O


def K(c):
    return np.array([[1.0, 0.0], [-c, 1.0]])


def D(g):
    return np.array([[1.0, g], [0.0, 1.0]])


def kdk(f, g, e):
    return K(f) @ D(g) @ K(e)


@pytest.mark.parametrize("mu,omega,t", [(1.0, 1.0, 0.3), (1.0, 1.0, -3.0), (1.0, 2.5, 1.1),
                                        (0.7, 1.3, -0.9), (2.0, 0.4, 5.0), (1.0, 1.0, 1e-6)])
def test_lemma2_matrix_identity(mu, omega, t):
    f, g, e = O.coef_lemma2(mu, omega, t)
    J = np.array([[0.0, 1.0 / mu], [-mu * omega ** 2, 0.0]])
    exact = sl.expm(t * J)
    assert np.abs(kdk(f, g, e) - exact).max() <= 2e-15 * max(1.0, np.abs(exact).max(), abs(f), abs(g))


@pytest.mark.parametrize("mu,wl,wr,t", [(1.0, 1.0, 1.0, 0.5), (1.0, 0.8, 1.7, 1.2), (1.0, 2.3, 0.4, -1.0),
                                        (1.0, -0.05, 1.1, 0.8), (0.5, 1.4, 0.9, 0.7), (1.0, 0.0, 2.0, 0.3),
                                        (1.0, 4.0, 4.2, 1e-5)])
def test_theorem2_matrix_identity(mu, wl, wr, t):
    f, g, e = O.coef_thm2(mu, wl, wr, t)
    JL = np.array([[0.0, 1.0 / mu], [-mu * wl, 0.0]])
    JR = np.array([[0.0, 1.0 / mu], [-mu * wr, 0.0]])
    exact = sl.expm(0.5 * t * JL) @ sl.expm(0.5 * t * JR)  # R applied first
    assert np.abs(kdk(f, g, e) - exact).max() <= 4e-15 * max(1.0, abs(f), abs(e))
    if abs(wl - wr) > 0.1:
        # the reversed kick order is a different operator (reading 3)
        assert np.abs(kdk(e, g, f) - exact).max() > 0.05 * t * t * abs(wl - wr)


@pytest.mark.parametrize("al,be,ga,t", [(1.0, 0.0, 1.0, 0.7), (2.0, 0.3, 1.1, 0.9), (0.5, -0.2, 0.9, -1.3),
                                        (-0.1, 0.05, 1.0, 0.6), (4.0, 0.01, 1.0, 1e-4)])
def test_theorem1_matrix_identity(al, be, ga, t):
    f, g, e = O.coef_thm1(al, be, ga, t)
    J = np.array([[be, ga], [-al, -be]])  # classical flow of (al x^2 + 2 be x p + ga p^2)/2
    exact = sl.expm(t * J)
    assert np.abs(kdk(f, g, e) - exact).max() <= 4e-15 * max(1.0, abs(f), abs(e), 1 / abs(t))


def _classical_flow(w2, t0, s):
    def rhs(t, y):
        m = y.reshape(2, 2)
        J = np.array([[0.0, 1.0], [-w2(t), 0.0]])
        return (J @ m).ravel()
    sol = solve_ivp(rhs, (t0, t0 + s), np.eye(2).ravel(), method="DOP853", rtol=1e-13, atol=1e-15)
    return sol.y[:, -1].reshape(2, 2)


@pytest.mark.parametrize("flow,order", [(O.FLOW_CF4, 5), (O.FLOW_M6, 7)])
def test_magnus_local_order(flow, order):
    prob = O.Problem(n=[8], a=[-1.0], b=[1.0], omega_law=O.OMEGA_SIN, w0=1.0, law=[0.5, 2.0, 0.3],
                     ho_flow=flow)

    def w2(t):
        return (1.0 + 0.5 * math.sin(2.0 * t + 0.3)) ** 2

    t0 = 0.37
    errs = []
    hs = [0.4, 0.2, 0.1] if flow == O.FLOW_CF4 else [0.8, 0.4, 0.2]
    for s in hs:
        f, g, e = O.stage_coeffs(prob, t0, s)
        errs.append(np.abs(kdk(f, g, e) - _classical_flow(w2, t0, s)).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(abs(r - order) < 0.35 for r in rates), (errs, rates)
    # negative steps are the inverse flow's approximation as well
    f, g, e = O.stage_coeffs(prob, t0 + 0.1, -0.1)
    assert np.abs(kdk(f, g, e) - _classical_flow(w2, t0 + 0.1, -0.1)).max() < 2 * errs[-1]


def test_m6_reading_omega_squared_and_beta_sign():
    """The sixth-order Magnus printed with omega_i is read with omega^2 at the
    nodes and beta as printed; flipping beta's sign destroys the order."""
    prob = O.Problem(n=[8], a=[-1.0], b=[1.0], omega_law=O.OMEGA_SIN, w0=1.0, law=[0.5, 2.0, 0.0],
                     ho_flow=O.FLOW_M6)

    def w2(t):
        return (1.0 + 0.5 * math.sin(2.0 * t)) ** 2
    s, t0 = 0.2, 0.1
    f, g, e = O.stage_coeffs(prob, t0, s)
    good = np.abs(kdk(f, g, e) - _classical_flow(w2, t0, s)).max()
    assert good < 2e-7
    # swapping f and e is the same as flipping beta's sign (Theorem 1)
    bad = np.abs(kdk(e, g, f) - _classical_flow(w2, t0, s)).max()
    assert bad > 1e3 * good


def test_cf4_constant_omega_is_exact():
    prob = O.Problem(n=[8], a=[-1.0], b=[1.0], omega_law=O.OMEGA_CONST, w0=1.7, ho_flow=O.FLOW_CF4)
    for s in (0.1, 0.9, -1.5):
        f, g, e = O.stage_coeffs(prob, 0.0, s)
        f2, g2, e2 = O.coef_lemma2(1.0, 1.7, s)
        assert abs(f - f2) < 1e-14 and abs(g - g2) < 1e-14 and abs(e - e2) < 1e-14


# --- Table 1 ----------------------------------------------------------------

def _nodes(a):
    return np.concatenate([[0.0], np.cumsum(a)])


@pytest.mark.parametrize("name", ["strang", "srkn6_4", "ni4_82", "ni5_84"])
def test_composition_consistency(name):
    a, b = O.composition(name)
    assert len(b) == len(a) + 1
    assert abs(sum(a) - 1.0) < 1e-15 and abs(sum(b) - 1.0) < 1e-15
    # symmetric (time-reversible) compositions
    assert np.allclose(a, a[::-1], atol=1e-15) and np.allclose(b, b[::-1], atol=1e-15)


@pytest.mark.parametrize("name,kmax", [("ni4_82", 7), ("ni5_84", 7), ("srkn6_4", 3), ("strang", 1)])
def test_composition_quadrature_conditions(name, kmax):
    """The perturbation part of a BAB composition is a quadrature rule with
    weights b_i at nodes c_i = a_1 + ... + a_{i-1}; the (8,2) and (8,4)
    methods integrate polynomials through degree 7 exactly, the fourth-order
    SRKN through degree 3."""
    a, b = O.composition(name)
    c = _nodes(a)
    for k in range(kmax + 1):
        assert abs(sum(bi * ci ** k for bi, ci in zip(b, c)) - 1.0 / (k + 1)) < 1e-14, k
    assert abs(sum(bi * ci ** (kmax + 1) for bi, ci in zip(b, c)) - 1.0 / (kmax + 2)) > 1e-6


def test_ni4_printed_b2_is_garbled():
    """Table 1 prints b_2 = 49/18 for NI_4; with it the degree-2 condition fails
    by O(1), so the printed value is read as 49/180."""
    a, _ = O.composition("ni4_82")
    b1, b2 = 1 / 20, 49 / 18
    b = [b1, b2, 1 - 2 * (b1 + b2), b2, b1]
    c = _nodes(a)
    assert abs(sum(bi * ci ** 2 for bi, ci in zip(b, c)) - 1 / 3) > 0.1


@pytest.mark.parametrize("name,order", [("strang", 2), ("srkn6_4", 4), ("ni4_82", 2), ("ni5_84", 4)])
def test_composition_order_on_matrices(name, order):
    rng = np.random.default_rng(7)
    n = 6
    A = np.diag(np.arange(n) + 0.5).astype(complex)
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    B = (M + M.conj().T) / 2
    a, b = O.composition(name)

    def comp(h):
        U = np.eye(n, dtype=complex)
        for i in range(len(a)):
            U = sl.expm(-1j * h * b[i] * B) @ U
            U = sl.expm(-1j * h * a[i] * A) @ U
        return sl.expm(-1j * h * b[-1] * B) @ U

    errs = [np.abs(comp(h) - sl.expm(-1j * h * (A + B))).max() for h in (0.2, 0.1)]
    assert abs(math.log2(errs[0] / errs[1]) - (order + 1)) < 0.35


def test_table1_printed_values():
    """Compare with the decimals printed in Table 1 (golden fixture)."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_coefficients.json")
    with open(path) as fh:
        gold = json.load(fh)
    for name, ent in gold["methods"].items():
        a, b = O.composition(name)
        for k, v in ent["b"].items():
            assert abs(b[int(k) - 1] - v) < 1e-15, (name, k)
        for k, v in ent["a"].items():
            assert abs(a[int(k) - 1] - v) < 1e-15, (name, k)


def test_explicit_composition_coefficients():
    """The oracle's explicit (a, b) coefficients: a named scheme's own
    coefficients reproduce it exactly; a wrong count is refused; and the order
    follows the order conditions.  With a = (0.3, 0.7) the second-order
    condition sum_i a_i (b_1 + ... + b_i) = 1/2 holds for b = (0.15, 0.5, 0.35)
    and fails for b = (0.25, 0.5, 0.25) (0.6): global errors fall as h^2 and
    as h respectively."""
    import dataclasses
    base = O.Problem(n=[128], a=[-10.0], b=[10.0], w0=1.0, eps=0.05, vi_kind=O.VI_COS, vi_k=1.5, sigma=2.0,
                     ho_flow=O.FLOW_LEMMA2, scheme="srkn6_4", h=0.05)
    x = np.linspace(-10, 10, 128, endpoint=False)
    psi0 = (np.pi ** -0.25 * np.exp(-(x - 0.5) ** 2 / 2)).astype(complex)
    named = O.run(base, psi0, 10)
    same = O.run(dataclasses.replace(base, coeffs=O.composition("srkn6_4")), psi0, 10)
    assert np.array_equal(named, same)
    with pytest.raises(ValueError):
        O.run(dataclasses.replace(base, coeffs=([0.5, 0.5], [1.0, 0.0])), psi0, 1)
    T = 1.0
    ref = O.run(dataclasses.replace(base, scheme="ni5_84", h=T / 200), psi0, 200)

    def rate(coeffs):
        e = [O.rel_l2(O.run(dataclasses.replace(base, coeffs=coeffs, h=T / k), psi0, k), ref) for k in (20, 40)]
        return math.log2(e[0] / e[1])

    for b, order in (([0.15, 0.5, 0.35], 2.0), ([0.25, 0.5, 0.25], 1.0)):
        assert abs(sum(ai * sum(b[: i + 1]) for i, ai in enumerate([0.3, 0.7])) - 0.5) < 1e-12 or order == 1.0
        assert abs(rate(([0.3, 0.7], b)) - order) < 0.3
