"""Pins of the Hermite-basis cross-check (oracle/hermite.py):

* the basis sizes printed in Sec. 4 for the displaced ground state (golden
  fixture tests/golden/e2_hermite_basis_sizes.json): the smallest M whose
  error against the coherent-state closed form is below 1e-11 is 8 for
  delta = 0.1 and 29 for delta = 2;
* for constant omega and no perturbation the split-step oracle (Lemma 2,
  chirp-kinetic-chirp) and the Hermite solution agree to round-off.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import hermite as H
from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "e2_hermite_basis_sizes.json")


def coherent(x, x0, t):
    q, p = x0 * math.cos(t), -x0 * math.sin(t)
    return math.pi ** -0.25 * np.exp(-(x - q) ** 2 / 2 + 1j * p * (x - q / 2) - 0.5j * t)


def test_hermite_functions_orthonormal():
    x = np.linspace(-12, 12, 1024, endpoint=False)
    K = H.hermite_functions(30, x)
    G = (x[1] - x[0]) * K @ K.T
    assert np.abs(G - np.eye(30)).max() < 1e-12


@pytest.mark.parametrize("delta", ["0.1", "2"])
def test_e2_printed_basis_sizes(delta):
    gold = json.load(open(GOLD))
    M_printed = gold["printed"][delta]
    d = float(delta)
    x = -10.0 + 20.0 / 512 * np.arange(512)
    dx = x[1] - x[0]
    u0 = math.pi ** -0.25 * np.exp(-(x - d) ** 2 / 2)
    exact = coherent(x, d, 10.0)

    def err(M):
        return math.sqrt(dx) * np.linalg.norm(H.evolve(u0, x, 10.0, M) - exact)

    errs = {M: err(M) for M in range(2, 40)}
    M_min = min(M for M, e in errs.items() if e < 1e-11)
    assert M_min == M_printed, (M_min, errs[M_min - 1], errs[M_min])


def test_hermite_matches_split_step_oracle():
    """Constant omega = 1, eps = sigma = 0: the exact chirp-kinetic-chirp flow
    of Lemma 2 and the Hermite expansion give the same state."""
    prob = O.Problem(n=[512], a=[-12.0], b=[12.0], w0=1.0, ho_flow=O.FLOW_LEMMA2, h=0.5)
    x = prob.x()
    u0 = math.pi ** -0.25 * np.exp(-(x - 1.3) ** 2 / 2 + 0.4j * x)
    split = O.run(prob, u0, 20)
    herm = H.evolve(u0, x, 10.0, 60)
    assert O.rel_l2(split, herm) < 1e-11
