"""Hermite-basis solution of the harmonic oscillator on a grid (Eq. Hermite2)
-- FP64, CPU, TEST INFRASTRUCTURE ONLY.

u(T) = K^T exp(-i T D_1) (dx K u_0), with K_{n,j} = h_n(x_j) the normalised
Hermite functions of Eq. EigenHarm on the equidistant mesh, D_1 = diag(n + 1/2),
n < M.  The quadrature weight dx of the projection c_n = int h_n phi_0 dx is
written out (the printed formula leaves it implicit).  This is the paper's
comparison method, used here only as an independent cross-check of the
split-step oracle for constant omega and to pin the basis sizes the paper
prints for the displaced ground state (Sec. 4).
"""
from __future__ import annotations

import math

import numpy as np


def hermite_functions(M: int, x: np.ndarray) -> np.ndarray:
    """K[n, j] = h_n(x_j), n < M, by the normalised three-term recursion
    h_{n+1} = sqrt(2/(n+1)) x h_n - sqrt(n/(n+1)) h_{n-1}, which is the
    recursion H_{k+1} = 2x H_k - 2k H_{k-1} of Eq. EigenHarm with the
    normalisation 1/(pi^{1/4} sqrt(2^n n!)) carried along."""
    K = np.zeros((M, x.size))
    K[0] = math.pi ** -0.25 * np.exp(-x * x / 2)
    if M > 1:
        K[1] = math.sqrt(2.0) * x * K[0]
    for n in range(1, M - 1):
        K[n + 1] = math.sqrt(2.0 / (n + 1)) * x * K[n] - math.sqrt(n / (n + 1)) * K[n - 1]
    return K


def evolve(u0: np.ndarray, x: np.ndarray, T: float, M: int) -> np.ndarray:
    """Harmonic flow (omega = mu = 1) of u0 over time T with M basis functions."""
    dx = x[1] - x[0]
    K = hermite_functions(M, x)
    c = dx * (K @ u0)
    E = np.arange(M) + 0.5
    return K.T @ (np.exp(-1j * T * E) * c)
