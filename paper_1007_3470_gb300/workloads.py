"""Seeded synthetic workloads shared by the CUDA path's tests/benchmark and
the oracle's.

This module holds only input generation -- grids, parameter draws and
initial wave functions -- and none of the split-step arithmetic, so that both
sides of a parity test start from identical bytes without sharing any of the
method.  All draws come from ``numpy.random.default_rng`` with fixed seeds
and in a fixed order.

Workloads (the problems of Sec. 4 of Bader & Blanes, and the batched,
3D and surrogate families built on the same equations):

* ``coherent_1d``   N=256 on [-16,16), mu=omega=1, eps x^4 (eps=0.05),
  sigma=0, psi0 = ground state shifted to x0=1 (a coherent state), Strang
  with the exact harmonic flow (Lemma 2), dt=0.01, 1000 steps.
* ``gpe_tdep_1d``   N=1024 on [-20,20), omega(t)=1+0.5 sin 2t, sigma=10,
  eps=0.1 with V_I=cos 2x, psi0 = ground Gaussian, commutator-free Magnus-4
  + Theorem 2 inside the NI_5(8,4) composition, dt in {0.04,...,0.005}, T=10.
* ``batch_1d``      4096 (or any count) independent 1D GPE instances with
  N ~ U{128,...,4096}, half-width 8+N/64, omega0 ~ U[0.5,2] with
  omega(t)=omega0(1+0.3 sin t), sigma ~ U[-1,20], eps ~ U[0,0.1],
  V_I=cos(kx) with k ~ U[1,4], psi0 = omega0-ground Gaussian with offset
  x0 ~ U[-1,1]; Strang + Magnus-4, dt=0.005, 500 steps.
* ``gpe_3d``        128^3 (or 32^3) on [-12,12)^3, omega_d = c_d (1+0.3 sin t)
  with c=(1,1.5,2), sigma=100, eps=0.05, V_I = sum_d cos 2x_d, anisotropic
  Gaussian psi0, Strang + Magnus-4, dt=0.005, 200 steps.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np

SEED = 20100703

# integer codes shared by both sides' parameter structs (names only, no arithmetic)
OMEGA_CONST, OMEGA_SIN, OMEGA_COS_SQ, OMEGA_PULSE = 0, 1, 2, 3
VI_NONE, VI_X4, VI_COS = 0, 1, 2
SPLIT_HO, SPLIT_FOURIER = 0, 1
FLOW_LEMMA2, FLOW_CF4, FLOW_M6 = 0, 1, 2


@dataclass
class Instance:
    """Parameters of one problem instance (plain data)."""
    n: List[int]
    a: List[float]
    b: List[float]
    mu: float = 1.0
    omega_law: int = OMEGA_CONST
    w0: float = 1.0
    law: List[float] = field(default_factory=lambda: [0.0, 0.0, 0.0])
    axis_scale: List[float] = field(default_factory=lambda: [1.0, 1.0, 1.0])
    eps: float = 0.0
    vi_kind: int = VI_NONE
    vi_k: float = 0.0
    sigma: float = 0.0
    split: int = SPLIT_HO
    ho_flow: int = FLOW_LEMMA2
    scheme: str = "strang"
    h: float = 0.01
    t0: float = 0.0

    @property
    def dim(self) -> int:
        return len(self.n)

    def x(self, d: int = 0) -> np.ndarray:
        n = int(self.n[d])
        return self.a[d] + (self.b[d] - self.a[d]) / n * np.arange(n, dtype=np.float64)

    def npoints(self) -> int:
        p = 1
        for v in self.n:
            p *= int(v)
        return p

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k in self.__dataclass_fields__}


def _normalise(psi: np.ndarray, dv: float) -> np.ndarray:
    return psi / np.sqrt(dv * np.sum(np.abs(psi) ** 2))


def gaussian_1d(inst: Instance, x0: float = 0.0, width2: float = 1.0, p0: float = 0.0) -> np.ndarray:
    """exp(-(x-x0)^2/(2 width2) + i p0 x), normalised so dx sum |psi|^2 = 1."""
    x = inst.x(0)
    psi = np.exp(-((x - x0) ** 2) / (2.0 * width2) + 1j * p0 * x)
    return _normalise(psi, (inst.b[0] - inst.a[0]) / inst.n[0])


# ---------------------------------------------------------------------------
# single-instance 1D workloads
# ---------------------------------------------------------------------------

def coherent_1d(n: int = 256, steps: int = 1000, h: float = 0.01):
    inst = Instance(n=[n], a=[-16.0], b=[16.0], omega_law=OMEGA_CONST, w0=1.0,
                    eps=0.05, vi_kind=VI_X4, sigma=0.0, ho_flow=FLOW_LEMMA2,
                    scheme="strang", h=h)
    return inst, gaussian_1d(inst, x0=1.0), steps


def gpe_tdep_1d(h: float = 0.01, n: int = 1024, T: float = 10.0, scheme: str = "ni5_84",
                ho_flow: int = FLOW_CF4):
    inst = Instance(n=[n], a=[-20.0], b=[20.0], omega_law=OMEGA_SIN, w0=1.0,
                    law=[0.5, 2.0, 0.0], eps=0.1, vi_kind=VI_COS, vi_k=2.0, sigma=10.0,
                    ho_flow=ho_flow, scheme=scheme, h=h)
    steps = int(round(T / h))
    return inst, gaussian_1d(inst), steps


def split_comparison_1d(sigma: float, n: int = 1024, h: float = 0.01, split: int = SPLIT_HO):
    """The HO-split vs F-split experiment of Sec. 4: mu = omega = 1, V_I = 0,
    psi0 = rho exp(-(x-1)^2/2), x in [-20,20) for sigma = 0.01 and [-30,30)
    otherwise (the paper's intervals), leap-frog BAB composition."""
    half = 20.0 if sigma < 0.1 else 30.0
    inst = Instance(n=[n], a=[-half], b=[half], omega_law=OMEGA_CONST, w0=1.0, sigma=sigma,
                    split=split, ho_flow=FLOW_LEMMA2, scheme="strang", h=h)
    return inst, gaussian_1d(inst, x0=1.0)


# ---------------------------------------------------------------------------
# batched 1D workload
# ---------------------------------------------------------------------------

BATCH_SIZES = (128, 256, 512, 1024, 2048, 4096)


def batch_1d(count: int = 4096, seed: int = SEED, h: float = 0.005, steps: int = 500,
             sizes: Sequence[int] = BATCH_SIZES):
    """Returns (instances, psi0 list (complex128), steps).  Draw order: N,
    omega0, sigma, eps, k, x0."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=count)
    w0 = rng.uniform(0.5, 2.0, size=count)
    sig = rng.uniform(-1.0, 20.0, size=count)
    eps = rng.uniform(0.0, 0.1, size=count)
    kk = rng.uniform(1.0, 4.0, size=count)
    x0 = rng.uniform(-1.0, 1.0, size=count)
    insts, psis = [], []
    for i in range(count):
        n = int(ns[i])
        hw = 8.0 + n / 64.0
        inst = Instance(n=[n], a=[-hw], b=[hw], omega_law=OMEGA_SIN, w0=float(w0[i]),
                        law=[0.3, 1.0, 0.0], eps=float(eps[i]), vi_kind=VI_COS, vi_k=float(kk[i]),
                        sigma=float(sig[i]), ho_flow=FLOW_CF4, scheme="strang", h=h)
        insts.append(inst)
        psis.append(gaussian_1d(inst, x0=float(x0[i]), width2=1.0 / float(w0[i])))
    return insts, psis, steps


# ---------------------------------------------------------------------------
# 3D workload
# ---------------------------------------------------------------------------

def gpe_3d(n: int = 128, h: float = 0.005, steps: int = 200, half_width: float = 12.0):
    inst = Instance(n=[n, n, n], a=[-half_width] * 3, b=[half_width] * 3, omega_law=OMEGA_SIN,
                    w0=1.0, law=[0.3, 1.0, 0.0], axis_scale=[1.0, 1.5, 2.0], eps=0.05,
                    vi_kind=VI_COS, vi_k=2.0, sigma=100.0, ho_flow=FLOW_CF4, scheme="strang", h=h)
    xs = [inst.x(d) for d in range(3)]
    # numpy C order: shape (nz, ny, nx), axis 0 of the problem (x) fastest
    X = xs[0][None, None, :]
    Y = xs[1][None, :, None]
    Z = xs[2][:, None, None]
    psi = np.exp(-(1.0 * X ** 2 + 1.5 * Y ** 2 + 2.0 * Z ** 2) / 2.0).astype(np.complex128)
    dv = ((2 * half_width) / n) ** 3
    return inst, _normalise(psi, dv), steps
