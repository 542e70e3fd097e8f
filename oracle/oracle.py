"""FP64 CPU oracle for the Hermite-Fourier split step (Bader & Blanes,
arXiv 1007.3470) -- Python side.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg use it; the product library never imports it.  It shares no
code with the CUDA path.  The arithmetic lives in ``hfs_oracle.c`` (plain C,
double precision, unmerged stage-by-stage application of the scheme); this
module compiles it with gcc, wraps it with ctypes, and holds the oracle's own
copy of the composition coefficients of Table 1 and the Strang/leapfrog
scheme of Eq. LeapFrogB.

Parity is pinned by ``tests/test_oracle_*.py`` (see the header of
``hfs_oracle.c`` for the list of pins).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hfs_oracle.c")
_HDR = os.path.join(_HERE, "hfs_oracle.h")
_LIB = os.path.join(_HERE, "_build", "libhfs_oracle.so")

OMEGA_CONST, OMEGA_SIN, OMEGA_COS_SQ, OMEGA_PULSE = 0, 1, 2, 3
VI_NONE, VI_X4, VI_COS = 0, 1, 2
SPLIT_HO, SPLIT_FOURIER = 0, 1
FLOW_LEMMA2, FLOW_CF4, FLOW_M6 = 0, 1, 2


# ---------------------------------------------------------------------------
# composition coefficients (Eq. LeapFrogB and Table 1); BAB form: m a's, m+1 b's
# ---------------------------------------------------------------------------

def composition(name: str) -> tuple[list[float], list[float]]:
    """(a, b) with len(b) == len(a) + 1; b_1 is applied first.

    Table 1 prints NI_4's b_2 as 49/18; it is read as 49/180 (the Lobatto
    weights 1/20, 49/180, 16/45 of the (8,2) method), which the quadrature
    pin in the tests confirms.
    """
    if name == "strang":
        return [1.0], [0.5, 0.5]
    if name == "srkn6_4":
        b1, b2, b3 = 0.0829844064174052, 0.396309801498368, -0.0390563049223486
        b4 = 1.0 - 2.0 * (b1 + b2 + b3)
        a1, a2 = 0.245298957184271, 0.604872665711080
        a3 = 0.5 - (a1 + a2)
        return [a1, a2, a3, a3, a2, a1], [b1, b2, b3, b4, b3, b2, b1]
    if name == "ni4_82":
        b1, b2 = 1.0 / 20.0, 49.0 / 180.0
        b3 = 1.0 - 2.0 * (b1 + b2)
        a1 = 0.5 - math.sqrt(3.0 / 28.0)
        a2 = 0.5 - a1
        return [a1, a2, a2, a1], [b1, b2, b3, b2, b1]
    if name == "ni5_84":
        b1, b2 = 0.811862738544516, -0.677480399532169
        b3 = 0.5 - (b1 + b2)
        a1, a2 = -0.00758691311877447, 0.317218277973169
        a3 = 1.0 - 2.0 * (a1 + a2)
        return [a1, a2, a3, a2, a1], [b1, b2, b3, b3, b2, b1]
    raise ValueError(f"unknown composition {name!r}")


# ---------------------------------------------------------------------------
# build + load
# ---------------------------------------------------------------------------

def build(force: bool = False) -> str:
    """Compile hfs_oracle.c into oracle/_build/libhfs_oracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("a", ctypes.c_double * 3),
        ("b", ctypes.c_double * 3),
        ("mu", ctypes.c_double),
        ("omega_law", ctypes.c_int),
        ("w0", ctypes.c_double),
        ("law", ctypes.c_double * 3),
        ("axis_scale", ctypes.c_double * 3),
        ("eps", ctypes.c_double),
        ("vi_kind", ctypes.c_int),
        ("vi_k", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("split", ctypes.c_int),
        ("ho_flow", ctypes.c_int),
        ("m", ctypes.c_int),
        ("acoef", ctypes.POINTER(ctypes.c_double)),
        ("bcoef", ctypes.POINTER(ctypes.c_double)),
        ("h", ctypes.c_double),
        ("t0", ctypes.c_double),
        ("naive_dft", ctypes.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        L.or_dft.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int]
        L.or_fft.argtypes = [ctypes.c_int, dp, ctypes.c_int]
        L.or_fft.restype = ctypes.c_int
        L.or_omega2.argtypes = [ctypes.POINTER(_Problem), ctypes.c_double]
        L.or_omega2.restype = ctypes.c_double
        for nm in ("or_coef_lemma2",):
            getattr(L, nm).argtypes = [ctypes.c_double] * 3 + [dp] * 3
        L.or_coef_thm2.argtypes = [ctypes.c_double] * 4 + [dp] * 3
        L.or_coef_thm1.argtypes = [ctypes.c_double] * 4 + [dp] * 3
        L.or_stage_coeffs.argtypes = [ctypes.POINTER(_Problem), ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, dp, dp, dp]
        L.or_stage_coeffs.restype = ctypes.c_int
        L.or_run.argtypes = [ctypes.POINTER(_Problem), dp, ctypes.c_long]
        L.or_run.restype = ctypes.c_int
        L.or_run_batch.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(dp), ctypes.c_long,
                                   ctypes.c_long, ctypes.c_int]
        L.or_run_batch.restype = ctypes.c_int
        L.or_max_threads.restype = ctypes.c_int
        L.or_norm.argtypes = [ctypes.POINTER(_Problem), dp]
        L.or_norm.restype = ctypes.c_double
        L.or_energy.argtypes = [ctypes.POINTER(_Problem), dp, ctypes.c_double]
        L.or_energy.restype = ctypes.c_double
        _lib = L
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---------------------------------------------------------------------------
# problem description
# ---------------------------------------------------------------------------

@dataclass
class Problem:
    """One instance of Eq. GP1 (1D) or its d-dimensional form with a diagonal trap."""
    n: Sequence[int]
    a: Sequence[float]
    b: Sequence[float]
    mu: float = 1.0
    omega_law: int = OMEGA_CONST
    w0: float = 1.0
    law: Sequence[float] = (0.0, 0.0, 0.0)
    axis_scale: Sequence[float] = (1.0, 1.0, 1.0)
    eps: float = 0.0
    vi_kind: int = VI_NONE
    vi_k: float = 0.0
    sigma: float = 0.0
    split: int = SPLIT_HO
    ho_flow: int = FLOW_LEMMA2
    scheme: str = "strang"
    h: float = 0.01
    t0: float = 0.0
    naive_dft: bool = False
    # explicit composition coefficients (a[m], b[m+1], b_1 applied first)
    # instead of a named scheme
    coeffs: Optional[tuple] = None
    _keep: list = field(default_factory=list, repr=False)

    @property
    def dim(self) -> int:
        return len(self.n)

    def shape(self) -> tuple[int, ...]:
        """numpy shape of psi, C order with axis 0 of the problem fastest."""
        return tuple(int(v) for v in reversed(list(self.n)))

    def to_c(self) -> _Problem:
        p = _Problem()
        p.dim = self.dim
        for d in range(3):
            p.n[d] = int(self.n[d]) if d < self.dim else 1
            p.a[d] = float(self.a[d]) if d < self.dim else 0.0
            p.b[d] = float(self.b[d]) if d < self.dim else 1.0
            p.law[d] = float(self.law[d])
            p.axis_scale[d] = float(self.axis_scale[d])
        p.mu = self.mu
        p.omega_law = self.omega_law
        p.w0 = self.w0
        p.eps = self.eps
        p.vi_kind = self.vi_kind
        p.vi_k = self.vi_k
        p.sigma = self.sigma
        p.split = self.split
        p.ho_flow = self.ho_flow
        a, b = composition(self.scheme) if self.coeffs is None else (list(self.coeffs[0]), list(self.coeffs[1]))
        if len(b) != len(a) + 1:
            raise ValueError("a composition has m a's and m + 1 b's")
        av = np.ascontiguousarray(a, dtype=np.float64)
        bv = np.ascontiguousarray(b, dtype=np.float64)
        self._keep[:] = [av, bv]
        p.m = len(a)
        p.acoef = _dptr(av)
        p.bcoef = _dptr(bv)
        p.h = self.h
        p.t0 = self.t0
        p.naive_dft = 1 if self.naive_dft else 0
        return p

    # grid of Eq. GP1ODE
    def x(self, d: int = 0) -> np.ndarray:
        n = int(self.n[d])
        dx = (self.b[d] - self.a[d]) / n
        return self.a[d] + dx * np.arange(n, dtype=np.float64)

    def dv(self) -> float:
        v = 1.0
        for d in range(self.dim):
            v *= (self.b[d] - self.a[d]) / self.n[d]
        return v


# ---------------------------------------------------------------------------
# wrappers
# ---------------------------------------------------------------------------

def _as_c128(psi) -> np.ndarray:
    return np.ascontiguousarray(psi, dtype=np.complex128)


def dft(x, sign: int = -1) -> np.ndarray:
    x = _as_c128(x)
    out = np.empty_like(x)
    lib().or_dft(x.size, _dptr(x.view(np.float64)), _dptr(out.view(np.float64)), sign)
    return out


def fft(x, sign: int = -1) -> np.ndarray:
    x = _as_c128(x).copy()
    if lib().or_fft(x.size, _dptr(x.view(np.float64)), sign) != 0:
        raise ValueError("radix-2 FFT needs a power-of-two length")
    return x


def coef_lemma2(mu: float, omega: float, t: float):
    f, g, e = (ctypes.c_double() for _ in range(3))
    lib().or_coef_lemma2(mu, omega, t, ctypes.byref(f), ctypes.byref(g), ctypes.byref(e))
    return f.value, g.value, e.value


def coef_thm2(mu: float, wl: float, wr: float, t: float):
    f, g, e = (ctypes.c_double() for _ in range(3))
    lib().or_coef_thm2(mu, wl, wr, t, ctypes.byref(f), ctypes.byref(g), ctypes.byref(e))
    return f.value, g.value, e.value


def coef_thm1(alpha: float, beta: float, gamma: float, t: float):
    f, g, e = (ctypes.c_double() for _ in range(3))
    lib().or_coef_thm1(alpha, beta, gamma, t, ctypes.byref(f), ctypes.byref(g), ctypes.byref(e))
    return f.value, g.value, e.value


def stage_coeffs(prob: Problem, t0: float, s: float, axis: int = 0):
    f, g, e = (ctypes.c_double() for _ in range(3))
    pc = prob.to_c()
    rc = lib().or_stage_coeffs(ctypes.byref(pc), axis, t0, s, ctypes.byref(f), ctypes.byref(g), ctypes.byref(e))
    if rc:
        raise ValueError("unknown HO flow")
    return f.value, g.value, e.value


def omega2(prob: Problem, t: float) -> float:
    pc = prob.to_c()
    return lib().or_omega2(ctypes.byref(pc), t)


def run(prob: Problem, psi0, nsteps: int) -> np.ndarray:
    """Advance psi0 by nsteps steps of size prob.h from prob.t0; returns a new array."""
    psi = _as_c128(psi0).copy()
    pc = prob.to_c()
    rc = lib().or_run(ctypes.byref(pc), _dptr(psi.view(np.float64)), int(nsteps))
    if rc:
        raise RuntimeError(f"oracle run failed ({rc})")
    return psi


def run_batch(probs: Sequence[Problem], psis: Sequence[np.ndarray], nsteps: int, nthreads: int = 0):
    """Run independent instances in parallel (OpenMP over instances)."""
    arrs = [_as_c128(p).copy() for p in psis]
    cp = (_Problem * len(probs))()
    for i, pr in enumerate(probs):
        cp[i] = pr.to_c()
    ptrs = (ctypes.POINTER(ctypes.c_double) * len(arrs))(*[_dptr(a.view(np.float64)) for a in arrs])
    rc = lib().or_run_batch(cp, ptrs, len(arrs), int(nsteps), int(nthreads))
    if rc:
        raise RuntimeError("oracle batch run failed")
    return arrs


def max_threads() -> int:
    return lib().or_max_threads()


def norm(prob: Problem, psi) -> float:
    psi = _as_c128(psi)
    pc = prob.to_c()
    return lib().or_norm(ctypes.byref(pc), _dptr(psi.view(np.float64)))


def energy(prob: Problem, psi, t: float) -> float:
    psi = _as_c128(psi)
    pc = prob.to_c()
    return lib().or_energy(ctypes.byref(pc), _dptr(psi.view(np.float64)), t)


def rel_l2(u, ref) -> float:
    """Relative discrete 2-norm error ||u - ref|| / ||ref|| (Sec. 4 error metric)."""
    u = np.asarray(u, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    return float(np.linalg.norm((u - ref).ravel()) / np.linalg.norm(ref.ravel()))
