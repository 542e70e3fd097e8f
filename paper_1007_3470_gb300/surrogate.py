"""The learned surrogate around the solver: training data from the
Hermite-Fourier solver, training and inference of the FNO (fno.py), its error
distribution judged by the solver, and the comparison with the solver itself
at equal accuracy.

Problem family: the batched 1D GPE family at N = 256 (half-width 12,
omega(t) = omega0 (1 + 0.3 sin t), omega0 ~ U[0.5,2], sigma ~ U[-1,20],
eps ~ U[0,0.1], V_I = cos(k x), k ~ U[1,4], Gaussian psi0 of width
1/sqrt(omega0) at x0 ~ U[-1,1]), map psi0 -> psi(T = 1) (200 Strang /
Magnus-4 steps of 0.005).  Input channels per grid point: Re psi0, Im psi0,
x / 12, omega0, sigma / 20, eps / 0.1, k / 4.
"""
from __future__ import annotations

import time

import numpy as np

from . import hfs
from . import workloads as W
from .fno import Fno, FnoConfig

N, T, DT = 256, 1.0, 0.005


def family(count: int, seed: int):
    return W.batch_1d(count=count, seed=seed, h=DT, steps=int(round(T / DT)), sizes=(N,))


def features(insts, psis) -> np.ndarray:
    X = np.zeros((len(insts), N, 7), dtype=np.float32)
    for i, (inst, p) in enumerate(zip(insts, psis)):
        X[i, :, 0] = p.real
        X[i, :, 1] = p.imag
        X[i, :, 2] = inst.x() / 12.0
        X[i, :, 3] = inst.w0
        X[i, :, 4] = inst.sigma / 20.0
        X[i, :, 5] = inst.eps / 0.1
        X[i, :, 6] = inst.vi_k / 4.0
    return X


def solve(insts, psis, dt: float = DT, precision: str = "c64", chunk: int = 4096) -> np.ndarray:
    """psi(T) of every instance with the plain solver (batched), [count, N, 2]."""
    steps = int(round(T / dt))
    out = np.zeros((len(insts), N, 2), dtype=np.float32)
    for s0 in range(0, len(insts), chunk):
        sub, ps = insts[s0:s0 + chunk], psis[s0:s0 + chunk]
        sv = hfs.Solver(sub, precision=precision, chunk_steps=steps)
        sv.set_schedule(dt, "strang", hfs.HFS_FLOW_CF4)
        sv.set_psi(ps)
        sv.step(steps)
        y = sv.get_psi().reshape(len(sub), N)
        sv.close()
        out[s0:s0 + chunk, :, 0] = y.real
        out[s0:s0 + chunk, :, 1] = y.imag
    return out


def rel_errors(pred: np.ndarray, ref: np.ndarray) -> np.ndarray:
    d = np.sqrt(np.sum((pred - ref) ** 2, axis=(1, 2)))
    return d / np.sqrt(np.sum(ref ** 2, axis=(1, 2)))


def train(model: Fno, X: np.ndarray, Y: np.ndarray, epochs: int, batch: int, lr: float, seed: int = 0,
          log=None) -> list[float]:
    torch = model.torch
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y).cuda()
    rng = np.random.default_rng(seed)
    history = []
    nb = len(X) // batch
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(len(X))).cuda()
        # cosine-decayed learning rate
        lr_ep = lr * 0.5 * (1.0 + np.cos(np.pi * ep / max(epochs, 1)))
        torch.cuda.synchronize()
        losses = []
        for bi in range(nb):
            idx = perm[bi * batch:(bi + 1) * batch]
            xb = Xd.index_select(0, idx).contiguous()
            yb = Yd.index_select(0, idx).contiguous()
            torch.cuda.synchronize()
            losses.append(model.train_step(xb, yb, float(lr_ep), want_loss=(bi == nb - 1)))
        history.append(losses[-1])
        if log:
            log(f"epoch {ep} loss {losses[-1]:.4e}")
    return history


def predict(model: Fno, X: np.ndarray, batch: int) -> np.ndarray:
    out = []
    for s0 in range(0, len(X), batch):
        out.append(model.forward(model.torch.from_numpy(X[s0:s0 + batch])).cpu().numpy())
    return np.concatenate(out)


def time_inference(model: Fno, X: np.ndarray, reps: int = 5) -> float:
    """Surrogate solves per second at batch len(X) (device time of the forward)."""
    torch = model.torch
    xd = torch.from_numpy(X).cuda()
    y = torch.empty((len(X), N, 2), device="cuda")
    import ctypes
    from .fno import _lib
    L = _lib()
    for _ in range(2):
        L.hfs_fno_forward(model.h, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(y.data_ptr()), len(X))
    model.stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(model.stream)
    for _ in range(reps):
        L.hfs_fno_forward(model.h, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(y.data_ptr()), len(X))
    e1.record(model.stream)
    e1.synchronize()
    return len(X) * reps / (e0.elapsed_time(e1) * 1e-3)


def time_solver(insts, psis, dt: float, reps: int = 3) -> float:
    """Plain solver solves per second for the same batch (device time)."""
    torch = __import__("torch")
    steps = int(round(T / dt))
    sv = hfs.Solver(insts, precision="c64", chunk_steps=steps)
    sv.set_schedule(dt, "strang", hfs.HFS_FLOW_CF4)
    sv.set_graphs(True)
    hfs.hfs_set_profiling(sv.h, True)
    sv.set_psi(psis)
    sv.step(steps)
    best = 1e30
    for _ in range(reps):
        sv.set_psi(psis)
        sv.step(steps)
        best = min(best, hfs.hfs_last_step_kernel_ms(sv.h))
    sv.close()
    del torch
    return len(insts) / (best * 1e-3)


def equal_accuracy_solver(insts, psis, ref: np.ndarray, target_err: float):
    """Coarsest solver step (T/dt integer) whose median relative error against
    the reference is at most target_err; returns (dt, median error)."""
    best = None
    for steps in (2, 4, 5, 8, 10, 20, 25, 40, 50, 100, 200):
        dt = T / steps
        pred = solve(insts, psis, dt=dt)
        med = float(np.median(rel_errors(pred, ref)))
        if med <= target_err:
            best = (dt, med)
            break
    return best
