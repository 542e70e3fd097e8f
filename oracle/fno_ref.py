"""FP64 numpy reference of the Fourier-neural-operator surrogate -- forward,
relative-L2 loss and hand-derived backward.  TEST INFRASTRUCTURE ONLY: the
GPU kernels' forward and gradients are checked against it, and its own
backward is checked against finite differences.  It shares no code with the
CUDA path.

Architecture (channels last, one sample = L grid points):
  H0  = X P_in + b_in                               (lift, in_ch -> C)
  for l = 1..layers:
      S   = truncated DFT of H_{l-1} over x: modes k < M (real and imaginary parts)
      Y_k = S_k R_k (complex C x C mixing per retained mode)
      U   = real inverse DFT of Y from the retained modes
      Z   = H_{l-1} W_l + b_l + U
      H_l = GELU(Z) for l < layers, Z for the last layer
  Q = GELU(H P1 + c1); O = Q P2 + c2                (projection C -> P -> out)
  loss = mean over samples of ||O - Y|| / ||Y||     (relative L2)

Parameter vector layout (float, in this order): P_in[in_ch][C], b_in[C], then per
layer R_re[M][C][C], R_im[M][C][C], W[C][C], b[C]; then P1[C][P], c1[P],
P2[P][out], c2[out].
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


class Config:
    def __init__(self, L=256, C=64, M=32, layers=4, in_ch=7, P=128, out=2):
        self.L, self.C, self.M, self.layers, self.in_ch, self.P, self.out = L, C, M, layers, in_ch, P, out

    def shapes(self):
        s = [("P_in", (self.in_ch, self.C)), ("b_in", (self.C,))]
        for l in range(self.layers):
            s += [(f"Rre{l}", (self.M, self.C, self.C)), (f"Rim{l}", (self.M, self.C, self.C)),
                  (f"W{l}", (self.C, self.C)), (f"b{l}", (self.C,))]
        s += [("P1", (self.C, self.P)), ("c1", (self.P,)), ("P2", (self.P, self.out)), ("c2", (self.out,))]
        return s

    def count(self):
        return sum(int(np.prod(sh)) for _, sh in self.shapes())


def unpack(cfg: Config, vec: np.ndarray) -> dict:
    out, o = {}, 0
    for name, sh in cfg.shapes():
        n = int(np.prod(sh))
        out[name] = vec[o:o + n].reshape(sh)
        o += n
    return out


def pack(cfg: Config, d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in cfg.shapes()])


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def dft_mats(cfg: Config):
    """Forward truncated DFT e^{-2 pi i k x / L} (k < M) and the real inverse
    from the half spectrum: u(x) = (1/L) sum_k w_k Re(Y_k e^{2 pi i k x/L}),
    w_0 = 1, w_k = 2 for k >= 1."""
    x = np.arange(cfg.L)
    k = np.arange(cfg.M)
    ang = 2.0 * math.pi * np.outer(k, x) / cfg.L        # [M, L]
    Fre, Fim = np.cos(ang), -np.sin(ang)                 # S = F H  (rows k)
    w = np.where(k == 0, 1.0, 2.0)[:, None]
    Gre, Gim = (w * np.cos(ang)).T / cfg.L, (-w * np.sin(ang)).T / cfg.L   # [L, M]
    return Fre, Fim, Gre, Gim


def forward(cfg: Config, p: dict, X: np.ndarray, keep=False):
    """X: [B, L, in_ch] -> O: [B, L, out] (and the saved activations)."""
    Fre, Fim, Gre, Gim = dft_mats(cfg)
    H = X @ p["P_in"] + p["b_in"]
    cache = {"X": X, "H": [H], "S": [], "pre": []}
    for l in range(cfg.layers):
        Sre = np.einsum("kx,bxc->bkc", Fre, H)
        Sim = np.einsum("kx,bxc->bkc", Fim, H)
        Rre, Rim = p[f"Rre{l}"], p[f"Rim{l}"]
        Yre = np.einsum("bkc,kco->bko", Sre, Rre) - np.einsum("bkc,kco->bko", Sim, Rim)
        Yim = np.einsum("bkc,kco->bko", Sre, Rim) + np.einsum("bkc,kco->bko", Sim, Rre)
        U = np.einsum("xk,bko->bxo", Gre, Yre) + np.einsum("xk,bko->bxo", Gim, Yim)
        Z = H @ p[f"W{l}"] + p[f"b{l}"] + U
        H = gelu(Z) if l < cfg.layers - 1 else Z
        cache["S"].append((Sre, Sim))
        cache["pre"].append(Z)
        cache["H"].append(H)
    Qpre = H @ p["P1"] + p["c1"]
    Q = gelu(Qpre)
    O = Q @ p["P2"] + p["c2"]
    cache.update(Qpre=Qpre, Q=Q)
    return (O, cache) if keep else O


def rel_l2_loss(O, Y):
    num = np.sqrt(np.sum((O - Y) ** 2, axis=(1, 2)))
    den = np.sqrt(np.sum(Y ** 2, axis=(1, 2)))
    return float(np.mean(num / den))


def loss_and_grad(cfg: Config, p: dict, X: np.ndarray, Ytarget: np.ndarray):
    O, c = forward(cfg, p, X, keep=True)
    B = X.shape[0]
    diff = O - Ytarget
    num = np.sqrt(np.sum(diff ** 2, axis=(1, 2)))
    den = np.sqrt(np.sum(Ytarget ** 2, axis=(1, 2)))
    loss = float(np.mean(num / den))
    dO = diff / (num * den)[:, None, None] / B
    g = {}
    g["P2"] = np.einsum("bxp,bxo->po", c["Q"], dO)
    g["c2"] = dO.sum(axis=(0, 1))
    dQ = dO @ p["P2"].T
    dQpre = dQ * gelu_grad(c["Qpre"])
    H = c["H"][-1]
    g["P1"] = np.einsum("bxc,bxp->cp", H, dQpre)
    g["c1"] = dQpre.sum(axis=(0, 1))
    dH = dQpre @ p["P1"].T
    Fre, Fim, Gre, Gim = dft_mats(cfg)
    for l in reversed(range(cfg.layers)):
        Z = c["pre"][l]
        dZ = dH * gelu_grad(Z) if l < cfg.layers - 1 else dH
        Hin = c["H"][l]
        g[f"W{l}"] = np.einsum("bxc,bxo->co", Hin, dZ)
        g[f"b{l}"] = dZ.sum(axis=(0, 1))
        dHin = dZ @ p[f"W{l}"].T
        dYre = np.einsum("xk,bxo->bko", Gre, dZ)
        dYim = np.einsum("xk,bxo->bko", Gim, dZ)
        Sre, Sim = c["S"][l]
        Rre, Rim = p[f"Rre{l}"], p[f"Rim{l}"]
        g[f"Rre{l}"] = np.einsum("bkc,bko->kco", Sre, dYre) + np.einsum("bkc,bko->kco", Sim, dYim)
        g[f"Rim{l}"] = -np.einsum("bkc,bko->kco", Sim, dYre) + np.einsum("bkc,bko->kco", Sre, dYim)
        dSre = np.einsum("bko,kco->bkc", dYre, Rre) + np.einsum("bko,kco->bkc", dYim, Rim)
        dSim = -np.einsum("bko,kco->bkc", dYre, Rim) + np.einsum("bko,kco->bkc", dYim, Rre)
        dHin += np.einsum("kx,bkc->bxc", Fre, dSre) + np.einsum("kx,bkc->bxc", Fim, dSim)
        dH = dHin
    g["P_in"] = np.einsum("bxi,bxc->ic", c["X"], dH)
    g["b_in"] = dH.sum(axis=(0, 1))
    return loss, g


def init_params(cfg: Config, seed: int) -> dict:
    """Deterministic initial parameters (uniform fan-in scaling)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, sh in cfg.shapes():
        if name.startswith(("b", "c")):
            p[name] = np.zeros(sh)
        elif name.startswith("R"):
            p[name] = rng.uniform(-1, 1, sh) / (cfg.C * cfg.C) ** 0.5
        else:
            p[name] = rng.uniform(-1, 1, sh) / math.sqrt(sh[0])
    return p
