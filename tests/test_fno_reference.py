"""Pins of the FP64 FNO reference (oracle/fno_ref.py): its hand-derived
backward equals central finite differences of its loss; the truncated DFT
pair is the identity on fields band-limited to the retained modes; the
mixing is the complex product it claims to be."""
import numpy as np
import pytest

from oracle import fno_ref as F


def small():
    return F.Config(L=16, C=4, M=3, layers=2, in_ch=3, P=5, out=2)


def test_gradient_matches_finite_differences():
    cfg = small()
    rng = np.random.default_rng(0)
    p = F.init_params(cfg, 1)
    for k in p:
        p[k] = p[k] + 0.1 * rng.standard_normal(p[k].shape)
    X = rng.standard_normal((3, cfg.L, cfg.in_ch))
    Y = rng.standard_normal((3, cfg.L, cfg.out))
    loss, g = F.loss_and_grad(cfg, p, X, Y)
    vec = F.pack(cfg, p)
    gvec = F.pack(cfg, g)
    idx = rng.choice(vec.size, size=60, replace=False)
    for i in idx:
        e = np.zeros_like(vec)
        e[i] = 1e-6
        lp = F.rel_l2_loss(F.forward(cfg, F.unpack(cfg, vec + e), X), Y)
        lm = F.rel_l2_loss(F.forward(cfg, F.unpack(cfg, vec - e), X), Y)
        fd = (lp - lm) / 2e-6
        assert abs(fd - gvec[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, gvec[i])


def test_truncated_dft_pair_is_identity_on_band_limited_fields():
    cfg = F.Config(L=32, M=5)
    Fre, Fim, Gre, Gim = F.dft_mats(cfg)
    x = np.arange(32)
    u = 0.3 + np.cos(2 * np.pi * 2 * x / 32) - 0.7 * np.sin(2 * np.pi * 4 * x / 32)
    S = (Fre @ u, Fim @ u)
    assert np.allclose(Gre @ S[0] + Gim @ S[1], u, atol=1e-12)
    # a mode above the cut is removed
    v = np.cos(2 * np.pi * 7 * x / 32)
    assert np.allclose(Gre @ (Fre @ v) + Gim @ (Fim @ v), 0.0, atol=1e-12)


def test_mixing_is_complex_product():
    cfg = F.Config(L=16, C=3, M=2, layers=1, in_ch=2, P=4, out=2)
    rng = np.random.default_rng(3)
    p = F.init_params(cfg, 0)
    p["Rre0"] = rng.standard_normal(p["Rre0"].shape)
    p["Rim0"] = rng.standard_normal(p["Rim0"].shape)
    X = rng.standard_normal((1, 16, 2))
    O, c = F.forward(cfg, p, X, keep=True)
    H0 = c["H"][0][0]
    S = np.fft.fft(H0, axis=0)[:2]              # library FFT, first two modes
    Yc = np.einsum("kc,kco->ko", S, p["Rre0"] + 1j * p["Rim0"])
    full = np.zeros((16, 3), complex)
    full[:2] = Yc
    full[-1] = np.conj(Yc[1])                    # Hermitian completion of mode 1
    U = np.fft.ifft(full, axis=0).real
    Z = H0 @ p["W0"] + p["b0"] + U
    assert np.allclose(c["pre"][0][0], Z, atol=1e-12)
