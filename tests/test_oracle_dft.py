"""Pin P1: the oracle's naive DFT and its radix-2 FFT agree with each other
and with numpy's FFT (a library routine) -- the transform of Eq. GP1ODE_T."""
import numpy as np
import pytest

from oracle import oracle as O


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16])
def test_dft_equals_fft_bruteforce(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    naive = O.dft(x, -1)
    fast = O.fft(x, -1)
    assert np.abs(naive - fast).max() <= 1e-15 * max(1, n) * 4
    # inverse (sign +1, unnormalised) undoes the forward up to the factor n
    back = O.fft(fast, +1) / n
    assert np.abs(back - x).max() <= 1e-15 * max(1, n) * 4


@pytest.mark.parametrize("n", [16, 64, 1024])
def test_transforms_match_numpy(n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = np.fft.fft(x)
    assert np.abs(O.fft(x, -1) - ref).max() <= 1e-13 * np.log2(n) * np.abs(ref).max()
    if n <= 64:
        assert np.abs(O.dft(x, -1) - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(O.fft(x, +1) - n * np.fft.ifft(x)).max() <= 1e-13 * np.log2(n) * np.abs(ref).max()


def test_delta_and_plane_wave():
    # closed forms: DFT of a delta is flat; of a plane wave is a delta
    n = 32
    d = np.zeros(n, complex)
    d[0] = 1.0
    assert np.allclose(O.fft(d), np.ones(n), atol=1e-15)
    j = np.arange(n)
    w = np.exp(2j * np.pi * 5 * j / n)
    out = O.fft(w)
    expect = np.zeros(n, complex)
    expect[5] = n
    assert np.abs(out - expect).max() < 1e-12


def test_non_power_of_two_rejected():
    with pytest.raises(ValueError):
        O.fft(np.ones(12, complex))


def test_naive_drift_equals_fft_drift():
    # the whole unmerged step with the naive DFT equals the FFT path
    from paper_1007_3470_gb300 import workloads as W
    inst, psi0, _ = W.gpe_tdep_1d(h=0.02, n=64)
    inst.a, inst.b = [-8.0], [8.0]
    psi0 = W.gaussian_1d(inst)
    p_fast = O.Problem(**inst.as_dict())
    p_slow = O.Problem(**inst.as_dict(), naive_dft=True)
    u1 = O.run(p_fast, psi0, 5)
    u2 = O.run(p_slow, psi0, 5)
    assert O.rel_l2(u1, u2) < 1e-13
