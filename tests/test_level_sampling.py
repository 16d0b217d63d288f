"""The two sampling identities the level convolutions rest on, checked with
numpy's FFT on random data (no oracle, no CUDA): a coarse level's samples on the
finest lattice have a spectrum that repeats with the compact period (times the
half-sample phase), and a coarse target level's samples of an inverse transform
are the inverse transform of the folded spectrum at the compact length. The
sign conventions are the kernels': forward exp(-2 pi i k n / P), inverse
exp(+2 pi i k n / P) unnormalised, psi(k) = exp(-i pi k / M)."""
import numpy as np
import pytest


def _psi(k, m):
    return np.exp(-1j * np.pi * k / m)


@pytest.mark.parametrize("p, c, half", [(64, 1, False), (64, 1, True), (256, 2, True), (256, 3, False),
                                        (1024, 2, True)])
def test_source_spectrum_repeats_with_the_compact_period(p, c, half):
    """x sampled at r + 2^c j on a length-p lattice (r = 0, or half a compact
    sample 2^(c-1)) has X(k) = psi(k)^(2 r / 2^c) X_c(k mod M), M = p / 2^c, where
    X_c is the length-M transform of the compact samples."""
    rng = np.random.default_rng(p + c)
    m = p >> c
    r = (1 << (c - 1)) if half else 0
    xc = np.zeros(m, complex)
    xc[: m // 2] = rng.standard_normal(m // 2) + 1j * rng.standard_normal(m // 2)
    x = np.zeros(p, complex)
    x[r + (np.arange(m) << c)] = xc
    X = np.fft.fft(x)
    Xc = np.fft.fft(xc)
    k = np.arange(p)
    phase = _psi(k, m) if half else np.ones(p)  # exp(-2 pi i k r / p) with r = 2^(c-1)
    assert np.allclose(X, phase * Xc[k % m], atol=1e-10 * np.abs(X).max())


@pytest.mark.parametrize("p, c, half", [(64, 1, False), (64, 1, True), (256, 2, True), (512, 3, True),
                                        (2048, 1, False)])
def test_target_samples_are_the_folded_inverse(p, c, half):
    """y = inverse transform of X (length p); y at r + 2^c n equals the length-M
    inverse transform of Z(k) = conj(psi(k))^h sum_q s_q X(k + q M), s_q = (-1)^q
    when r = 2^(c-1) (h = 1), 1 when r = 0 (h = 0)."""
    rng = np.random.default_rng(7 * p + c)
    m = p >> c
    r = (1 << (c - 1)) if half else 0
    X = rng.standard_normal(p) + 1j * rng.standard_normal(p)
    y = np.fft.ifft(X) * p
    q = np.arange(1 << c)
    s = (-1.0) ** q if half else np.ones(1 << c)
    k = np.arange(m)
    Z = (s[:, None] * X[k[None, :] + q[:, None] * m]).sum(axis=0)
    if half:
        Z = Z * np.conj(_psi(k, m))
    z = np.fft.ifft(Z) * m
    assert np.allclose(y[r + (np.arange(m) << c)], z, atol=1e-10 * np.abs(y).max())


def test_folding_a_wrong_sign_fails():
    """The alternating signs are needed for the half-sample offset (a plain sum
    samples the even positions instead)."""
    p, c = 256, 2
    m, r = p >> c, 1 << (c - 1)
    X = np.random.default_rng(3).standard_normal(p) + 0j
    y = np.fft.ifft(X) * p
    k = np.arange(m)
    Z = X.reshape(1 << c, m).sum(axis=0) * np.conj(_psi(k, m))
    assert not np.allclose(y[r + (np.arange(m) << c)], np.fft.ifft(Z) * m)
