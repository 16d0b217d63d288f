"""Uniform-grid force as a zero-padded FFT convolution (FP64, numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

On a uniform grid of square cells the cell integrals of Section 2 depend only
on the offset (m, n) between source and target cells (K^{.,0} is scale-free;
K^{.,x} and K^{.,y} are proportional to h), so
    F_x[t] = G sum_s sigma0[s] K^{x,0}[s - t] + deltax[s] K^{x,x}[s - t] + deltay[s] K^{x,y}[s - t]
is a correlation of the three input fields with three tables. Zero padding to
P >= 2N - 1 in each direction makes the circular convolution equal to the linear
one; the paper's introduction and conclusion describe this FFT route for uniform
grids (after Yen et al. 2012). The FFT itself is numpy's (a library routine).
"""
import numpy as np

from .kernels import offset_tables, offset_tables_z


def _wrap_correlation_kernel(table, py, px):
    """Place K[-e] at index e mod P so that F = sigma (*) wrapped is the correlation."""
    ky, kx = table.shape
    my, mx = (ky + 1) // 2, (kx + 1) // 2
    out = np.zeros((py, px), dtype=np.float64)
    n = np.arange(-(my - 1), my)
    m = np.arange(-(mx - 1), mx)
    # table[n + my - 1, m + mx - 1] = K(m, n); K~(e) = K(-e)
    rows = (-n) % py
    cols = (-m) % px
    out[np.ix_(rows, cols)] = table
    return out


def uniform_fft_force(sigma, dx, dy, h, G=1.0, pad=None):
    """Fx, Fy at every cell of a uniform nx-by-ny grid by zero-padded FFT.

    sigma, dx, dy: arrays [ny, nx] (dx, dy may be None: order-0 sum).
    pad: (py, px) padded sizes, default (2 ny, 2 nx); each must be >= 2n - 1.
    """
    sigma = np.asarray(sigma, dtype=np.float64)
    ny, nx = sigma.shape
    py, px = pad if pad is not None else (2 * ny, 2 * nx)
    if py < 2 * ny - 1 or px < 2 * nx - 1:
        raise ValueError("padding too small for a linear convolution")
    tabs = offset_tables(nx, ny, h)

    def spec(a):
        return np.fft.rfft2(a, s=(py, px))

    def kspec(name):
        return np.fft.rfft2(_wrap_correlation_kernel(tabs[name], py, px))

    s_hat = spec(sigma)
    fx_hat = s_hat * kspec("x0")
    fy_hat = s_hat * kspec("y0")
    if dx is not None:
        dx_hat = spec(np.asarray(dx, dtype=np.float64))
        fx_hat += dx_hat * kspec("xx")
        fy_hat += dx_hat * kspec("yx")
    if dy is not None:
        dy_hat = spec(np.asarray(dy, dtype=np.float64))
        fx_hat += dy_hat * kspec("xy")
        fy_hat += dy_hat * kspec("yy")
    fx = np.fft.irfft2(fx_hat, s=(py, px))[:ny, :nx]
    fy = np.fft.irfft2(fy_hat, s=(py, px))[:ny, :nx]
    return G * fx, G * fy


def central_slopes(sigma, h):
    """deltax, deltay by central differences with sigma = 0 outside the grid.

    The paper does not say how the slopes of Eq. eqnGamma are obtained; this is
    the reading used for the 'central' slope mode: (sigma[i+1] - sigma[i-1]) / 2h
    along each axis, the neighbours beyond the grid edge counting as zero.
    """
    s = np.asarray(sigma, dtype=np.float64)
    p = np.pad(s, 1)
    dx = (p[1:-1, 2:] - p[1:-1, :-2]) / (2.0 * h)
    dy = (p[2:, 1:-1] - p[:-2, 1:-1]) / (2.0 * h)
    return dx, dy


def uniform_fft_force3(sigma, dx, dy, h, z, G=1.0, pad=None):
    """Fx, Fy, Fz at height z != 0 above every cell centre, by zero-padded FFT
    with the nine off-plane kernel tables."""
    sigma = np.asarray(sigma, dtype=np.float64)
    ny, nx = sigma.shape
    py, px = pad if pad is not None else (2 * ny, 2 * nx)
    tabs = offset_tables_z(nx, ny, h, z)

    def spec(a):
        return np.fft.rfft2(a, s=(py, px))

    def kspec(name):
        return np.fft.rfft2(_wrap_correlation_kernel(tabs[name], py, px))

    fields = [(spec(sigma), "0")]
    if dx is not None:
        fields.append((spec(np.asarray(dx, np.float64)), "x"))
    if dy is not None:
        fields.append((spec(np.asarray(dy, np.float64)), "y"))
    out = []
    for comp in ("x", "y", "z"):
        acc = sum(f * kspec(comp + k) for f, k in fields)
        out.append(G * np.fft.irfft2(acc, s=(py, px))[:ny, :nx])
    return tuple(out)
