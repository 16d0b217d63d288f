"""The benchmark's torch.fft comparison computes the same convolution (CPU).

bench.TorchFFTConv is timed beside the library's transforms; here it runs on
the CPU with the oracle's FP64 tables and is held to the oracle's FFT route
(oracle.fftconv, Section 2 closed forms) on ragged grids in every slope mode,
so that the timed comparison is known to do the same work.
"""
import numpy as np
import pytest
import torch

import bench
from oracle.fftconv import central_slopes, uniform_fft_force
from oracle.kernels import offset_tables
from oracle.norms import rel_l2

NAMES = ("x0", "xx", "xy", "y0", "yx", "yy")


def _case(nx, ny, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(0.5, 1.5, (ny, nx)), rng.normal(size=(ny, nx)), rng.normal(size=(ny, nx))


@pytest.mark.parametrize("nx, ny", [(13, 9), (32, 32), (40, 17)])
@pytest.mark.parametrize("slope_mode", [0, 1, 2])
def test_matches_the_oracle_fft_route(nx, ny, slope_mode):
    h, G = 0.05, 1.7
    sigma, dx, dy = _case(nx, ny, nx * 100 + ny)
    tabs = offset_tables(nx, ny, h)
    pad = (bench._pad(ny), bench._pad(nx))
    conv = bench.TorchFFTConv([tabs[k] for k in NAMES], nx, ny, h, G, slope_mode, pad, torch.float64, "cpu")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel())
    if slope_mode == 0:
        fx, fy = conv(t(sigma))
        ox, oy = uniform_fft_force(sigma, None, None, h, G=G, pad=pad)
    elif slope_mode == 1:
        fx, fy = conv(t(sigma))
        cx, cy = central_slopes(sigma, h)
        ox, oy = uniform_fft_force(sigma, cx, cy, h, G=G, pad=pad)
    else:
        fx, fy = conv(t(sigma), t(dx), t(dy))
        ox, oy = uniform_fft_force(sigma, dx, dy, h, G=G, pad=pad)
    err = rel_l2(fx.numpy().ravel(), fy.numpy().ravel(), ox.ravel(), oy.ravel())
    assert err < 1e-12, err


def test_fp32_form_within_single_precision():
    nx, ny, h = 48, 48, 1.0 / 24
    sigma, _, _ = _case(nx, ny, 7)
    tabs = offset_tables(nx, ny, h)
    pad = (bench._pad(ny), bench._pad(nx))
    conv = bench.TorchFFTConv([tabs[k] for k in NAMES], nx, ny, h, 1.0, 1, pad, torch.float32, "cpu")
    fx, fy = conv(torch.from_numpy(sigma.astype(np.float32).ravel()))
    cx, cy = central_slopes(sigma.astype(np.float32).astype(np.float64), h)
    ox, oy = uniform_fft_force(sigma.astype(np.float32).astype(np.float64), cx, cy, h, pad=pad)
    err = rel_l2(fx.double().numpy().ravel(), fy.double().numpy().ravel(), ox.ravel(), oy.ravel())
    assert err < 1e-5, err
