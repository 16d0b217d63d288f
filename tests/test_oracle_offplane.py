"""Pins of the oracle's off-plane forces (targets at height z != 0; Section 2,
the antiderivatives with the arctan terms)."""
import math

import numpy as np
import pytest

from oracle.direct import uniform_direct_force3
from oracle.disks import kuzmin_force_xyz
from oracle.fftconv import uniform_fft_force3
from oracle.kernels import cell_kernels, cell_kernels_z
from oracle.norms import rel_l2
from paper_2001_02765_gb300 import workloads as W


def _quad(f, xl, xr, yd, yu):
    from scipy.integrate import dblquad
    val, _ = dblquad(lambda yb, xb: f(xb, yb), xl, xr, yd, yu, epsabs=1e-13, epsrel=1e-12)
    return val


@pytest.mark.parametrize("z", [0.25, -0.4, 0.03])
@pytest.mark.parametrize("cell", [(0.3, 0.7, 0.2, 0.5), (-2.0, -1.5, 3.0, 3.5), (-0.1, 0.1, -0.1, 0.1),
                                  (0.0, 0.4, -0.3, 0.3)])
def test_offplane_closed_forms_match_quadrature(cell, z):
    pytest.importorskip("scipy")
    xl, xr, yd, yu = cell
    x = y = 0.0
    xc, yc = (xl + xr) / 2, (yd + yu) / 2
    k = cell_kernels_z(x, y, z, *cell)
    r3 = lambda a, b: ((a - x) ** 2 + (b - y) ** 2 + z * z) ** 1.5
    ref = {
        "x0": lambda a, b: (a - x) / r3(a, b), "xx": lambda a, b: (a - xc) * (a - x) / r3(a, b),
        "xy": lambda a, b: (b - yc) * (a - x) / r3(a, b), "y0": lambda a, b: (b - y) / r3(a, b),
        "yx": lambda a, b: (a - xc) * (b - y) / r3(a, b), "yy": lambda a, b: (b - yc) * (b - y) / r3(a, b),
        "z0": lambda a, b: -z / r3(a, b), "zx": lambda a, b: (a - xc) * -z / r3(a, b),
        "zy": lambda a, b: (b - yc) * -z / r3(a, b),
    }
    for name, f in ref.items():
        v = _quad(f, *cell)
        assert abs(float(k[name]) - v) <= 2e-9 * max(1.0, abs(v)), (name, float(k[name]), v)


def test_offplane_reduces_to_plane_and_solid_angle_limit():
    cell = (0.3, 0.7, -0.2, 0.5)
    inplane = cell_kernels(0.0, 0.0, *cell)
    near = cell_kernels_z(0.0, 0.0, 1e-9, *cell)
    for name in inplane:
        assert abs(float(inplane[name]) - float(near[name])) < 1e-7, name
    # just above / below a cell the normal force density is -/+ 2 pi (the half-space solid angle)
    h = 0.2
    above = cell_kernels_z(0.0, 0.0, 1e-9, -h / 2, h / 2, -h / 2, h / 2)
    below = cell_kernels_z(0.0, 0.0, -1e-9, -h / 2, h / 2, -h / 2, h / 2)
    assert abs(float(above["z0"]) + 2 * math.pi) < 1e-7 and abs(float(below["z0"]) - 2 * math.pi) < 1e-7


def test_offplane_parity_in_z():
    cell = (0.3, 0.7, -0.2, 0.5)
    a = cell_kernels_z(0.1, -0.05, 0.37, *cell)
    b = cell_kernels_z(0.1, -0.05, -0.37, *cell)
    for name in a:
        sgn = -1.0 if name.startswith("z") else 1.0
        assert abs(float(a[name]) - sgn * float(b[name])) < 1e-14, name


def test_offplane_fft_route_equals_plain_sum():
    ny, nx = 11, 14
    s, sx, sy = W.random_fields(ny, nx, seed=41)
    h, z = 0.07, 0.13
    f = uniform_fft_force3(s, sx, sy, h, z, G=0.9)
    g = uniform_direct_force3(s, sx, sy, h, z, G=0.9)
    num = sum(np.sum((a - b) ** 2) for a, b in zip(f, g))
    den = sum(np.sum(b ** 2) for b in g)
    assert math.sqrt(num / den) < 1e-13


def test_kuzmin_off_plane_converges_second_order():
    """Kuzmin a = 0.2 on a [-8,8]^2 grid, targets at height z = 0.1 above the
    cells with |x|, |y| < 1: closed form -G M (x, y, a + z) / (R^2 + (a + z)^2)^{3/2}."""
    errs = []
    z = 0.1
    for n_unit in (32, 64):
        n = 8 * n_unit
        h = 16.0 / n
        X, Y = W.cell_centres(n, n, -8.0, -8.0, h)
        s, sx, sy = W.kuzmin_sigma(X, Y, 0.2)
        fx, fy, fz = uniform_fft_force3(s, sx, sy, h, z)
        inner = (np.abs(X) < 1.0) & (np.abs(Y) < 1.0)
        kx, ky, kz = kuzmin_force_xyz(X[inner], Y[inner], z, 0.2)
        num = np.sum((fx[inner] - kx) ** 2 + (fy[inner] - ky) ** 2 + (fz[inner] - kz) ** 2)
        den = np.sum(kx ** 2 + ky ** 2 + kz ** 2)
        errs.append(math.sqrt(num / den))
    assert errs[0] < 1e-2
    assert math.log2(errs[0] / errs[1]) > 1.8, errs
