"""Error bounds of the far-field evaluations the FP32 direct sums use (CPU).

The FP32 cross-patch sums evaluate the cells at least 6 cell widths from a
target (along some axis) not by their closed forms but by approximations of
the same integrals:
  * in the plane, the expansion of each cell's force integrals about its
    centre through H^6 (within 32 widths) or H^4 (beyond), in complex form;
  * for the potential, the moments of 1/r over the cell (p = 1/rho, through p^7
    within 32 widths, p^3 beyond);
  * off the plane, tensor Gauss-Legendre quadrature (3 x 3 nodes within 32
    widths, 2 x 2 beyond).
Here each approximation, restated from its stated form, is compared with the
oracle's FP64 closed forms of Section 2 (oracle.kernels, oracle.potential) over
a spread of offsets, and held to the truncation bound the kernels rely on, so
that a wrong coefficient or sign in the stated forms fails here.
"""
import numpy as np
import pytest

from oracle.kernels import cell_kernels, cell_kernels_z
from oracle.potential import cell_potentials


def _offsets(lo, hi, n=400, seed=0):
    """Cell-centre offsets (a, b) with lo <= max(|a|, |b|) < hi (unit cells)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    while len(out) < n:
        a, b = rng.uniform(-hi, hi, 2)
        if lo <= max(abs(a), abs(b)) < hi:
            out.append((a, b))
    return np.array(out)


def _exact_force(a, b, m, dx, dy):
    k = cell_kernels(0.0, 0.0, a - 0.5, a + 0.5, b - 0.5, b + 0.5)
    fx = m * k["x0"] + dx * k["xx"] + dy * k["xy"]
    fy = m * k["y0"] + dx * k["yx"] + dy * k["yy"]
    return fx, fy


def _expansion_force(a, b, m, dx, dy, order):
    """Fx - i Fy of the cell-centred expansion (unit cell, G = 1)."""
    w = 1.0 / (a + 1j * b)
    s = 1.0 / (a * a + b * b)
    D = dx + 1j * dy
    Db = np.conj(D)
    wb = np.conj(w)
    if order == 4:
        q = m * w * (1 + s / 8) - D * w ** 2 / 8 - Db * s / 24
    else:
        q = (m * (w * (1 + s / 8 + 7 * s * s / 256) - 21 * w ** 5 / 512 - 7 * s * wb ** 3 / 1536)
             - D * w ** 2 / 8 - Db * s / 24 + 7 * Db * w ** 4 / 384 + D * s * (wb ** 2 - 7 * w ** 2) / 384
             - 7 * Db * s * s / 640)
    q = q * np.sqrt(s)
    return q.real, -q.imag


# (sigma0 bound, slope bound), relative to 1/rho^2 per unit sigma0 or unit delta H;
# measured maxima on a half-cell grid: 1.3e-7 / 1.02e-6 (H^6), 3e-8 / 7.6e-7 (H^4)
@pytest.mark.parametrize("lo, hi, order, bounds", [(6, 32, 6, (2e-7, 1.5e-6)), (32, 200, 4, (1e-7, 1e-6))])
@pytest.mark.parametrize("m, dx, dy", [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)])
def test_in_plane_expansion_within_bound(lo, hi, order, bounds, m, dx, dy):
    bound = bounds[0] if m else bounds[1]
    ab = _offsets(lo, hi)
    worst = 0.0
    for a, b in ab:
        ex, ey = _exact_force(a, b, m, dx, dy)
        gx, gy = _expansion_force(a, b, m, dx, dy, order)
        scale = 1.0 / (a * a + b * b)  # the size of a unit cell's sigma0 term
        worst = max(worst, abs(gx - ex) / scale, abs(gy - ey) / scale)
    assert worst < bound, worst


def _moments(a, b, order):
    p = 1.0 / np.hypot(a, b)
    i0 = p + p ** 3 / 24
    ix = -a * p ** 3 / 12
    iy = -b * p ** 3 / 12
    if order >= 6:
        i0 = i0 + p ** 5 * (-7.0 / 1920 + (7.0 / 96) * a * a * b * b * p ** 4)
        ix = ix + (7.0 / 240) * a * p ** 5 - a * p ** 7 * (a * a / 32 + 5 * b * b / 96)
        iy = iy + (7.0 / 240) * b * p ** 5 - b * p ** 7 * (b * b / 32 + 5 * a * a / 96)
    return i0, ix, iy


# relative to p = 1/rho; measured maxima 1.6e-8 / 1.5e-7 (through p^7), 5e-9 / 1.8e-7 (p^3)
@pytest.mark.parametrize("lo, hi, order, bounds", [(6, 32, 6, (5e-8, 3e-7)), (32, 200, 4, (2e-8, 3e-7))])
def test_potential_moments_within_bound(lo, hi, order, bounds):
    ab = _offsets(lo, hi, seed=1)
    w0 = ws = 0.0
    for a, b in ab:
        ex = cell_potentials(0.0, 0.0, a - 0.5, a + 0.5, b - 0.5, b + 0.5)
        i0, ix, iy = _moments(a, b, order)
        p = 1.0 / np.hypot(a, b)
        w0 = max(w0, abs(i0 - ex["p0"]) / p)
        ws = max(ws, abs(ix - ex["px"]) / p, abs(iy - ex["py"]) / p)
    assert w0 < bounds[0] and ws < bounds[1], (w0, ws)


def _quadrature_force(a, b, zeta, m, dx, dy, n):
    """Gauss-Legendre tensor rule on the unit cell of (m + dx xi + dy eta)(a + xi, b + eta, -zeta)/R^3."""
    x, w = np.polynomial.legendre.leggauss(n)
    x, w = x / 2.0, w / 2.0
    f = np.zeros(3)
    for xi, wi in zip(x, w):
        for eta, wj in zip(x, w):
            da, db = a + xi, b + eta
            r3 = (da * da + db * db + zeta * zeta) ** 1.5
            dens = m + dx * xi + dy * eta
            f += wi * wj * dens * np.array([da, db, -zeta]) / r3
    return f


# relative to 1/R^2; measured maxima 2e-8 / 1.7e-7 (3 x 3 from 6 widths), 3.4e-8 / 6.5e-7 (2 x 2 from 32)
@pytest.mark.parametrize("zeta", [0.25, 1.0, -3.0])
@pytest.mark.parametrize("lo, hi, n, bounds", [(6, 32, 3, (5e-8, 3e-7)), (32, 200, 2, (1e-7, 1e-6))])
@pytest.mark.parametrize("m, dx, dy", [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)])
def test_offplane_quadrature_within_bound(zeta, lo, hi, n, bounds, m, dx, dy):
    bound = bounds[0] if m else bounds[1]
    ab = _offsets(lo, hi, n=200, seed=2)
    worst = 0.0
    for a, b in ab:
        k = cell_kernels_z(0.0, 0.0, zeta, a - 0.5, a + 0.5, b - 0.5, b + 0.5)
        exact = np.array([m * k["x0"] + dx * k["xx"] + dy * k["xy"],
                          m * k["y0"] + dx * k["yx"] + dy * k["yy"],
                          m * k["z0"] + dx * k["zx"] + dy * k["zy"]])
        got = _quadrature_force(a, b, zeta, m, dx, dy, n)
        scale = 1.0 / (a * a + b * b + zeta * zeta)
        worst = max(worst, np.max(np.abs(got - exact)) / scale)
    assert worst < bound, worst
