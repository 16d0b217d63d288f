"""Pins of the oracle's mid-plane potential (Section 2, K = 1/r) against
quadrature, the D_2 closed form of Section 3, reciprocity, the force (F = -grad
Phi) and a second route (FFT)."""
import math

import numpy as np
import pytest

from oracle.direct import uniform_direct_force
from oracle.disks import d2_potential
from oracle.norms import norms
from oracle import amr as oamr
from oracle.potential import amr_direct_potential, cell_potentials, uniform_direct_potential, uniform_fft_potential
from paper_2001_02765_gb300 import workloads as W


def _quad(f, xl, xr, yd, yu):
    from scipy.integrate import dblquad
    val, _ = dblquad(lambda yb, xb: f(xb, yb), xl, xr, yd, yu, epsabs=1e-13, epsrel=1e-12)
    return val


@pytest.mark.parametrize("cell", [(0.3, 0.7, 0.2, 0.5), (-2.0, -1.5, 3.0, 3.5), (0.0, 0.4, -0.3, 0.3),
                                  (-0.3, 0.5, 0.1, 0.6), (0.2, 0.6, 0.0, 0.3)])
def test_cell_potentials_match_quadrature(cell):
    """Far, near, on a vertical edge line, and on a horizontal edge line (target at the origin)."""
    pytest.importorskip("scipy")
    xl, xr, yd, yu = cell
    xc, yc = (xl + xr) / 2, (yd + yu) / 2
    k = cell_potentials(0.0, 0.0, *cell)
    r = lambda a, b: math.hypot(a, b)
    ref = {"p0": lambda a, b: 1.0 / r(a, b), "px": lambda a, b: (a - xc) / r(a, b),
           "py": lambda a, b: (b - yc) / r(a, b)}
    for name, f in ref.items():
        assert abs(float(k[name]) - _quad(f, *cell)) < 1e-11, name


def test_self_cell_closed_form():
    """The integral of 1/r over a square of side h centred on the target is 4 h ln(1 + sqrt 2)."""
    for h in (1.0, 0.03):
        k = cell_potentials(0.0, 0.0, -h / 2, h / 2, -h / 2, h / 2)
        assert abs(float(k["p0"]) / (4 * h * math.log(1 + math.sqrt(2))) - 1) < 1e-14
        assert float(k["px"]) == 0.0 and float(k["py"]) == 0.0


def test_far_cell_is_point_mass():
    h, d = 0.1, (7.0, -4.0)
    k = cell_potentials(d[0], d[1], -h / 2, h / 2, -h / 2, h / 2)
    assert abs(float(k["p0"]) / (h * h / math.hypot(*d)) - 1) < 1e-4


def test_d2_potential_converges_second_order():
    """Uniform D_2 (radius 0.5) with analytic slopes against the closed form of Section 3."""
    errs = []
    for n in (64, 128):
        nx, ny, x0, y0, h = W.unit_grid(n)
        X, Y = W.cell_centres(nx, ny, x0, y0, h)
        s, sx, sy = W.d2_sigma(X, Y, 0.5)
        phi = uniform_fft_potential(s, sx, sy, h)
        errs.append(norms(phi - d2_potential(np.hypot(X, Y), 0.5), h * h)[0])
    assert errs[1] < 2e-4
    assert math.log2(errs[0] / errs[1]) > 1.8, errs


def test_reciprocity_order0():
    """For piecewise-constant densities the pair integral is symmetric:
    sum_i a_i Phi[b]_i = sum_i b_i Phi[a]_i."""
    a, _, _ = W.random_fields(20, 24, seed=5)
    b, _, _ = W.random_fields(20, 24, seed=6)
    pa = uniform_direct_potential(a, None, None, 0.05)
    pb = uniform_direct_potential(b, None, None, 0.05)
    lhs, rhs = float(np.sum(a * pb)), float(np.sum(b * pa))
    assert abs(lhs - rhs) < 1e-13 * (abs(lhs) + 1.0)


def test_force_is_minus_gradient():
    """Central differences of Phi against the force, at cells away from the grid
    edge: the discrepancy falls at second order."""
    errs = []
    for n in (48, 96):
        nx, ny, x0, y0, h = W.unit_grid(n)
        X, Y = W.cell_centres(nx, ny, x0, y0, h)
        s, sx, sy = W.kuzmin_sigma(X, Y, 0.3)
        phi = uniform_fft_potential(s, sx, sy, h)
        fx, fy = uniform_direct_force(s, sx, sy, h)
        gx = -(phi[1:-1, 2:] - phi[1:-1, :-2]) / (2 * h)
        gy = -(phi[2:, 1:-1] - phi[:-2, 1:-1]) / (2 * h)
        inner = (np.abs(X[1:-1, 1:-1]) < 0.5) & (np.abs(Y[1:-1, 1:-1]) < 0.5)
        e = np.hypot(gx - fx[1:-1, 1:-1], gy - fy[1:-1, 1:-1])[inner]
        errs.append(float(np.sqrt(np.mean(e * e))) / float(np.sqrt(np.mean(fx[1:-1, 1:-1][inner] ** 2))))
    assert errs[0] < 2e-2
    assert math.log2(errs[0] / errs[1]) > 1.8, errs


@pytest.mark.parametrize("shape", [(9, 13), (16, 16)])
def test_fft_route_equals_plain_sum(shape):
    s, sx, sy = W.random_fields(*shape, seed=sum(shape))
    a = uniform_direct_potential(s, sx, sy, 0.07, x0=0.3, y0=-0.2)
    b = uniform_fft_potential(s, sx, sy, 0.07)
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(a))


def test_amr_refinement_invariance():
    """Refining coarse cells into children that carry the parent's linear
    reconstruction (sigma0 + delta . offset, same delta) leaves the potential at
    the coarse leaves equal to the uniform-grid sum: the integrand is identical."""
    n = 16
    nx, ny, x0, y0, h = W.unit_grid(n)
    s, sx, sy = W.random_fields(n, n, seed=23)
    ref = uniform_direct_potential(s, sx, sy, h, x0=x0, y0=y0)
    patches = oamr.make_patches([(0, nx, ny, x0, y0, h), (1, 16, 16, -0.5, -0.5, h / 2)])
    fs, fsx, fsy = (np.zeros((16, 16)) for _ in range(3))
    for J in range(16):
        for I in range(16):
            pj, pi = 4 + J // 2, 4 + I // 2
            fs[J, I] = s[pj, pi] + sx[pj, pi] * (I % 2 - 0.5) * h / 2 + sy[pj, pi] * (J % 2 - 0.5) * h / 2
            fsx[J, I], fsy[J, I] = sx[pj, pi], sy[pj, pi]
    leaves, phi = amr_direct_potential(patches, [s, fs], [sx, fsx], [sy, fsy])
    coarse = leaves["patch"] == 0
    got, want = phi[coarse], ref[leaves["j"][coarse], leaves["i"][coarse]]
    assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want))
    # the refined region's leaves see the same potential at their own centres as
    # the plain sum over the unrefined grid's cells
    fine = ~coarse
    tx, ty = leaves["xc"][fine], leaves["yc"][fine]
    I, J = np.meshgrid(np.arange(nx), np.arange(ny))
    from oracle.potential import direct_potential
    cells = (x0 + I * h, x0 + (I + 1) * h, y0 + J * h, y0 + (J + 1) * h)
    want_f = direct_potential(cells, s, sx, sy, tx, ty)
    assert np.max(np.abs(phi[fine] - want_f)) < 1e-13 * np.max(np.abs(want_f))
