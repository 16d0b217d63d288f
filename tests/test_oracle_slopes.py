"""Pins of the oracle's neighbour-leaf slope rule for AMR hierarchies
(oracle/slopes.py; the reading of Section 2's slopes when only sigma0 is given).

* On a single uniform grid the rule is the central difference with zero
  outside the grid: numpy's gradient of the zero-padded array (a library
  routine), at every cell.
* A linear density sigma = a + b x + c y is reproduced exactly (b, c) at every
  leaf none of whose sides faces the outside of the level-0 grid, on nested
  patches, ragged off-centre patches, the Table-10 hierarchy and ILR/VLR band
  hierarchies: same-level, finer and coarser neighbours all enter.
* The patch form equals the zone form of the same hierarchy.
* Mirror symmetry: reflecting the density and the hierarchy in x negates deltax
  and keeps deltay.
"""
import numpy as np
import pytest

from oracle import amr as oamr
from oracle import slopes as S
from paper_2001_02765_gb300 import workloads as W


def _full_grid(nx, ny):
    jj, ii = np.mgrid[0:ny, 0:nx]
    return np.zeros(nx * ny, int), ii.ravel(), jj.ravel(), np.ones(nx * ny, bool)


def test_one_level_is_central_difference_with_zero_outside():
    rng = np.random.Generator(np.random.PCG64(1))
    nx, ny, h = 13, 9, 0.125
    s = rng.uniform(-1, 1, (ny, nx))
    level, ix, iy, leaf = _full_grid(nx, ny)
    dx, dy = S.zone_neighbour_slopes(-0.5, 0.25, h, level, ix, iy, leaf, s.ravel())
    padded = np.pad(s, 1)
    gy, gx = np.gradient(padded, h)
    assert np.allclose(dx.reshape(ny, nx), gx[1:-1, 1:-1], rtol=0, atol=1e-13)
    assert np.allclose(dy.reshape(ny, nx), gy[1:-1, 1:-1], rtol=0, atol=1e-13)


def _interior(x0, y0, h0, level, ix, iy, nx0, ny0):
    """Zones farther from the outside of the level-0 grid than one level-0 cell
    per level: a leaf's slope may rest on a coarser neighbour's slope, which
    may rest on the next coarser one's, each one cell further out, and a slope
    next to the outside sees the zero there."""
    xl, xr, yd, yu, _, _ = oamr.zone_bounds(x0, y0, h0, level, ix, iy)
    m = (int(np.max(level)) + 1) * h0 + 1e-12
    return (xl > x0 + m) & (xr < x0 + nx0 * h0 - m) & (yd > y0 + m) & (yu < y0 + ny0 * h0 - m)


def _check_linear(x0, y0, h0, level, ix, iy, leaf, nx0, ny0):
    a, b, c = 0.3, -1.7, 2.4
    _, _, _, _, xc, yc = oamr.zone_bounds(x0, y0, h0, level, ix, iy)
    s = a + b * xc + c * yc
    dx, dy = S.zone_neighbour_slopes(x0, y0, h0, level, ix, iy, leaf, s)
    sel = np.asarray(leaf, bool) & _interior(x0, y0, h0, level, ix, iy, nx0, ny0)
    assert sel.sum() > 0
    assert np.max(np.abs(dx[sel] - b)) < 1e-11
    assert np.max(np.abs(dy[sel] - c)) < 1e-11
    # the levels really mix: some leaf has a neighbour of another level
    assert len(set(np.asarray(level)[np.asarray(leaf, bool)].tolist())) > 1


@pytest.mark.parametrize("spec", ["nested", "ragged", "table10"])
def test_linear_density_exact_on_patch_hierarchies(spec):
    if spec == "nested":
        patches = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(16, 3))]
        n0 = (16, 16)
    elif spec == "ragged":
        patches = [(0, 37, 29, -1.0, -0.8, 0.05), (1, 22, 14, -0.6, -0.3, 0.025), (1, 6, 8, 0.2, 0.1, 0.025),
                   (2, 10, 12, -0.5, -0.25, 0.0125)]
        n0 = (37, 29)
    else:
        # the refined patches of Fig. 1 / Table 10 inside a level-0 grid widened
        # by four cells on every side, so that they lie away from its outside
        patches = [(0, 12, 12, -1.0, -1.0, 0.25), (1, 2, 2, 0.25, 0.25, 0.125), (1, 2, 2, 0.5, 0.5, 0.125),
                   (2, 2, 2, 0.25, 0.375, 0.0625), (2, 2, 2, 0.375, 0.25, 0.0625)]
        n0 = (12, 12)
    x0, y0, h0, level, ix, iy, leaf = S.patches_as_zones(oamr.make_patches(patches))
    _check_linear(x0, y0, h0, level, ix, iy, leaf, *n0)


@pytest.mark.parametrize("rule, disk", [("ilr", "d2"), ("vlr", "d22")])
def test_linear_density_exact_on_band_hierarchies(rule, disk):
    hier = W.band_hierarchy(32, 3, rule, disk)
    _check_linear(hier["x0"], hier["y0"], hier["h0"], hier["level"], hier["ix"], hier["iy"], hier["leaf"],
                  hier["n"], hier["n"])


def test_patch_form_equals_zone_form():
    patches = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(8, 3))]
    P = oamr.make_patches(patches)
    rng = np.random.Generator(np.random.PCG64(2))
    sig = [rng.uniform(0, 1, (p.ny, p.nx)) for p in P]
    px, py = S.patch_neighbour_slopes(P, sig)
    x0, y0, h0, level, ix, iy, leaf = S.patches_as_zones(P)
    zx, zy = S.zone_neighbour_slopes(x0, y0, h0, level, ix, iy, leaf, np.concatenate([a.ravel() for a in sig]))
    assert np.array_equal(np.concatenate([a.ravel() for a in px]), zx)
    assert np.array_equal(np.concatenate([a.ravel() for a in py]), zy)


def test_mirror_symmetry():
    hier = W.band_hierarchy(24, 3, "ilr", "d2")
    x0, h0, n = hier["x0"], hier["h0"], hier["n"]
    level, ix, iy, leaf = hier["level"], hier["ix"], hier["iy"], hier["leaf"]
    rng = np.random.Generator(np.random.PCG64(3))
    s = rng.uniform(0, 1, level.size)
    dx, dy = S.zone_neighbour_slopes(x0, hier["y0"], h0, level, ix, iy, leaf, s)
    # reflect in x about the domain centre: zone (l, i, j) -> (l, n 2^l - 1 - i, j)
    mix = (n * 2 ** level.astype(np.int64) - 1 - ix).astype(ix.dtype)
    keys = {(int(l), int(i), int(j)): k for k, (l, i, j) in enumerate(zip(level, mix, iy))}
    perm = np.array([keys[(int(l), int(i), int(j))] for l, i, j in zip(level, ix, iy)])
    mx, my = S.zone_neighbour_slopes(x0, hier["y0"], h0, level[perm], ix, iy[perm], leaf[perm], s[perm])
    assert np.allclose(mx, -dx[perm], atol=1e-12) and np.allclose(my, dy[perm], atol=1e-12)
