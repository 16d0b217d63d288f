"""Pins of the FP64 oracle against values the paper prints and facts mathematics fixes.

Each test pins the oracle to something other than itself: a printed table, a
closed-form force, numerical quadrature of the integrand, a symmetry, an exact
cancellation, or a second independent route (library FFT vs plain sum).
"""
import math
import os

import numpy as np
import pytest

from oracle import amr as oamr
from oracle.direct import direct_force, uniform_direct_force
from oracle.disks import d2_force_xy, kuzmin_force_xy
from oracle.fftconv import central_slopes, uniform_fft_force
from oracle.kernels import cell_kernels, offset_tables
from oracle.norms import amr_norms, norms, radial_error, rel_l2
from paper_2001_02765_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([float(t) for t in line.split()])
    return rows


def _sig3(a, b):
    """True when a, rounded to three significant digits, equals the printed b."""
    e = math.floor(math.log10(abs(b)))
    return abs(round(a / 10 ** e, 2) - round(b / 10 ** e, 2)) < 1e-9


def _near3(a, b, units=0.51):
    """True when a lies within `units` of the printed b's third digit (the default,
    half a unit plus 2 %, admits a rounding tie: 3.50499e-3 printed as 3.51e-3)."""
    e = math.floor(math.log10(abs(b)))
    return abs(a / 10 ** e - b / 10 ** e) <= 0.01 * units


# --------------------------------------------------------------- Table 1 --

@pytest.mark.parametrize("n", [128, 256, 512])
def test_table1_d2_uniform_reproduced(n):
    """Table 1 (Section 3): uniform D_2 errors, all six printed norms to 3 digits.

    Readings: attractive sign, order-1 Taylor terms with the analytic gradient,
    D_2 radius 0.5 on [-1,1]^2 (the text's alpha = 0.25 does not reproduce the
    table), norms over all cells.
    """
    row = {int(r[0]): r[1:] for r in _load_table("table1_d2_uniform.txt")}[n]
    nx, ny, x0, y0, h = W.unit_grid(n)
    X, Y = W.cell_centres(nx, ny, x0, y0, h)
    s, sx, sy = W.d2_sigma(X, Y, 0.5)
    fx, fy = uniform_fft_force(s, sx, sy, h)
    ex, ey = d2_force_xy(X, Y, 0.5)
    got = norms(fx - ex, h * h) + norms(radial_error(X, Y, fx - ex, fy - ey), h * h)
    for g, p in zip(got, row):
        assert _sig3(g, p), (n, got, row)


@pytest.mark.parametrize("n", [128, 256, 512])
def test_table2_d22_uniform_reproduced(n):
    """Table 2 (Section 3): uniform D_2,2 errors, all nine printed norms to 3 digits
    (N = 512 without its misprinted L_Rinf).

    Reading: the two D_2 disks at (0, +-0.5) have radius 0.4 (the text gives
    only alpha = 0.25; radius 0.4 also reproduces the D_2,2 zone counts of
    Tables 8 and 9)."""
    row = {int(r[0]): r[1:] for r in _load_table("table2_d22_uniform.txt")}[n]
    nx, ny, x0, y0, h = W.unit_grid(n)
    X, Y = W.cell_centres(nx, ny, x0, y0, h)
    s, sx, sy = W.d22_sigma(X, Y)
    fx, fy = uniform_fft_force(s, sx, sy, h)
    ax, ay = d2_force_xy(X, Y, W.D22_RADIUS, xc=0.0, yc=0.5)
    bx, by = d2_force_xy(X, Y, W.D22_RADIUS, xc=0.0, yc=-0.5)
    ex, ey = fx - ax - bx, fy - ay - by
    got = norms(ex, h * h) + norms(ey, h * h) + norms(radial_error(X, Y, ex, ey), h * h)
    skip = {8} if n == 512 else set()
    for k, (g, p) in enumerate(zip(got, row)):
        if k not in skip:
            assert _sig3(g, p), (n, k, got, row)


# ------------------------------------------------ closed-form convergence --

def test_kuzmin_converges_second_order():
    """Kuzmin disk a = 0.2: F on a [-8,8]^2 grid vs the closed form at |x|,|y| < 1.

    The truncation beyond 8 leaves ~1e-5; the discretisation error must fall at
    second order under refinement (order-1 Taylor terms)."""
    errs = []
    for n_unit in (32, 64):
        n = 8 * n_unit
        h = 16.0 / n
        X, Y = W.cell_centres(n, n, -8.0, -8.0, h)
        s, sx, sy = W.kuzmin_sigma(X, Y, 0.2)
        fx, fy = uniform_fft_force(s, sx, sy, h)
        inner = (np.abs(X) < 1.0) & (np.abs(Y) < 1.0)
        kx, ky = kuzmin_force_xy(X[inner], Y[inner], 0.2)
        errs.append(rel_l2(fx[inner], fy[inner], kx, ky))
    assert errs[0] < 2e-2
    assert math.log2(errs[0] / errs[1]) > 1.8, errs


def test_order0_is_first_order_only():
    """Without the Taylor slopes the same D_2 problem converges at first order."""
    e = []
    for n in (64, 128):
        nx, ny, x0, y0, h = W.unit_grid(n)
        X, Y = W.cell_centres(nx, ny, x0, y0, h)
        s, _, _ = W.d2_sigma(X, Y, 0.5)
        fx, fy = uniform_fft_force(s, None, None, h)
        ex, ey = d2_force_xy(X, Y, 0.5)
        e.append(norms(fx - ex, h * h)[0])
    assert 0.8 < math.log2(e[0] / e[1]) < 1.3


def test_single_cell_far_field_is_point_mass():
    """A uniform cell of mass sigma h^2 seen from far away pulls like a point mass."""
    h, s0 = 0.1, 3.0
    tx, ty = 7.3, -4.1
    fx, fy = direct_force(([-h / 2], [h / 2], [-h / 2], [h / 2]), [s0], None, None, [tx], [ty], G=2.0)
    d3 = (tx * tx + ty * ty) ** 1.5
    m = s0 * h * h
    assert abs(fx[0] / (-2.0 * m * tx / d3) - 1) < 1e-4
    assert abs(fy[0] / (-2.0 * m * ty / d3) - 1) < 1e-4


# ------------------------------------------------------------- quadrature --

def _quad(f, xl, xr, yd, yu):
    from scipy.integrate import dblquad
    val, _ = dblquad(lambda yb, xb: f(xb, yb), xl, xr, yd, yu, epsabs=1e-13, epsrel=1e-12)
    return val


@pytest.mark.parametrize("cell", [
    (0.3, 0.7, 0.2, 0.5),     # near, off-axis
    (-2.0, -1.5, 3.0, 3.5),   # far
    (0.0, 0.4, 0.1, 0.3),     # target on the vertical edge line (u1 = 0), outside the span
    (0.1, 0.5, -0.9, 0.0),    # target on the horizontal edge line (v2 = 0), outside the span
    (-0.6, 0.0, -0.5, -0.2),  # u2 = 0 and both v < 0
])
def test_closed_forms_match_quadrature(cell):
    pytest.importorskip("scipy")
    xl, xr, yd, yu = cell
    x, y = 0.0, 0.0
    xc, yc = (xl + xr) / 2, (yd + yu) / 2
    k = cell_kernels(x, y, xl, xr, yd, yu)

    def r3(xb, yb):
        return ((xb - x) ** 2 + (yb - y) ** 2) ** 1.5

    ref = {
        "x0": _quad(lambda a, b: (a - x) / r3(a, b), *cell),
        "xx": _quad(lambda a, b: (a - xc) * (a - x) / r3(a, b), *cell),
        "xy": _quad(lambda a, b: (b - yc) * (a - x) / r3(a, b), *cell),
        "y0": _quad(lambda a, b: (b - y) / r3(a, b), *cell),
        "yx": _quad(lambda a, b: (a - xc) * (b - y) / r3(a, b), *cell),
        "yy": _quad(lambda a, b: (b - yc) * (b - y) / r3(a, b), *cell),
    }
    for name, v in ref.items():
        assert abs(float(k[name]) - v) <= 1e-9 * max(1.0, abs(v)), (name, float(k[name]), v)


def test_self_cell_values():
    """Target at the centre of its own cell: K^{x,0} = K^{x,y} = 0 by symmetry,
    K^{x,x} = integral of u^2/r^3 over the square = 2 h ln(1 + sqrt 2)."""
    h = 0.37
    k = cell_kernels(0.0, 0.0, -h / 2, h / 2, -h / 2, h / 2)
    assert abs(float(k["x0"])) < 1e-15 and abs(float(k["xy"])) < 1e-15
    assert abs(float(k["xx"]) - 2 * h * math.log(1 + math.sqrt(2))) < 1e-14
    assert abs(float(k["yy"]) - float(k["xx"])) < 1e-15


def test_coincident_line_form_is_the_limit():
    """The paper's sgn(v) ln|v| form on u = 0 equals the limit u -> 0 of the general form."""
    cell = (0.0, 0.25, 0.125, 0.5)
    on = cell_kernels(0.0, 0.0, *cell)
    for eps in (1e-9, -1e-9):
        near = cell_kernels(eps, 0.0, *cell)
        for name in on:
            assert abs(float(on[name]) - float(near[name])) < 1e-7, name


def test_divergent_pairs_raise():
    with pytest.raises(ValueError):
        cell_kernels(0.0, 0.0, 0.0, 0.5, -0.25, 0.25)   # strictly inside an edge span
    with pytest.raises(ValueError):
        cell_kernels(0.0, 0.0, 0.0, 0.5, 0.0, 0.25)     # on a corner


# ---------------------------------------------------------- table symmetry --

def test_table_symmetries():
    t = offset_tables(9, 9, h=1.0)
    flipm = lambda a: a[:, ::-1]
    flipn = lambda a: a[::-1, :]
    assert np.allclose(flipm(t["x0"]), -t["x0"], atol=1e-15)
    assert np.allclose(flipn(t["x0"]), t["x0"], atol=1e-15)
    assert np.allclose(flipm(t["xx"]), t["xx"], atol=1e-15) and np.allclose(flipn(t["xx"]), t["xx"], atol=1e-15)
    assert np.allclose(flipm(t["xy"]), -t["xy"], atol=1e-15) and np.allclose(flipn(t["xy"]), -t["xy"], atol=1e-15)
    assert np.allclose(t["y0"], t["x0"].T, atol=1e-15)
    assert np.allclose(t["yy"], t["xx"].T, atol=1e-15)
    assert np.allclose(t["yx"], t["xy"].T, atol=1e-15)
    assert t["x0"][8, 8] == 0.0


def test_table_scaling_and_asymptotics():
    t1 = offset_tables(41, 41, h=1.0)
    t2 = offset_tables(41, 41, h=0.25)
    assert np.allclose(t1["x0"], t2["x0"], rtol=0, atol=1e-14)
    # the double differences of O(d ln d) corner terms leave ~1e-16 d ln d of
    # absolute rounding in the order-1 tables (d = distance in cells)
    assert np.allclose(0.25 * t1["xx"], t2["xx"], rtol=1e-10, atol=1e-13)
    m, n = 30, 25
    kx0 = t1["x0"][n + 40, m + 40]
    assert abs(kx0 / (m / (m * m + n * n) ** 1.5) - 1) < 1e-3


# --------------------------------------------------------- invariants ------

def test_order0_momentum_cancels():
    """Order 0: K^{x,0} is odd, so sum_t sigma_t F_t dA = 0 to rounding."""
    s, _, _ = W.random_fields(20, 20, seed=11)
    s = np.abs(s)
    h = 0.1
    fx, fy = uniform_direct_force(s, None, None, h)
    px = np.sum(s * fx) * h * h
    py = np.sum(s * fy) * h * h
    scale = np.sum(np.abs(s * fx)) * h * h
    assert abs(px) < 1e-13 * scale and abs(py) < 1e-13 * scale


@pytest.mark.parametrize("shape", [(16, 16), (9, 13)])
def test_fft_route_equals_plain_sum(shape):
    ny, nx = shape
    s, sx, sy = W.random_fields(ny, nx, seed=5)
    h = 0.05
    fx, fy = uniform_fft_force(s, sx, sy, h, G=1.5)
    dx_, dy_ = uniform_direct_force(s, sx, sy, h, G=1.5)
    assert rel_l2(fx, fy, dx_, dy_) < 1e-13


def test_central_slopes_definition():
    s = np.arange(12, dtype=float).reshape(3, 4) ** 2
    dx, dy = central_slopes(s, 0.5)
    assert dx[1, 1] == (s[1, 2] - s[1, 0]) / 1.0
    assert dx[1, 0] == (s[1, 1] - 0.0) / 1.0
    assert dy[2, 3] == (0.0 - s[1, 3]) / 1.0


# ----------------------------------------------------------------- AMR -----

TABLE10_PATCHES = [(0, 4, 4, 0.0, 0.0, 0.25),
                   (1, 2, 2, 0.25, 0.25, 0.125), (1, 2, 2, 0.5, 0.5, 0.125),
                   (2, 2, 2, 0.25, 0.375, 0.0625), (2, 2, 2, 0.375, 0.25, 0.0625)]


def test_table10_hierarchy_leaves():
    """Fig. 1 / Table 10: 32 zones, 28 leaves; leaf centres and levels as printed."""
    rows = _load_table("table10_amr_cells.txt")
    patches = oamr.make_patches(TABLE10_PATCHES)
    masks = oamr.leaf_masks(patches)
    zones = []
    for p, m in zip(patches, masks):
        for j in range(p.ny):
            for i in range(p.nx):
                zones.append((p.x0 + (i + .5) * p.h, p.y0 + (j + .5) * p.h, p.level + 1, int(m[j, i])))
    half_up = lambda v: math.floor(v * 100 + 0.5) / 100
    mine = sorted((half_up(x), half_up(y), L, el) for x, y, L, el in zones)
    printed = sorted((r[1], r[2], int(r[3]), int(r[5])) for r in rows)
    assert len(mine) == 32 and sum(z[3] for z in zones) == 28
    for a, b in zip(mine, printed):
        assert abs(a[0] - b[0]) < 1e-9 and abs(a[1] - b[1]) < 1e-9 and a[2:] == b[2:], (a, b)


def _nested_random(base=16, levels=3, seed=3):
    patches = oamr.make_patches([(lev,) + p for lev, p in enumerate(W.centred_nested_patches(base, levels))])
    sig, sx, sy = [], [], []
    for k, p in enumerate(patches):
        a, b, c = W.random_fields(p.ny, p.nx, seed=seed + k)
        sig.append(a)
        sx.append(b)
        sy.append(c)
    return patches, sig, sx, sy


def test_amr_routes_agree():
    """Flattened leaf-pair sum == per-patch FFT + cross-patch direct (3 levels)."""
    patches, sig, sx, sy = _nested_random()
    leaves, fx, fy = oamr.amr_direct_force(patches, sig, sx, sy)
    gx, gy = oamr.amr_patchfft_plus_direct(patches, sig, sx, sy)
    fxs = oamr.scatter(patches, leaves, fx)
    fys = oamr.scatter(patches, leaves, fy)
    a = np.concatenate([v[np.isfinite(v)] for v in fxs] + [v[np.isfinite(v)] for v in fys])
    b = np.concatenate([v[np.isfinite(v)] for v in gx] + [v[np.isfinite(v)] for v in gy])
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-12


def test_amr_table10_hierarchy_routes_agree():
    patches = oamr.make_patches(TABLE10_PATCHES)
    rng = np.random.Generator(np.random.PCG64(8))
    sig = [rng.uniform(0, 1, (p.ny, p.nx)) for p in patches]
    sx = [rng.uniform(-1, 1, (p.ny, p.nx)) for p in patches]
    sy = [rng.uniform(-1, 1, (p.ny, p.nx)) for p in patches]
    leaves, fx, fy = oamr.amr_direct_force(patches, sig, sx, sy)
    gx, gy = oamr.amr_patchfft_plus_direct(patches, sig, sx, sy)
    fxs = oamr.scatter(patches, leaves, fx)
    for a, b in zip(fxs, gx):
        m = np.isfinite(a)
        assert np.allclose(a[m], b[m], rtol=1e-12, atol=1e-13)


def test_refinement_invariance():
    """Refining a coarse cell into 4 children that carry the parent's linear
    reconstruction (sigma0 + delta . offset, same delta) leaves the force at the
    coarse leaves unchanged: the integrand is identical. This exercises the
    coincident-line form, since coarse centres lie on fine edge lines."""
    n = 16
    nx, ny, x0, y0, h = W.unit_grid(n)
    s, sx, sy = W.random_fields(n, n, seed=21)
    ux, uy = uniform_direct_force(s, sx, sy, h)
    # refine the central 8x8 coarse cells
    fine = (1, 16, 16, -0.5, -0.5, h / 2)
    patches = oamr.make_patches([(0, nx, ny, x0, y0, h), fine])
    fs = np.zeros((16, 16)); fsx = np.zeros((16, 16)); fsy = np.zeros((16, 16))
    for J in range(16):
        for I in range(16):
            pj, pi = 4 + J // 2, 4 + I // 2
            ox = (I % 2 - 0.5) * h / 2
            oy = (J % 2 - 0.5) * h / 2
            fs[J, I] = s[pj, pi] + sx[pj, pi] * ox + sy[pj, pi] * oy
            fsx[J, I] = sx[pj, pi]
            fsy[J, I] = sy[pj, pi]
    leaves, fx, fy = oamr.amr_direct_force(patches, [s, fs], [sx, fsx], [sy, fsy])
    coarse = leaves["patch"] == 0
    j, i = leaves["j"][coarse], leaves["i"][coarse]
    assert rel_l2(fx[coarse], fy[coarse], ux[j, i], uy[j, i]) < 1e-12


# ------------------------------------------- refined hierarchies (Section 4) --

def test_tables8_9_zone_and_leaf_counts():
    """Every zone and leaf count of Tables 8 (ILR) and 9 (VLR), N = 128 ... 2048,
    L = 2, 3, D_2 and D_2,2, from the band refinement rules."""
    rows = _load_table("tables8_9_zone_counts.txt")
    assert len(rows) == 40
    for table, rule, disk, L, n, zones, leaves in rows:
        hier = W.band_hierarchy(int(n), int(L), ("ilr", "vlr")[int(rule)], ("d2", "d22")[int(disk)])
        assert (hier["level"].size, int(hier["leaf"].sum())) == (int(zones), int(leaves)), (table, rule, disk, L, n)


def _children_complete(hier):
    """Every non-leaf zone has exactly its four children on the next level."""
    lev, ix, iy, leaf = hier["level"], hier["ix"], hier["iy"], hier["leaf"]
    keys = set(zip(lev.tolist(), ix.tolist(), iy.tolist()))
    for l, i, j, f in zip(lev.tolist(), ix.tolist(), iy.tolist(), leaf.tolist()):
        kids = [(l + 1, 2 * i + a, 2 * j + b) for a in (0, 1) for b in (0, 1)]
        assert all(k in keys for k in kids) != f
        if l > 0:
            assert (l - 1, i // 2, j // 2) in keys


def test_band_hierarchy_structure():
    for rule in ("ilr", "vlr"):
        for disk in ("d2", "d22"):
            _children_complete(W.band_hierarchy(32, 3, rule, disk))


def _d_sigma(disk, X, Y):
    return W.d2_sigma(X, Y, 0.5) if disk == "d2" else W.d22_sigma(X, Y)


def _d_force(disk, X, Y):
    if disk == "d2":
        return d2_force_xy(X, Y, 0.5)
    ax, ay = d2_force_xy(X, Y, W.D22_RADIUS, yc=0.5)
    bx, by = d2_force_xy(X, Y, W.D22_RADIUS, yc=-0.5)
    return ax + bx, ay + by


def amr_table_norms(hier, disk, fx, fy):
    """Norms of Tables 3-6 at the leaves (finest-area weights) from per-zone forces."""
    xc, yc, h = W.zone_geometry(hier)
    m = hier["leaf"]
    ex, ey = _d_force(disk, xc[m], yc[m])
    ex, ey = fx[m] - ex, fy[m] - ey
    eR = radial_error(xc[m], yc[m], ex, ey)
    if disk == "d2":
        return amr_norms(ex, h[m]) + amr_norms(eR, h[m])
    return amr_norms(ex, h[m]) + amr_norms(ey, h[m]) + amr_norms(eR, h[m])


# Entries of Tables 3-6 pinned: D_2,2 every norm; D_2 the Linf norms only (its
# L1, L2 entries differ from the finest-area norms by inconsistent powers of 2).
# (table, L, N, column) entries that are misprints: exponents (8.72E-04 for
# 8.72E-05, 2.72E-05 for 2.72E-04) and a digit (3.31E-03 for 3.11E-03).
AMR_MISPRINTS = {(4, 3, 128, 0), (6, 2, 128, 2), (5, 3, 256, 2)}


def amr_pinned_columns(table, disk, L, n):
    cols = range(9) if disk == 1 else (2, 5)
    return [c for c in cols if (table, L, n, c) not in AMR_MISPRINTS]


@pytest.mark.parametrize("table, L", [(3, 2), (3, 3), (4, 2), (6, 2)])
def test_tables3_6_amr_errors_reproduced(table, L):
    """Tables 3-6 (Section 4), N = 128: the oracle's leaf sum on the ILR/VLR
    hierarchy with the analytic density and gradient at every leaf centre
    reproduces the printed errors to three digits."""
    rows = {(int(r[0]), int(r[3]), int(r[4])): r for r in _load_table("tables3_6_amr_norms.txt")}
    r = rows[(table, L, 128)]
    rule, disk = ("ilr", "vlr")[int(r[1])], ("d2", "d22")[int(r[2])]
    hier = W.band_hierarchy(128, L, rule, disk)
    xc, yc, _ = W.zone_geometry(hier)
    s, sx, sy = _d_sigma(disk, xc, yc)
    fx, fy = oamr.zone_leaf_force(hier["x0"], hier["y0"], hier["h0"], hier["level"], hier["ix"], hier["iy"],
                                  hier["leaf"], s, sx, sy)
    got = amr_table_norms(hier, disk, fx, fy)
    printed = r[5:]
    for c in amr_pinned_columns(table, int(r[2]), L, 128):
        assert _near3(got[c], printed[c]), (table, L, c, got, printed)


def test_zone_sum_refinement_invariance():
    """Zones split into children that carry the parent's linear reconstruction
    (sigma0 + delta . offset, same delta) leave the force at the unsplit zones
    equal to the uniform-grid sum (same integrand), through two levels."""
    n = 16
    nx, ny, x0, y0, h = W.unit_grid(n)
    s, sx, sy = W.random_fields(n, n, seed=31)
    ux, uy = uniform_direct_force(s, sx, sy, h)
    hier = W.band_hierarchy(n, 3, "ilr", "d2")
    lev, ix, iy = hier["level"], hier["ix"], hier["iy"]
    # each zone's value: the level-0 ancestor's linear function at the zone centre
    anc_i, anc_j = ix >> lev, iy >> lev
    xc, yc, _ = W.zone_geometry(hier)
    pxc = x0 + (anc_i + 0.5) * h
    pyc = y0 + (anc_j + 0.5) * h
    zs = s[anc_j, anc_i] + sx[anc_j, anc_i] * (xc - pxc) + sy[anc_j, anc_i] * (yc - pyc)
    fx, fy = oamr.zone_leaf_force(x0, y0, h, lev, ix, iy, hier["leaf"], zs, sx[anc_j, anc_i], sy[anc_j, anc_i])
    coarse = (lev == 0) & hier["leaf"]
    assert np.count_nonzero(lev > 0) > 0 and np.count_nonzero(coarse) > 0
    assert rel_l2(fx[coarse], fy[coarse], ux[iy[coarse], ix[coarse]], uy[iy[coarse], ix[coarse]]) < 1e-12


def test_zone_sum_equals_patch_sum_table10():
    """The Fig. 1 hierarchy given zone by zone gives the patch-list leaf sum."""
    patches = oamr.make_patches(TABLE10_PATCHES)
    rng = np.random.Generator(np.random.PCG64(8))
    sig = [rng.uniform(0, 1, (p.ny, p.nx)) for p in patches]
    leaves, fx, fy = oamr.amr_direct_force(patches, sig)
    lev, zi, zj, zs, zl = [], [], [], [], []
    masks = oamr.leaf_masks(patches)
    for p, m, sg in zip(patches, masks, sig):
        oi, oj = int(round(p.x0 / p.h)), int(round(p.y0 / p.h))
        for j in range(p.ny):
            for i in range(p.nx):
                lev.append(p.level); zi.append(oi + i); zj.append(oj + j); zs.append(sg[j, i]); zl.append(m[j, i])
    gx, gy = oamr.zone_leaf_force(0.0, 0.0, 0.25, lev, zi, zj, zl, zs)
    zl = np.array(zl)
    assert np.allclose(np.sort(gx[zl]), np.sort(fx), rtol=1e-13, atol=1e-14)
    assert np.allclose(np.sort(gy[zl]), np.sort(fy), rtol=1e-13, atol=1e-14)
