"""Seeded synthetic inputs: surface densities, their analytic slopes, and grids.

This module generates inputs only. It holds none of the force method's
arithmetic (no kernel integrals, transforms or sums) and is shared by the
tests, the oracle comparisons and the benchmark so that both sides of every
comparison see the same arrays.

Conventions: arrays are row-major [y][x]; cell (j, i) of a patch with origin
(x0, y0) and cell width h has centre (x0 + (i + 1/2) h, y0 + (j + 1/2) h).

Disks (Section 3 of Tseng, Shang & Yen for D_2; the others are the workloads
of the benchmark configurations):
* D_2:   sigma0 (1 - R^2/alpha^2)^{3/2} for R < alpha, else 0 (alpha = 0.5 on [-1, 1]^2;
         D_2,2 is two of them of radius 0.4 centred at (0, +-0.5)).
* Kuzmin: a M / (2 pi (R^2 + a^2)^{3/2}).
* two-armed logarithmic spiral: Kuzmin(a) (1 + A cos(2 theta - ln(R) / tan 15deg)).
* exponential: exp(-R / r0).
"""
import math

import numpy as np


# ---------------------------------------------------------------- geometry --

def cell_centres(nx, ny, x0, y0, h):
    """Centre coordinates (X, Y), each [ny, nx], of a uniform patch."""
    x = x0 + (np.arange(nx) + 0.5) * h
    y = y0 + (np.arange(ny) + 0.5) * h
    return np.meshgrid(x, y)


def unit_grid(n):
    """A uniform n-by-n grid on [-1, 1]^2: returns (nx, ny, x0, y0, h)."""
    return (n, n, -1.0, -1.0, 2.0 / n)


def centred_nested_patches(base_n, nlevels, cells_per_level=None):
    """Nested, centred ratio-2 patches: level l covers [-2^-l, 2^-l]^2.

    Level 0 is base_n^2 cells on [-1, 1]^2; every finer level has the same number
    of cells per side (cells_per_level, default base_n), i.e. half the extent at
    half the cell width. Returns a list of (nx, ny, x0, y0, h).
    """
    n = base_n if cells_per_level is None else cells_per_level
    out = []
    for lev in range(nlevels):
        h = (2.0 / base_n) / (2 ** lev)
        nl = base_n if lev == 0 else n
        half = nl * h / 2.0
        out.append((nl, nl, -half, -half, h))
    return out


def covered_mask(patches, level):
    """Boolean [ny, nx] mask of cells of patch `level` covered by patch `level+1`."""
    nx, ny, x0, y0, h = patches[level]
    mask = np.zeros((ny, nx), dtype=bool)
    if level + 1 < len(patches):
        fx, fy, fx0, fy0, fh = patches[level + 1]
        i0 = int(round((fx0 - x0) / h))
        j0 = int(round((fy0 - y0) / h))
        i1 = i0 + int(round(fx * fh / h))
        j1 = j0 + int(round(fy * fh / h))
        mask[j0:j1, i0:i1] = True
    return mask


# ------------------------------------------------------------------ disks --

def d2_sigma(X, Y, alpha, sigma0=1.0, xc=0.0, yc=0.0):
    """D_2 surface density and its analytic gradient (sigma, dsdx, dsdy)."""
    dx = X - xc
    dy = Y - yc
    q = 1.0 - (dx * dx + dy * dy) / (alpha * alpha)
    inside = q > 0.0
    qp = np.where(inside, q, 0.0)
    s = sigma0 * qp ** 1.5
    g = -3.0 * sigma0 * np.sqrt(qp) / (alpha * alpha)
    return s, g * dx, g * dy


D22_RADIUS = 0.4


def d22_sigma(X, Y, alpha=D22_RADIUS, sigma0=1.0):
    """Two D_2 disks centred at (0, 0.5) and (0, -0.5) (Section 3), radius 0.4 each
    (the radius that reproduces Table 2 and the D_2,2 zone counts of Tables 8-9)."""
    a = d2_sigma(X, Y, alpha, sigma0, 0.0, 0.5)
    b = d2_sigma(X, Y, alpha, sigma0, 0.0, -0.5)
    return tuple(p + q for p, q in zip(a, b))


def kuzmin_sigma(X, Y, a, M=1.0):
    """Kuzmin surface density and its analytic gradient."""
    q = X * X + Y * Y + a * a
    s = a * M / (2.0 * math.pi * q ** 1.5)
    g = -3.0 * s / q
    return s, g * X, g * Y


def spiral_sigma(X, Y, a, amp, pitch_deg=15.0, M=1.0):
    """Kuzmin(a) modulated by a two-armed logarithmic spiral, with its gradient.

    The spiral phase is undefined at R = 0; a cell centred there (odd grids)
    gets the unmodulated Kuzmin value and gradient."""
    s, sx, sy = kuzmin_sigma(X, Y, a, M)
    R2 = X * X + Y * Y
    origin = R2 == 0.0
    R2s = np.where(origin, 1.0, R2)
    th = np.arctan2(Y, X)
    k = 1.0 / math.tan(math.radians(pitch_deg))
    ph = 2.0 * th - k * 0.5 * np.log(R2s)
    c = np.where(origin, 0.0, np.cos(ph))
    sn = np.where(origin, 0.0, np.sin(ph))
    # d(ph)/dx = 2 d(theta)/dx - k x / R^2 = (-2 y - k x) / R^2 ; d(ph)/dy = (2 x - k y) / R^2
    dphx = (-2.0 * Y - k * X) / R2s
    dphy = (2.0 * X - k * Y) / R2s
    m = 1.0 + amp * c
    return s * m, sx * m - s * amp * sn * dphx, sy * m - s * amp * sn * dphy


def exponential_sigma(X, Y, r0):
    """exp(-R / r0) and its gradient (the cusp at R = 0 gets gradient 0)."""
    R = np.hypot(X, Y)
    s = np.exp(-R / r0)
    g = np.where(R > 0.0, -s / (r0 * np.where(R > 0.0, R, 1.0)), 0.0)
    return s, g * X, g * Y


# --------------------------------------------------------- configurations --

def kuzmin_64(a=0.2):
    """64^2 grid on [-1,1]^2, Kuzmin a = 0.2, G = M = 1."""
    nx, ny, x0, y0, h = unit_grid(64)
    X, Y = cell_centres(nx, ny, x0, y0, h)
    s, sx, sy = kuzmin_sigma(X, Y, a)
    return dict(geom=(nx, ny, x0, y0, h), sigma=s, dx=sx, dy=sy, X=X, Y=Y)


def spiral_1024(seed=2, n=1024, a=0.1, amp=0.1, noise=1e-3):
    """n^2 grid on [-1,1]^2: Kuzmin(a) x (1 + amp cos(2 theta - ln R / tan 15deg)) + U(-noise, noise).

    The noise is absolute, drawn from numpy's PCG64 with the given seed; the
    analytic gradient returned ignores the noise.
    """
    nx, ny, x0, y0, h = unit_grid(n)
    X, Y = cell_centres(nx, ny, x0, y0, h)
    s, sx, sy = spiral_sigma(X, Y, a, amp)
    rng = np.random.Generator(np.random.PCG64(seed))
    s = s + rng.uniform(-noise, noise, size=s.shape)
    return dict(geom=(nx, ny, x0, y0, h), sigma=s, dx=sx, dy=sy, X=X, Y=Y)


def exponential_hierarchy(base_n=256, nlevels=3, r0=0.1):
    """Centred nested ratio-2 patches of base_n^2 cells each, sigma = exp(-R/r0).

    Covered cells (those refined by the next level) hold sigma = slopes = 0.
    Returns dict(patches=[...], sigma=[...], dx=[...], dy=[...], leaf=[...]).
    """
    patches = centred_nested_patches(base_n, nlevels)
    sig, sxs, sys_, leaf = [], [], [], []
    for lev, (nx, ny, x0, y0, h) in enumerate(patches):
        X, Y = cell_centres(nx, ny, x0, y0, h)
        s, sx, sy = exponential_sigma(X, Y, r0)
        cov = covered_mask(patches, lev)
        for a in (s, sx, sy):
            a[cov] = 0.0
        sig.append(s)
        sxs.append(sx)
        sys_.append(sy)
        leaf.append(~cov)
    return dict(patches=patches, sigma=sig, dx=sxs, dy=sys_, leaf=leaf)


def batch_sizes(count=64, lo=64, hi=512, seed=4):
    """Grid sizes N = round(exp U(ln lo, ln hi)) and disk parameters, seeded."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(int)
    a = rng.uniform(0.05, 0.3, size=count)
    amp = rng.uniform(0.0, 0.2, size=count)
    return ns, a, amp


def bumps_on_patches(patches, seed, nbumps=6):
    """Seeded smooth density: a sum of Gaussian bumps (random centres in
    [-0.6, 0.6]^2, widths in [0.08, 0.3], amplitudes in [0.2, 1]) at the cell
    centres of every patch, with its analytic gradient. Returns lists
    (sigma, dx, dy) of per-patch [ny, nx] arrays."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cx = rng.uniform(-0.6, 0.6, nbumps)
    cy = rng.uniform(-0.6, 0.6, nbumps)
    w = rng.uniform(0.08, 0.3, nbumps)
    a = rng.uniform(0.2, 1.0, nbumps)
    sig, gx, gy = [], [], []
    for p in patches:
        nx, ny, x0, y0, h = p[-5:]
        X, Y = cell_centres(nx, ny, x0, y0, h)
        s = np.zeros_like(X)
        sx = np.zeros_like(X)
        sy = np.zeros_like(X)
        for k in range(nbumps):
            e = a[k] * np.exp(-((X - cx[k]) ** 2 + (Y - cy[k]) ** 2) / (2 * w[k] ** 2))
            s += e
            sx += -e * (X - cx[k]) / w[k] ** 2
            sy += -e * (Y - cy[k]) / w[k] ** 2
        sig.append(s)
        gx.append(sx)
        gy.append(sy)
    return sig, gx, gy


def random_fields(ny, nx, seed, scale=1.0):
    """Seeded uniform random sigma, dx, dy in [-scale, scale] (parity inputs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return tuple(rng.uniform(-scale, scale, size=(ny, nx)) for _ in range(3))


# ------------------------------------------------ refined hierarchies (AMR) --

def d2_edge_distance(X, Y):
    """Distance of (X, Y) from the edge of the D_2 disk (radius 0.5 at the origin)."""
    return np.abs(np.hypot(X, Y) - 0.5)


def d22_edge_distance(X, Y):
    """Distance of (X, Y) from the nearer edge of the two D_2,2 disks."""
    a = np.abs(np.hypot(X, Y - 0.5) - D22_RADIUS)
    b = np.abs(np.hypot(X, Y + 0.5) - D22_RADIUS)
    return np.minimum(a, b)


def refinement_band(rule, n, level):
    """Half-width of the band around a disk edge inside which a zone of `level`
    (0 = the n x n grid on [-1, 1]^2) is split into four (Section 4):

    * "ilr" (independent level refinement): 0.025 / 2^level, a fixed distance
      that halves per level;
    * "vlr" (variable level refinement): 0.1 (128 / n) / 2^level, i.e. 6.4 cells
      of the zone's own level whatever n is.

    These constants reproduce every zone and leaf count of Tables 8 and 9."""
    if rule == "ilr":
        return 0.025 / 2.0 ** level
    if rule == "vlr":
        return 0.1 * (128.0 / n) / 2.0 ** level
    raise ValueError("rule must be 'ilr' or 'vlr'")


def band_hierarchy(n, nlevels, rule, disk="d2"):
    """Quadtree hierarchy of Section 4: an n x n grid on [-1, 1]^2 (level 0)
    whose zones near the disk edge(s) are split into four children, level by
    level, up to nlevels levels (the paper's L; L = 1 is the uniform grid).

    A level-l zone is split when the distance of its centre from the edge is
    below refinement_band(rule, n, l). Zones are listed level by level: level 0
    row-major, then the four children of every split zone of the previous
    level in that level's order, each as (SW, SE, NW, NE).

    Returns dict(n, x0, y0, h0, level, ix, iy, leaf): int32 arrays level, ix, iy
    (zone (ix, iy) of level l spans [x0 + ix h_l, x0 + (ix + 1) h_l] with
    h_l = h0 / 2^l, likewise in y) and a boolean leaf flag per zone.
    """
    dist = {"d2": d2_edge_distance, "d22": d22_edge_distance}[disk]
    h0 = 2.0 / n
    x0 = y0 = -1.0
    J, I = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ix, iy = I.ravel().astype(np.int64), J.ravel().astype(np.int64)
    levels, xs, ys, leaves = [], [], [], []
    for lev in range(nlevels):
        h = h0 / 2.0 ** lev
        split = np.zeros(ix.size, dtype=bool)
        if lev + 1 < nlevels:
            split = dist(x0 + (ix + 0.5) * h, y0 + (iy + 0.5) * h) < refinement_band(rule, n, lev)
        levels.append(np.full(ix.size, lev))
        xs.append(ix)
        ys.append(iy)
        leaves.append(~split)
        pi, pj = ix[split], iy[split]
        ix = np.stack([2 * pi, 2 * pi + 1, 2 * pi, 2 * pi + 1], axis=1).ravel()
        iy = np.stack([2 * pj, 2 * pj, 2 * pj + 1, 2 * pj + 1], axis=1).ravel()
        if ix.size == 0:
            break
    return dict(n=n, x0=x0, y0=y0, h0=h0,
                level=np.concatenate(levels).astype(np.int32), ix=np.concatenate(xs).astype(np.int32),
                iy=np.concatenate(ys).astype(np.int32), leaf=np.concatenate(leaves))


def zone_geometry(hier):
    """Centres and widths (xc, yc, h) of every zone of a band_hierarchy dict."""
    h = hier["h0"] / 2.0 ** hier["level"]
    return hier["x0"] + (hier["ix"] + 0.5) * h, hier["y0"] + (hier["iy"] + 0.5) * h, h
