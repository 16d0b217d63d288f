"""AMR hierarchies of rectangular patches and the flattened leaf-pair force (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 3 of Tseng, Shang & Yen refines each parent zone into four children
(ratio 2, Fig. 1) and evaluates the force at the centres of leaf zones only,
summing over all leaf zones as sources (Eq. eqnXforce2). Here a hierarchy is a
list of patches (level, nx, ny, x0, y0, h): uniform blocks of square cells.
A cell is a leaf when no patch of the next level covers it. The force at every
leaf centre is the plain sum over every leaf cell, evaluated by the C oracle.
"""
import numpy as np

from .direct import direct_force
from .fftconv import uniform_fft_force


class Patch:
    def __init__(self, level, nx, ny, x0, y0, h):
        self.level, self.nx, self.ny = int(level), int(nx), int(ny)
        self.x0, self.y0, self.h = float(x0), float(y0), float(h)

    @property
    def x1(self):
        return self.x0 + self.nx * self.h

    @property
    def y1(self):
        return self.y0 + self.ny * self.h


def make_patches(spec):
    """spec: iterable of (level, nx, ny, x0, y0, h) tuples."""
    return [Patch(*p) for p in spec]


def leaf_masks(patches):
    """Per patch, a boolean [ny, nx] mask: True where the cell is a leaf."""
    masks = []
    for p in patches:
        m = np.ones((p.ny, p.nx), dtype=bool)
        xc = p.x0 + (np.arange(p.nx) + 0.5) * p.h
        yc = p.y0 + (np.arange(p.ny) + 0.5) * p.h
        X, Y = np.meshgrid(xc, yc)
        for c in patches:
            if c.level == p.level + 1:
                m &= ~((X > c.x0) & (X < c.x1) & (Y > c.y0) & (Y < c.y1))
        masks.append(m)
    return masks


def leaf_cells(patches, masks=None):
    """Flattened leaf list: dict of arrays (patch, j, i, xl, xr, yd, yu, xc, yc)."""
    masks = leaf_masks(patches) if masks is None else masks
    cols = {k: [] for k in ("patch", "j", "i", "xl", "xr", "yd", "yu", "xc", "yc")}
    for k, (p, m) in enumerate(zip(patches, masks)):
        J, I = np.nonzero(m)
        xl = p.x0 + I * p.h
        yd = p.y0 + J * p.h
        cols["patch"].append(np.full(J.size, k))
        cols["j"].append(J)
        cols["i"].append(I)
        cols["xl"].append(xl)
        cols["xr"].append(xl + p.h)
        cols["yd"].append(yd)
        cols["yu"].append(yd + p.h)
        cols["xc"].append(p.x0 + (I + 0.5) * p.h)
        cols["yc"].append(p.y0 + (J + 0.5) * p.h)
    return {k: np.concatenate(v) for k, v in cols.items()}


def _gather(fields, leaves):
    return np.array([fields[k][j, i] for k, j, i in zip(leaves["patch"], leaves["j"], leaves["i"])],
                    dtype=np.float64) if fields is not None else None


def amr_direct_force(patches, sigma, dx=None, dy=None, G=1.0, target_index=None, nthreads=0):
    """Force at leaf centres from all leaf cells (the plain leaf-pair sum).

    sigma, dx, dy: lists of per-patch [ny, nx] arrays (values at covered cells
    are ignored). target_index: optional integer array selecting targets from
    the flattened leaf list (default: all leaves).
    Returns (leaves, fx, fy): the flattened leaf list and the forces at the
    selected targets.
    """
    leaves = leaf_cells(patches)
    s0 = _gather(sigma, leaves)
    sx = _gather(dx, leaves)
    sy = _gather(dy, leaves)
    tsel = np.arange(leaves["xc"].size) if target_index is None else np.asarray(target_index)
    fx, fy = direct_force((leaves["xl"], leaves["xr"], leaves["yd"], leaves["yu"]), s0, sx, sy,
                          leaves["xc"][tsel], leaves["yc"][tsel], G=G, nthreads=nthreads)
    return leaves, fx, fy


def scatter(patches, leaves, values, fill=np.nan):
    """Per-patch dense arrays holding `values` at leaf cells and `fill` elsewhere."""
    out = [np.full((p.ny, p.nx), fill, dtype=np.float64) for p in patches]
    for k, j, i, v in zip(leaves["patch"], leaves["j"], leaves["i"], values):
        out[k][j, i] = v
    return out


def amr_patchfft_plus_direct(patches, sigma, dx=None, dy=None, G=1.0):
    """Second route: same-patch pairs by FFT convolution, all other pairs directly.

    Each patch's own leaves act on its own leaves through the uniform FFT route
    with covered cells set to zero; every pair of cells in different patches is
    summed directly. Returns per-patch dense (fx, fy) lists, NaN at covered cells.
    """
    masks = leaf_masks(patches)
    leaves = leaf_cells(patches, masks)
    fx_out, fy_out = [], []
    for k, (p, m) in enumerate(zip(patches, masks)):
        s = np.where(m, sigma[k], 0.0)
        sx = None if dx is None else np.where(m, dx[k], 0.0)
        sy = None if dy is None else np.where(m, dy[k], 0.0)
        fx, fy = uniform_fft_force(s, sx, sy, p.h, G=G)
        other = leaves["patch"] != k
        sel = leaves["patch"] == k
        if np.any(other):
            cells = (leaves["xl"][other], leaves["xr"][other], leaves["yd"][other], leaves["yu"][other])
            o = np.nonzero(other)[0]
            s0 = np.array([sigma[a][b, c] for a, b, c in zip(leaves["patch"][o], leaves["j"][o], leaves["i"][o])])
            ox = None if dx is None else np.array([dx[a][b, c] for a, b, c in zip(leaves["patch"][o], leaves["j"][o], leaves["i"][o])])
            oy = None if dy is None else np.array([dy[a][b, c] for a, b, c in zip(leaves["patch"][o], leaves["j"][o], leaves["i"][o])])
            cx, cy = direct_force(cells, s0, ox, oy, leaves["xc"][sel], leaves["yc"][sel], G=G)
            fx[leaves["j"][sel], leaves["i"][sel]] += cx
            fy[leaves["j"][sel], leaves["i"][sel]] += cy
        fx_out.append(np.where(m, fx, np.nan))
        fy_out.append(np.where(m, fy, np.nan))
    return fx_out, fy_out


# ------------------------------------------------ zone-by-zone hierarchies --
#
# A quadtree hierarchy given zone by zone (Fig. 1, Table 10): level l, column
# ix and row iy on the level-l grid of cell width h_l = h0 / 2^l, and a leaf
# flag. Only leaf zones carry density and receive the force (Section 2: the
# sum of Eq. eqnXforce2 runs over the leaf zones).

def zone_bounds(x0, y0, h0, level, ix, iy):
    """Edges (xl, xr, yd, yu) and centres (xc, yc) of zones (level, ix, iy)."""
    h = h0 / 2.0 ** np.asarray(level, np.float64)
    xl = x0 + np.asarray(ix, np.float64) * h
    yd = y0 + np.asarray(iy, np.float64) * h
    return xl, xl + h, yd, yd + h, xl + 0.5 * h, yd + 0.5 * h


def zone_leaf_force(x0, y0, h0, level, ix, iy, leaf, sigma, dx=None, dy=None, G=1.0, targets=None, nthreads=0):
    """Force at leaf centres from every leaf zone (plain sum, C oracle).

    sigma, dx, dy: per-zone arrays (values at non-leaf zones are ignored).
    targets: optional zone indices (leaf zones) to evaluate; default all leaves.
    Returns (fx, fy): per zone (0 at non-leaf zones), or per entry of targets.
    """
    leaf = np.asarray(leaf, bool)
    xl, xr, yd, yu, xc, yc = zone_bounds(x0, y0, h0, level, ix, iy)
    pick = lambda a: None if a is None else np.asarray(a, np.float64)[leaf]
    tsel = np.nonzero(leaf)[0] if targets is None else np.asarray(targets)
    fx, fy = direct_force((xl[leaf], xr[leaf], yd[leaf], yu[leaf]), pick(sigma), pick(dx), pick(dy), xc[tsel],
                          yc[tsel], G=G, nthreads=nthreads)
    if targets is not None:
        return fx, fy
    ox = np.zeros(leaf.size)
    oy = np.zeros(leaf.size)
    ox[leaf] = fx
    oy[leaf] = fy
    return ox, oy
