"""Neighbour-leaf slopes of AMR hierarchies (FP64, plain Python loops).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 2 reconstructs every leaf's density linearly, sigma0 + deltax (x - xc)
+ deltay (y - yc) (Eq. eqnGamma), but does not say how the slopes are obtained
when only sigma0 is known. The reading used here, for a leaf t of width h and
each axis (x shown; y likewise):

    deltax_t = (v_R - v_L) / (x_R - x_L)

where (x_L, v_L) and (x_R, v_R) describe what lies across t's left and right
sides, found at the midpoint of the side:
  * a leaf of t's level: its sigma0 at its centre;
  * a refined cell of t's level: the mean of the two children that touch the
    side (their own value, or for refined children the mean of theirs, and so
    on down), at the mean of their centres (3h/4 from t's centre);
  * a coarser leaf c (no cell of t's level there): c's linear reconstruction
    at the point of c's centre line level with t, sigma0_c + deltay_c (y_t -
    y_c), at x_c (its slopes are those of this rule: levels are done from the
    coarsest up, and a leaf's slopes never depend on a finer leaf's slopes);
  * nothing (outside the level-0 grid): 0, at one cell width h from t.
On a single uniform grid this is the central difference with zero outside the
grid; on any hierarchy it reproduces a linear density exactly at every leaf
whose sides all have a neighbour.
"""
import numpy as np


def _centre(x0, y0, h0, l, i, j):
    h = h0 / 2.0 ** l
    return x0 + (i + 0.5) * h, y0 + (j + 0.5) * h


def zone_filled_values(level, ix, iy, leaf, sigma):
    """sigma0 at every zone: the leaf's own value, or for a refined zone the
    mean of its four children's values (finest first). Returns a dict
    (l, i, j) -> value."""
    val = {}
    order = np.argsort(-np.asarray(level), kind="stable")
    zones = {(int(level[k]), int(ix[k]), int(iy[k])): k for k in range(len(level))}
    for k in order:
        l, i, j = int(level[k]), int(ix[k]), int(iy[k])
        if leaf[k]:
            val[(l, i, j)] = float(sigma[k])
        else:
            kids = [(l + 1, 2 * i + a, 2 * j + b) for b in (0, 1) for a in (0, 1)]
            assert all(c in zones for c in kids), "a refined zone must have four children"
            val[(l, i, j)] = sum(val[c] for c in kids) / 4.0
    return val


def zone_neighbour_slopes(x0, y0, h0, level, ix, iy, leaf, sigma):
    """Slopes (dx, dy) of every leaf zone of a zone list by the rule above
    (0 at non-leaf zones). level, ix, iy: zone coordinates on the level grids;
    leaf: leaf flags; sigma: sigma0 per zone (read at leaf zones)."""
    level = np.asarray(level)
    leaf = np.asarray(leaf, bool)
    zones = {(int(level[k]), int(ix[k]), int(iy[k])): k for k in range(len(level))}
    val = zone_filled_values(level, ix, iy, leaf, sigma)
    dx = np.zeros(len(level))
    dy = np.zeros(len(level))

    def across(l, i, j, axis, side):
        """(position along the axis, value) of what lies across one side of zone (l, i, j)."""
        h = h0 / 2.0 ** l
        xc, yc = _centre(x0, y0, h0, l, i, j)
        tc = xc if axis == 0 else yc
        di, dj = (side, 0) if axis == 0 else (0, side)
        n = (l, i + di, j + dj)
        if n in zones:
            if leaf[zones[n]]:
                return tc + side * h, val[n]
            # the two children of the neighbour that touch the side
            if axis == 0:
                kids = [(l + 1, 2 * n[1] + (0 if side > 0 else 1), 2 * n[2] + b) for b in (0, 1)]
            else:
                kids = [(l + 1, 2 * n[1] + a, 2 * n[2] + (0 if side > 0 else 1)) for a in (0, 1)]
            return tc + side * 0.75 * h, 0.5 * (val[kids[0]] + val[kids[1]])
        # a coarser leaf containing the point just across the side's midpoint
        px, py = (xc + side * 0.75 * h, yc) if axis == 0 else (xc, yc + side * 0.75 * h)
        for m in range(l - 1, -1, -1):
            hm = h0 / 2.0 ** m
            c = (m, int(np.floor((px - x0) / hm)), int(np.floor((py - y0) / hm)))
            if c in zones:
                k = zones[c]
                assert leaf[k], "the first listed zone across a side is a leaf"
                cx, cy = _centre(x0, y0, h0, *c)
                if axis == 0:
                    return cx, val[c] + dy[k] * (yc - cy)
                return cy, val[c] + dx[k] * (xc - cx)
        return tc + side * h, 0.0

    for l in sorted(set(int(v) for v in level)):
        for k in np.nonzero(leaf & (level == l))[0]:
            i, j = int(ix[k]), int(iy[k])
            for axis, out in ((0, dx), (1, dy)):
                pl, vl = across(l, i, j, axis, -1)
                pr, vr = across(l, i, j, axis, +1)
                out[k] = (vr - vl) / (pr - pl)
    return dx, dy


def patches_as_zones(patches):
    """Zone coordinates of every cell of a patch hierarchy (patches as in
    oracle.amr), in field-array order: (x0, y0, h0, level, ix, iy, leaf)."""
    from .amr import leaf_masks
    lev0 = [p for p in patches if p.level == 0]
    x0 = min(p.x0 for p in lev0)
    y0 = min(p.y0 for p in lev0)
    h0 = lev0[0].h
    L, I, J, F = [], [], [], []
    for p, m in zip(patches, leaf_masks(patches)):
        h = h0 / 2.0 ** p.level
        gi = int(round((p.x0 - x0) / h))
        gj = int(round((p.y0 - y0) / h))
        jj, ii = np.mgrid[0:p.ny, 0:p.nx]
        L.append(np.full(p.nx * p.ny, p.level))
        I.append((gi + ii).ravel())
        J.append((gj + jj).ravel())
        F.append(m.ravel())
    return x0, y0, h0, np.concatenate(L), np.concatenate(I), np.concatenate(J), np.concatenate(F)


def patch_neighbour_slopes(patches, sigma):
    """The rule above on a patch hierarchy: sigma is a list of per-patch
    [ny, nx] arrays; returns per-patch (dx, dy) lists (0 at covered cells)."""
    x0, y0, h0, level, ix, iy, leaf = patches_as_zones(patches)
    s = np.concatenate([np.asarray(a, np.float64).ravel() for a in sigma])
    dx, dy = zone_neighbour_slopes(x0, y0, h0, level, ix, iy, leaf, s)
    out_x, out_y, o = [], [], 0
    for p in patches:
        n = p.nx * p.ny
        out_x.append(dx[o:o + n].reshape(p.ny, p.nx))
        out_y.append(dy[o:o + n].reshape(p.ny, p.nx))
        o += n
    return out_x, out_y
