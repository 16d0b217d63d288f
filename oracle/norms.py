"""Error norms of Section 3 (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

    |e|_1 = sum_i |e_i| dA_i,   |e|_2 = (sum_i e_i^2 dA_i)^{1/2},   |e|_inf = max_i |e_i|

over all cells i of the domain, dA_i the cell area. The radial error is
e_R = (x e_x + y e_y) / R. The order of accuracy between successive sizes is
log2(L(N_k) / L(N_{k+1})).
"""
import numpy as np


def norms(e, dA):
    e = np.asarray(e, dtype=np.float64).ravel()
    dA = np.broadcast_to(np.asarray(dA, dtype=np.float64), e.shape).ravel() if np.ndim(dA) else np.full(e.shape, float(dA))
    return (float(np.sum(np.abs(e) * dA)), float(np.sqrt(np.sum(e * e * dA))), float(np.max(np.abs(e))))


def radial_error(x, y, ex, ey):
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    R = np.hypot(x, y)
    return (x * ex + y * ey) / R


def order(l_coarse, l_fine):
    return float(np.log2(l_coarse / l_fine))


def rel_l2(fx, fy, rx, ry):
    """Relative L2 error over both components: ||F - F_ref|| / ||F_ref||."""
    num = np.sum((np.asarray(fx, np.float64) - rx) ** 2) + np.sum((np.asarray(fy, np.float64) - ry) ** 2)
    den = np.sum(np.asarray(rx, np.float64) ** 2) + np.sum(np.asarray(ry, np.float64) ** 2)
    return float(np.sqrt(num / den))


def amr_norms(e, h_leaf):
    """Norms over the leaf zones of a refined hierarchy, every leaf weighted by
    the area of the finest zone, min(h)^2 (the weighting with which the L1, L2
    norms of Tables 4 and 6 come out; the text's 'area of sub-region D_i' does
    not reproduce them)."""
    h = float(np.min(np.asarray(h_leaf, np.float64)))
    return norms(e, h * h)
