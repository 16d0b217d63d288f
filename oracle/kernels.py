"""Closed-form cell integrals of the thin-disk force kernel at z = 0 (FP64, numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Source: Section 2 of Tseng, Shang & Yen, the list of antiderivatives for
K^{x,0}, K^{x,x}, K^{x,y}, K^{y,0}, K^{y,x}, K^{y,y} (evaluated at z = 0), and
the coincident-line modification that follows it.

Notation: the target is (x, y); the source cell is [xl, xr] x [yd, yu] with
centre (xc, yc); u = xbar - x, v = ybar - y, r = sqrt(u^2 + v^2); and
"dd f" is the double difference f(u2, v2) - f(u1, v2) - f(u2, v1) + f(u1, v1)
over the cell corners (u1 = xl - x, u2 = xr - x, v1 = yd - y, v2 = yu - y).

    K^{x,0} = -dd ln(v + r)
    K^{x,x} = (x - xc) K^{x,0} + dd [v ln(u + r)]
    K^{x,y} = (y - yc) K^{x,0} - dd r
    K^{y,0} = -dd ln(u + r)
    K^{y,x} = (x - xc) K^{y,0} - dd r
    K^{y,y} = (y - yc) K^{y,0} + dd [u ln(v + r)]

Readings (the paper's printed arctan terms vanish at z = 0):

* ln(v + r) for v < 0 is evaluated as 2 ln|u| - ln(r - v), an algebraic
  identity ((v + r)(r - v) = u^2) that avoids cancellation; it changes no value.
* Where u == 0 (the target lies on the line of a vertical source edge) the
  paper replaces ln(v + r) by sgn(v) ln|v|; the same replacement with the roles
  of u and v swapped is used for ln(u + r) where v == 0 (the y-family).
* v ln(u + r) and u ln(v + r) are 0 where their prefactor is 0 (their limit).
* A target on a source corner, or strictly inside a source edge span, makes
  the integral log-divergent; such pairs raise ValueError.

With these K the force is attractive:
    F_x = G sum_i [sigma0_i K^{x,0}_i + deltax_i K^{x,x}_i + deltay_i K^{x,y}_i]
    F_y = G sum_i [sigma0_i K^{y,0}_i + deltax_i K^{y,x}_i + deltay_i K^{y,y}_i]
(the paper writes the sum with a leading minus sign; with K defined as the
integral of (xbar - x)/r^3 that sign would make gravity repulsive, so the
attractive sign is taken, which is the one that matches the D_2 closed form).
"""
import numpy as np


def ln_s_plus_r(t, s):
    """ln(s + sqrt(t^2 + s^2)) with the paper's coincident-line form at t == 0.

    For t == 0 the value is sgn(s) ln|s| (the modification in Section 2).
    Raises ValueError where t == 0 and s == 0.
    """
    t = np.asarray(t, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    t, s = np.broadcast_arrays(t, s)
    if np.any((t == 0.0) & (s == 0.0)):
        raise ValueError("target on a source-cell corner: the kernel integral diverges")
    out = np.empty(t.shape, dtype=np.float64)
    on_line = t == 0.0
    pos = (~on_line) & (s >= 0.0)
    neg = (~on_line) & (s < 0.0)
    r = np.sqrt(t * t + s * s)
    out[pos] = np.log(s[pos] + r[pos])
    out[neg] = 2.0 * np.log(np.abs(t[neg])) - np.log(r[neg] - s[neg])
    out[on_line] = np.sign(s[on_line]) * np.log(np.abs(s[on_line]))
    return out


def _dd(f, u1, u2, v1, v2):
    return f(u2, v2) - f(u1, v2) - f(u2, v1) + f(u1, v1)


def _check_edges(u1, u2, v1, v2):
    """Reject targets strictly inside the span of a source edge line."""
    on_v_edge = ((u1 == 0.0) | (u2 == 0.0)) & (v1 < 0.0) & (v2 > 0.0)
    on_h_edge = ((v1 == 0.0) | (v2 == 0.0)) & (u1 < 0.0) & (u2 > 0.0)
    if np.any(on_v_edge | on_h_edge):
        raise ValueError("target strictly inside a source edge span: the kernel integral diverges")


def _v_ln_u_plus_r(u, v):
    u, v = np.broadcast_arrays(np.asarray(u, np.float64), np.asarray(v, np.float64))
    out = np.zeros(u.shape, dtype=np.float64)
    nz = v != 0.0
    out[nz] = v[nz] * ln_s_plus_r(v[nz], u[nz])
    return out


def _u_ln_v_plus_r(u, v):
    u, v = np.broadcast_arrays(np.asarray(u, np.float64), np.asarray(v, np.float64))
    out = np.zeros(u.shape, dtype=np.float64)
    nz = u != 0.0
    out[nz] = u[nz] * ln_s_plus_r(u[nz], v[nz])
    return out


def _r(u, v):
    return np.sqrt(np.asarray(u, np.float64) ** 2 + np.asarray(v, np.float64) ** 2)


def cell_kernels(x, y, xl, xr, yd, yu):
    """All six cell integrals for targets (x, y) and source cells [xl,xr]x[yd,yu].

    Arguments broadcast against each other. Returns a dict with keys
    'x0', 'xx', 'xy', 'y0', 'yx', 'yy' (K^{x,0}, K^{x,x}, ... of Section 2).
    """
    x, y, xl, xr, yd, yu = np.broadcast_arrays(*[np.asarray(a, np.float64) for a in (x, y, xl, xr, yd, yu)])
    u1, u2, v1, v2 = xl - x, xr - x, yd - y, yu - y
    _check_edges(u1, u2, v1, v2)
    xc = 0.5 * (xl + xr)
    yc = 0.5 * (yd + yu)
    kx0 = -_dd(lambda u, v: ln_s_plus_r(u, v), u1, u2, v1, v2)
    ky0 = -_dd(lambda u, v: ln_s_plus_r(v, u), u1, u2, v1, v2)
    ddr = _dd(_r, u1, u2, v1, v2)
    return {
        "x0": kx0,
        "xx": (x - xc) * kx0 + _dd(_v_ln_u_plus_r, u1, u2, v1, v2),
        "xy": (y - yc) * kx0 - ddr,
        "y0": ky0,
        "yx": (x - xc) * ky0 - ddr,
        "yy": (y - yc) * ky0 + _dd(_u_ln_v_plus_r, u1, u2, v1, v2),
    }


def offset_tables(mx, my, h=1.0):
    """Kernel tables of a uniform grid with square cells of width h.

    Entry [n + my - 1, m + mx - 1] holds the integrals for a source cell whose
    centre is offset by (m h, n h) from the target centre, for
    m in [-(mx-1), mx-1] and n in [-(my-1), my-1]. Returns the dict of
    ``cell_kernels``. K^{x,0} and K^{y,0} do not depend on h; the other four
    scale linearly with h.
    """
    m = np.arange(-(mx - 1), mx, dtype=np.float64)
    n = np.arange(-(my - 1), my, dtype=np.float64)
    M, Nn = np.meshgrid(m, n)
    return cell_kernels(0.0, 0.0, (M - 0.5) * h, (M + 0.5) * h, (Nn - 0.5) * h, (Nn + 0.5) * h)


# ----------------------------------------------------------- off the plane --
#
# Targets at height z != 0 above the disk plane (Section 2, the antiderivative
# list with the arctan terms; the printed "sgn(x) x y" is read as u v, and the
# z-family as below). With r = sqrt(u^2 + v^2 + z^2):
#   K^{x,0} = -dd ln(v + r)
#   K^{x,x} = (x - xc) K^{x,0} + dd[v ln(u + r) - |z| atan(u v / (|z| r))]
#   K^{x,y} = (y - yc) K^{x,0} - dd r
#   (y-family with u <-> v)
#   K^{z,0} = integral of (zbar - z) / r^3 over the cell = -dd atan(u v / (z r))
#   K^{z,x} = (x - xc) K^{z,0} - z K^{x,0}
#   K^{z,y} = (y - yc) K^{z,0} - z K^{y,0}
# so that F_z = G sum_i [sigma0_i K^{z,0}_i + deltax_i K^{z,x}_i + deltay_i K^{z,y}_i]
# (attractive: towards the plane). The paper's z-family differs from these by
# the overall sign convention discussed for the in-plane force.

def _ln_s_plus_rz(t, s, z):
    """ln(s + sqrt(t^2 + s^2 + z^2)) for z != 0 (never singular)."""
    t, s = np.broadcast_arrays(np.asarray(t, np.float64), np.asarray(s, np.float64))
    r = np.sqrt(t * t + s * s + z * z)
    out = np.empty(t.shape, dtype=np.float64)
    pos = s >= 0.0
    out[pos] = np.log(s[pos] + r[pos])
    neg = ~pos
    out[neg] = np.log(t[neg] ** 2 + z * z) - np.log(r[neg] - s[neg])
    return out


def cell_kernels_z(x, y, z, xl, xr, yd, yu):
    """All nine cell integrals at height z != 0: keys x0 xx xy y0 yx yy z0 zx zy."""
    if z == 0.0:
        raise ValueError("cell_kernels_z needs z != 0 (use cell_kernels in the plane)")
    x, y, xl, xr, yd, yu = np.broadcast_arrays(*[np.asarray(a, np.float64) for a in (x, y, xl, xr, yd, yu)])
    u1, u2, v1, v2 = xl - x, xr - x, yd - y, yu - y
    xc = 0.5 * (xl + xr)
    yc = 0.5 * (yd + yu)
    az = abs(z)
    rr = lambda u, v: np.sqrt(u * u + v * v + z * z)
    kx0 = -_dd(lambda u, v: _ln_s_plus_rz(u, v, z), u1, u2, v1, v2)
    ky0 = -_dd(lambda u, v: _ln_s_plus_rz(v, u, z), u1, u2, v1, v2)
    solid = _dd(lambda u, v: np.arctan(u * v / (az * rr(u, v))), u1, u2, v1, v2)
    ddr = _dd(rr, u1, u2, v1, v2)
    kz0 = -np.sign(z) * solid
    return {
        "x0": kx0,
        "xx": (x - xc) * kx0 + _dd(lambda u, v: v * _ln_s_plus_rz(v, u, z), u1, u2, v1, v2) - az * solid,
        "xy": (y - yc) * kx0 - ddr,
        "y0": ky0,
        "yx": (x - xc) * ky0 - ddr,
        "yy": (y - yc) * ky0 + _dd(lambda u, v: u * _ln_s_plus_rz(u, v, z), u1, u2, v1, v2) - az * solid,
        "z0": kz0,
        "zx": (x - xc) * kz0 - z * kx0,
        "zy": (y - yc) * kz0 - z * ky0,
    }


def offset_tables_z(mx, my, h, z):
    """Nine kernel tables of a uniform grid at height z (layout of offset_tables)."""
    m = np.arange(-(mx - 1), mx, dtype=np.float64)
    n = np.arange(-(my - 1), my, dtype=np.float64)
    M, Nn = np.meshgrid(m, n)
    return cell_kernels_z(0.0, 0.0, z, (M - 0.5) * h, (M + 0.5) * h, (Nn - 0.5) * h, (Nn + 0.5) * h)
