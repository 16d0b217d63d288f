"""Mid-plane potential of the thin disk (FP64, numpy and the plain C sum).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 2 gives the mid-plane potential as the singular kernel integral
    Phi(x, y, 0) = -G integral K(xbar - x, ybar - y, 0) sigma(xbar, ybar) dxbar dybar,  K = 1/r.
With the order-1 reconstruction of Eq. eqnGamma on cell i,
    Phi(t) = -G sum_i [sigma0_i P^0_i(t) + deltax_i P^x_i(t) + deltay_i P^y_i(t)],
    P^0 = integral of 1/r,  P^x = integral of (xbar - xc)/r,  P^y = integral of (ybar - yc)/r
over the cell, u = xbar - x, v = ybar - y, r = sqrt(u^2 + v^2). Antiderivatives
(d^2/du dv of each equals the integrand):
    1/r  :  u ln(v + r) + v ln(u + r)
    u/r  :  (v r + u^2 ln(v + r)) / 2
    v/r  :  (u r + v^2 ln(u + r)) / 2
and P^x = dd[u/r antiderivative] + (x - xc) P^0, P^y likewise, dd the double
difference over the cell corners. Every term carries a factor that vanishes
where its logarithm is singular (u ln(v + r) at u = 0, u^2 ln(v + r) at u = 0),
so the integrals are finite everywhere, the target's own cell included; those
terms are 0 there (their limits). ln(v + r) for v < 0 uses 2 ln|u| - ln(r - v).
The force is minus the gradient of this potential. On an AMR hierarchy the
sum runs over every leaf cell (Eq. eqnXforce2 with K = 1/r), evaluated at leaf
centres.
"""
import numpy as np

from .direct import _load, _ptr
from .kernels import _dd


def _ln_v_plus_r(u, v):
    """ln(v + sqrt(u^2 + v^2)) for u != 0 (cancellation-free for v < 0)."""
    r = np.sqrt(u * u + v * v)
    return np.where(v >= 0.0, np.log(np.where(v >= 0.0, v + r, 1.0)),
                    2.0 * np.log(np.abs(np.where(u != 0.0, u, 1.0))) - np.log(np.where(v < 0.0, r - v, 1.0)))


def _f_one(u, v):
    """u ln(v + r) + v ln(u + r), with each term 0 where its prefactor is 0."""
    u, v = np.broadcast_arrays(np.asarray(u, np.float64), np.asarray(v, np.float64))
    a = np.where(u != 0.0, u * _ln_v_plus_r(np.where(u != 0.0, u, 1.0), v), 0.0)
    b = np.where(v != 0.0, v * _ln_v_plus_r(np.where(v != 0.0, v, 1.0), u), 0.0)
    return a + b


def _f_u(u, v):
    """(v r + u^2 ln(v + r)) / 2."""
    u, v = np.broadcast_arrays(np.asarray(u, np.float64), np.asarray(v, np.float64))
    r = np.sqrt(u * u + v * v)
    a = np.where(u != 0.0, u * u * _ln_v_plus_r(np.where(u != 0.0, u, 1.0), v), 0.0)
    return 0.5 * (v * r + a)


def _f_v(u, v):
    return _f_u(v, u)


def cell_potentials(x, y, xl, xr, yd, yu):
    """P^0, P^x, P^y for targets (x, y) and cells [xl, xr] x [yd, yu] (broadcast)."""
    x, y, xl, xr, yd, yu = np.broadcast_arrays(*[np.asarray(a, np.float64) for a in (x, y, xl, xr, yd, yu)])
    u1, u2, v1, v2 = xl - x, xr - x, yd - y, yu - y
    p0 = _dd(_f_one, u1, u2, v1, v2)
    xc = 0.5 * (xl + xr)
    yc = 0.5 * (yd + yu)
    return {"p0": p0, "px": _dd(_f_u, u1, u2, v1, v2) + (x - xc) * p0,
            "py": _dd(_f_v, u1, u2, v1, v2) + (y - yc) * p0}


def offset_potentials(mx, my, h=1.0):
    """Potential tables of a uniform grid (layout of kernels.offset_tables)."""
    m = np.arange(-(mx - 1), mx, dtype=np.float64)
    n = np.arange(-(my - 1), my, dtype=np.float64)
    M, Nn = np.meshgrid(m, n)
    return cell_potentials(0.0, 0.0, (M - 0.5) * h, (M + 0.5) * h, (Nn - 0.5) * h, (Nn + 0.5) * h)


def direct_potential(cells, s0, sx, sy, tx, ty, G=1.0, nthreads=0):
    """Phi at targets (tx, ty) from cells (xl, xr, yd, yu) by the plain C sum."""
    import ctypes
    lib = _load()
    if not hasattr(lib, "_pot_ready"):
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_direct_potential.argtypes = [ctypes.c_long, dp, dp, dp, dp, dp, dp, dp, ctypes.c_long, dp, dp,
                                                ctypes.c_double, dp, ctypes.c_int]
        lib.oracle_direct_potential.restype = ctypes.c_int
        lib._pot_ready = True
    xl, xr, yd, yu = [np.ascontiguousarray(c, dtype=np.float64).ravel() for c in cells]
    s0 = np.ascontiguousarray(s0, dtype=np.float64).ravel()
    sx = None if sx is None else np.ascontiguousarray(sx, dtype=np.float64).ravel()
    sy = None if sy is None else np.ascontiguousarray(sy, dtype=np.float64).ravel()
    tx = np.ascontiguousarray(tx, dtype=np.float64).ravel()
    ty = np.ascontiguousarray(ty, dtype=np.float64).ravel()
    phi = np.zeros(tx.size)
    lib.oracle_direct_potential(xl.size, _ptr(xl), _ptr(xr), _ptr(yd), _ptr(yu), _ptr(s0), _ptr(sx), _ptr(sy),
                                tx.size, _ptr(tx), _ptr(ty), float(G), _ptr(phi), int(nthreads))
    return phi


def uniform_direct_potential(sigma, dx, dy, h, x0=-1.0, y0=-1.0, G=1.0, targets=None, nthreads=0):
    """Plain-sum potential on a uniform grid (layout of direct.uniform_direct_force)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    ny, nx = sigma.shape
    I, J = np.meshgrid(np.arange(nx), np.arange(ny))
    xl = x0 + I * h
    yd = y0 + J * h
    if targets is None:
        tj, ti = J.ravel(), I.ravel()
        shape = sigma.shape
    else:
        tj, ti = (np.asarray(a).ravel() for a in targets)
        shape = np.asarray(targets[0]).shape
    phi = direct_potential((xl, xl + h, yd, yd + h), sigma, dx, dy, x0 + (ti + 0.5) * h, y0 + (tj + 0.5) * h, G=G,
                           nthreads=nthreads)
    return phi.reshape(shape)


def uniform_fft_potential(sigma, dx, dy, h, G=1.0):
    """Second route: the same sum as a zero-padded FFT convolution (numpy FFT)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    ny, nx = sigma.shape
    py, px = 2 * ny, 2 * nx
    tab = offset_potentials(nx, ny, h)

    def wrap(t):
        # correlation phi[t] = sum_s q[s] P[s - t] = convolution with P[-e], placed at e mod P
        out = np.zeros((py, px))
        for j in range(2 * ny - 1):
            for i in range(2 * nx - 1):
                ex, ey = -(i - (nx - 1)), -(j - (ny - 1))
                out[ey % py, ex % px] = t[j, i]
        return np.fft.rfft2(out)

    spec = lambda a: np.fft.rfft2(np.asarray(a, np.float64), s=(py, px))
    acc = spec(sigma) * wrap(tab["p0"])
    if dx is not None:
        acc = acc + spec(dx) * wrap(tab["px"])
    if dy is not None:
        acc = acc + spec(dy) * wrap(tab["py"])
    return -G * np.fft.irfft2(acc, s=(py, px))[:ny, :nx]


def amr_direct_potential(patches, sigma, dx=None, dy=None, G=1.0, target_index=None, nthreads=0):
    """Potential at leaf centres of an AMR hierarchy (oracle.amr patches) from
    all leaf cells, by the plain C sum. sigma, dx, dy: per-patch [ny, nx] arrays
    (covered cells ignored). Returns (leaves, phi) as amr.amr_direct_force does."""
    from .amr import _gather, leaf_cells
    leaves = leaf_cells(patches)
    s0 = _gather(sigma, leaves)
    sx = _gather(dx, leaves)
    sy = _gather(dy, leaves)
    tsel = np.arange(leaves["xc"].size) if target_index is None else np.asarray(target_index)
    phi = direct_potential((leaves["xl"], leaves["xr"], leaves["yd"], leaves["yu"]), s0, sx, sy,
                           leaves["xc"][tsel], leaves["yc"][tsel], G=G, nthreads=nthreads)
    return leaves, phi
