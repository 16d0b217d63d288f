"""ctypes wrapper of the plain C direct sum (``direct.c``) and its build step.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "direct.c")
_LIB = os.path.join(_HERE, "liboracle_direct.so")
_lib = None


def build(force=False):
    """Compile direct.c into liboracle_direct.so with gcc and OpenMP (IEEE FP64)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_direct_force.argtypes = [ctypes.c_long, dp, dp, dp, dp, dp, dp, dp,
                                            ctypes.c_long, dp, dp, ctypes.c_double, dp, dp, ctypes.c_int]
        lib.oracle_direct_force.restype = ctypes.c_int
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_direct_force3.argtypes = [ctypes.c_long, dp, dp, dp, dp, dp, dp, dp, ctypes.c_long, dp, dp,
                                             ctypes.c_double, ctypes.c_double, dp, dp, dp, ctypes.c_int]
        lib.oracle_direct_force3.restype = ctypes.c_int
        _lib = lib
    return _lib


def max_threads():
    return _load().oracle_max_threads()


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def direct_force(cells, s0, sx, sy, tx, ty, G=1.0, nthreads=0):
    """F at targets (tx, ty) from source cells (xl, xr, yd, yu) by the plain sum.

    cells: tuple of four 1-D arrays (xl, xr, yd, yu). s0, sx, sy: per-cell
    sigma0, deltax, deltay (sx, sy may be None for the order-0 sum).
    Returns (fx, fy) as float64 arrays. Raises ValueError on a log-divergent pair.
    """
    lib = _load()
    xl, xr, yd, yu = [np.ascontiguousarray(c, dtype=np.float64).ravel() for c in cells]
    s0 = np.ascontiguousarray(s0, dtype=np.float64).ravel()
    sx = None if sx is None else np.ascontiguousarray(sx, dtype=np.float64).ravel()
    sy = None if sy is None else np.ascontiguousarray(sy, dtype=np.float64).ravel()
    tx = np.ascontiguousarray(tx, dtype=np.float64).ravel()
    ty = np.ascontiguousarray(ty, dtype=np.float64).ravel()
    ns, nt = xl.size, tx.size
    for a in (xr, yd, yu, s0) + tuple(a for a in (sx, sy) if a is not None):
        if a.size != ns:
            raise ValueError("source arrays differ in length")
    if ty.size != nt:
        raise ValueError("target arrays differ in length")
    fx = np.zeros(nt, dtype=np.float64)
    fy = np.zeros(nt, dtype=np.float64)
    st = lib.oracle_direct_force(ns, _ptr(xl), _ptr(xr), _ptr(yd), _ptr(yu), _ptr(s0), _ptr(sx), _ptr(sy),
                                 nt, _ptr(tx), _ptr(ty), float(G), _ptr(fx), _ptr(fy), int(nthreads))
    if st != 0:
        raise ValueError("log-divergent target/source pair (target on a source edge span or corner)")
    return fx, fy


def uniform_direct_force(sigma, dx, dy, h, x0=-1.0, y0=-1.0, G=1.0, targets=None, nthreads=0):
    """Direct sum on a uniform grid, sigma[j, i] at centre (x0+(i+1/2)h, y0+(j+1/2)h).

    targets: optional (j_idx, i_idx) integer arrays of target cells; default all.
    Returns (fx, fy) shaped like sigma (all targets) or like the index arrays.
    """
    sigma = np.asarray(sigma, dtype=np.float64)
    ny, nx = sigma.shape
    i = np.arange(nx)
    j = np.arange(ny)
    I, J = np.meshgrid(i, j)
    xl = x0 + I * h
    yd = y0 + J * h
    cells = (xl, xl + h, yd, yd + h)
    if targets is None:
        tj, ti = J.ravel(), I.ravel()
        shape = sigma.shape
    else:
        tj, ti = (np.asarray(a).ravel() for a in targets)
        shape = np.asarray(targets[0]).shape
    tx = x0 + (ti + 0.5) * h
    ty = y0 + (tj + 0.5) * h
    fx, fy = direct_force(cells, sigma, dx, dy, tx, ty, G=G, nthreads=nthreads)
    return fx.reshape(shape), fy.reshape(shape)


def direct_force3(cells, s0, sx, sy, tx, ty, z, G=1.0, nthreads=0):
    """Fx, Fy, Fz at targets (tx, ty, z), z != 0, by the plain sum over cells."""
    lib = _load()
    xl, xr, yd, yu = [np.ascontiguousarray(c, dtype=np.float64).ravel() for c in cells]
    s0 = np.ascontiguousarray(s0, dtype=np.float64).ravel()
    sx = None if sx is None else np.ascontiguousarray(sx, dtype=np.float64).ravel()
    sy = None if sy is None else np.ascontiguousarray(sy, dtype=np.float64).ravel()
    tx = np.ascontiguousarray(tx, dtype=np.float64).ravel()
    ty = np.ascontiguousarray(ty, dtype=np.float64).ravel()
    out = [np.zeros(tx.size) for _ in range(3)]
    st = lib.oracle_direct_force3(xl.size, _ptr(xl), _ptr(xr), _ptr(yd), _ptr(yu), _ptr(s0), _ptr(sx), _ptr(sy),
                                  tx.size, _ptr(tx), _ptr(ty), float(z), float(G), _ptr(out[0]), _ptr(out[1]),
                                  _ptr(out[2]), int(nthreads))
    if st != 0:
        raise ValueError("direct_force3 needs z != 0")
    return tuple(out)


def uniform_direct_force3(sigma, dx, dy, h, z, x0=-1.0, y0=-1.0, G=1.0, targets=None, nthreads=0):
    """Off-plane direct sum on a uniform grid (layout as uniform_direct_force)."""
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
    f = direct_force3((xl, xl + h, yd, yd + h), sigma, dx, dy, x0 + (ti + 0.5) * h, y0 + (tj + 0.5) * h, z, G=G,
                      nthreads=nthreads)
    return tuple(a.reshape(shape) for a in f)
