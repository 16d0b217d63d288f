"""Off-plane forces on the GPU (targets at height z above the cell centres;
Section 2, the antiderivatives with the arctan terms) against the oracle.
Tolerances as for the in-plane path: relative L2 over all three components,
1e-12 (FP64) and 1e-5 (FP32)."""
import math

import numpy as np
import pytest

from oracle.direct import uniform_direct_force3
from oracle.fftconv import uniform_fft_force3
from oracle.kernels import offset_tables_z
from paper_2001_02765_gb300 import workloads as W
from tests._lib import ensure_built, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available()
    ensure_built()
    from paper_2001_02765_gb300 import sg as mod
    return mod


def _rel(a, b):
    num = sum(float(np.sum((x - y) ** 2)) for x, y in zip(a, b))
    den = sum(float(np.sum(y ** 2)) for y in b)
    return math.sqrt(num / den)


def _solve3(sg, geom, z, prec, mode, s, sx, sy):
    import torch
    nx, ny, x0, y0, h = geom
    dt = np.float64 if prec == "fp64" else np.float32
    plan = sg.Plan([(0, nx, ny, x0, y0, h)], precision=prec, slope_mode=mode, z=z)
    a = to_dev(s, dt)
    b = to_dev(sx, dt) if mode == sg.SG_SLOPES_CALLER else None
    c = to_dev(sy, dt) if mode == sg.SG_SLOPES_CALLER else None
    out = plan.force3(a, b, c)
    torch.cuda.synchronize()
    res = tuple(t.cpu().numpy().astype(np.float64).reshape(ny, nx) for t in out)
    plan.close()
    return res


@pytest.mark.parametrize("z", [0.3, -0.05, 1e-3])
def test_offplane_tables_match_oracle(sg, z):
    nx, ny, h = 13, 9, 0.1
    plan = sg.Plan([(0, nx, ny, 0.0, 0.0, h)], precision="fp64", z=z)
    ref = offset_tables_z(nx, ny, h, z)
    for name in sg.KERNEL_NAMES:
        got = plan.kernel_table(0, name)
        assert np.max(np.abs(got - ref[name])) < 1e-12, name
    plan.close()


@pytest.mark.parametrize("shape", [(32, 32), (45, 20), (1, 1)])
@pytest.mark.parametrize("z", [0.2, -0.07, 2e-3])
@pytest.mark.parametrize("prec, tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_offplane_parity(sg, shape, z, prec, tol):
    ny, nx = shape
    geom = (nx, ny, -0.5, -0.3, 0.04)
    patches = [(0,) + geom]
    s, sx, sy = (a[0] for a in W.bumps_on_patches(patches, seed=nx + ny))
    dt = np.float64 if prec == "fp64" else np.float32
    r = lambda a: np.asarray(a, dt).astype(np.float64)
    got = _solve3(sg, geom, z, prec, sg.SG_SLOPES_CALLER, s, sx, sy)
    ref = uniform_fft_force3(r(s), r(sx), r(sy), geom[4], z)
    assert _rel(got, ref) < tol


def test_offplane_central_slopes_and_plain_sum(sg):
    """Central slopes at height z, against the oracle's plain sum (FP64)."""
    from oracle.fftconv import central_slopes
    ny, nx, h, z = 24, 30, 0.05, 0.11
    geom = (nx, ny, -1.0, -0.6, h)
    s, _, _ = W.random_fields(ny, nx, seed=77)
    got = _solve3(sg, geom, z, "fp64", sg.SG_SLOPES_CENTRAL, s, None, None)
    cx, cy = central_slopes(s, h)
    ref = uniform_direct_force3(s, cx, cy, h, z, x0=-1.0, y0=-0.6)
    assert _rel(got, ref) < 1e-12


def test_in_plane_fz_is_the_limit_from_above(sg):
    import torch
    ny, nx = 16, 16
    s, sx, sy = W.random_fields(ny, nx, seed=3)
    plan = sg.Plan([(0, nx, ny, 0.0, 0.0, 0.1)], precision="fp64", G=1.3)
    a, b, c = to_dev(s, np.float64), to_dev(sx, np.float64), to_dev(sy, np.float64)
    fx, fy, fz = plan.force3(a, b, c)
    gx, gy = plan.force(a, b, c)
    torch.cuda.synchronize()
    assert torch.equal(fx, gx) and torch.equal(fy, gy)
    assert np.allclose(fz.cpu().numpy(), -2 * math.pi * 1.3 * s.ravel(), rtol=1e-15, atol=0)
    plan.close()


def _amr_force3(sg, patches, prec, z, sig, sx, sy, masks=None):
    import torch
    from tests._lib import concat_dev
    dt = np.float64 if prec == "fp64" else np.float32
    plan = sg.Plan(patches, precision=prec, slope_mode=sg.SG_SLOPES_CALLER, z=z, masks=masks)
    assert plan.info["cross_mode"] == sg.SG_CROSS_DIRECT  # level convolutions are for the plane
    out = plan.force3(concat_dev(sig, dt), concat_dev(sx, dt), concat_dev(sy, dt))
    torch.cuda.synchronize()
    res = [t.cpu().numpy().astype(np.float64) for t in out]
    return plan, res


@pytest.mark.parametrize("z", [0.02, -0.3])
@pytest.mark.parametrize("prec, tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_offplane_hierarchy_parity(sg, prec, tol, z):
    """Three nested levels of 16^2 cells off the plane (each patch's own FFT
    convolution with its height-z tables, the cross-patch sum in the corner
    form of the off-plane antiderivatives), random signed densities and slopes:
    Fx, Fy, Fz at every leaf equal the oracle's plain sum over the leaf cells."""
    from oracle import amr as oamr
    from oracle.direct import direct_force3
    from tests._lib import gather_leaves
    patches = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(16, 3))]
    rng = np.random.Generator(np.random.PCG64(21))
    sig = [rng.uniform(-1, 1, (p[2], p[1])) for p in patches]
    sx = [rng.uniform(-1, 1, (p[2], p[1])) for p in patches]
    sy = [rng.uniform(-1, 1, (p[2], p[1])) for p in patches]
    plan, (fx, fy, fz) = _amr_force3(sg, patches, prec, z, sig, sx, sy)
    dt = np.float64 if prec == "fp64" else np.float32
    P = oamr.make_patches(patches)
    leaves = oamr.leaf_cells(P)
    c = lambda a: np.concatenate([np.asarray(x, dt).astype(np.float64).ravel() for x in a])
    flat = lambda a: c(a)[_leaf_index(P, leaves)]
    ref = direct_force3((leaves["xl"], leaves["xr"], leaves["yd"], leaves["yu"]), flat(sig), flat(sx), flat(sy),
                        leaves["xc"], leaves["yc"], z)
    got = tuple(gather_leaves(plan, f, leaves) for f in (fx, fy, fz))
    plan.close()
    err = _rel(got, ref)
    print("rel L2 off-plane hierarchy %s z=%g: %.3e (tolerance %.0e)" % (prec, z, err, tol))
    assert err < tol


def _leaf_index(P, leaves):
    """Index of every leaf in the concatenated per-patch field arrays."""
    off = np.cumsum([0] + [p.nx * p.ny for p in P])
    return np.array([off[k] + j * P[k].nx + i for k, j, i in zip(leaves["patch"], leaves["j"], leaves["i"])])


def test_offplane_hierarchies_are_valid(sg):
    pat = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(16, 2))]
    assert sg.sg_geom_validate(pat, z=0.1) == sg.SG_OK
    assert sg.sg_geom_validate(pat[:1], z=0.1) == sg.SG_OK
