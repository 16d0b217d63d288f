"""Parity of the CUDA mid-plane potential (sg_potential; Section 2, K = 1/r) with
the oracle. Tolerances (relative L2 over all cells): FP64 1e-12, FP32 1e-5."""
import math

import numpy as np
import pytest

from oracle.disks import d2_potential
from oracle.fftconv import central_slopes
from oracle.norms import norms, rel_l2
from oracle.potential import uniform_direct_potential, uniform_fft_potential
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


def _phi(sg, geom, prec, mode, s, sx=None, sy=None, G=1.0):
    import torch
    nx, ny, x0, y0, h = geom
    dt = np.float64 if prec == "fp64" else np.float32
    plan = sg.Plan([(0, nx, ny, x0, y0, h)], precision=prec, slope_mode=mode, G=G)
    b = to_dev(sx, dt) if mode == sg.SG_SLOPES_CALLER else None
    c = to_dev(sy, dt) if mode == sg.SG_SLOPES_CALLER else None
    phi = plan.potential(to_dev(s, dt), b, c)
    torch.cuda.synchronize()
    out = phi.cpu().numpy().astype(np.float64).reshape(ny, nx)
    plan.close()
    return out


def _oracle(sg, h, mode, s, sx, sy, dt, G=1.0):
    c = lambda a: np.asarray(a, dt).astype(np.float64)
    s = c(s)
    if mode == sg.SG_SLOPES_NONE:
        return uniform_fft_potential(s, None, None, h, G=G)
    if mode == sg.SG_SLOPES_CENTRAL:
        return uniform_fft_potential(s, *central_slopes(s, h), h, G=G)
    return uniform_fft_potential(s, c(sx), c(sy), h, G=G)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("shape", [(16, 16), (64, 64), (37, 53), (1, 1), (2, 7), (100, 100)])
@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("prec, tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_potential_parity(sg, shape, mode, prec, tol):
    ny, nx = shape
    h = 0.05
    s, sx, sy = W.random_fields(ny, nx, seed=nx * 3 + ny)
    s = np.abs(s)
    got = _phi(sg, (nx, ny, -0.3, 0.1, h), prec, mode, s, sx, sy, G=1.7)
    ref = _oracle(sg, h, mode, s, sx, sy, np.float64 if prec == "fp64" else np.float32, G=1.7)
    assert _rel(got, ref) < tol


def test_potential_against_plain_sum(sg):
    """Against the oracle's plain C sum (not the FFT route), FP64, 48 x 40."""
    ny, nx, h = 40, 48, 0.04
    s, sx, sy = W.random_fields(ny, nx, seed=77)
    got = _phi(sg, (nx, ny, -1.0, -0.7, h), "fp64", 2, s, sx, sy)
    ref = uniform_direct_potential(s, sx, sy, h, x0=-1.0, y0=-0.7)
    assert _rel(got, ref) < 1e-12


def test_d2_potential_second_order(sg):
    """The D_2 disk of Section 3 (radius 0.5) with analytic slopes: the CUDA FP64
    potential converges to the closed form at second order."""
    errs = []
    for n in (128, 256):
        geom = W.unit_grid(n)
        nx, ny, x0, y0, h = geom
        X, Y = W.cell_centres(nx, ny, x0, y0, h)
        s, sx, sy = W.d2_sigma(X, Y, 0.5)
        phi = _phi(sg, geom, "fp64", 2, s, sx, sy)
        errs.append(norms(phi - d2_potential(np.hypot(X, Y), 0.5), h * h)[0])
    assert math.log2(errs[0] / errs[1]) > 1.8, errs


def test_force_is_minus_gradient_on_gpu(sg):
    """Central differences of the CUDA potential against the CUDA force (FP64),
    a smooth disk: agreement to O(h^2) away from the grid edge."""
    import torch
    n = 128
    nx, ny, x0, y0, h = W.unit_grid(n)
    X, Y = W.cell_centres(nx, ny, x0, y0, h)
    s, sx, sy = W.kuzmin_sigma(X, Y, 0.3)
    plan = sg.Plan([(0, nx, ny, x0, y0, h)], precision="fp64", slope_mode=sg.SG_SLOPES_CALLER)
    a, b, c = to_dev(s, np.float64), to_dev(sx, np.float64), to_dev(sy, np.float64)
    phi = plan.potential(a, b, c)
    fx, fy = plan.force(a, b, c)
    torch.cuda.synchronize()
    phi = phi.cpu().numpy().reshape(ny, nx)
    fx = fx.cpu().numpy().reshape(ny, nx)
    fy = fy.cpu().numpy().reshape(ny, nx)
    plan.close()
    gx = -(phi[1:-1, 2:] - phi[1:-1, :-2]) / (2 * h)
    gy = -(phi[2:, 1:-1] - phi[:-2, 1:-1]) / (2 * h)
    inner = (np.abs(X[1:-1, 1:-1]) < 0.5) & (np.abs(Y[1:-1, 1:-1]) < 0.5)
    assert rel_l2(gx[inner], gy[inner], fx[1:-1, 1:-1][inner], fy[1:-1, 1:-1][inner]) < 5e-3


def test_potential_large_fp32_sampled(sg):
    """The 1024^2 spiral disk with central slopes, FP32: 48 sampled cells against
    the oracle's plain sum."""
    case = W.spiral_1024()
    nx, ny, x0, y0, h = case["geom"]
    got = _phi(sg, case["geom"], "fp32", sg.SG_SLOPES_CENTRAL, case["sigma"])
    rng = np.random.Generator(np.random.PCG64(18))
    tj, ti = rng.integers(0, ny, 48), rng.integers(0, nx, 48)
    s32 = np.asarray(case["sigma"], np.float32).astype(np.float64)
    cx, cy = central_slopes(s32, h)
    ref = uniform_direct_potential(s32, cx, cy, h, x0=x0, y0=y0, targets=(tj, ti))
    assert _rel(got[tj, ti], ref) < 1e-5


def test_potential_repeatable_and_errors(sg):
    import torch
    plan = sg.Plan([(0, 32, 32, 0.0, 0.0, 0.1)], precision="fp32", slope_mode=sg.SG_SLOPES_NONE)
    s = torch.rand(1024, device="cuda")
    a = plan.potential(s).clone()
    b = plan.potential(s)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    plan.close()
    amr = sg.Plan([(lev,) + p for lev, p in enumerate(W.centred_nested_patches(16, 2))])
    x = torch.zeros(amr.ncells, device="cuda")
    with pytest.raises(sg.SgError) as e:
        sg.sg_potential(amr.handle, x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr())
    assert e.value.status == sg.SG_EINVAL and "one unmasked patch" in str(e.value)
    amr.close()
