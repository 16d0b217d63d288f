"""Parity of the CUDA uniform-grid path (tables, spectra, FFT convolution) with the FP64 oracle.

Tolerances: relative L2 over both components and all cells. FP64 plans: 1e-12
(the oracle's own table rounding is ~1e-16 d ln d per entry, well below this at
these sizes). FP32 plans: 1e-5 (FP32 transforms of length P lose about
eps32 * log2(P^2) ~ 1e-6 in relative L2; kernel spectra are built in FP64).
"""
import math

import numpy as np
import pytest

from oracle.direct import uniform_direct_force
from oracle.disks import d2_force_xy
from oracle.fftconv import central_slopes, uniform_fft_force
from oracle.kernels import offset_tables
from oracle.norms import norms, radial_error, rel_l2
from paper_2001_02765_gb300 import workloads as W
from tests._lib import ensure_built, to_dev

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 1e-5


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available()
    ensure_built()
    from paper_2001_02765_gb300 import sg as mod
    return mod


def _solve(sg, geom, prec, mode, s, sx=None, sy=None):
    import torch
    nx, ny, x0, y0, h = geom
    dt = np.float64 if prec == "fp64" else np.float32
    plan = sg.Plan([(0, nx, ny, x0, y0, h)], precision=prec, slope_mode=mode)
    a = to_dev(s, dt)
    b = to_dev(sx, dt) if mode == sg.SG_SLOPES_CALLER else None
    c = to_dev(sy, dt) if mode == sg.SG_SLOPES_CALLER else None
    fx, fy = plan.force(a, b, c)
    torch.cuda.synchronize()
    out = fx.cpu().numpy().astype(np.float64).reshape(ny, nx), fy.cpu().numpy().astype(np.float64).reshape(ny, nx)
    plan.close()
    return out


def _oracle(sg, geom, mode, s, sx, sy, dt):
    nx, ny, x0, y0, h = geom
    s = np.asarray(s, dt).astype(np.float64)
    if mode == sg.SG_SLOPES_NONE:
        return uniform_fft_force(s, None, None, h)
    if mode == sg.SG_SLOPES_CENTRAL:
        cx, cy = central_slopes(s, h)
        return uniform_fft_force(s, cx, cy, h)
    return uniform_fft_force(s, np.asarray(sx, dt).astype(np.float64), np.asarray(sy, dt).astype(np.float64), h)


@pytest.mark.parametrize("nx, ny", [(33, 17), (5, 9), (1, 1)])
def test_kernel_tables_match_oracle(sg, nx, ny):
    h = 0.07
    plan = sg.Plan([(0, nx, ny, 0.0, 0.0, h)], precision="fp64")
    ref = offset_tables(nx, ny, h)
    for name in sg.KERNEL_NAMES[:6]:
        got = plan.kernel_table(0, name)
        assert got.shape == ref[name].shape
        assert np.max(np.abs(got - ref[name])) < 1e-13, name
    plan.close()


@pytest.mark.parametrize("shape", [(16, 16), (64, 64), (100, 100), (37, 53), (1, 1), (2, 7), (200, 3)])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_uniform_fp64_parity(sg, shape, mode):
    ny, nx = shape
    geom = (nx, ny, -0.3, 0.1, 0.05)
    s, sx, sy = W.random_fields(ny, nx, seed=nx * 7 + ny)
    fx, fy = _solve(sg, geom, "fp64", mode, s, sx, sy)
    rx, ry = _oracle(sg, geom, mode, s, sx, sy, np.float64)
    if np.all(rx == 0) and np.all(ry == 0):
        assert np.max(np.abs(fx)) < 1e-14 and np.max(np.abs(fy)) < 1e-14
    else:
        assert rel_l2(fx, fy, rx, ry) < F64_TOL


@pytest.mark.parametrize("shape", [(16, 16), (64, 64), (100, 100), (37, 53), (2, 7)])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_uniform_fp32_parity(sg, shape, mode):
    ny, nx = shape
    geom = (nx, ny, -0.3, 0.1, 0.05)
    s, sx, sy = W.random_fields(ny, nx, seed=nx * 5 + ny)
    s = np.abs(s)
    fx, fy = _solve(sg, geom, "fp32", mode, s, sx, sy)
    rx, ry = _oracle(sg, geom, mode, s, sx, sy, np.float32)
    assert rel_l2(fx, fy, rx, ry) < F32_TOL


def test_single_cell_self_force(sg):
    """One cell: F = G deltax K^{x,x}(0,0) with K^{x,x}(0,0) = 2 h ln(1 + sqrt 2)."""
    h = 0.3
    fx, fy = _solve(sg, (1, 1, 0.0, 0.0, h), "fp64", 2, [[2.0]], [[0.5]], [[-0.25]])
    k = 2 * h * math.log(1 + math.sqrt(2))
    assert abs(fx[0, 0] - 0.5 * k) < 1e-14 and abs(fy[0, 0] + 0.25 * k) < 1e-14


def test_uniform_matches_plain_sum(sg):
    """Against the oracle's plain direct sum (not the FFT route), FP64, 48 x 40."""
    ny, nx = 40, 48
    geom = (nx, ny, -1.0, -0.7, 0.04)
    s, sx, sy = W.random_fields(ny, nx, seed=99)
    fx, fy = _solve(sg, geom, "fp64", 2, s, sx, sy)
    rx, ry = uniform_direct_force(s, sx, sy, 0.04, x0=-1.0, y0=-0.7)
    assert rel_l2(fx, fy, rx, ry) < F64_TOL


def test_table1_reproduced_by_cuda_path(sg):
    """Table 1 row N = 128 (Section 3) from the CUDA FP64 path, all six norms to 3 digits."""
    n = 128
    geom = W.unit_grid(n)
    nx, ny, x0, y0, h = geom
    X, Y = W.cell_centres(nx, ny, x0, y0, h)
    s, sx, sy = W.d2_sigma(X, Y, 0.5)
    fx, fy = _solve(sg, geom, "fp64", 2, s, sx, sy)
    ex, ey = d2_force_xy(X, Y, 0.5)
    got = norms(fx - ex, h * h) + norms(radial_error(X, Y, fx - ex, fy - ey), h * h)
    printed = (8.48e-4, 9.31e-4, 5.26e-3, 1.32e-3, 1.31e-3, 5.91e-3)
    for g, p in zip(got, printed):
        e = math.floor(math.log10(p))
        assert round(g / 10 ** e, 2) == round(p / 10 ** e, 2), (got, printed)


def test_spiral_1024_fp32_full_field(sg):
    """The 1024^2 spiral workload (P = 2048), FP32 with central slopes, every cell vs the oracle."""
    case = W.spiral_1024()
    geom = case["geom"]
    fx, fy = _solve(sg, geom, "fp32", sg.SG_SLOPES_CENTRAL, case["sigma"])
    rx, ry = _oracle(sg, geom, sg.SG_SLOPES_CENTRAL, case["sigma"], None, None, np.float32)
    assert rel_l2(fx, fy, rx, ry) < F32_TOL


def test_spiral_1024_fp64_sampled(sg):
    """The same workload in FP64, 48 seeded sample cells vs the oracle's plain direct sum."""
    case = W.spiral_1024()
    nx, ny, x0, y0, h = case["geom"]
    fx, fy = _solve(sg, case["geom"], "fp64", sg.SG_SLOPES_CENTRAL, case["sigma"])
    rng = np.random.Generator(np.random.PCG64(12))
    tj = rng.integers(0, ny, 48)
    ti = rng.integers(0, nx, 48)
    cx, cy = central_slopes(case["sigma"], h)
    rx, ry = uniform_direct_force(case["sigma"], cx, cy, h, x0=x0, y0=y0, targets=(tj, ti))
    assert rel_l2(fx[tj, ti], fy[tj, ti], rx, ry) < 1e-11


def test_largest_patch_2048_fp32_sampled(sg):
    """Maximum patch side 2048 (P = 4096), FP32, 16 sampled cells vs the plain sum."""
    n = 2048
    geom = W.unit_grid(n)
    nx, ny, x0, y0, h = geom
    X, Y = W.cell_centres(nx, ny, x0, y0, h)
    s, sx, sy = W.kuzmin_sigma(X, Y, 0.15)
    fx, fy = _solve(sg, geom, "fp32", sg.SG_SLOPES_CALLER, s, sx, sy)
    rng = np.random.Generator(np.random.PCG64(13))
    tj = rng.integers(0, ny, 16)
    ti = rng.integers(0, nx, 16)
    s32 = [np.asarray(a, np.float32).astype(np.float64) for a in (s, sx, sy)]
    rx, ry = uniform_direct_force(*s32, h, x0=x0, y0=y0, targets=(tj, ti))
    assert rel_l2(fx[tj, ti], fy[tj, ti], rx, ry) < F32_TOL


@pytest.mark.parametrize("mode", ["central", "caller"])
def test_fp64_4096_point_columns_sampled(sg, mode):
    """FP64 plans whose padded length is 4096 (sides 1100 x 1030; one exchange
    buffer in the column pass there, the shared-memory limit): 24 sampled
    cells vs the plain sum."""
    nx, ny = 1100, 1030
    geom = (nx, ny, -1.0, -0.95, 2.0 / nx)
    h = geom[4]
    X, Y = W.cell_centres(*geom)
    s, sx, sy = W.kuzmin_sigma(X, Y, 0.15)
    if mode == "central":
        fx, fy = _solve(sg, geom, "fp64", sg.SG_SLOPES_CENTRAL, s)
        sx, sy = central_slopes(s, h)
    else:
        fx, fy = _solve(sg, geom, "fp64", sg.SG_SLOPES_CALLER, s, sx, sy)
    rng = np.random.Generator(np.random.PCG64(14))
    tj = rng.integers(0, ny, 24)
    ti = rng.integers(0, nx, 24)
    rx, ry = uniform_direct_force(s, sx, sy, h, x0=geom[2], y0=geom[3], targets=(tj, ti))
    err = rel_l2(fx[tj, ti], fy[tj, ti], rx, ry)
    print("rel L2 fp64 4096-point %s: %.3e" % (mode, err))
    assert err < 1e-11


def test_host_entry_point_equals_device_entry_point(sg):
    import torch
    ny, nx = 96, 80
    s, sx, sy = W.random_fields(ny, nx, seed=4)
    plan = sg.Plan([(0, nx, ny, 0.0, 0.0, 0.01)], precision="fp32", slope_mode=sg.SG_SLOPES_CALLER)
    hx, hy = plan.force_host(s.astype(np.float32), sx.astype(np.float32), sy.astype(np.float32))
    dx_, dy_ = plan.force(to_dev(s, np.float32), to_dev(sx, np.float32), to_dev(sy, np.float32))
    torch.cuda.synchronize()
    assert np.array_equal(hx, dx_.cpu().numpy()) and np.array_equal(hy, dy_.cpu().numpy())
    plan.close()


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_host_entry_point_pinned_in_place(sg, mode, prec):
    """Pinned host output buffers are written in place by the kernels; the
    result equals the device entry point bit for bit."""
    import torch
    ny, nx = 70, 90
    dt = np.float64 if prec == "fp64" else np.float32
    tdt = torch.float64 if prec == "fp64" else torch.float32
    s, sx, sy = W.random_fields(ny, nx, seed=5 + mode)
    plan = sg.Plan([(0, nx, ny, 0.0, 0.0, 0.01)], precision=prec, slope_mode=mode)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dt).ravel()).pin_memory()
    hs, hdx, hdy = pin(s), pin(sx) if mode == 2 else None, pin(sy) if mode == 2 else None
    hfx = torch.empty(nx * ny, dtype=tdt).pin_memory()
    hfy = torch.empty(nx * ny, dtype=tdt).pin_memory()
    plan.force_host(hs, hdx, hdy, hfx, hfy)
    dfx, dfy = plan.force(to_dev(s, dt), to_dev(sx, dt) if mode == 2 else None, to_dev(sy, dt) if mode == 2 else None)
    torch.cuda.synchronize()
    assert torch.equal(hfx, dfx.cpu()) and torch.equal(hfy, dfy.cpu())
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_host_async_two_plans_pipelined(sg, prec):
    """Solves enqueued by sg_force_host_async alternately on two plans and two
    streams, each waited for one step later (the pipelined host loop), give
    every input set's device-entry result bit for bit."""
    import torch
    ny, nx = 100, 84
    dt = np.float64 if prec == "fp64" else np.float32
    tdt = torch.float64 if prec == "fp64" else torch.float32
    plans = [sg.Plan([(0, nx, ny, 0.0, 0.0, 0.01)], precision=prec, slope_mode=sg.SG_SLOPES_CENTRAL)
             for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    sets = 5
    hs = [torch.from_numpy(np.ascontiguousarray(W.random_fields(ny, nx, seed=20 + k)[0], dt).ravel()).pin_memory()
          for k in range(sets)]
    outs = [(torch.empty(nx * ny, dtype=tdt).pin_memory(), torch.empty(nx * ny, dtype=tdt).pin_memory())
            for _ in range(sets)]
    for k in range(sets):
        j = k % 2
        if k >= 2:
            plans[j].wait(streams[j])
        plans[j].force_host_async(hs[k], None, None, outs[k][0], outs[k][1], stream=streams[j])
    for j in range(2):
        plans[j].wait(streams[j])
    for k in range(sets):
        dfx, dfy = plans[0].force(hs[k].cuda())
        torch.cuda.synchronize()
        assert torch.equal(outs[k][0], dfx.cpu()) and torch.equal(outs[k][1], dfy.cpu())
    for p in plans:
        p.close()


def test_repeatable_bitwise(sg):
    import torch
    ny, nx = 128, 128
    s, _, _ = W.random_fields(ny, nx, seed=6)
    plan = sg.Plan([(0, nx, ny, 0.0, 0.0, 0.01)], precision="fp32", slope_mode=sg.SG_SLOPES_CENTRAL)
    a = to_dev(s, np.float32)
    f1 = [t.clone() for t in plan.force(a)]
    f2 = plan.force(a)
    torch.cuda.synchronize()
    assert torch.equal(f1[0], f2[0]) and torch.equal(f1[1], f2[1])
    plan.close()


def test_errors_are_reported(sg):
    import torch
    with pytest.raises(sg.SgError) as e:
        sg.Plan([(0, 0, 4, 0.0, 0.0, 1.0)])
    assert e.value.status == sg.SG_EINVAL
    plan = sg.Plan([(0, 8, 8, 0.0, 0.0, 1.0)], slope_mode=sg.SG_SLOPES_CALLER)
    a = torch.zeros(64, device="cuda")
    with pytest.raises(sg.SgError) as e:
        sg.sg_force(plan.handle, a.data_ptr(), 0, 0, a.data_ptr(), a.data_ptr(), 0)  # slopes missing
    assert e.value.status == sg.SG_EINVAL
    with pytest.raises(sg.SgError):
        sg.sg_plan_create([(0, 2048, 2048, 0.0, 0.0, 1.0)], hbm_budget=1 << 20)
    with pytest.raises(sg.SgError) as e:
        plan.kernel_table(0, "z0")  # the z-family exists for off-plane plans only
    assert e.value.status == sg.SG_EINVAL and "table" in str(e.value)
    plan.close()
