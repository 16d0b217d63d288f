"""The allocation-free entry point sg_direct_force_static against sg_force.

sg_direct_force_static serves callers that cannot let a library allocate
device memory (an application that owns the whole device budget, or a step
loop that must avoid cudaMalloc's latency and synchronisation): it keeps its
corner weights in a fixed array inside the library. This test calls it through
the C ABI twice in a row (the second call reuses the array the first one left
behind) and compares both results with the plan-based entry point sg_force on
the same grid, within the FP32 tolerance of the other parity tests (relative L2
1e-5), and, on small grids with random densities and slopes, with the FP64
oracle's plain sum over every cell pair. It sits in a file of its own,
collected last.
"""
import numpy as np
import pytest

from oracle.direct import uniform_direct_force
from oracle.norms import rel_l2
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


@pytest.mark.parametrize("nx, ny, slopes", [(64, 64, True), (100, 37, True), (48, 48, False)])
def test_static_entry_point_matches_sg_force(sg, nx, ny, slopes):
    import torch
    h = 2.0 / max(nx, ny)
    x0, y0 = -1.0, -1.0
    patches = [(0, nx, ny, x0, y0, h)]
    sig, sx, sy = (a[0] for a in W.bumps_on_patches(patches, seed=nx + ny))
    mode = sg.SG_SLOPES_CALLER if slopes else sg.SG_SLOPES_NONE
    plan = sg.Plan(patches, precision="fp32", slope_mode=mode, G=1.7)
    s, dx, dy = to_dev(sig, np.float32), to_dev(sx, np.float32), to_dev(sy, np.float32)
    rx, ry = plan.force(s, dx if slopes else None, dy if slopes else None)
    torch.cuda.synchronize()
    rx, ry = rx.cpu().numpy().astype(np.float64), ry.cpu().numpy().astype(np.float64)
    plan.close()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        fx = torch.full((nx * ny,), float("nan"), device="cuda")
        fy = torch.full((nx * ny,), float("nan"), device="cuda")
        sg.sg_direct_force_static(nx, ny, h, 1.7, s.data_ptr(), dx.data_ptr() if slopes else 0,
                                  dy.data_ptr() if slopes else 0, fx.data_ptr(), fy.data_ptr(), stream)
        torch.cuda.synchronize()
        gx, gy = fx.cpu().numpy().astype(np.float64), fy.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(gx)) and np.all(np.isfinite(gy)), call
        assert rel_l2(gx, gy, rx, ry) < 1e-5, (call, rel_l2(gx, gy, rx, ry))


@pytest.mark.parametrize("nx, ny, slopes", [(16, 16, True), (31, 9, True), (24, 40, False)])
def test_static_entry_point_matches_oracle(sg, nx, ny, slopes):
    """Random density and slopes on a small grid: both of two consecutive calls
    against the oracle's FP64 plain sum (Section 2 closed forms), 1e-5."""
    import torch
    h = 0.0625
    x0, y0 = -0.5, -0.75
    sig, sx, sy = W.random_fields(ny, nx, seed=nx * ny)
    s32 = [np.asarray(a, np.float32) for a in (sig, sx, sy)]
    ox, oy = uniform_direct_force(s32[0].astype(np.float64), s32[1].astype(np.float64) if slopes else None,
                                  s32[2].astype(np.float64) if slopes else None, h, x0=x0, y0=y0, G=0.8)
    s, dx, dy = (to_dev(a, np.float32) for a in s32)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        fx = torch.full((nx * ny,), float("nan"), device="cuda")
        fy = torch.full((nx * ny,), float("nan"), device="cuda")
        sg.sg_direct_force_static(nx, ny, h, 0.8, s.data_ptr(), dx.data_ptr() if slopes else 0,
                                  dy.data_ptr() if slopes else 0, fx.data_ptr(), fy.data_ptr(), stream)
        torch.cuda.synchronize()
        err = rel_l2(fx.cpu().numpy().astype(np.float64), fy.cpu().numpy().astype(np.float64), ox.ravel(), oy.ravel())
        print("rel L2 vs oracle, call %d: %.3e" % (call, err))
        assert err < 1e-5, (call, err)


def test_static_entry_point_rejects_oversize(sg):
    import torch
    a = torch.zeros(4, device="cuda")
    with pytest.raises(sg.SgError) as e:
        sg.sg_direct_force_static(513, 4, 0.1, 1.0, a.data_ptr(), 0, 0, a.data_ptr(), a.data_ptr(), 0)
    assert e.value.status == sg.SG_EINVAL and "512" in str(e.value)
