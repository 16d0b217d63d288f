"""Parity of the CUDA mid-plane potential (sg_potential; Section 2, K = 1/r) with
the oracle. Tolerances (relative L2 over all cells): FP64 1e-12, FP32 1e-5."""
import math

import numpy as np
import pytest

from oracle.disks import d2_potential
from oracle.fftconv import central_slopes
from oracle.norms import norms, rel_l2
from oracle import amr as oamr
from oracle.potential import amr_direct_potential, uniform_direct_potential, uniform_fft_potential
from paper_2001_02765_gb300 import workloads as W
from tests._lib import concat_dev, ensure_built, gather_leaves, to_dev

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
    off = sg.Plan([(0, 16, 16, 0.0, 0.0, 0.1)], z=0.05)
    x = torch.zeros(off.ncells, device="cuda")
    with pytest.raises(sg.SgError) as e:
        sg.sg_potential(off.handle, x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr())
    assert e.value.status == sg.SG_EINVAL and "in the plane" in str(e.value)
    off.close()


# ----------------- hierarchies (level convolutions, and the direct-sum path) --

TABLE10 = [(0, 4, 4, 0.0, 0.0, 0.25), (1, 2, 2, 0.25, 0.25, 0.125), (1, 2, 2, 0.5, 0.5, 0.125),
           (2, 2, 2, 0.25, 0.375, 0.0625), (2, 2, 2, 0.375, 0.25, 0.0625)]


def _amr_phi(sg, patches, prec, mode, sig, sx, sy, G=1.0, cross="levels"):
    import torch
    dt = np.float64 if prec == "fp64" else np.float32
    cm = sg.SG_CROSS_LEVELS if cross == "levels" else sg.SG_CROSS_DIRECT
    plan = sg.Plan(patches, precision=prec, slope_mode=mode, G=G, cross_mode=cm)
    assert plan.info["cross_mode"] == cm
    a = concat_dev(sig, dt)
    b = concat_dev(sx, dt) if mode == sg.SG_SLOPES_CALLER else None
    c = concat_dev(sy, dt) if mode == sg.SG_SLOPES_CALLER else None
    phi = plan.potential(a, b, c)
    torch.cuda.synchronize()
    return plan, phi.cpu().numpy().astype(np.float64)


def _amr_check(sg, patches, prec, mode, sig, sx, sy, tol, G=1.0, target_index=None, cross="levels"):
    dt = np.float64 if prec == "fp64" else np.float32
    plan, phi = _amr_phi(sg, patches, prec, mode, sig, sx, sy, G, cross)
    r = lambda a: [np.asarray(x, dt).astype(np.float64) for x in a]
    slopes = mode == sg.SG_SLOPES_CALLER
    leaves, ref = amr_direct_potential(oamr.make_patches(patches), r(sig), r(sx) if slopes else None,
                                       r(sy) if slopes else None, G=G, target_index=target_index)
    if target_index is not None:
        leaves = {k: v[target_index] for k, v in leaves.items()}
    got = gather_leaves(plan, phi, leaves)
    plan.close()
    err = _rel(got, ref)
    print("rel L2 potential %s %s: %.3e (tolerance %.0e)" % (prec, cross, err, tol))
    assert err < tol, err
    return err


CROSS = pytest.mark.parametrize("cross", ["levels", "direct"])


@CROSS
@pytest.mark.parametrize("prec, tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("mode", [0, 2])
def test_amr_potential_nested(sg, prec, tol, mode, cross):
    """Three centred nested levels of 16^2 cells, smooth bumps: the leaf-sum potential."""
    patches = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(16, 3))]
    sig, sx, sy = W.bumps_on_patches(patches, 3)
    _amr_check(sg, patches, prec, mode, sig, sx, sy, tol, G=2.5, cross=cross)


@CROSS
@pytest.mark.parametrize("prec, tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_amr_potential_table10(sg, prec, tol, cross):
    """Fig. 1 / Table 10: two patches per refined level, 28 leaves, random positive data."""
    rng = np.random.Generator(np.random.PCG64(8))
    sig = [rng.uniform(0, 1, (p[2], p[1])) for p in TABLE10]
    sx = [rng.uniform(-1, 1, (p[2], p[1])) for p in TABLE10]
    sy = [rng.uniform(-1, 1, (p[2], p[1])) for p in TABLE10]
    _amr_check(sg, TABLE10, prec, 2, sig, sx, sy, tol, cross=cross)


@CROSS
@pytest.mark.parametrize("prec, tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_amr_potential_ragged(sg, prec, tol, cross):
    """Non-square, off-centre patches (two on level 1), sizes not powers of two."""
    patches = [(0, 37, 29, -1.0, -0.8, 0.05), (1, 22, 14, -0.6, -0.3, 0.025), (1, 6, 8, 0.2, 0.1, 0.025),
               (2, 10, 12, -0.5, -0.25, 0.0125)]
    sig, sx, sy = W.bumps_on_patches(patches, 5)
    _amr_check(sg, patches, prec, 2, sig, sx, sy, tol, cross=cross)


@CROSS
@pytest.mark.parametrize("prec, tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_amr_potential_rough(sg, prec, tol, cross):
    """Three nested levels of 24^2 cells with independent uniform noise in
    sigma0 and both slopes (signed): every far-field and near-field term."""
    patches = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(24, 3))]
    rng = np.random.Generator(np.random.PCG64(17))
    sig = [rng.uniform(-1, 1, (p[2], p[1])) for p in patches]
    sx = [rng.uniform(-1, 1, (p[2], p[1])) for p in patches]
    sy = [rng.uniform(-1, 1, (p[2], p[1])) for p in patches]
    _amr_check(sg, patches, prec, 2, sig, sx, sy, tol, cross=cross)


@CROSS
def test_amr_potential_config3_sampled(sg, cross):
    """The 3 x 256^2 exponential-disk hierarchy, FP32: 64 sampled leaves against the plain sum."""
    case = W.exponential_hierarchy(256, 3, 0.1)
    patches = [(lev,) + p for lev, p in enumerate(case["patches"])]
    sig, sx, sy = case["sigma"], case["dx"], case["dy"]
    n = len(oamr.leaf_cells(oamr.make_patches(patches))["xc"])
    idx = np.random.Generator(np.random.PCG64(33)).choice(n, 64, replace=False)
    _amr_check(sg, patches, "fp32", 2, sig, sx, sy, 1e-5, target_index=idx, cross=cross)


def test_amr_potential_matches_force(sg):
    """Central differences of the hierarchy's potential on the finest patch
    against its force (FP64): agreement to O(h^2) inside the patch."""
    import torch
    patches = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(32, 3))]
    sig, sx, sy = W.bumps_on_patches(patches, 3)
    plan = sg.Plan(patches, precision="fp64", slope_mode=sg.SG_SLOPES_CALLER, cross_mode=sg.SG_CROSS_LEVELS)
    a, b, c = (concat_dev(f, np.float64) for f in (sig, sx, sy))
    phi = plan.potential(a, b, c)
    fx, fy = plan.force(a, b, c)
    torch.cuda.synchronize()
    P = plan.split(phi.cpu().numpy())[-1]
    FX = plan.split(fx.cpu().numpy())[-1]
    FY = plan.split(fy.cpu().numpy())[-1]
    h = patches[-1][5]
    plan.close()
    gx = -(P[1:-1, 2:] - P[1:-1, :-2]) / (2 * h)
    gy = -(P[2:, 1:-1] - P[:-2, 1:-1]) / (2 * h)
    err = np.hypot(gx - FX[1:-1, 1:-1], gy - FY[1:-1, 1:-1])
    assert float(np.sqrt(np.mean(err ** 2))) < 2e-2 * float(np.sqrt(np.mean(FX[1:-1, 1:-1] ** 2 + FY[1:-1, 1:-1] ** 2)))


def _exp_levels(sg, n, levels):
    patches = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(n, levels))]
    sig, sx, sy = [], [], []
    for p in patches:
        X, Y = W.cell_centres(*p[1:])
        a, b, c = W.exponential_sigma(X, Y, 0.1)
        sig.append(a)
        sx.append(b)
        sy.append(c)
    return patches, sig, sx, sy


def _per_level_sample(counts, k, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    off = np.concatenate([[0], np.cumsum(counts)])
    return np.sort(np.concatenate([off[i] + rng.choice(c, k, replace=False) for i, c in enumerate(counts)]))


@pytest.mark.parametrize("prec, tol, levels", [("fp32", 1e-5, 4), ("fp64", 1e-11, 3)])
def test_amr_potential_long_transforms_sampled(sg, prec, tol, levels):
    """Nested 512^2 levels of an exponential disk: four in FP32 (8192-point
    transforms), three in FP64 (4096, its limit), where the coarse target levels
    take the folded inverse transforms; 48 sampled leaves per level against the
    plain leaf sum."""
    patches, sig, sx, sy = _exp_levels(sg, 512, levels)
    n0 = 512 * 512 - 256 * 256
    counts = [n0] * (levels - 1) + [512 * 512]
    idx = _per_level_sample(counts, 48, 46 + levels)
    _amr_check(sg, patches, prec, 2, sig, sx, sy, tol, target_index=idx)
