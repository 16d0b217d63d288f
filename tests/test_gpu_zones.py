"""Parity of the CUDA path on zone-by-zone hierarchies (Fig. 1 / Table 10 and the
ILR/VLR hierarchies of Section 4) and on masked patches, against the oracle's
plain leaf sum; and the printed errors of Tables 3-6 from the CUDA path.

Tolerances (relative L2 over both components and all leaves): FP64 1e-12;
FP32 1e-5, for smooth densities and for uniform random fields alike.
"""
import numpy as np
import pytest

from oracle import amr as oamr
from oracle.direct import uniform_direct_force
from oracle.norms import rel_l2
from paper_2001_02765_gb300 import workloads as W
from tests._lib import ensure_built, to_dev
from tests.test_oracle_pins import (_d_sigma, _load_table, _near3, amr_pinned_columns, amr_table_norms)
from tests.test_zones_host import T10_GRID

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


def _hier_args(hier):
    n = hier["n"]
    return (n, n, hier["x0"], hier["y0"], hier["h0"], hier["level"], hier["ix"], hier["iy"])


def _solve(sg, args, prec, s, sx=None, sy=None, cross=0):
    import torch
    dt = np.float64 if prec == "fp64" else np.float32
    mode = sg.SG_SLOPES_CALLER if sx is not None else sg.SG_SLOPES_NONE
    plan = sg.ZonePlan(*args, precision=prec, slope_mode=mode, cross_mode=cross)
    if cross:
        assert plan.info["cross_mode"] == cross
    fx, fy = plan.force_zones(to_dev(s, dt), None if sx is None else to_dev(sx, dt),
                              None if sy is None else to_dev(sy, dt))
    torch.cuda.synchronize()
    out = fx.cpu().numpy().astype(np.float64), fy.cpu().numpy().astype(np.float64)
    info = plan.info
    plan.close()
    return out, info


def _oracle(args, leaf, s, sx, sy, dt, targets=None):
    nx0, ny0, x0, y0, h0, level, ix, iy = args
    c = lambda a: None if a is None else np.asarray(a, dt).astype(np.float64)
    return oamr.zone_leaf_force(x0, y0, h0, level, ix, iy, leaf, c(s), c(sx), c(sy), targets=targets)


def _table10(sg):
    rec = np.array(_load_table("table10_amr_cells.txt"))
    level, ix, iy = sg.sg_zones_from_records(rec, *T10_GRID)
    leaf = rec[:, 5] == 1
    return T10_GRID + (level, ix, iy), leaf


@pytest.mark.parametrize("cross", [1, 2], ids=["direct", "levels"])
@pytest.mark.parametrize("prec, tol", [("fp64", F64_TOL), ("fp32", F32_TOL)])
def test_table10_zones(sg, prec, tol, cross):
    args, leaf = _table10(sg)
    rng = np.random.Generator(np.random.PCG64(14))
    s = rng.uniform(0.5, 1.5, 32)
    sx = rng.uniform(-1, 1, 32)
    sy = rng.uniform(-1, 1, 32)
    (fx, fy), info = _solve(sg, args, prec, s, sx, sy, cross=cross)
    rx, ry = _oracle(args, leaf, s, sx, sy, np.float64 if prec == "fp64" else np.float32)
    assert info["nleaves"] == 28 and info["nzones"] == 32
    assert rel_l2(fx[leaf], fy[leaf], rx[leaf], ry[leaf]) < tol
    assert np.all(fx[~leaf] == 0) and np.all(fy[~leaf] == 0)


@pytest.mark.parametrize("cross", [1, 2], ids=["direct", "levels"])
@pytest.mark.parametrize("rule", ["ilr", "vlr"])
@pytest.mark.parametrize("disk", ["d2", "d22"])
@pytest.mark.parametrize("prec, tol", [("fp64", F64_TOL), ("fp32", F32_TOL)])
def test_band_hierarchy_disk_parity(sg, rule, disk, prec, tol, cross):
    hier = W.band_hierarchy(48, 3, rule, disk)
    args = _hier_args(hier)
    xc, yc, _ = W.zone_geometry(hier)
    s, sx, sy = _d_sigma(disk, xc, yc)
    (fx, fy), info = _solve(sg, args, prec, s, sx, sy, cross=cross)
    leaf = hier["leaf"]
    rx, ry = _oracle(args, leaf, s, sx, sy, np.float64 if prec == "fp64" else np.float32)
    assert info["nleaves"] == leaf.sum() and info["nzones"] == leaf.size
    assert rel_l2(fx[leaf], fy[leaf], rx[leaf], ry[leaf]) < tol


@pytest.mark.parametrize("cross", [1, 2], ids=["direct", "levels"])
@pytest.mark.parametrize("prec, tol", [("fp64", F64_TOL), ("fp32", F32_TOL)])
def test_band_hierarchy_random_fields(sg, prec, tol, cross):
    """Four levels, a ragged level-0 grid, random densities and slopes (order 1)."""
    hier = W.band_hierarchy(40, 4, "vlr", "d22")
    args = _hier_args(hier)
    rng = np.random.Generator(np.random.PCG64(15))
    n = hier["level"].size
    s, sx, sy = rng.uniform(0, 1, n), rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    (fx, fy), _ = _solve(sg, args, prec, s, sx, sy, cross=cross)
    leaf = hier["leaf"]
    rx, ry = _oracle(args, leaf, s, sx, sy, np.float64 if prec == "fp64" else np.float32)
    err = rel_l2(fx[leaf], fy[leaf], rx[leaf], ry[leaf])
    print("rel L2 %s cross=%d: %.3e (tolerance %.0e)" % (prec, cross, err, tol))
    assert err < tol


def test_band_hierarchy_order0(sg):
    hier = W.band_hierarchy(32, 3, "ilr", "d2")
    args = _hier_args(hier)
    xc, yc, _ = W.zone_geometry(hier)
    s, _, _ = _d_sigma("d2", xc, yc)
    (fx, fy), _ = _solve(sg, args, "fp64", s)
    leaf = hier["leaf"]
    rx, ry = _oracle(args, leaf, s, None, None, np.float64)
    assert rel_l2(fx[leaf], fy[leaf], rx[leaf], ry[leaf]) < F64_TOL


def test_large_hierarchy_fp32_sampled(sg):
    """AMR(3, D_2,2) ILR at N = 512 (410,272 leaves, several patches per level):
    FP32, 64 sampled leaves against the plain sum over every leaf."""
    hier = W.band_hierarchy(512, 3, "ilr", "d22")
    args = _hier_args(hier)
    xc, yc, _ = W.zone_geometry(hier)
    s, sx, sy = _d_sigma("d22", xc, yc)
    (fx, fy), info = _solve(sg, args, "fp32", s, sx, sy)
    leaf = hier["leaf"]
    assert info["nleaves"] == 410272 and info["nzones"] == 459648
    rng = np.random.Generator(np.random.PCG64(16))
    t = rng.choice(np.nonzero(leaf)[0], 64, replace=False)
    rx, ry = _oracle(args, leaf, s, sx, sy, np.float32, targets=t)
    assert rel_l2(fx[t], fy[t], rx, ry) < F32_TOL


def test_ilr_1024_levels_fp32_sampled(sg):
    """AMR(3, D_2) ILR at N = 1024 (1,419,424 leaves; finest extent 4096, 8192-point
    level convolutions), FP32, 64 sampled leaves against the plain sum."""
    hier = W.band_hierarchy(1024, 3, "ilr", "d2")
    args = _hier_args(hier)
    xc, yc, _ = W.zone_geometry(hier)
    s, sx, sy = _d_sigma("d2", xc, yc)
    (fx, fy), info = _solve(sg, args, "fp32", s, sx, sy)
    assert info["cross_mode"] == sg.SG_CROSS_LEVELS and info["nleaves"] == 1419424
    leaf = hier["leaf"]
    rng = np.random.Generator(np.random.PCG64(17))
    t = rng.choice(np.nonzero(leaf)[0], 64, replace=False)
    rx, ry = _oracle(args, leaf, s, sx, sy, np.float32, targets=t)
    assert rel_l2(fx[t], fy[t], rx, ry) < F32_TOL


@pytest.mark.parametrize("n", [128, 256])
@pytest.mark.parametrize("table, L", [(3, 2), (3, 3), (4, 2), (4, 3), (5, 2), (5, 3), (6, 2), (6, 3)])
def test_tables3_6_from_cuda_path(sg, table, L, n):
    """Tables 3-6 (Section 4), FP64 CUDA path: at N = 128 the printed entries the
    oracle reproduces (see test_oracle_pins) come out the same to half a unit of
    the third digit; at N = 256 to one unit (three D_2,2 entries differ from the
    paper's by one in the last digit)."""
    rows = {(int(r[0]), int(r[3]), int(r[4])): r for r in _load_table("tables3_6_amr_norms.txt")}
    r = rows[(table, L, n)]
    rule, disk = ("ilr", "vlr")[int(r[1])], ("d2", "d22")[int(r[2])]
    hier = W.band_hierarchy(n, L, rule, disk)
    xc, yc, _ = W.zone_geometry(hier)
    s, sx, sy = _d_sigma(disk, xc, yc)
    (fx, fy), _ = _solve(sg, _hier_args(hier), "fp64", s, sx, sy)
    got = amr_table_norms(hier, disk, fx, fy)
    printed = r[5:]
    for c in amr_pinned_columns(table, int(r[2]), L, n):
        assert _near3(got[c], printed[c], 0.51 if n == 128 else 1.01), (table, L, n, c, got, printed)


def test_zone_refinement_invariance(sg):
    """Zones carrying their level-0 ancestor's linear density: the force at the
    unrefined zones equals the uniform CUDA solve (FP64)."""
    import torch
    n = 32
    nx, ny, x0, y0, h = W.unit_grid(n)
    s, sx, sy = W.random_fields(n, n, seed=33)
    plan = sg.Plan([(0, nx, ny, x0, y0, h)], precision="fp64", slope_mode=sg.SG_SLOPES_CALLER)
    ux, uy = plan.force(to_dev(s, np.float64), to_dev(sx, np.float64), to_dev(sy, np.float64))
    torch.cuda.synchronize()
    ux = ux.cpu().numpy().reshape(n, n)
    uy = uy.cpu().numpy().reshape(n, n)
    plan.close()
    hier = W.band_hierarchy(n, 3, "vlr", "d2")
    lev, ix, iy = hier["level"], hier["ix"], hier["iy"]
    ai, aj = ix >> lev, iy >> lev
    xc, yc, _ = W.zone_geometry(hier)
    zs = s[aj, ai] + sx[aj, ai] * (xc - (x0 + (ai + 0.5) * h)) + sy[aj, ai] * (yc - (y0 + (aj + 0.5) * h))
    (fx, fy), _ = _solve(sg, _hier_args(hier), "fp64", zs, sx[aj, ai], sy[aj, ai])
    c = (lev == 0) & hier["leaf"]
    assert rel_l2(fx[c], fy[c], ux[iy[c], ix[c]], uy[iy[c], ix[c]]) < F64_TOL


def test_zone_slots_and_counts(sg):
    rows = _load_table("tables8_9_zone_counts.txt")
    for table, rule, disk, L, n, zones, leaves in rows:
        if n > 256:
            continue
        hier = W.band_hierarchy(int(n), int(L), ("ilr", "vlr")[int(rule)], ("d2", "d22")[int(disk)])
        plan = sg.ZonePlan(*_hier_args(hier), precision="fp32")
        assert (plan.nzones, plan.info["nleaves"]) == (int(zones), int(leaves))
        slots = plan.slots()
        assert np.unique(slots).size == slots.size and slots.min() >= 0 and slots.max() < plan.ncells
        plan.close()


@pytest.mark.parametrize("prec, tol", [("fp64", F64_TOL), ("fp32", F32_TOL)])
def test_masked_single_patch(sg, prec, tol):
    """One patch with holes (absent cells carry no density, get no force)."""
    import torch
    n = 40
    nx, ny, x0, y0, h = W.unit_grid(n)
    X, Y = W.cell_centres(nx, ny, x0, y0, h)
    mask = (np.hypot(X, Y) < 0.9) & ~((np.abs(X) < 0.2) & (np.abs(Y - 0.3) < 0.1))
    s, sx, sy = W.kuzmin_sigma(X, Y, 0.2)
    dt = np.float64 if prec == "fp64" else np.float32
    plan = sg.Plan([(0, nx, ny, x0, y0, h)], precision=prec, slope_mode=sg.SG_SLOPES_CALLER, masks=[mask])
    assert plan.info["nleaves"] == mask.sum()
    fx, fy = plan.force(to_dev(s, dt), to_dev(sx, dt), to_dev(sy, dt))
    torch.cuda.synchronize()
    fx = fx.cpu().numpy().astype(np.float64).reshape(ny, nx)
    fy = fy.cpu().numpy().astype(np.float64).reshape(ny, nx)
    plan.close()
    J, I = np.nonzero(mask)
    c = lambda a: np.asarray(a, dt).astype(np.float64)[J, I]
    rx, ry = oamr.zone_leaf_force(x0, y0, h, np.zeros(J.size), I, J, np.ones(J.size, bool), c(s), c(sx), c(sy))
    assert rel_l2(fx[J, I], fy[J, I], rx, ry) < tol


def test_force_zones_errors(sg):
    import torch
    plan = sg.Plan([(0, 8, 8, 0.0, 0.0, 1.0)], slope_mode=sg.SG_SLOPES_NONE)
    a = torch.zeros(64, device="cuda")
    with pytest.raises(sg.SgError) as e:
        sg.sg_force_zones(plan.handle, a.data_ptr(), 0, 0, a.data_ptr(), a.data_ptr())
    assert e.value.status == sg.SG_EINVAL and "zone plan" in str(e.value)
    plan.close()
    args, _ = _table10(sg)
    zp = sg.ZonePlan(*args, precision="fp32", slope_mode=sg.SG_SLOPES_CALLER)
    b = torch.zeros(32, device="cuda")
    with pytest.raises(sg.SgError) as e:
        sg.sg_force_zones(zp.handle, b.data_ptr(), 0, 0, b.data_ptr(), b.data_ptr())  # slopes missing
    assert e.value.status == sg.SG_EINVAL
    zp.close()


@pytest.mark.parametrize("cross", [1, 2], ids=["direct", "levels"])
@pytest.mark.parametrize("prec, tol", [("fp64", F64_TOL), ("fp32", F32_TOL)])
def test_band_hierarchy_central_slopes(sg, prec, tol, cross):
    """Zone plans with SG_SLOPES_CENTRAL (the neighbour-leaf rule across zones of
    every level): against the oracle's rule and the plain leaf sum."""
    from oracle import slopes as S
    hier = W.band_hierarchy(40, 3, "ilr", "d22")
    args = _hier_args(hier)
    xc, yc, _ = W.zone_geometry(hier)
    s, _, _ = _d_sigma("d22", xc, yc)
    dt = np.float64 if prec == "fp64" else np.float32
    import torch
    plan = sg.ZonePlan(*args, precision=prec, slope_mode=sg.SG_SLOPES_CENTRAL, cross_mode=cross)
    assert plan.info["cross_mode"] == cross
    fx, fy = plan.force_zones(to_dev(s, dt))
    torch.cuda.synchronize()
    fx, fy = fx.cpu().numpy().astype(np.float64), fy.cpu().numpy().astype(np.float64)
    plan.close()
    leaf = hier["leaf"]
    s64 = np.asarray(s, dt).astype(np.float64)
    ox, oy = S.zone_neighbour_slopes(hier["x0"], hier["y0"], hier["h0"], hier["level"], hier["ix"], hier["iy"], leaf,
                                     s64)
    rx, ry = _oracle(args, leaf, s64, ox, oy, np.float64)
    err = rel_l2(fx[leaf], fy[leaf], rx[leaf], ry[leaf])
    print("rel L2 %s cross=%d central: %.3e (tolerance %.0e)" % (prec, cross, err, tol))
    assert err < tol


def test_ilr2048_fp32_sampled(sg):
    """AMR(3, D_2) ILR at N = 2048 (Table 8's largest hierarchy: 5,677,336
    leaves, finest extent 8192 cells, beyond the level convolutions: the direct
    path), FP32: 96 sampled leaves (32 per level) against the plain sum over
    every leaf."""
    import torch
    hier = W.band_hierarchy(2048, 3, "ilr", "d2")
    args = _hier_args(hier)
    xc, yc, _ = W.zone_geometry(hier)
    s, sx, sy = _d_sigma("d2", xc, yc)
    leaf = hier["leaf"]
    assert int(leaf.sum()) == 5677336
    plan = sg.ZonePlan(*args, precision="fp32", slope_mode=sg.SG_SLOPES_CALLER)
    assert plan.info["cross_mode"] == sg.SG_CROSS_DIRECT
    fx, fy = plan.force_zones(to_dev(s, np.float32), to_dev(sx, np.float32), to_dev(sy, np.float32))
    torch.cuda.synchronize()
    fx, fy = fx.cpu().numpy().astype(np.float64), fy.cpu().numpy().astype(np.float64)
    assert sg.sg_plan_check_error(plan.handle) == sg.SG_OK
    plan.close()
    rng = np.random.Generator(np.random.PCG64(2048))
    t = np.concatenate([rng.choice(np.nonzero(leaf & (hier["level"] == l))[0], 32, replace=False) for l in range(3)])
    rx, ry = _oracle(args, leaf, s, sx, sy, np.float32, targets=t)
    err = rel_l2(fx[t], fy[t], rx, ry)
    print("rel L2 fp32 ILR N=2048: %.3e" % err)
    assert err < F32_TOL


@pytest.mark.parametrize("cross", [1, 2], ids=["direct", "levels"])
@pytest.mark.parametrize("prec, tol", [("fp64", F64_TOL), ("fp32", F32_TOL)])
def test_band_hierarchy_potential_zones(sg, prec, tol, cross):
    """sg_potential_zones on a four-level VLR hierarchy (level convolutions or
    the direct-sum path), random densities and slopes: the leaf potentials
    equal the oracle's plain sum of Section 2's 1/r cell integrals over the
    leaf cells; non-leaf zones get 0."""
    import torch
    from oracle.potential import direct_potential
    hier = W.band_hierarchy(32, 4, "vlr", "d22")
    args = _hier_args(hier)
    nx0, ny0, x0, y0, h0, level, ix, iy = args
    leaf = hier["leaf"]
    rng = np.random.Generator(np.random.PCG64(16))
    n = level.size
    s, sx, sy = rng.uniform(0, 1, n), rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    dt = np.float64 if prec == "fp64" else np.float32
    plan = sg.ZonePlan(*args, precision=prec, slope_mode=sg.SG_SLOPES_CALLER, cross_mode=cross)
    assert plan.info["cross_mode"] == cross
    phi = plan.potential_zones(to_dev(s, dt), to_dev(sx, dt), to_dev(sy, dt))
    torch.cuda.synchronize()
    phi = phi.cpu().numpy().astype(np.float64)
    plan.close()
    xl, xr, yd, yu, xc, yc = oamr.zone_bounds(x0, y0, h0, level, ix, iy)
    c = lambda a: np.asarray(a, dt).astype(np.float64)[leaf]
    ref = direct_potential((xl[leaf], xr[leaf], yd[leaf], yu[leaf]), c(s), c(sx), c(sy), xc[leaf], yc[leaf])
    err = np.linalg.norm(phi[leaf] - ref) / np.linalg.norm(ref)
    print("rel L2 potential %s cross=%d: %.3e (tolerance %.0e)" % (prec, cross, err, tol))
    assert err < tol
    assert np.all(phi[~leaf] == 0.0)
