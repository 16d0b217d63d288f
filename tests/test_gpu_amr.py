"""Parity of the CUDA AMR paths with the oracle's plain leaf-pair sum: per-patch
FFT + cross-patch direct sum (cross mode 1), and level convolutions on the
finest lattice (cross mode 2). Tolerances as for the uniform path: relative L2
over all leaf targets, 1e-12 (FP64 plans) and 1e-5 (FP32 plans), on smooth
densities (disks, Gaussian bumps) and on rough ones (independent uniform noise
in every cell), where the FP32 direct sum relies on its FP64 near field and the
cell-centred expansion of the far field. Every check prints its measured error."""
import numpy as np
import pytest

from oracle import amr as oamr
from oracle.norms import rel_l2
from paper_2001_02765_gb300 import workloads as W
from tests._lib import concat_dev, ensure_built, gather_leaves

pytestmark = pytest.mark.gpu

TABLE10 = [(0, 4, 4, 0.0, 0.0, 0.25), (1, 2, 2, 0.25, 0.25, 0.125), (1, 2, 2, 0.5, 0.5, 0.125),
           (2, 2, 2, 0.25, 0.375, 0.0625), (2, 2, 2, 0.375, 0.25, 0.0625)]


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available()
    ensure_built()
    from paper_2001_02765_gb300 import sg as mod
    return mod


def _fields(patches, seed, positive=False):
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = 0.0 if positive else -1.0
    sig = [rng.uniform(lo, 1, (p[2], p[1])) for p in patches]
    sx = [rng.uniform(-1, 1, (p[2], p[1])) for p in patches]
    sy = [rng.uniform(-1, 1, (p[2], p[1])) for p in patches]
    return sig, sx, sy


CROSS = pytest.mark.parametrize("cross", [1, 2], ids=["direct", "levels"])


def _run(sg, patches, prec, mode, sig, sx, sy, G=1.0, cross=0):
    import torch
    dt = np.float64 if prec == "fp64" else np.float32
    plan = sg.Plan(patches, precision=prec, slope_mode=mode, G=G, cross_mode=cross)
    if cross:
        assert plan.info["cross_mode"] == cross
    a = concat_dev(sig, dt)
    b = concat_dev(sx, dt) if mode == sg.SG_SLOPES_CALLER else None
    c = concat_dev(sy, dt) if mode == sg.SG_SLOPES_CALLER else None
    fx, fy = plan.force(a, b, c)
    torch.cuda.synchronize()
    return plan, fx.cpu().numpy(), fy.cpu().numpy()


def _check(sg, patches, prec, mode, sig, sx, sy, tol, G=1.0, target_index=None, cross=0):
    dt = np.float64 if prec == "fp64" else np.float32
    plan, fx, fy = _run(sg, patches, prec, mode, sig, sx, sy, G, cross)
    r = lambda a: [np.asarray(x, dt).astype(np.float64) for x in a]
    use_slopes = mode == sg.SG_SLOPES_CALLER
    leaves, rx, ry = oamr.amr_direct_force(oamr.make_patches(patches), r(sig), r(sx) if use_slopes else None,
                                           r(sy) if use_slopes else None, G=G, target_index=target_index)
    if target_index is not None:
        leaves = {k: v[target_index] for k, v in leaves.items()}
    gx = gather_leaves(plan, fx, leaves)
    gy = gather_leaves(plan, fy, leaves)
    plan.close()
    err = rel_l2(gx, gy, rx, ry)
    print("rel L2 %s cross=%d: %.3e (tolerance %.0e)" % (prec, cross, err, tol))
    assert err < tol, err
    return err


@CROSS
@pytest.mark.parametrize("prec, tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("mode", [0, 2])
def test_nested_three_levels(sg, prec, tol, mode, cross):
    patches = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(16, 3))]
    sig, sx, sy = W.bumps_on_patches(patches, 3)
    _check(sg, patches, prec, mode, sig, sx, sy, tol, G=2.5, cross=cross)


@CROSS
@pytest.mark.parametrize("prec, tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_nested_three_levels_rough(sg, prec, tol, cross):
    """Independent noise in every cell."""
    patches = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(16, 3))]
    sig, sx, sy = _fields(patches, 3, positive=True)
    _check(sg, patches, prec, 2, sig, sx, sy, tol, G=2.5, cross=cross)


@CROSS
@pytest.mark.parametrize("n, positive", [(64, True), (128, True), (128, False)], ids=["64", "128", "128signed"])
def test_nested_rough_sampled_fp32(sg, n, positive, cross):
    """Three n^2 levels of independent noise (signed or not), FP32 at 1e-5 on 384
    seeded leaves: the sizes at which a corner-form FP32 sum exceeds the bound."""
    patches = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(n, 3))]
    sig, sx, sy = _fields(patches, 3, positive=positive)
    nleaf = 3 * n * n - 2 * (n * n // 4)
    rng = np.random.Generator(np.random.PCG64(7))
    idx = np.sort(rng.choice(nleaf, 384, replace=False))
    _check(sg, patches, "fp32", 2, sig, sx, sy, 1e-5, target_index=idx, cross=cross)


def _boundary_leaf_index(patches):
    """Indices (in the oracle's leaf order) of the leaves next to every
    coarse/fine boundary: the coarse leaves whose centre is within one coarse
    cell of a refined patch, and the leaves of the refined patch along its edge
    (where target centres lie on source edge lines: the coincident-line form)."""
    leaves = oamr.leaf_cells(oamr.make_patches(patches))
    sel = []
    for k in range(len(leaves["patch"])):
        p = leaves["patch"][k]
        lp, _, _, _, _, h = patches[p]
        xc, yc = leaves["xc"][k], leaves["yc"][k]
        for q, (lq, qnx, qny, qx0, qy0, qh) in enumerate(patches):
            if lq == 0:
                continue
            dx = max(qx0 - xc, xc - (qx0 + qnx * qh), 0.0)
            dy = max(qy0 - yc, yc - (qy0 + qny * qh), 0.0)
            if q == p:
                edge = min(xc - qx0, qx0 + qnx * qh - xc, yc - qy0, qy0 + qny * qh - yc)
                hit = edge < qh
            else:
                hit = lq == lp + 1 and (dx > 0.0 or dy > 0.0) and max(dx, dy) < h
            if hit:
                sel.append(k)
                break
    return np.array(sorted(set(sel)))


@CROSS
@pytest.mark.parametrize("prec, tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_exponential_hierarchy_boundary_leaves(sg, prec, tol, cross):
    """Config-3 hierarchy (three 256^2 levels, exp(-R/0.1), analytic slopes):
    192 seeded leaves among those adjacent to the coarse/fine boundaries, on
    both sides of each, against the plain leaf-pair sum."""
    case = W.exponential_hierarchy(256, 3, 0.1)
    patches = [(lev,) + p for lev, p in enumerate(case["patches"])]
    cand = _boundary_leaf_index(patches)
    assert len(cand) > 3000
    rng = np.random.Generator(np.random.PCG64(32))
    idx = np.sort(rng.choice(cand, 192, replace=False))
    _check(sg, patches, prec, 2, case["sigma"], case["dx"], case["dy"], tol, target_index=idx, cross=cross)


@CROSS
@pytest.mark.parametrize("prec, tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_table10_hierarchy(sg, prec, tol, cross):
    """Fig. 1 / Table 10: two patches per refined level, 28 leaves."""
    sig, sx, sy = _fields(TABLE10, 8, positive=True)
    _check(sg, TABLE10, prec, 2, sig, sx, sy, tol, cross=cross)


@CROSS
@pytest.mark.parametrize("prec, tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_ragged_off_centre_patches(sg, prec, tol, cross):
    """Non-square, off-centre patches whose sizes are not tile multiples."""
    patches = [(0, 37, 29, -1.0, -0.8, 0.05), (1, 22, 14, -0.6, -0.3, 0.025), (1, 6, 8, 0.2, 0.1, 0.025),
               (2, 10, 12, -0.5, -0.25, 0.0125)]
    assert sg.sg_geom_validate(patches) == sg.SG_OK
    sig, sx, sy = W.bumps_on_patches(patches, 17)
    _check(sg, patches, prec, 2, sig, sx, sy, tol, cross=cross)


@CROSS
def test_refinement_invariance_on_gpu(sg, cross):
    """A fine patch carrying the coarse linear reconstruction leaves the force at
    the coarse leaves equal to the uniform coarse force (FP64)."""
    import torch
    n = 16
    nx, ny, x0, y0, h = W.unit_grid(n)
    s, sx, sy = W.random_fields(n, n, seed=21)
    fine = np.zeros((16, 16)), np.zeros((16, 16)), np.zeros((16, 16))
    for J in range(16):
        for I in range(16):
            pj, pi = 4 + J // 2, 4 + I // 2
            fine[0][J, I] = s[pj, pi] + sx[pj, pi] * (I % 2 - 0.5) * h / 2 + sy[pj, pi] * (J % 2 - 0.5) * h / 2
            fine[1][J, I] = sx[pj, pi]
            fine[2][J, I] = sy[pj, pi]
    patches = [(0, nx, ny, x0, y0, h), (1, 16, 16, -0.5, -0.5, h / 2)]
    plan, fx, fy = _run(sg, patches, "fp64", 2, [s, fine[0]], [sx, fine[1]], [sy, fine[2]], cross=cross)
    uni, ux, uy = _run(sg, patches[:1], "fp64", 2, [s], [sx], [sy])
    leaf = np.ones((n, n), bool)
    leaf[4:12, 4:12] = False
    ax = fx[:n * n].reshape(n, n)[leaf]
    ay = fy[:n * n].reshape(n, n)[leaf]
    assert rel_l2(ax, ay, ux.reshape(n, n)[leaf], uy.reshape(n, n)[leaf]) < 1e-12
    plan.close()
    uni.close()
    torch.cuda.synchronize()


@CROSS
@pytest.mark.parametrize("prec, tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_exponential_hierarchy_full_size_sampled(sg, prec, tol, cross):
    """Three 256^2 levels on [-1,1]^2, [-.5,.5]^2, [-.25,.25]^2, exp(-R/0.1),
    analytic slopes: 192 seeded leaf targets vs the plain leaf-pair sum."""
    case = W.exponential_hierarchy(256, 3, 0.1)
    patches = [(lev,) + p for lev, p in enumerate(case["patches"])]
    nleaf = sum(int(m.sum()) for m in case["leaf"])
    rng = np.random.Generator(np.random.PCG64(31))
    idx = np.sort(rng.choice(nleaf, 192, replace=False))
    _check(sg, patches, prec, 2, case["sigma"], case["dx"], case["dy"], tol, target_index=idx, cross=cross)


@CROSS
def test_covered_cells_are_ignored(sg, cross):
    """Garbage in covered cells must not change any leaf result."""
    patches = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(16, 2))]
    sig, sx, sy = _fields(patches, 5, positive=True)
    _, a, b = _run(sg, patches, "fp64", 2, sig, sx, sy, cross=cross)
    sig2 = [x.copy() for x in sig]
    sig2[0][4:12, 4:12] = 1e6
    plan, c, d = _run(sg, patches, "fp64", 2, sig2, sx, sy, cross=cross)
    leaves = oamr.leaf_cells(oamr.make_patches(patches))
    assert np.allclose(gather_leaves(plan, a, leaves), gather_leaves(plan, c, leaves), rtol=1e-13, atol=1e-13)
    plan.close()


def test_levels_equal_direct(sg):
    """The two AMR paths on the same hierarchy agree to FP64 rounding at every leaf."""
    patches = [(0, 40, 40, -1.0, -1.0, 0.05), (1, 24, 32, -0.6, -0.7, 0.025), (2, 16, 20, -0.5, -0.5, 0.0125),
               (3, 12, 8, -0.45, -0.4, 0.00625)]
    assert sg.sg_geom_validate(patches) == sg.SG_OK
    sig, sx, sy = _fields(patches, 41, positive=True)
    p1, a1, b1 = _run(sg, patches, "fp64", 2, sig, sx, sy, cross=1)
    p2, a2, b2 = _run(sg, patches, "fp64", 2, sig, sx, sy, cross=2)
    leaves = oamr.leaf_cells(oamr.make_patches(patches))
    g1 = gather_leaves(p1, a1, leaves), gather_leaves(p1, b1, leaves)
    g2 = gather_leaves(p2, a2, leaves), gather_leaves(p2, b2, leaves)
    assert rel_l2(g2[0], g2[1], g1[0], g1[1]) < 1e-12
    assert p2.info["cross_pairs"] == 0 and p1.info["cross_pairs"] > 0
    p1.close()
    p2.close()


def test_levels_mode_limits(sg):
    """Level convolutions take finest-lattice extents up to 4096 cells (FP32) or
    2048 (FP64); beyond, SG_CROSS_LEVELS is refused and SG_CROSS_AUTO falls back
    to the direct sum."""
    big = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(1536, 3))]  # 6144 finest cells
    with pytest.raises(sg.SgError) as e:
        sg.Plan(big, cross_mode=sg.SG_CROSS_LEVELS)
    assert e.value.status == sg.SG_EINVAL and "level convolutions" in str(e.value)
    plan = sg.Plan(big, cross_mode=sg.SG_CROSS_AUTO)
    assert plan.info["cross_mode"] == sg.SG_CROSS_DIRECT
    plan.close()
    mid = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(768, 3))]  # 3072 finest cells
    with pytest.raises(sg.SgError):
        sg.Plan(mid, precision="fp64", cross_mode=sg.SG_CROSS_LEVELS)
    plan = sg.Plan(mid, precision="fp32", cross_mode=sg.SG_CROSS_AUTO)
    assert plan.info["cross_mode"] == sg.SG_CROSS_LEVELS and plan.info["max_pad"] == 8192
    plan.close()


def test_levels_8192_four_levels_sampled(sg):
    """Four nested 512^2 levels (finest extent 4096, 8192-point transforms),
    exponential disk, FP32: 96 sampled leaves against the plain leaf-pair sum."""
    patches = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(512, 4))]
    sig, sx, sy = [], [], []
    for p in patches:
        X, Y = W.cell_centres(*p[1:])
        a, b, c = W.exponential_sigma(X, Y, 0.1)
        sig.append(a)
        sx.append(b)
        sy.append(c)
    nleaf = 3 * (512 * 512 - 256 * 256) + 512 * 512
    rng = np.random.Generator(np.random.PCG64(44))
    idx = np.sort(rng.choice(nleaf, 96, replace=False))
    _check(sg, patches, "fp32", 2, sig, sx, sy, 1e-5, target_index=idx, cross=2)


def test_levels_4096_fp64_sampled(sg):
    """Three nested 512^2 levels (finest extent 2048, 4096-point transforms, the
    FP64 limit), exponential disk, FP64: 64 sampled leaves on every level against
    the plain leaf-pair sum (coarse targets take the folded inverse transforms)."""
    patches = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(512, 3))]
    sig, sx, sy = [], [], []
    for p in patches:
        X, Y = W.cell_centres(*p[1:])
        a, b, c = W.exponential_sigma(X, Y, 0.1)
        sig.append(a)
        sx.append(b)
        sy.append(c)
    n0 = 512 * 512 - 256 * 256
    rng = np.random.Generator(np.random.PCG64(45))
    idx = np.sort(np.concatenate([rng.choice(n0, 64, replace=False), n0 + rng.choice(n0, 64, replace=False),
                                  2 * n0 + rng.choice(512 * 512, 64, replace=False)]))
    _check(sg, patches, "fp64", 2, sig, sx, sy, 1e-11, target_index=idx, cross=2)


CENTRAL_CASES = {
    "nested": [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(16, 3))],
    "ragged": [(0, 37, 29, -1.0, -0.8, 0.05), (1, 22, 14, -0.6, -0.3, 0.025), (1, 6, 8, 0.2, 0.1, 0.025),
               (2, 10, 12, -0.5, -0.25, 0.0125)],
    "table10": TABLE10,
}


@CROSS
@pytest.mark.parametrize("prec, tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("case", sorted(CENTRAL_CASES))
def test_central_slopes_on_hierarchies(sg, case, prec, tol, cross):
    """SG_SLOPES_CENTRAL on a hierarchy: the neighbour-leaf slope rule computed
    on the GPU, against the oracle's rule (oracle.slopes) fed to the plain
    leaf-pair sum."""
    from oracle import slopes as S
    patches = CENTRAL_CASES[case]
    sig, _, _ = W.bumps_on_patches(patches, 23)
    dt = np.float64 if prec == "fp64" else np.float32
    plan, fx, fy = _run(sg, patches, prec, sg.SG_SLOPES_CENTRAL, sig, None, None, cross=cross)
    P = oamr.make_patches(patches)
    s64 = [np.asarray(a, dt).astype(np.float64) for a in sig]
    ox, oy = S.patch_neighbour_slopes(P, s64)
    leaves, rx, ry = oamr.amr_direct_force(P, s64, ox, oy)
    err = rel_l2(gather_leaves(plan, fx, leaves), gather_leaves(plan, fy, leaves), rx, ry)
    plan.close()
    print("rel L2 %s cross=%d central: %.3e (tolerance %.0e)" % (prec, cross, err, tol))
    assert err < tol


def test_central_slopes_fp32_config3_sampled(sg):
    """The config-3 hierarchy (three 256^2 levels, exp(-R/0.1)) with slopes from
    the neighbour-leaf rule, FP32 level convolutions: 128 leaves next to the
    coarse/fine boundaries and 64 elsewhere against the oracle."""
    from oracle import slopes as S
    case = W.exponential_hierarchy(256, 3, 0.1)
    patches = [(lev,) + p for lev, p in enumerate(case["patches"])]
    plan, fx, fy = _run(sg, patches, "fp32", sg.SG_SLOPES_CENTRAL, case["sigma"], None, None)
    P = oamr.make_patches(patches)
    s64 = [np.asarray(a, np.float32).astype(np.float64) for a in case["sigma"]]
    ox, oy = S.patch_neighbour_slopes(P, s64)
    cand = _boundary_leaf_index(patches)
    nleaf = sum(int(m.sum()) for m in case["leaf"])
    rng = np.random.Generator(np.random.PCG64(33))
    idx = np.unique(np.concatenate([rng.choice(cand, 128, replace=False), rng.choice(nleaf, 64, replace=False)]))
    leaves, rx, ry = oamr.amr_direct_force(P, s64, ox, oy, target_index=idx)
    leaves = {k: v[idx] for k, v in leaves.items()}
    err = rel_l2(gather_leaves(plan, fx, leaves), gather_leaves(plan, fy, leaves), rx, ry)
    plan.close()
    print("rel L2 fp32 central config 3: %.3e" % err)
    assert err < 1e-5


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_plan_autotune_direct_sum(sg, prec):
    """sg_plan_autotune picks the direct sum's split and far-field grid among
    its candidates; the solve afterwards agrees with the solve before to FP64
    rounding of the regrouped partial sums (FP32 plans: to FP32 rounding) and
    still matches the oracle."""
    import torch
    patches = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(64, 3))]
    sig, sx, sy = _fields(patches, 9, positive=True)
    dt = np.float64 if prec == "fp64" else np.float32
    plan, fx0, fy0 = _run(sg, patches, prec, 2, sig, sx, sy, cross=1)
    ns0, fg0 = sg.sg_plan_direct_shape(plan.handle)
    ms = sg.sg_plan_autotune(plan.handle, 3)
    ns1, fg1 = sg.sg_plan_direct_shape(plan.handle)
    assert ms > 0 and ns1 in (ns0, ns0 // 2, ns0 // 4) and ns1 >= 1
    if prec == "fp32":
        nsm = torch.cuda.get_device_properties(0).multi_processor_count
        assert 1 <= fg1 <= 8 * nsm
    fx, fy = plan.force(concat_dev(sig, dt), concat_dev(sx, dt), concat_dev(sy, dt))
    torch.cuda.synchronize()
    fx, fy = fx.cpu().numpy(), fy.cpu().numpy()
    scale = max(np.abs(fx0).max(), np.abs(fy0).max())
    tol = 1e-13 if prec == "fp64" else 1e-6
    assert np.abs(fx - fx0).max() <= tol * scale and np.abs(fy - fy0).max() <= tol * scale
    plan.close()
