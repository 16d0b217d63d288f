"""Graph-captured batches of uneven solves equal sg_force bit for bit."""
import numpy as np
import pytest

from paper_2001_02765_gb300 import workloads as W
from tests._lib import concat_dev, ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available()
    ensure_built()
    from paper_2001_02765_gb300 import sg as mod
    return mod


def test_batch_equals_individual_solves(sg):
    import torch
    ns, a, amp = W.batch_sizes(count=12, lo=20, hi=300, seed=4)
    members = []
    for k, n in enumerate(ns):
        patches = [(0,) + W.unit_grid(int(n))]
        X, Y = W.cell_centres(*patches[0][1:])
        s, sx, sy = W.spiral_sigma(X, Y, a[k], amp[k])
        members.append((patches, sg.SG_SLOPES_CENTRAL, [s], None, None))
    amr = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(32, 3))]
    sig, sx, sy = W.bumps_on_patches(amr, seed=9)
    members.append((amr, sg.SG_SLOPES_CALLER, sig, sx, sy))
    plans, ins, outs, refs = [], [], [], []
    for patches, mode, s, sx, sy in members:
        plan = sg.Plan(patches, precision="fp32", slope_mode=mode)
        i = (concat_dev(s, np.float32), concat_dev(sx, np.float32) if sx else None,
             concat_dev(sy, np.float32) if sy else None)
        rx, ry = plan.force(*i)
        torch.cuda.synchronize()
        refs.append((rx.clone(), ry.clone()))
        plans.append(plan)
        ins.append(i)
        outs.append((torch.full_like(i[0], float("nan")), torch.full_like(i[0], float("nan"))))
    ptr = lambda t: t.data_ptr() if t is not None else 0
    batch = sg.sg_batch_create([p.handle for p in plans], [ptr(i[0]) for i in ins], [ptr(i[1]) for i in ins],
                               [ptr(i[2]) for i in ins], [ptr(o[0]) for o in outs], [ptr(o[1]) for o in outs])
    try:
        for _ in range(2):
            sg.sg_batch_launch(batch, torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            for o, r in zip(outs, refs):
                assert torch.equal(o[0], r[0]) and torch.equal(o[1], r[1])
            for o in outs:
                o[0].fill_(float("nan"))
                o[1].fill_(float("nan"))
    finally:
        sg.sg_batch_destroy(batch)
        for p in plans:
            p.close()


def test_batch_argument_errors(sg):
    with pytest.raises(sg.SgError) as e:
        sg.sg_batch_create([0], [0], [0], [0], [0], [0])
    assert e.value.status == sg.SG_EINVAL


@pytest.mark.parametrize("layout", ["persistent", "grouped", "auto"])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_batch_groups_equal_individual_solves(sg, prec, mode, layout):
    """Single-patch members of any padded length up to 2048 run in one
    persistent kernel launch, or as one launch per pass per group of equal
    lengths, or whichever of the two replays faster (slope modes none,
    central, caller; both precisions); results equal sg_force bit for bit,
    including members whose row counts differ, on two replays in a row."""
    import torch
    dt = np.float64 if prec == "fp64" else np.float32
    ns = [33, 40, 47, 64, 20, 30, 90, 100, 128, 17]  # padded lengths 128, 128, 128, 128, 64, 64, 256, 256, 256, 64
    rng = np.random.Generator(np.random.PCG64(40 + mode))
    plans, ins, outs, refs = [], [], [], []
    for n in ns:
        nx, ny = n, max(1, n - int(rng.integers(0, 8)))  # ragged rows
        plan = sg.Plan([(0, nx, ny, -1.0, -1.0, 2.0 / n)], precision=prec, slope_mode=mode)
        s, sx, sy = W.random_fields(ny, nx, seed=int(rng.integers(0, 1 << 30)))
        i = (concat_dev([s], dt), concat_dev([sx], dt) if mode == 2 else None,
             concat_dev([sy], dt) if mode == 2 else None)
        rx, ry = plan.force(*i)
        torch.cuda.synchronize()
        refs.append((rx.clone(), ry.clone()))
        plans.append(plan)
        ins.append(i)
        outs.append((torch.full_like(i[0], float("nan")), torch.full_like(i[0], float("nan"))))
    ptr = lambda t: t.data_ptr() if t is not None else 0
    want = {"persistent": sg.SG_BATCH_PERSISTENT, "grouped": sg.SG_BATCH_GROUPED, "auto": sg.SG_BATCH_AUTO}[layout]
    batch = sg.sg_batch_create([p.handle for p in plans], [ptr(i[0]) for i in ins], [ptr(i[1]) for i in ins],
                               [ptr(i[2]) for i in ins], [ptr(o[0]) for o in outs], [ptr(o[1]) for o in outs],
                               mode=want)
    try:
        got, ms_p, ms_g = sg.sg_batch_layout(batch)
        if layout == "auto":
            assert got in (sg.SG_BATCH_PERSISTENT, sg.SG_BATCH_GROUPED) and ms_p > 0 and ms_g > 0
            assert (got == sg.SG_BATCH_PERSISTENT) == (ms_p <= ms_g)
            for o in outs:  # the timing replays ran on the bound buffers
                o[0].fill_(float("nan"))
                o[1].fill_(float("nan"))
        else:
            assert got == want and ms_p == 0 and ms_g == 0
        # persistent: one kernel; grouped: one launch per pass of each group of
        # equal padded lengths (and a solve's launches for a member alone)
        nl = sg.sg_batch_launches(batch)
        assert nl == 1 if got == sg.SG_BATCH_PERSISTENT else nl >= (4 if mode == 1 else 3)
        for _ in range(2):
            sg.sg_batch_launch(batch, torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            for o, r in zip(outs, refs):
                assert torch.equal(o[0], r[0]) and torch.equal(o[1], r[1])
                o[0].fill_(float("nan"))
                o[1].fill_(float("nan"))
        assert sg.sg_batch_check_error(batch) == sg.SG_OK
    finally:
        sg.sg_batch_destroy(batch)
        for p in plans:
            p.close()
