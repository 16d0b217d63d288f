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
