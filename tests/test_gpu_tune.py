"""Launch-shape tuning: every compiled shape of every uniform pass gives the
same result bit for bit (only the grouping of sequences into CTAs changes), and
the autotuner keeps compiled candidates."""
import itertools

import numpy as np
import pytest

from paper_2001_02765_gb300 import workloads as W
from tests._lib import ensure_built, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available()
    ensure_built()
    from paper_2001_02765_gb300 import sg as mod
    yield mod
    for prec in (mod.SG_FP32, mod.SG_FP64):
        p = 64
        while p <= 4096:
            mod.sg_tune_set(prec, p, [0, 0, 0, 0])
            p *= 2


def _candidates(d):
    return sorted({v for v in (d // 2, d, 2 * d) if v >= 1})


@pytest.mark.parametrize("n, prec", [(100, "fp32"), (300, "fp32"), (700, "fp32"), (300, "fp64")])
@pytest.mark.parametrize("mode", [1, 2])
def test_every_shape_gives_identical_results(sg, n, prec, mode):
    import torch
    precision = sg.SG_FP32 if prec == "fp32" else sg.SG_FP64
    dt = np.float32 if prec == "fp32" else np.float64
    nx, ny, x0, y0, h = W.unit_grid(n)
    s, sx, sy = W.random_fields(n, n, seed=n)
    plan = sg.Plan([(0, nx, ny, x0, y0, h)], precision=prec, slope_mode=mode)
    pad = plan.info["max_pad"]
    a, b, c = to_dev(s, dt), to_dev(sx, dt), to_dev(sy, dt)
    ref = [t.clone() for t in plan.force(a, b, c)]
    torch.cuda.synchronize()
    d = sg.sg_tune_get(precision, pad)
    knobs = ["row_fwd", "row_inv", "col_central" if mode == 1 else "col"]
    tried = 0
    for combo in itertools.product(*[_candidates(d[k]) for k in knobs]):
        shape = dict(zip(knobs, combo))
        try:
            sg.sg_tune_set(precision, pad, shape)
        except sg.SgError:
            continue  # not a compiled candidate at this length
        out = plan.force(a, b, c)
        torch.cuda.synchronize()
        assert torch.equal(out[0], ref[0]) and torch.equal(out[1], ref[1]), shape
        tried += 1
    sg.sg_tune_set(precision, pad, [0, 0, 0, 0])
    plan.close()
    assert tried >= 4


def test_autotune_keeps_candidates(sg):
    res = sg.sg_autotune(sg.SG_FP32, 64, 512, reps=3)
    assert sorted(res) == [64, 128, 256, 512]
    for pad, (shape, ms) in res.items():
        assert ms > 0
        for k, v in shape.items():
            base = {"row_fwd": 4096 // pad if pad < 4096 else 2, "row_inv": 4096 // pad,
                    "col": 2048 // pad, "col_central": 2048 // pad}[k]
            assert v in (base // 2, base, 2 * base), (pad, k, v)
