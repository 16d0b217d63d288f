"""Bounded waits: a wait that runs out is reported, and the GPU stays usable.

Kernels that wait for bulk copies into shared memory (the column passes'
kernel spectra; the FP32 direct sum's source tiles) give up after the plan's
wait limit, set the workspace's device error word, wait for their copies in
flight with the default limit and return. A wait limit of 0 attempts makes the
first wait give up at once, deterministically, with no copy left in flight and
no fault: these tests use it to check that the status reaches the caller
through sg_plan_check_error, a server request's result and a batch's check,
and that solves with the default limit afterwards are correct again."""
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


def _uniform(sg, n=64):
    patches = [(0,) + W.unit_grid(n)]
    sig, sx, sy = W.bumps_on_patches(patches, seed=5)
    plan = sg.Plan(patches, precision="fp32", slope_mode=sg.SG_SLOPES_CALLER)
    return plan, [concat_dev(a, np.float32) for a in (sig, sx, sy)]


def test_plan_wait_runs_out_and_recovers(sg):
    import torch
    plan, ins = _uniform(sg)
    ref = [t.clone() for t in plan.force(*ins)]
    torch.cuda.synchronize()
    assert sg.sg_plan_check_error(plan.handle) == sg.SG_OK
    sg.sg_plan_set_wait_limit(plan.handle, 0)
    plan.force(*ins)
    assert sg.sg_plan_check_error(plan.handle) == sg.SG_ETIMEOUT
    assert sg.sg_plan_check_error(plan.handle) == sg.SG_OK  # the check clears the word
    sg.sg_plan_set_wait_limit(plan.handle, -1)
    out = plan.force(*ins)
    assert sg.sg_plan_check_error(plan.handle) == sg.SG_OK
    assert torch.equal(out[0], ref[0]) and torch.equal(out[1], ref[1])
    with pytest.raises(sg.SgError):
        sg.sg_plan_set_wait_limit(plan.handle, -2)
    plan.close()


def test_host_entry_reports_wait_run_out(sg):
    """The host entry points read the error word copied after the solve: a
    wait that ran out raises SG_ETIMEOUT from sg_force_host and from
    sg_plan_wait, once, and the next solve is correct."""
    import torch
    n = 64
    patches = [(0,) + W.unit_grid(n)]
    sig, _, _ = W.bumps_on_patches(patches, seed=6)
    plan = sg.Plan(patches, precision="fp32", slope_mode=sg.SG_SLOPES_CENTRAL)
    hs = torch.from_numpy(np.ascontiguousarray(sig[0], np.float32).ravel()).pin_memory()
    hfx = torch.empty(n * n, dtype=torch.float32).pin_memory()
    hfy = torch.empty(n * n, dtype=torch.float32).pin_memory()
    plan.force_host(hs, None, None, hfx, hfy)
    ref = (hfx.clone(), hfy.clone())
    sg.sg_plan_set_wait_limit(plan.handle, 0)
    with pytest.raises(sg.SgError) as e:
        plan.force_host(hs, None, None, hfx, hfy)
    assert e.value.status == sg.SG_ETIMEOUT
    plan.force_host_async(hs, None, None, hfx, hfy)
    with pytest.raises(sg.SgError) as e:
        plan.wait()
    assert e.value.status == sg.SG_ETIMEOUT
    sg.sg_plan_set_wait_limit(plan.handle, -1)
    plan.force_host_async(hs, None, None, hfx, hfy)
    plan.wait()
    assert torch.equal(hfx, ref[0]) and torch.equal(hfy, ref[1])
    plan.close()


def test_direct_sum_wait_runs_out_and_recovers(sg):
    """The persistent far-field launch of an FP32 hierarchy on the direct path."""
    import torch
    patches = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(32, 3))]
    sig, sx, sy = W.bumps_on_patches(patches, seed=6)
    plan = sg.Plan(patches, precision="fp32", slope_mode=sg.SG_SLOPES_CALLER, cross_mode=sg.SG_CROSS_DIRECT)
    ins = [concat_dev(a, np.float32) for a in (sig, sx, sy)]
    ref = [t.clone() for t in plan.force(*ins)]
    torch.cuda.synchronize()
    sg.sg_plan_set_wait_limit(plan.handle, 0)
    plan.force(*ins)
    assert sg.sg_plan_check_error(plan.handle) == sg.SG_ETIMEOUT
    sg.sg_plan_set_wait_limit(plan.handle, -1)
    out = plan.force(*ins)
    assert sg.sg_plan_check_error(plan.handle) == sg.SG_OK
    assert torch.equal(out[0], ref[0]) and torch.equal(out[1], ref[1])
    plan.close()


def test_server_reports_wait_run_out(sg):
    import torch
    plan, ins = _uniform(sg)
    good, gins = _uniform(sg, 96)
    server = sg.sg_server_create(0, 2)
    try:
        sg.sg_plan_set_wait_limit(plan.handle, 0)
        fx, fy = torch.empty_like(ins[0]), torch.empty_like(ins[0])
        t = sg.sg_submit(server, plan.handle, *(a.data_ptr() for a in ins), fx.data_ptr(), fy.data_ptr())
        gx, gy = torch.empty_like(gins[0]), torch.empty_like(gins[0])
        t2 = sg.sg_submit(server, good.handle, *(a.data_ptr() for a in gins), gx.data_ptr(), gy.data_ptr())
        st, res, _ = sg.sg_wait(server, t, 10000.0)
        assert st == sg.SG_OK and res == sg.SG_ETIMEOUT
        st, res, _ = sg.sg_wait(server, t2, 10000.0)
        assert st == sg.SG_OK and res == sg.SG_OK
        rx, ry = good.force(*gins)
        torch.cuda.synchronize()
        assert torch.equal(gx, rx) and torch.equal(gy, ry)
        stats = sg.sg_server_get_stats(server)
        assert stats["failed"] == 1 and stats["completed"] == 1
    finally:
        sg.sg_server_destroy(server)
        plan.close()
        good.close()


def test_batch_reports_wait_run_out(sg):
    import torch
    plan, ins = _uniform(sg)
    sg.sg_plan_set_wait_limit(plan.handle, 0)
    fx, fy = torch.empty_like(ins[0]), torch.empty_like(ins[0])
    batch = sg.sg_batch_create([plan.handle], [ins[0].data_ptr()], [ins[1].data_ptr()], [ins[2].data_ptr()],
                               [fx.data_ptr()], [fy.data_ptr()])
    try:
        sg.sg_batch_launch(batch, torch.cuda.current_stream().cuda_stream)
        assert sg.sg_batch_check_error(batch) == sg.SG_ETIMEOUT
        assert sg.sg_batch_check_error(batch) == sg.SG_OK
    finally:
        sg.sg_batch_destroy(batch)
        plan.close()
