"""The request server: continuous batching, admission by device-memory budget,
and host-side failure paths (no GPU fault is provoked anywhere).

A result must be bit-for-bit the same alone (sg_force, one at a time) and in a
mix of overlapping requests on several streams."""
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


def _cases():
    out = []
    for n in (64, 128, 250):
        out.append(("u%d" % n, [(0,) + W.unit_grid(n)]))
    out.append(("rect", [(0, 200, 96, -1.0, -0.5, 0.01)]))
    out.append(("amr2", [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(32, 2))]))
    out.append(("t10", [(0, 4, 4, 0.0, 0.0, 0.25), (1, 2, 2, 0.25, 0.25, 0.125), (1, 2, 2, 0.5, 0.5, 0.125),
                        (2, 2, 2, 0.25, 0.375, 0.0625), (2, 2, 2, 0.375, 0.25, 0.0625)]))
    return out


def _prepare(sg, precision="fp32"):
    import torch
    dt = np.float32 if precision == "fp32" else np.float64
    reqs = []
    for k, (name, patches) in enumerate(_cases()):
        plan = sg.Plan(patches, precision=precision, slope_mode=sg.SG_SLOPES_CALLER)
        sig, sx, sy = W.bumps_on_patches(patches, seed=100 + k)
        ins = [concat_dev(a, dt) for a in (sig, sx, sy)]
        fx, fy = plan.force(*ins)
        torch.cuda.synchronize()
        reqs.append(dict(name=name, plan=plan, ins=ins, ref=(fx.clone(), fy.clone())))
    return reqs


def test_mixed_results_equal_solo_results_bitwise(sg):
    import torch
    reqs = _prepare(sg)
    server = sg.sg_server_create(0, 4)
    try:
        outs = []
        for rnd in range(3):
            for r in reqs:
                fx = torch.full_like(r["ins"][0], float("nan"))
                fy = torch.full_like(r["ins"][0], float("nan"))
                t = sg.sg_submit(server, r["plan"].handle, *(a.data_ptr() for a in r["ins"]), fx.data_ptr(),
                                 fy.data_ptr())
                outs.append((r, t, fx, fy))
        for r, t, fx, fy in outs:
            st, res, lat = sg.sg_wait(server, t, 60000.0)
            assert st == sg.SG_OK and res == sg.SG_OK and lat > 0.0, (r["name"], st, res)
            assert torch.equal(fx, r["ref"][0]) and torch.equal(fy, r["ref"][1]), r["name"]
        stats = sg.sg_server_get_stats(server)
        assert stats["completed"] == len(outs) and stats["failed"] == 0
        assert stats["latency_count"] == len(outs) and stats["latency_p99_ms"] >= stats["latency_p50_ms"] > 0
        assert stats["queued"] == 0 and stats["running"] == 0 and stats["bytes_in_use"] == 0
    finally:
        sg.sg_server_destroy(server)
        for r in reqs:
            r["plan"].close()


def test_admission_respects_budget(sg):
    import torch
    reqs = _prepare(sg)
    big = max(reqs, key=lambda r: r["plan"].info["scratch_bytes"])
    budget = int(1.5 * big["plan"].info["scratch_bytes"])  # at most one copy of the largest in flight
    server = sg.sg_server_create(budget, 8)
    try:
        outs = []
        for _ in range(4):
            fx = torch.empty_like(big["ins"][0])
            fy = torch.empty_like(big["ins"][0])
            t = sg.sg_submit(server, big["plan"].handle, *(a.data_ptr() for a in big["ins"]), fx.data_ptr(),
                             fy.data_ptr())
            outs.append((t, fx, fy))
        for t, fx, fy in outs:
            st, res, _ = sg.sg_wait(server, t, 60000.0)
            assert st == sg.SG_OK and res == sg.SG_OK
            assert torch.equal(fx, big["ref"][0])
        stats = sg.sg_server_get_stats(server)
        assert 0 < stats["peak_bytes"] <= budget
        # a request whose workspace alone exceeds the budget is rejected at submit
        small = sg.sg_server_create(1024, 2)
        try:
            with pytest.raises(sg.SgError) as e:
                sg.sg_submit(small, big["plan"].handle, *(a.data_ptr() for a in big["ins"]), 1, 1)
            assert e.value.status == sg.SG_EBUDGET
            assert sg.sg_server_get_stats(small)["rejected"] == 1
        finally:
            sg.sg_server_destroy(small)
    finally:
        sg.sg_server_destroy(server)
        for r in reqs:
            r["plan"].close()


def test_poll_cancel_timeout_and_unknown_tickets(sg):
    import torch
    n = 1024
    plan = sg.Plan([(0,) + W.unit_grid(n)], precision="fp64", slope_mode=sg.SG_SLOPES_CENTRAL)
    s = torch.rand(n * n, dtype=torch.float64, device="cuda")
    outs = [(torch.empty_like(s), torch.empty_like(s)) for _ in range(3)]
    server = sg.sg_server_create(0, 1)  # one slot: the second and third requests queue
    sg.sg_server_set_group_limit(server, 1)  # and are not admitted together with the first
    try:
        assert sg.sg_poll(server, 12345)[0] == sg.SG_ENOTFOUND
        t1 = sg.sg_submit(server, plan.handle, s.data_ptr(), 0, 0, outs[0][0].data_ptr(), outs[0][1].data_ptr())
        t2 = sg.sg_submit(server, plan.handle, s.data_ptr(), 0, 0, outs[1][0].data_ptr(), outs[1][1].data_ptr())
        t3 = sg.sg_submit(server, plan.handle, s.data_ptr(), 0, 0, outs[2][0].data_ptr(), outs[2][1].data_ptr())
        # t3 is still queued behind t1 (running) and t2: cancel it
        assert sg.sg_cancel(server, t3) == sg.SG_OK
        st, res, _ = sg.sg_poll(server, t3)
        assert st == sg.SG_OK and res == sg.SG_ECANCELLED
        assert sg.sg_poll(server, t3)[0] == sg.SG_ENOTFOUND  # retired
        # a zero timeout on a queued or running request times out without side effects
        st, _, _ = sg.sg_wait(server, t2, 0.0)
        assert st in (sg.SG_ETIMEOUT, sg.SG_OK)
        if st == sg.SG_ETIMEOUT:
            st, res, _ = sg.sg_wait(server, t2, 60000.0)
            assert st == sg.SG_OK and res == sg.SG_OK
        st, res, _ = sg.sg_wait(server, t1, 60000.0)
        assert st == sg.SG_OK and res == sg.SG_OK
        assert torch.equal(outs[0][0], outs[1][0])
        stats = sg.sg_server_get_stats(server)
        assert stats["cancelled"] == 1 and stats["completed"] == 2
        # invalid submissions fail on the host
        with pytest.raises(sg.SgError) as e:
            sg.sg_submit(server, plan.handle, 0, 0, 0, 0, 0)
        assert e.value.status == sg.SG_EINVAL
    finally:
        sg.sg_server_destroy(server)
        plan.close()


def test_destroy_cancels_queued_requests(sg):
    import torch
    n = 1024
    plan = sg.Plan([(0,) + W.unit_grid(n)], precision="fp64", slope_mode=sg.SG_SLOPES_CENTRAL)
    s = torch.rand(n * n, dtype=torch.float64, device="cuda")
    f = [torch.empty_like(s) for _ in range(8)]
    server = sg.sg_server_create(0, 1)
    for k in range(4):
        sg.sg_submit(server, plan.handle, s.data_ptr(), 0, 0, f[2 * k].data_ptr(), f[2 * k + 1].data_ptr())
    sg.sg_server_destroy(server)  # waits for the running one, cancels the rest
    torch.cuda.synchronize()
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_queued_requests_of_one_length_run_grouped(sg, prec):
    """Requests of one padded length queued behind a long one are admitted
    together (one grouped launch per pass); each result equals its solo
    sg_force bit for bit, with ragged row counts and two slope modes; with a
    group limit of 1 nothing is grouped."""
    import torch
    dt = np.float32 if prec == "fp32" else np.float64
    big = sg.Plan([(0,) + W.unit_grid(1024)], precision=prec, slope_mode=sg.SG_SLOPES_CENTRAL)
    bs = concat_dev([np.random.Generator(np.random.PCG64(3)).uniform(0, 1, (1024, 1024))], dt)
    shapes = [(100, 100), (120, 96), (110, 90)]  # padded 256 x 256 each
    reqs = []
    for k in range(9):
        nx, ny = shapes[k % 3]
        mode = sg.SG_SLOPES_CALLER if k % 2 == 0 else sg.SG_SLOPES_CENTRAL
        plan = sg.Plan([(0, nx, ny, -1.0, -1.0, 2.0 / nx)], precision=prec, slope_mode=mode)
        s, sx, sy = W.random_fields(ny, nx, seed=60 + k)
        ins = [concat_dev([a], dt) for a in (s, sx, sy)]
        if mode != sg.SG_SLOPES_CALLER:
            ins = [ins[0], None, None]
        fx, fy = plan.force(*ins)
        torch.cuda.synchronize()
        reqs.append((plan, ins, fx.clone(), fy.clone()))
    ptr = lambda t: 0 if t is None else t.data_ptr()
    for limit in (16, 1):
        server = sg.sg_server_create(0, 1)  # one slot: everything queues behind the first request
        try:
            sg.sg_server_set_group_limit(server, limit)
            bfx, bfy = torch.empty_like(bs), torch.empty_like(bs)
            tickets = [sg.sg_submit(server, big.handle, bs.data_ptr(), 0, 0, bfx.data_ptr(), bfy.data_ptr())]
            outs = []
            for plan, ins, rx, ry in reqs:
                fx = torch.full_like(ins[0], float("nan"))
                fy = torch.full_like(ins[0], float("nan"))
                tickets.append(sg.sg_submit(server, plan.handle, *(ptr(a) for a in ins), fx.data_ptr(), fy.data_ptr()))
                outs.append((fx, fy, rx, ry))
            for t in tickets:
                st, res, _ = sg.sg_wait(server, t, 60000.0)
                assert st == sg.SG_OK and res == sg.SG_OK
            for fx, fy, rx, ry in outs:
                assert torch.equal(fx, rx) and torch.equal(fy, ry)
            stats = sg.sg_server_get_stats(server)
            if limit == 1:
                assert stats["groups_started"] == 0
            else:
                # the caller-slope and central-slope requests form one group each
                assert stats["groups_started"] >= 2 and stats["grouped_requests"] >= 4
            assert stats["bytes_in_use"] == 0 and stats["running"] == 0
        finally:
            sg.sg_server_destroy(server)
    for plan, *_ in reqs:
        plan.close()
    big.close()
