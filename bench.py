"""Benchmark of the thin-disk self-gravity force solve on GB300.

Workload (one "step" = one force solve through the C ABI): the uniform
1024 x 1024 grid on [-1,1]^2 with the two-armed spiral Kuzmin disk
(a = 0.1, amplitude 0.1, pitch 15 deg) plus seeded uniform noise +-1e-3,
FP32 fields and transforms, FP64-built kernel spectra, central-difference
slopes, zero padding to 2048 x 2048. The L2 cache is flushed (a 512 MB
write) before every timed solve; each solve is timed with CUDA events on the
stream it runs on.

Reported: value = solves/s (whole job, N ranks), p50/p99 latency per solve,
target-cells/s, the plain FP64 per-solve path on the same GPU, the relative L2
force error of the FP32 path against the FP64 path, a roofline entry for the
dominant kernel, the end-to-end rate through the host-buffer entry point, and
the FP64 CPU oracle timed on the host cores on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload amr3]

Multi-GPU (torchrun): every rank solves its own independent stream of
problems (replicas, no collective on the data path); the slowest rank's time
sets the rate.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "force solves/sec and target-cells/sec (p50/p99 latency) vs FP64 plain, ≤1e-5 rel err"
METRIC_POTENTIAL = "potential solves/sec and target-cells/sec (p50/p99 latency) vs FP64 plain, ≤1e-5 rel err"
L2_FLUSH_BYTES = 512 << 20


_ALU = {}


def _alu_peaks():
    """Pipe throughput of this GPU measured by the library (sg_alu_peak: every
    SM, 8 CTAs x 256 threads each, independent chains, best of five launches):
    FP32 and FP64 FMA in TFLOP/s, FP32 base-2 logarithm in 1e12 results/s.
    Measured once per process."""
    if not _ALU:
        from paper_2001_02765_gb300 import sg
        _ALU["fp32_tflops"] = sg.sg_alu_peak(sg.SG_PEAK_FP32_FMA) / 1e12
        _ALU["fp64_tflops"] = sg.sg_alu_peak(sg.SG_PEAK_FP64_FMA) / 1e12
        _ALU["lg2_tops"] = sg.sg_alu_peak(sg.SG_PEAK_FP32_LG2) / 1e12
    return dict(_ALU)


def _peaks():
    """(HBM GB/s, its source, FP32 non-tensor TFLOP/s, its source). HBM: the
    driver's measured copy bandwidth (MEASURED_PEAKS.json); FP32: measured on
    this GPU by sg_alu_peak."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        hbm, src = float(p["hbm_gbs"]), "measured"
    except Exception:
        hbm, src = 6800.0, "fallback"
    alu = _alu_peaks()
    return hbm, src, alu["fp32_tflops"], "measured (sg_alu_peak: FP32 FMA on every SM, best of 5)"


class ClockSampler:
    """nvidia-smi clock / throttle sampling every 20 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.time()
            while not self.rows and time.time() - t0 < 5.0:  # wait for the first sample
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def job_rate(local_ms, local_solves):
    """Whole-job rate of independent replicas: solves summed over ranks divided
    by the slowest rank's time (max over ranks). Uses the initialised
    torch.distributed group when there is one (any backend)."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(local_ms)], dtype=torch.float64, device=dev)
        n = torch.tensor([float(local_solves)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
        local_ms, local_solves = float(t.item()), float(n.item())
    return local_solves / (local_ms / 1e3), local_ms, local_solves


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------- workloads --

def workload_spiral():
    from paper_2001_02765_gb300 import workloads as W
    case = W.spiral_1024(seed=2)
    nx, ny, x0, y0, h = case["geom"]
    return {
        "name": "uniform 1024x1024 spiral Kuzmin disk (a=0.1, m=2 amplitude 0.1, pitch 15 deg, noise 1e-3), "
                "central slopes, FFT on 2048x2048 padded grid",
        "patches": [(0, nx, ny, x0, y0, h)], "slope_mode": 1,
        "sigma": case["sigma"].ravel(), "dx": None, "dy": None, "targets": nx * ny,
        "config": {"workload": "spiral_1024_fft", "grid": [nx, ny], "padded": [2048, 2048], "precision": "fp32",
                   "slopes": "central", "l2": "flushed before every solve (512 MB write)"},
    }


def workload_amr3():
    from paper_2001_02765_gb300 import workloads as W
    case = W.exponential_hierarchy(256, 3, 0.1)
    patches = [(lev,) + p for lev, p in enumerate(case["patches"])]
    cat = lambda a: np.concatenate([x.ravel() for x in a])
    nleaf = int(sum(m.sum() for m in case["leaf"]))
    return {
        "name": "AMR 3 levels x 256^2 (ratio 2, centred nested), exponential disk exp(-R/0.1), caller slopes",
        "patches": patches, "slope_mode": 2, "sigma": cat(case["sigma"]), "dx": cat(case["dx"]),
        "dy": cat(case["dy"]), "targets": nleaf,
        "config": {"workload": "amr3_exponential", "levels": 3, "cells_per_level": [256, 256], "leaves": nleaf,
                   "precision": "fp32", "slopes": "caller",
                   "l2": "flushed before every solve (512 MB write)"},
    }


def workload_offplane():
    """The spiral 1024^2 disk with the targets one cell width above the plane
    (Fx, Fy, Fz; off-plane kernels with the arctan terms), central slopes."""
    wl = workload_spiral()
    h = wl["patches"][0][5]
    wl["z"] = h
    wl["name"] = wl["name"] + ", targets at z = h above the plane"
    wl["config"] = dict(wl["config"], workload="spiral_1024_offplane", z=h, outputs="Fx Fy Fz")
    return wl


def workload_offplane_amr3():
    """The config-3 hierarchy (3 x 256^2) with the targets one finest cell
    width above the plane (Fx, Fy, Fz): each patch's own convolution with its
    height-z tables plus the FP64 corner-form cross sum."""
    wl = workload_amr3()
    h = min(p[5] for p in wl["patches"])
    wl["z"] = h
    wl["name"] = wl["name"] + ", targets at z = finest h above the plane"
    wl["config"] = dict(wl["config"], workload="amr3_exponential_offplane", z=h, outputs="Fx Fy Fz")
    return wl


def workload_nested(base, levels, r0=0.1):
    """Centred nested ratio-2 patches of base^2 cells each (the largest AMR
    request of the serving mix at base 512, 4 levels), sigma = exp(-R/r0)."""
    from paper_2001_02765_gb300 import workloads as W
    case = W.exponential_hierarchy(base, levels, r0)
    patches = [(lev,) + p for lev, p in enumerate(case["patches"])]
    cat = lambda a: np.concatenate([x.ravel() for x in a])
    nleaf = int(sum(m.sum() for m in case["leaf"]))
    return {
        "name": "AMR %d levels x %d^2 (ratio 2, centred nested), exponential disk exp(-R/%g), caller slopes"
                % (levels, base, r0),
        "patches": patches, "slope_mode": 2, "sigma": cat(case["sigma"]), "dx": cat(case["dx"]),
        "dy": cat(case["dy"]), "targets": nleaf,
        "config": {"workload": "amr%d_exponential_%d" % (levels, base), "levels": levels,
                   "cells_per_level": [base, base], "leaves": nleaf, "precision": "fp32", "slopes": "caller",
                   "l2": "flushed before every solve (512 MB write)"},
    }


def workload_ilr(n=512, levels=3, rule="ilr", disk="d2"):
    """AMR(L, D_2) of Section 4: the n x n grid on [-1,1]^2 refined in bands
    around the disk edge (ILR rule), analytic density and gradient at every
    zone centre, solved zone by zone."""
    from paper_2001_02765_gb300 import workloads as W
    hier = W.band_hierarchy(n, levels, rule, disk)
    xc, yc, _ = W.zone_geometry(hier)
    s, sx, sy = W.d2_sigma(xc, yc, 0.5) if disk == "d2" else W.d22_sigma(xc, yc)
    nleaf = int(hier["leaf"].sum())
    return {
        "name": "AMR(%d, %s) %s hierarchy on a %d^2 grid, %d zones, %d leaves, analytic slopes"
                % (levels, disk.upper(), rule.upper(), n, hier["level"].size, nleaf),
        "patches": [], "zones": (n, n, hier["x0"], hier["y0"], hier["h0"], hier["level"], hier["ix"], hier["iy"]),
        "leaf": hier["leaf"], "slope_mode": 2, "sigma": s, "dx": sx, "dy": sy, "targets": nleaf,
        "config": {"workload": "amr%d_%s_%s_%d" % (levels, disk, rule, n), "zones": int(hier["level"].size),
                   "leaves": nleaf, "precision": "fp32", "slopes": "caller (analytic)",
                   "l2": "flushed before every solve (512 MB write)",
                   "paper_context": "Tables 8-9 give P100 wall times for the same hierarchies (direct O(EL^2) sum)"},
    }


WORKLOADS = {"spiral1024": workload_spiral, "amr3": workload_amr3, "offplane": workload_offplane,
             "offplane_amr3": workload_offplane_amr3,
             "ilr512": lambda: workload_ilr(512, 3, "ilr", "d2"), "ilr1024": lambda: workload_ilr(1024, 3, "ilr", "d2"),
             "ilr2048": lambda: workload_ilr(2048, 3, "ilr", "d2"),
             "amr4_512": lambda: workload_nested(512, 4)}


# -------------------------------------------------------------- batch run --

def sg_pad(n):
    p = 64
    while p < 2 * n - 1:
        p *= 2
    return p


def run_batch(args):
    """64 independent spiral disks (N log-uniform 64..512, seed 4), one CUDA
    graph launch per step, versus the same solves launched one by one."""
    import torch
    from paper_2001_02765_gb300 import sg
    from paper_2001_02765_gb300 import workloads as W
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    ns, a, amp = W.batch_sizes(count=args.batch_size, lo=64, hi=512, seed=4 + rank)
    # launch shapes picked by the library's autotuner for the padded lengths of the batch
    pads = sorted({sg_pad(int(n)) for n in ns})
    tuned, tune_s = None, 0.0
    if not args.no_autotune:
        t0 = time.perf_counter()
        res = sg.sg_autotune(sg.SG_FP32, pads[0], pads[-1], reps=15)
        tune_s = time.perf_counter() - t0
        tuned = {str(p): res[p][0] for p in pads}

    def build(precision):
        # the members' fields are views of one input and one output allocation, so
        # that a batch moves between host and device in one copy each way
        dt = torch.float32 if precision == "fp32" else torch.float64
        sizes = [int(n) * int(n) for n in ns]
        total = sum(sizes)
        flat_in = torch.empty(total, dtype=dt, device="cuda")
        flat_out = torch.empty(2 * total, dtype=dt, device="cuda")
        plans, ins, outs, off = [], [], [], 0
        for k, n in enumerate(ns):
            patches = [(0,) + W.unit_grid(int(n))]
            X, Y = W.cell_centres(*patches[0][1:])
            s, _, _ = W.spiral_sigma(X, Y, a[k], amp[k])
            plans.append(sg.Plan(patches, precision=precision, slope_mode=sg.SG_SLOPES_CENTRAL))
            m = sizes[k]
            ins.append(flat_in[off:off + m])
            ins[-1].copy_(torch.from_numpy(s.ravel()).to(dtype=dt))
            outs.append((flat_out[off:off + m], flat_out[total + off:total + off + m]))
            off += m
        return plans, ins, outs, flat_in, flat_out

    plans, ins, outs, flat_in, flat_out = build("fp32")
    batch = sg.sg_batch_create([p.handle for p in plans], [i.data_ptr() for i in ins], [0] * len(ins), [0] * len(ins),
                               [o[0].data_ptr() for o in outs], [o[1].data_ptr() for o in outs])
    batch_launches = sg.sg_batch_launches(batch)
    mode, ms_p, ms_g = sg.sg_batch_layout(batch)
    layout = {"chosen": "persistent" if mode == sg.SG_BATCH_PERSISTENT else "grouped",
              "replay_ms_persistent": ms_p, "replay_ms_grouped": ms_g,
              "note": "both layouts captured and replayed three times at creation; the faster is kept"}
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def timed(fn, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
                ev[k][0].record(stream)
            fn()
            with torch.cuda.stream(stream):
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        return [x.elapsed_time(y) for x, y in ev]

    graph = lambda: sg.sg_batch_launch(batch, stream.cuda_stream)

    def one_by_one(pl=plans, i_=ins, o_=outs):
        for p, i, o in zip(pl, i_, o_):
            p.force(i, None, None, o[0], o[1], stream=stream)

    timed(graph, args.warmup)
    timed(one_by_one, args.warmup)
    with ClockSampler(local) as clk:
        per = timed(graph, args.steps)
    per_seq = timed(one_by_one, args.steps)
    value, total_ms, solves = job_rate(sum(per), args.steps * len(plans))
    # end to end: all members' sigma copied in from pinned host memory (one
    # copy), the graph, all Fx, Fy copied back (one copy), in the timed region
    hin = flat_in.cpu().pin_memory()
    hout = torch.empty_like(flat_out, device="cpu").pin_memory()
    e2e_ms = 0.0
    for k in range(args.steps + 2):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            flat_in.copy_(hin, non_blocking=True)
            graph()
            hout.copy_(flat_out, non_blocking=True)
        stream.synchronize()
        if k >= 2:
            e2e_ms += 1e3 * (time.perf_counter() - t0)
    h2d = flat_in.numel() * 4
    d2h = flat_out.numel() * 4
    # FP64 plain per-solve path and the FP32 error against it
    plans64, ins64, outs64, _, _ = build("fp64")
    for p, i, o in zip(plans64, ins64, outs64):
        p.force(i, None, None, o[0], o[1])
    graph()
    torch.cuda.synchronize()
    num = sum(float(torch.sum((o[0].double() - q[0]) ** 2) + torch.sum((o[1].double() - q[1]) ** 2))
              for o, q in zip(outs, outs64))
    den = sum(float(torch.sum(q[0] ** 2) + torch.sum(q[1] ** 2)) for q in outs64)
    n64 = max(1, min(args.steps, 3))
    per64 = timed(lambda: one_by_one(plans64, ins64, outs64), n64)
    sg.sg_batch_destroy(batch)
    targets = int(sum(int(n) ** 2 for n in ns))
    for p in plans + plans64:
        p.close()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch64_graph", "members": len(ns), "sizes": "N = round(exp U(ln 64, ln 512)), seed 4",
                   "disk": "Kuzmin a~U[.05,.3] x (1 + A cos(2 theta - ln R / tan 15deg)), A~U[0,.2]",
                   "slopes": "central", "precision": "fp32", "l2": "flushed before every batch (512 MB write)",
                   "launch_shapes": "autotuned" if tuned else "defaults"},
        "autotune": {"seconds": tune_s, "shapes": tuned} if tuned else None,
        "target_cells_per_s": value / len(ns) * targets,
        "latency_ms": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99))},
        "one_by_one": {"solves_per_s": len(ns) * args.steps / (sum(per_seq) / 1e3)},
        "fp64_plain": {"solves_per_s": len(ns) * n64 / (sum(per64) / 1e3)},
        "rel_err_vs_fp64": float(np.sqrt(num / den)),
        "e2e": {"value": args.steps * len(ns) * world / (e2e_ms / 1e3), "unit": "solves/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "roofline": batch_roofline(ns, total_ms / args.steps),
        "gpu_launches": args.steps * batch_launches,
        "batch_layout": layout,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def batch_roofline(ns, ms_per_batch):
    """Whole-step roofline of a batch (every pass of every member; the batch has
    no per-stage timers): conventional FFT flops and algorithmic bytes of the
    spiral members (central slopes, FP32) against the FP32 and HBM peaks."""
    hbm_peak, hbm_src, fp32_peak, fp32_src = _peaks()
    flops = sum(algorithmic_flops({"patches": [(0, int(n), int(n))], "slope_mode": 1}, {}, st)
                for n in ns for st in ("row_fwd", "col_conv", "row_inv"))
    alg = sum(algorithmic_bytes({"patches": [(0, int(n), int(n))], "slope_mode": 1}, {}, st)
              for n in ns for st in ("row_fwd", "col_conv", "row_inv"))
    secs = ms_per_batch * 1e-3
    tflops = flops / secs / 1e12
    return {"kernel": "batch (all passes of all members, one graph)", "bound": "alu", "achieved": tflops,
            "peak": fp32_peak, "unit": "TFLOP/s", "frac": tflops / fp32_peak, "traffic": None,
            "algorithmic_flops": flops, "peak_source": fp32_src, "alu_peaks": _alu_peaks(),
            "hbm": {"algorithmic_bytes": alg, "achieved_gbs": alg / secs / 1e9, "peak_gbs": hbm_peak,
                    "frac": alg / secs / 1e9 / hbm_peak, "peak_source": hbm_src}}


# ------------------------------------------------------------ serving run --

def serve_requests(n, seed=5, amr_bases=(128, 256, 512), amr_levels=(1, 4)):
    """Seeded request mix: 70 % uniform grids N = round(exp U(ln 128, ln 2048)) to
    the nearest multiple of 64 (31 sizes), central slopes; 30 % centred nested
    ratio-2 hierarchies of 1-4 levels with base 128^2, 256^2 or 512^2, analytic
    slopes. Densities: Kuzmin (a in {0.05, 0.1, 0.2, 0.3}) or exponential
    (r0 in {0.05, 0.1, 0.15, 0.2}), eight variants per geometry. Plans are
    per geometry and shared by every request on it. Returns a list of
    (key, patches, slope_mode, density) tuples."""
    from paper_2001_02765_gb300 import workloads as W
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n):
        kuz = rng.uniform() < 0.5
        par = float((0.05, 0.1, 0.2, 0.3)[rng.integers(0, 4)] if kuz else (0.05, 0.1, 0.15, 0.2)[rng.integers(0, 4)])
        if rng.uniform() < 0.7:
            N = int(np.rint(np.exp(rng.uniform(np.log(128), np.log(2048)))))
            N = min(2048, max(128, 64 * int(round(N / 64.0))))
            patches = [(0,) + W.unit_grid(N)]
            mode = 1
        else:
            base = int(rng.choice(list(amr_bases)))
            lev = int(rng.integers(amr_levels[0], amr_levels[1] + 1))
            patches = [(k,) + p for k, p in enumerate(W.centred_nested_patches(base, lev))]
            mode = 2
        key = (tuple(patches), mode, kuz, par)
        out.append((key, patches, mode, ("kuzmin" if kuz else "exp", par)))
    return out


def _serve_inputs(patches, density):
    from paper_2001_02765_gb300 import workloads as W
    sig, gx, gy = [], [], []
    for p in patches:
        X, Y = W.cell_centres(*p[1:])
        if density[0] == "kuzmin":
            a, b, c = W.kuzmin_sigma(X, Y, density[1])
        else:
            a, b, c = W.exponential_sigma(X, Y, density[1])
        sig.append(a.ravel())
        gx.append(b.ravel())
        gy.append(c.ravel())
    return np.concatenate(sig), np.concatenate(gx), np.concatenate(gy)


def _leaf_mask(patches):
    """Leaf cells of a patch hierarchy in field-array order: a cell is covered
    when its centre lies inside a patch of the next level."""
    out = []
    for lev, nx, ny, x0, y0, h in patches:
        xc = x0 + (np.arange(nx) + 0.5) * h
        yc = y0 + (np.arange(ny) + 0.5) * h
        leaf = np.ones((ny, nx), bool)
        for lq, qnx, qny, qx0, qy0, qh in patches:
            if lq != lev + 1:
                continue
            ix = (xc > qx0) & (xc < qx0 + qnx * qh)
            iy = (yc > qy0) & (yc < qy0 + qny * qh)
            leaf &= ~(iy[:, None] & ix[None, :])
        out.append(leaf.ravel())
    return np.concatenate(out)


def run_serve(args):
    """Continuous-batching server on a seeded Poisson request stream."""
    import torch
    from paper_2001_02765_gb300 import sg
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    reqs = serve_requests(args.serve_requests, seed=5 + rank)
    plans, inputs, outputs = {}, {}, {}

    def prepare(precision, subset=None):
        dt = torch.float32 if precision == "fp32" else torch.float64
        dev = lambda v: torch.from_numpy(v).to(dtype=dt, device="cuda")
        for key, patches, mode, dens in (subset or reqs):
            g = (key[0], mode, precision)
            if g not in plans:
                plans[g] = sg.Plan(patches, precision=precision, slope_mode=mode)
                uses = sum(1 for r in reqs if r[0][:2] == key[:2])
                outputs[g] = [(torch.empty(plans[g].ncells, dtype=dt, device="cuda"),
                               torch.empty(plans[g].ncells, dtype=dt, device="cuda"))
                              for _ in range(min(uses, args.serve_inflight))]
                outputs[g + ("n",)] = 0
            if (key, precision) not in inputs:
                a, b, c = _serve_inputs(patches, dens)
                inputs[(key, precision)] = (dev(a), dev(b) if mode == 2 else None, dev(c) if mode == 2 else None)

    def submit(server, key, precision):
        g = (key[0], key[1], precision)
        outs = outputs[g]
        fx, fy = outs[outputs[g + ("n",)] % len(outs)]
        outputs[g + ("n",)] += 1
        ins = inputs[(key, precision)]
        return sg.sg_submit(server, plans[g].handle, ins[0].data_ptr(), ins[1].data_ptr() if ins[1] is not None else 0,
                            ins[2].data_ptr() if ins[2] is not None else 0, fx.data_ptr(), fy.data_ptr())

    prepare("fp32")
    torch.cuda.synchronize()
    budget = args.serve_budget_gb << 30
    server = sg.sg_server_create(budget, args.serve_inflight)
    # warm-up and closed-loop capacity (everything submitted at once)
    for key, *_ in reqs[: min(len(reqs), 16)]:
        sg.sg_wait(server, submit(server, key, "fp32"), 600000.0)
    t0 = time.perf_counter()
    tickets = [submit(server, key, "fp32") for key, *_ in reqs]
    for t in tickets:
        sg.sg_wait(server, t, 600000.0)
    capacity = len(reqs) / (time.perf_counter() - t0)
    def open_loop(stream, load, sampler=None):
        """Poisson arrivals at load x capacity; returns (wall, tickets, stats)."""
        rate = load * capacity
        rng = np.random.Generator(np.random.PCG64(55))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(stream)))
        sg.sg_server_get_stats(server, reset_latencies=True)
        t0 = time.perf_counter()
        tickets = []
        for (key, *_), at in zip(stream, arrivals):
            delay = at - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets.append(submit(server, key, "fp32"))
        for t in tickets:
            sg.sg_wait(server, t, 600000.0)
        return time.perf_counter() - t0, tickets, sg.sg_server_get_stats(server)

    sweep = []
    if args.serve_sweep:
        part = reqs[: max(1, len(reqs) // 10)]
        for load in (0.3, 0.5, 1.0):
            w, tk, st = open_loop(part, load)
            sweep.append({"load": load, "requests": len(tk), "solves_per_s": len(tk) / w,
                          "p50_ms": st["latency_p50_ms"], "p99_ms": st["latency_p99_ms"]})
    rate = args.serve_load * capacity
    with ClockSampler(local) as clk:
        wall, tickets, stats = open_loop(reqs, args.serve_load)

    # end to end, closed loop on a prefix: each request's inputs copied from
    # pinned host memory before it is submitted, its Fx, Fy copied back to pinned
    # host memory once it has finished (at most max_inflight requests in flight)
    part = reqs[: min(len(reqs), args.serve_e2e_requests)]
    host = {}
    for key, patches, mode, dens in part:
        if key not in host:
            n = plans[(key[0], key[1], "fp32")].ncells
            ins = inputs[(key, "fp32")]
            host[key] = ([t.cpu().pin_memory() if t is not None else None for t in ins],
                         torch.empty(n, dtype=torch.float32).pin_memory(),
                         torch.empty(n, dtype=torch.float32).pin_memory())
    copy = torch.cuda.Stream()
    h2d = d2h = 0
    pending = []
    t0 = time.perf_counter()

    def retire(item):
        nonlocal d2h
        t_, g_, hx, hy, outs_ = item
        sg.sg_wait(server, t_, 600000.0)
        with torch.cuda.stream(copy):
            hx.copy_(outs_[0], non_blocking=True)
            hy.copy_(outs_[1], non_blocking=True)
        copy.synchronize()
        d2h += 2 * hx.numel() * 4

    for key, patches, mode, dens in part:
        g = (key[0], key[1], "fp32")
        hin, hx, hy = host[key]
        din = inputs[(key, "fp32")]
        with torch.cuda.stream(copy):
            for dst, src in zip(din, hin):
                if dst is not None:
                    dst.copy_(src, non_blocking=True)
                    h2d += src.numel() * 4
        copy.synchronize()
        outs_ = outputs[g][outputs[g + ("n",)] % len(outputs[g])]
        pending.append((submit(server, key, "fp32"), g, hx, hy, outs_))
        if len(pending) >= args.serve_inflight:
            retire(pending.pop(0))
    while pending:
        retire(pending.pop(0))
    e2e_s = time.perf_counter() - t0
    sg.sg_server_destroy(server)
    value = len(tickets) / wall  # the open-loop requests, all completed
    targets = sum(plans[(key[0], key[1], "fp32")].info["nleaves"] for key, *_ in reqs)

    # the plain FP64 per-solve path on a time-bounded prefix of the same stream,
    # and every served result of that prefix against it: the FP32 plan's sg_force
    # on the same inputs (a request's result is the same bit for bit alone and in
    # any mix), relative L2 over the request's leaf cells
    t_budget = args.serve_fp64_seconds
    done64 = 0
    t64 = 0.0
    skipped64 = set()
    left_out = 0
    errs = []
    for key, patches, mode, dens in reqs:
        if t64 > t_budget:
            break
        if (key[0], mode) in skipped64:
            left_out += 1
            continue
        prepare("fp64", [(key, patches, mode, dens)])
        g = (key[0], mode, "fp64")
        info64 = plans[g].info
        if info64["cross_mode"] == 1 and info64["cross_pairs"] > 5e10:
            skipped64.add((key[0], mode))  # FP64 direct sum of minutes: left out of the comparison
            left_out += 1
            continue
        ins = inputs[(key, "fp64")]
        fx, fy = outputs[g][0]
        torch.cuda.synchronize()
        a = time.perf_counter()
        plans[g].force(ins[0], ins[1], ins[2], fx, fy)
        torch.cuda.synchronize()
        t64 += time.perf_counter() - a
        done64 += 1
        g32 = (key[0], mode, "fp32")
        i32 = inputs[(key, "fp32")]
        sx, sy = plans[g32].force(i32[0], i32[1], i32[2])
        leaf = torch.from_numpy(_leaf_mask(patches)).cuda()
        num = ((sx.double() - fx)[leaf] ** 2).sum() + ((sy.double() - fy)[leaf] ** 2).sum()
        den = (fx[leaf] ** 2).sum() + (fy[leaf] ** 2).sum()
        errs.append(float(torch.sqrt(num / den)))
    for p_ in plans.values():
        p_.close()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value * world, "unit": "solves/s", "n_gpus": world, "steps": len(reqs),
        "warmup": 16, "ms_per_step": 1e3 * wall / len(reqs), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serve_poisson_mix", "requests": len(reqs),
                   "uniform": "128^2..2048^2, multiples of 64 (70%)",
                   "amr": "1-4 levels, base 128^2/256^2/512^2 (30%)", "load": args.serve_load,
                   "plans": len([g for g in plans if g[2] == "fp32"]),
                   "budget_gb": args.serve_budget_gb, "max_inflight": args.serve_inflight, "precision": "fp32"},
        "target_cells_per_s": targets / wall * world,
        "latency_ms": {"p50": stats["latency_p50_ms"], "p99": stats["latency_p99_ms"],
                       "mean": stats["latency_mean_ms"]},
        "capacity_solves_per_s": capacity, "offered_rate": rate, "load_sweep": sweep,
        "peak_bytes": stats["peak_bytes"],
        "grouped": {"groups": stats["groups_started"], "requests": stats["grouped_requests"],
                    "note": "queued single-patch requests of one padded length, precision and slope handling "
                            "admitted together (one launch per pass over the group)"},
        "fp64_plain": {"solves_per_s": done64 / t64 if t64 else None, "requests": done64,
                       "left_out": left_out,
                       "note": "one solve at a time on a %.0f s prefix of the same stream; requests whose FP64 plan "
                               "would take the direct sum over > 5e10 pairs (hierarchies too wide for FP64 level "
                               "convolutions: %d geometries) are left out of the comparison" % (
                                   t_budget, len(skipped64))},
        "rel_err_vs_fp64": {"max": max(errs) if errs else None,
                            "median": float(np.median(errs)) if errs else None, "results": len(errs),
                            "note": "every FP32 result of the FP64 prefix against the FP64 plain path, relative L2 "
                                    "over the request's leaf cells"},
        "e2e": {"value": len(part) / e2e_s * world, "unit": "solves/s", "requests": len(part),
                "h2d_bytes_per_step": h2d / len(part), "d2h_bytes_per_step": d2h / len(part),
                "note": "closed loop, inputs copied from pinned host memory before each submit, Fx and Fy copied "
                        "back to pinned host memory when the request finishes, %d in flight" % args.serve_inflight},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- oracle --

class OracleSample:
    """The FP64 plain direct sum (the oracle) on a seeded sample of leaf targets
    of a workload; the leaf list is prepared once."""

    def __init__(self, wl, potential=False):
        from oracle import amr as oamr
        self.potential = potential
        self.z = wl.get("z", 0.0)  # off the plane: the three-component sum at height z
        from oracle.fftconv import central_slopes
        self.total_targets = wl["targets"]
        self.rng = np.random.Generator(np.random.PCG64(77))
        if "zones" in wl:
            nx0, ny0, x0, y0, h0, level, ix, iy = wl["zones"]
            m = wl["leaf"]
            xl, xr, yd, yu, xc, yc = (a[m] for a in oamr.zone_bounds(x0, y0, h0, level, ix, iy))
            self.cells = (xl, xr, yd, yu)
            self.tx, self.ty = xc, yc
            self.s0 = np.asarray(wl["sigma"], np.float64)[m]
            self.sx = np.asarray(wl["dx"], np.float64)[m]
            self.sy = np.asarray(wl["dy"], np.float64)[m]
            return
        patches = wl["patches"]
        sig, off = [], 0
        for p in patches:
            sig.append(np.asarray(wl["sigma"][off:off + p[1] * p[2]], np.float64).reshape(p[2], p[1]))
            off += p[1] * p[2]
        if wl["slope_mode"] == 1:
            sx, sy = central_slopes(sig[0], patches[0][5])
            sxs, sys_ = [sx], [sy]
        elif wl["slope_mode"] == 2:
            sxs, sys_, off = [], [], 0
            for p in patches:
                n = p[1] * p[2]
                sxs.append(np.asarray(wl["dx"][off:off + n], np.float64).reshape(p[2], p[1]))
                sys_.append(np.asarray(wl["dy"][off:off + n], np.float64).reshape(p[2], p[1]))
                off += n
        else:
            sxs = sys_ = None
        leaves = oamr.leaf_cells(oamr.make_patches(patches))
        k, j, i = leaves["patch"], leaves["j"], leaves["i"]

        def g(f):
            return np.concatenate([f[q][j[k == q], i[k == q]] for q in range(len(patches))])

        self.s0 = g(sig)
        self.sx = g(sxs) if sxs is not None else None
        self.sy = g(sys_) if sys_ is not None else None
        self.cells = (leaves["xl"], leaves["xr"], leaves["yd"], leaves["yu"])
        self.tx, self.ty = leaves["xc"], leaves["yc"]

    def run(self, sample_targets, nthreads=0):
        """Returns (solves/s, target-cells/s, seconds, threads, description)."""
        from oracle.direct import direct_force, direct_force3, max_threads
        from oracle.potential import direct_potential
        tsel = self.rng.choice(self.tx.size, sample_targets, replace=False)
        t0 = time.perf_counter()
        if self.z != 0.0 and not self.potential:
            direct_force3(self.cells, self.s0, self.sx, self.sy, self.tx[tsel], self.ty[tsel], self.z,
                          nthreads=nthreads)
        else:
            f = direct_potential if self.potential else direct_force
            f(self.cells, self.s0, self.sx, self.sy, self.tx[tsel], self.ty[tsel], nthreads=nthreads)
        dt = time.perf_counter() - t0
        threads = nthreads or max_threads()
        tps = sample_targets / dt
        return (tps / self.total_targets, tps, dt, threads,
                "%d seeded leaf targets of the full workload, plain FP64 direct sum over all sources" % sample_targets)


# ------------------------------------------------------- cuFFT comparison --

class TorchFFTConv:
    """The uniform-grid convolution through torch.fft (cuFFT on a GPU), timed
    beside the library's own transforms as a comparison only; no path of the
    library uses it.

    F_x[t] = G sum_s sigma0[s] K^{x,0}[s - t] + deltax[s] K^{x,x}[s - t]
    + deltay[s] K^{x,y}[s - t] (and F_y with K^{y,.}) is a correlation of the
    fields with the kernel tables; zero padding to P >= 2N - 1 per axis makes
    the circular form equal to the linear one. tables: the six tables K^{x,0},
    K^{x,x}, K^{x,y}, K^{y,0}, K^{y,x}, K^{y,y}, each (2 ny - 1) x (2 nx - 1)
    with entry [n + ny - 1][m + nx - 1] for a source offset (m h, n h). Their
    spectra are formed once, in FP64, and held in `dtype`'s complex type. Per
    call: central slopes by elementwise ops (slope_mode 1; sigma = 0 beyond the
    grid), R2C of the fields, six spectral products, two C2R, crop.
    """

    def __init__(self, tables, nx, ny, h, G, slope_mode, pad, dtype, device):
        import torch
        self.nx, self.ny, self.h, self.G, self.slope_mode = nx, ny, h, G, slope_mode
        self.py, self.px = pad
        self.dtype = dtype
        m = torch.arange(-(nx - 1), nx)
        n = torch.arange(-(ny - 1), ny)
        rows = ((-n) % self.py).to(device)
        cols = ((-m) % self.px).to(device)
        cdt = torch.complex64 if dtype == torch.float32 else torch.complex128
        self.spec = []
        for t in tables:
            w = torch.zeros(self.py, self.px, dtype=torch.float64, device=device)
            w[rows[:, None], cols[None, :]] = torch.as_tensor(np.asarray(t, np.float64), device=device)
            self.spec.append(torch.fft.rfft2(w).to(cdt))

    def __call__(self, sigma, dx=None, dy=None):
        import torch
        import torch.nn.functional as F
        s = sigma.reshape(self.ny, self.nx)
        if self.slope_mode == 1:
            p = F.pad(s, (1, 1, 1, 1))
            dx = (p[1:-1, 2:] - p[1:-1, :-2]) * (0.5 / self.h)
            dy = (p[2:, 1:-1] - p[:-2, 1:-1]) * (0.5 / self.h)
        elif self.slope_mode == 2:
            dx, dy = dx.reshape(self.ny, self.nx), dy.reshape(self.ny, self.nx)
        else:
            dx = dy = None
        size = (self.py, self.px)
        sh = torch.fft.rfft2(s, s=size)
        kx0, kxx, kxy, ky0, kyx, kyy = self.spec
        fxh, fyh = sh * kx0, sh * ky0
        if dx is not None:
            ah = torch.fft.rfft2(dx, s=size)
            bh = torch.fft.rfft2(dy, s=size)
            fxh = fxh + ah * kxx + bh * kxy
            fyh = fyh + ah * kyx + bh * kyy
        fx = torch.fft.irfft2(fxh, s=size)[: self.ny, : self.nx]
        fy = torch.fft.irfft2(fyh, s=size)[: self.ny, : self.nx]
        return self.G * fx, self.G * fy


def cufft_compare(plan, wl, steps, flush, ref):
    """Time TorchFFTConv on the workload (FP32, tables from the plan, L2 flushed
    before each solve, CUDA events on the current stream) and its relative L2
    error against `ref`, the FP64 plan's (Fx, Fy)."""
    import torch
    _, nx, ny, _, _, h = wl["patches"][0]
    tabs = [plan.kernel_table(0, w) for w in range(6)]
    conv = TorchFFTConv(tabs, nx, ny, h, plan.G, wl["slope_mode"], (_pad(ny), _pad(nx)), torch.float32, "cuda")
    dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    s, dx, dy = dev(wl["sigma"]), dev(wl["dx"]), dev(wl["dy"])
    for _ in range(3):  # cuFFT plans are made on first use
        fx, fy = conv(s, dx, dy)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(float(k))
        ev[k][0].record()
        fx, fy = conv(s, dx, dy)
        ev[k][1].record()
    torch.cuda.synchronize()
    per = [a.elapsed_time(b) for a, b in ev]
    rx, ry = ref[0].ravel(), ref[1].ravel()
    num = torch.sum((fx.double().ravel() - rx) ** 2) + torch.sum((fy.double().ravel() - ry) ** 2)
    den = torch.sum(rx ** 2) + torch.sum(ry ** 2)
    return {"solves_per_s": 1e3 * steps / sum(per), "ms_per_solve": sum(per) / steps,
            "p50_ms": float(np.percentile(per, 50)), "rel_err_vs_fp64": float(torch.sqrt(num / den)),
            "note": "torch.fft (cuFFT) in FP32, a comparison only: %s, R2C of the fields, products with the "
                    "spectra of the plan's six kernel tables (formed once, untimed), two C2R, crop; L2 flushed "
                    "before each solve" % ("central slopes by elementwise ops" if wl["slope_mode"] == 1 else
                                           "caller slopes" if wl["slope_mode"] == 2 else "order 0")}


# -------------------------------------------------------------- GPU arm --

def run_gpu(args):
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2001_02765_gb300 import sg

    wl = WORKLOADS[args.workload]()
    dt = torch.float32
    zt = wl.get("z", 0.0)
    zones = wl.get("zones")
    pot = args.quantity == "potential"
    if pot and (zt or zones is not None):
        raise SystemExit("--quantity potential takes the in-plane patch workloads")

    cross = {"auto": sg.SG_CROSS_AUTO, "direct": sg.SG_CROSS_DIRECT, "levels": sg.SG_CROSS_LEVELS}[args.cross]

    def make_plan(prec):
        # the FP32 plan takes --cross; the FP64 plain comparator the library's own choice
        c = cross if prec == "fp32" else sg.SG_CROSS_AUTO
        if zones is not None:
            return sg.ZonePlan(*zones, precision=prec, slope_mode=wl["slope_mode"], cross_mode=c)
        return sg.Plan(wl["patches"], precision=prec, slope_mode=wl["slope_mode"], z=zt, cross_mode=c)

    plan = make_plan("fp32")
    # launch shapes of the plan's transform lengths picked by the library's autotuner
    tuned = None
    if (not args.no_autotune and wl["patches"] and plan.info["max_pad"] <= 4096
            and plan.info["cross_mode"] != 2):
        t0 = time.perf_counter()
        pads = sorted({_pad(p[1]) for p in wl["patches"]} | {_pad(p[2]) for p in wl["patches"]})
        res = sg.sg_autotune(sg.SG_FP32, pads[0], pads[-1], reps=15)
        tuned = {"seconds": time.perf_counter() - t0, "shapes": {str(p): res[p][0] for p in pads}}
    # the cross-patch direct sum's split and far-field grid (skipped where one
    # solve takes seconds: the candidates would take minutes)
    if not args.no_autotune and plan.info["cross_mode"] == 1 and plan.info["cross_pairs"] < 1e11:
        t0 = time.perf_counter()
        before = sg.sg_plan_direct_shape(plan.handle)
        best = sg.sg_plan_autotune(plan.handle, 3)
        after = sg.sg_plan_direct_shape(plan.handle)
        tuned = dict(tuned or {}, direct={"seconds": time.perf_counter() - t0, "split_and_far_grid_built": before,
                                          "split_and_far_grid_chosen": after, "best_ms": best})
    stream = torch.cuda.Stream()
    dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    sigma, dxs, dys = dev(wl["sigma"]), dev(wl["dx"]), dev(wl["dy"])
    fx = torch.empty_like(sigma)
    fy = torch.empty_like(sigma)
    fz = torch.empty_like(sigma) if zt else None
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def solve():
        with torch.cuda.stream(stream):
            if zt:
                sg.sg_force3(plan.handle, sigma.data_ptr(), dxs.data_ptr() if dxs is not None else 0,
                             dys.data_ptr() if dys is not None else 0, fx.data_ptr(), fy.data_ptr(), fz.data_ptr(),
                             stream.cuda_stream)
            elif zones is not None:
                plan.force_zones(sigma, dxs, dys, fx, fy, stream=stream)
            else:
                if pot:
                    plan.potential(sigma, dxs, dys, phi=fx, stream=stream)
                else:
                    plan.force(sigma, dxs, dys, fx, fy, stream=stream)

    torch.cuda.synchronize()
    for _ in range(args.warmup):
        flush.fill_(1.0)
        solve()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    # the timed solves run with the library's stage timers off (their events would
    # sit between the passes); the stage split comes from a second, shorter pass
    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
                ev[k][0].record(stream)
            solve()
            with torch.cuda.stream(stream):
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    per = [a.elapsed_time(b) for a, b in ev]
    value, total_ms, solves = job_rate(sum(per), args.steps)
    p50 = float(np.percentile(per, 50))
    p99 = float(np.percentile(per, 99))
    stage_ms = {k: [] for k in sg.STAGE_NAMES}
    sg.sg_plan_set_timing(plan.handle, True)
    for k in range(min(args.steps, 20)):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
        solve()
        t = sg.sg_plan_get_timing(plan.handle)  # waits for this solve's events
        for name, v in t.items():
            stage_ms[name].append(v)
    sg.sg_plan_set_timing(plan.handle, False)

    # FP64 plain per-solve path on the same GPU, and the FP32 error against it.
    # FP64 level convolutions stop at 4096-point transforms; beyond, the FP64
    # plan takes the direct sum, which is skipped above 5e10 leaf pairs (minutes).
    plan64 = make_plan("fp64")
    f64 = plan64.force_zones if zones is not None else plan64.force
    fp64_ms, rel_err, fp64_note = None, None, None
    if plan64.info["cross_mode"] == 1 and plan64.info["cross_pairs"] > 5e10:
        fp64_note = "skipped: the FP64 plan takes the direct sum over %.2e leaf pairs" % plan64.info["cross_pairs"]
    else:
        d64 = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a, np.float32).astype(np.float64)).cuda()
        s64, dx64, dy64 = d64(wl["sigma"]), d64(wl["dx"]), d64(wl["dy"])
        t0 = time.perf_counter()
        if pot:
            g64 = (plan64.potential(s64, dx64, dy64),)
        else:
            g64 = plan64.force3(s64, dx64, dy64) if zt else f64(s64, dx64, dy64)
        torch.cuda.synchronize()
        first = time.perf_counter() - t0
        ff = [x.double() for x in ((fx,) if pot else ((fx, fy, fz) if zt else (fx, fy)))]
        # over the leaf cells only: the output at covered cells is unspecified
        # (the FP32 and FP64 plans may take different paths)
        keep = None
        if zones is None and wl["patches"] and len(wl["patches"]) > 1:
            keep = torch.from_numpy(_leaf_mask(wl["patches"])).cuda()
        sel = (lambda a: a[keep]) if keep is not None else (lambda a: a)
        num = sum(torch.sum((sel(a) - sel(b)) ** 2) for a, b in zip(ff, g64))
        den = sum(torch.sum(sel(b) ** 2) for b in g64)
        rel_err = float(torch.sqrt(num / den))
        n64 = 1 if first > 1.0 else max(3, min(args.steps, 10))
        e64 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n64)]
        for k in range(n64):
            flush.fill_(1.0)
            e64[k][0].record()
            if zt:
                plan64.force3(s64, dx64, dy64)
            else:
                if pot:
                    plan64.potential(s64, dx64, dy64, phi=g64[0])
                else:
                    f64(s64, dx64, dy64, g64[0], g64[1])
            e64[k][1].record()
        torch.cuda.synchronize()
        fp64_ms = statistics.median([a.elapsed_time(b) for a, b in e64])
    fp64_path = plan64.info["cross_mode"]
    plan64.close()

    # the same convolution through torch.fft (cuFFT) in FP32, timed as a
    # comparison only (single in-plane patch force workloads)
    cufft = None
    if not pot and not zt and zones is None and len(wl["patches"]) == 1 and fp64_ms is not None:
        try:
            cufft = cufft_compare(plan, wl, args.steps, flush, g64)
        except Exception as e:  # the comparison never fails the benchmark
            cufft = {"unavailable": "%s: %s" % (type(e).__name__, e)}

    # end to end through the host-buffer entry point (pinned buffers)
    hs = torch.from_numpy(np.ascontiguousarray(wl["sigma"], np.float32)).pin_memory()
    hdx = torch.from_numpy(np.ascontiguousarray(wl["dx"], np.float32)).pin_memory() if wl["dx"] is not None else None
    hdy = torch.from_numpy(np.ascontiguousarray(wl["dy"], np.float32)).pin_memory() if wl["dy"] is not None else None
    nout = sigma.numel()
    hfx = torch.empty(nout, dtype=dt).pin_memory()
    hfy = torch.empty(nout, dtype=dt).pin_memory()
    sg.sg_plan_set_timing(plan.handle, False)
    e2e_ms, h2d, d2h = None, 0, 0
    e2e_sync_ms, e2e_mode = None, "one synchronous call per step"
    if zones is not None:
        # zone plans: pinned host arrays copied in, the zone solve, forces copied back, all in the timed region
        e2e_ms = 0.0
        for k in range(args.steps + 2):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                sigma.copy_(hs, non_blocking=True)
                dxs.copy_(hdx, non_blocking=True)
                dys.copy_(hdy, non_blocking=True)
                plan.force_zones(sigma, dxs, dys, fx, fy, stream=stream)
                hfx.copy_(fx, non_blocking=True)
                hfy.copy_(fy, non_blocking=True)
            stream.synchronize()
            if k >= 2:
                e2e_ms += 1e3 * (time.perf_counter() - t0)
        h2d = 3 * nout * 4
        d2h = 2 * nout * 4
    elif pot:
        # pinned host arrays copied in, the potential, phi copied back, all in the timed region
        e2e_ms = 0.0
        for k in range(args.steps + 2):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                sigma.copy_(hs, non_blocking=True)
                if dxs is not None:
                    dxs.copy_(hdx, non_blocking=True)
                    dys.copy_(hdy, non_blocking=True)
                plan.potential(sigma, dxs, dys, phi=fx, stream=stream)
                hfx.copy_(fx, non_blocking=True)
            stream.synchronize()
            if k >= 2:
                e2e_ms += 1e3 * (time.perf_counter() - t0)
        h2d = nout * 4 * (3 if dxs is not None else 1)
        d2h = nout * 4
    elif not zt:  # the host entry point returns Fx, Fy
        for _ in range(2):
            plan.force_host(hs, hdx, hdy, hfx, hfy, stream=stream)
        e2e_ms = 0.0
        for k in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan.force_host(hs, hdx, hdy, hfx, hfy, stream=stream)  # copies in, solve, copies out, waits
            e2e_ms += 1e3 * (time.perf_counter() - t0)
        nbytes = nout * 4
        h2d = nbytes * (3 if wl["dx"] is not None else 1)
        d2h = 2 * nbytes
        e2e_sync_ms = e2e_ms
        # pipelined: two plans on two streams, each solve enqueued by
        # sg_force_host_async and waited for one step later, so one solve's
        # results stream back over the CPU-GPU link while the next one's inputs
        # come in and transform; host buffers rotate over enough sets to exceed L2
        if e2e_ms:
            sets = max(4, -(-2 * (129 << 20) // (h2d + d2h)))
            pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32).ravel()).pin_memory()
            rot = [(pin(wl["sigma"]), pin(wl["dx"]) if wl["dx"] is not None else None,
                    pin(wl["dy"]) if wl["dy"] is not None else None,
                    torch.empty(nout, dtype=dt).pin_memory(), torch.empty(nout, dtype=dt).pin_memory())
                   for _ in range(sets)]
            plan2 = make_plan("fp32")
            sg.sg_plan_set_timing(plan2.handle, False)
            pair = [(plan, stream), (plan2, torch.cuda.Stream())]

            def pipelined(k_steps):
                for k in range(k_steps):
                    pl, st = pair[k % 2]
                    if k >= 2:
                        pl.wait(st)
                    pl.force_host_async(*rot[k % sets], stream=st)
                for pl, st in pair:
                    pl.wait(st)

            # warm-up over every buffer set; at least 200 timed solves, since
            # 50 pipelined solves last only a few ms and one host stall there
            # halves the figure
            e2e_steps = max(args.steps, 200)
            pipelined(sets + 2)
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pipelined(e2e_steps)
            e2e_ms = 1e3 * (time.perf_counter() - t0) * args.steps / e2e_steps
            e2e_mode = ("pipelined: sg_force_host_async on two plans and two streams, each solve waited for one "
                        "step later; %d rotating pinned host buffer sets (%.0f MB, more than L2), warmed up over "
                        "every set; %d solves timed" % (sets, sets * (h2d + d2h) / 2**20, e2e_steps))
            plan2.close()

    # roofline of the dominant kernel
    stage_mean = {k: (sum(v) / len(v) if v else 0.0) for k, v in stage_ms.items()}
    dom = max(stage_mean, key=stage_mean.get)
    hbm_peak, hbm_src, fp32_peak, fp32_src = _peaks()
    alu_peak, alu_src = fp32_peak, fp32_src
    if wl.get("precision", "fp32") == "fp64" and dom == "cross_direct":
        alu_peak = _alu_peaks()["fp64_tflops"]
        alu_src = "measured (sg_alu_peak: FP64 FMA on every SM, best of 5): an FP64 plan's cross sum"
    info = plan.info
    alg = algorithmic_bytes(wl, info, dom, nout=1 if pot else 2)
    flops = algorithmic_flops(wl, info, dom, nout=1 if pot else 2)
    secs = stage_mean[dom] * 1e-3
    tflops = flops / secs / 1e12 if secs > 0 else 0.0
    gbs = alg / secs / 1e9 if secs > 0 else 0.0
    plan.close()

    if rank != 0:
        return
    line = {
        "metric": METRIC_POTENTIAL if pot else METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(wl["config"], parallelism="replicas" if world > 1 else "single",
                       **({"cross": args.cross} if args.cross != "auto" else {}),
                       **({"quantity": "potential"} if pot else {})),
        "target_cells_per_s": value * wl["targets"],
        "latency_ms": {"p50": p50, "p99": p99},
        "fp64_plain": {"solves_per_s": 1e3 / fp64_ms * world if fp64_ms else None, "ms_per_solve": fp64_ms,
                       "cross_mode": fp64_path, "note": fp64_note},
        "rel_err_vs_fp64": rel_err,
        **({"cufft_comparison": cufft} if cufft is not None else {}),
        "stage_ms": stage_mean,
        "roofline": {"kernel": dom, "bound": "alu", "achieved": tflops, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": tflops / alu_peak, "traffic": TRAFFIC.get((args.workload, dom)),
                     "algorithmic_flops": flops, "peak_source": alu_src, "alu_peaks": _alu_peaks(),
                     "hbm": {"algorithmic_bytes": alg, "achieved_gbs": gbs, "peak_gbs": hbm_peak,
                             "frac": gbs / hbm_peak, "peak_source": hbm_src}},
        "e2e": ({"value": args.steps * world / (e2e_ms / 1e3), "unit": "solves/s", "h2d_bytes_per_step": h2d,
                 "d2h_bytes_per_step": d2h, "mode": e2e_mode,
                 **({"sync_value": args.steps * world / (e2e_sync_ms / 1e3)}
                    if e2e_sync_ms and e2e_sync_ms != e2e_ms else {})} if e2e_ms else None),
        "gpu_launches": args.steps * info["launches"],
        "autotune": tuned,
        "clocks": clk.summary(),
        "wall_s": wall,
    }
    if world == 1 and not args.no_cpu_baseline:
        sampler = OracleSample(wl, potential=pot)
        sps, tps, secs, thr, what = sampler.run(args.cpu_targets)
        line["cpu_baseline"] = {"value": sps, "unit": "solves/s", "cores": thr, "kind": "oracle", "sample": what,
                                "target_cells_per_s": tps, "seconds": secs}
        # the same sum on one core (a sixteenth of the sample)
        sps1, tps1, secs1, _, what1 = sampler.run(max(16, args.cpu_targets // 16), nthreads=1)
        line["cpu_baseline"]["single_core"] = {"value": sps1, "unit": "solves/s", "cores": 1, "sample": what1,
                                               "target_cells_per_s": tps1, "seconds": secs1}
        fft = oracle_fft_route(wl) if not pot and zones is None else None
        if fft is not None:
            line["cpu_baseline"]["fft_route"] = fft
    print(json.dumps(line), flush=True)


def oracle_fft_route(wl, reps=3):
    """The oracle's FP64 FFT route (numpy pocketfft, one thread) on the whole
    workload when it is one uniform patch (in the plane, or at height z): median
    of `reps` calls, each building its own kernel tables as the oracle does. None
    otherwise."""
    if "zones" in wl or len(wl["patches"]) != 1 or wl.get("masks") is not None:
        return None
    from oracle.fftconv import central_slopes, uniform_fft_force, uniform_fft_force3
    z = wl.get("z", 0.0)
    _, nx, ny, _, _, h = wl["patches"][0]
    s = np.asarray(wl["sigma"], np.float64).reshape(ny, nx)
    if wl["slope_mode"] == 1:
        dx, dy = central_slopes(s, h)
    elif wl["slope_mode"] == 2:
        dx = np.asarray(wl["dx"], np.float64).reshape(ny, nx)
        dy = np.asarray(wl["dy"], np.float64).reshape(ny, nx)
    else:
        dx = dy = None
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        if z != 0.0:
            uniform_fft_force3(s, dx, dy, h, z)
        else:
            uniform_fft_force(s, dx, dy, h)
        times.append(time.perf_counter() - t0)
    med = float(np.median(times))
    return {"value": 1.0 / med, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": "the whole workload through the oracle's FP64 FFT route (numpy pocketfft, one thread, its "
                      "kernel tables built in every call); median of %d calls" % reps,
            "target_cells_per_s": wl["targets"] / med, "seconds": med}


# DRAM bytes (read + write) per launch of a stage's kernel from the ncu capture
# of the current kernel build (see profiles/); None when not captured for it.
# amr3 col_conv: the stage's column-transform and column-MAC launches, one each
# per solve (profiles/k_lv_col_fwd_amr3.md, k_lv_col_mac_inv_amr3.md).
TRAFFIC = {("spiral1024", "col_conv"): 33.810e6 + 0.014e6,
           ("amr3", "col_conv"): (11.152e6 + 7.286e6) + (226.808e6 + 11.011e6),
           ("amr3", "cross_direct"): 5.882e6 + 3.741e6}


def _pad(n):
    p = 64
    while p < 2 * n - 1:
        p *= 2
    return p


def _lv_cexp(s, p):
    """Compression exponent of a level's source transforms (lengths p >> c >= 64)."""
    return min(s, p.bit_length() - 1 - 6)


def lv_geometry(wl):
    """Level-convolution layout of a workload: padded finest-lattice lengths and
    the (nx, ny, s) of every level's image (bounding box of its cells; cells
    2^s finest cells wide)."""
    if "zones" in wl:
        nx0, ny0, x0, y0, h0, level, ix, iy = wl["zones"]
        lmax = int(level.max())
        imgs = []
        for m in range(lmax + 1):
            sel = level == m
            imgs.append((int(ix[sel].max() - ix[sel].min() + 1), int(iy[sel].max() - iy[sel].min() + 1), lmax - m))
        wx, wy = nx0 << lmax, ny0 << lmax
    else:
        pats = wl["patches"]
        lmax = max(p[0] for p in pats)
        h0 = pats[0][5]
        X0 = min(p[3] for p in pats if p[0] == 0)
        Y0 = min(p[4] for p in pats if p[0] == 0)
        imgs = []
        for m in range(lmax + 1):
            ps = [p for p in pats if p[0] == m]
            h = h0 / 2 ** m
            gx0 = min(round((p[3] - X0) / h) for p in ps)
            gy0 = min(round((p[4] - Y0) / h) for p in ps)
            gx1 = max(round((p[3] - X0) / h) + p[1] for p in ps)
            gy1 = max(round((p[4] - Y0) / h) + p[2] for p in ps)
            imgs.append((gx1 - gx0, gy1 - gy0, lmax - m))
        wx = max(round((p[3] - X0) / h0) + p[1] for p in pats if p[0] == 0) << lmax
        wy = max(round((p[4] - Y0) / h0) + p[2] for p in pats if p[0] == 0) << lmax
    return _pad(wx), _pad(wy), imgs


def algorithmic_flops(wl, info, stage, nout=2):
    """Conventional flop counts: 5 L log2 L per complex FFT of length L, plus
    the spectral multiply-adds (8 flops per field per bin; about 60 per bin for
    the central-slope spectrum; 10 per field and target for level convolutions);
    the direct sum counts 28 FP32 operations per target-corner pair (FMA = 2).
    nout = 1: the potential (one output; slopes formed in the row pass)."""
    import math
    total = 0.0
    if info.get("cross_mode") == 2:
        px, py, imgs = lv_geometry(wl)
        qx = px // 2 + 1
        fft = lambda n: 5.0 * n * math.log2(n)
        L = len(imgs)
        for nx, ny, s in imgs:
            pcx, pcy = px >> _lv_cexp(s, px), py >> _lv_cexp(s, py)
            if stage == "row_fwd":
                total += 3 * (ny / 2) * fft(pcx)
            # as a target, the level's bins are folded onto its compact lengths
            # before the inverse transforms from 4096-point transforms up
            tcx = pcx if px >= 4096 else px
            tcy = pcy if py >= 4096 else py
            if stage == "col_conv":
                total += (pcx // 2 + 1) * 3 * fft(pcy) + qx * (nout * fft(tcy) + L * 3 * 5 * nout * py)
            elif stage == "row_inv":
                total += nout * (ny / 2) * fft(tcx)
        return total
    for p in wl["patches"]:
        nx, ny = p[1], p[2]
        px, py = _pad(nx), _pad(ny)
        qx = px // 2 + 1
        fft_x = 5.0 * px * math.log2(px)
        fft_y = 5.0 * py * math.log2(py)
        central = wl["slope_mode"] == 1 and nout == 2
        nfwd = 1 if wl["slope_mode"] == 0 or central else 3
        if stage == "row_fwd":
            total += nfwd * (ny / 2) * fft_x + (fft_y if central else 0)
        elif stage == "col_conv":
            total += qx * ((nfwd + nout) * fft_y + (60 if central else 4 * nout * nfwd) * py)
        elif stage == "row_inv":
            total += nout * (ny / 2) * fft_x  # two rows per transform
    if stage == "cross_direct":
        # FP32 plans: 30 flops per target-cell pair for the force (the far-field
        # expansion through H^4, FMA = 2), 16 for the potential (its moments
        # through p^3); FP64 plans: 28 per target-corner pair
        fp32 = wl.get("precision", "fp32") == "fp32"
        total = (30.0 if nout == 2 else 16.0) if fp32 else 28.0
        if wl.get("z"):
            # off the plane: FP32 plans 2 x 2 Gauss nodes per far pair at 16 flops each
            # (3 x 3 within SG_FAR_R4 cells); FP64 plans the corner form, 36 per target-corner pair
            total = 64.0 if fp32 else 36.0
        total *= info["cross_pairs"]
    return total


def algorithmic_bytes(wl, info, stage, nout=2):
    """Bytes a stage must move per solve (see the design notes): FP32 complex
    intermediates of (P/2+1) x ny bins per field, spectra planes, inputs, outputs.
    Level convolutions: the forward column pass writes compact source spectra
    (a level of cells 2^s finest cells wide: P/2^s per axis); the column-MAC
    launch of all target levels reads them once, and once each distinct set of
    compressed kernel planes (6 real quarter planes per (source width, sample
    shift); 3 for the potential, nout = 1, which has one output)."""
    es = 4
    cs = 8
    total = 0
    if info.get("cross_mode") == 2:
        px, py, imgs = lv_geometry(wl)
        qx, qy = px // 2 + 1, py // 2 + 1
        L = len(imgs)
        for nx, ny, s in imgs:
            qxc, pcy = (px >> _lv_cexp(s, px)) // 2 + 1, py >> _lv_cexp(s, py)
            if stage == "row_fwd":
                total += 3 * nx * ny * es + 3 * qxc * ny * cs
            elif stage == "col_conv":
                total += 3 * qxc * ny * cs + 3 * qxc * pcy * cs       # compact column transforms of this level
                total += 3 * qxc * pcy * cs                         # read once by the column-MAC launch
                total += nout * qx * ny * cs                        # this level's inverse columns
            elif stage == "row_inv":
                total += nout * qx * ny * cs + nout * nx * ny * es
        if stage == "col_conv":
            # kernel planes: one set of 6 (3) real quarter planes per distinct (source width, sample shift)
            keys = {(sm, (sm >= 1) - (sl >= 1)) for _, _, sm in imgs for _, _, sl in imgs}
            total += len(keys) * 3 * nout * qx * qy * es
        return total
    # central slopes are formed from sigma's transforms: one field is transformed
    # (the potential forms them in the row pass: three fields)
    nf = 1 if wl["slope_mode"] == 0 or (wl["slope_mode"] == 1 and nout == 2) else 3
    for p in wl["patches"]:
        nx, ny = p[1], p[2]
        px, py = _pad(nx), _pad(ny)
        qx, qy = px // 2 + 1, py // 2 + 1
        inputs = nx * ny * es * (1 if wl["slope_mode"] != 2 else 3)
        if stage == "row_fwd":
            total += inputs + nf * qx * ny * 2 * es
        elif stage == "col_conv":
            total += nf * qx * ny * 2 * es + 3 * nout * qx * qy * es + nout * qx * ny * 2 * es
        elif stage == "row_inv":
            total += nout * qx * ny * 2 * es + nout * nx * ny * es
    if stage in ("corner_weights", "cross_direct"):
        total = info["ncells"] * es * 3
    return total


# ---------------------------------------------------------- reference arm --

def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]()
    pot = args.quantity == "potential"
    orc = OracleSample(wl, potential=pot)
    for _ in range(args.warmup):
        orc.run(8)
    times, tps_all, thr, what = [], [], 0, ""
    for _ in range(args.steps):
        sps, tps, secs, thr, what = orc.run(args.ref_targets)
        times.append(secs)
        tps_all.append(tps)
    tps = args.steps * args.ref_targets / sum(times)
    value = tps / wl["targets"]
    line = {
        "impl": "reference", "metric": METRIC_POTENTIAL if pot else METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(wl["config"], precision="fp64", parallelism="host cores",
                       **({"quantity": "potential"} if pot else {})),
        "target_cells_per_s": tps,
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": thr, "kind": "oracle",
                         "sample": "each step: " + what},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="spiral1024", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-targets", type=int, default=2048)
    ap.add_argument("--ref-targets", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve", action="store_true", help="run the request-server workload instead")
    ap.add_argument("--batch", action="store_true", help="run the graph-captured batch workload instead")
    ap.add_argument("--batch-size", type=int, default=64)
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--cross", default="auto", choices=["auto", "direct", "levels"],
                    help="how the FP32 plan sums pairs of cells in different patches (hierarchies)")
    ap.add_argument("--quantity", default="force", choices=["force", "potential"],
                    help="what a step computes (the potential: in-plane patch workloads)")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-sweep", action="store_true", help="also run loads 0.3, 0.5, 1.0 on a tenth of the stream")
    ap.add_argument("--serve-inflight", type=int, default=8)
    ap.add_argument("--serve-budget-gb", type=int, default=64)
    ap.add_argument("--serve-load", type=float, default=0.8)
    ap.add_argument("--serve-fp64-seconds", type=float, default=20.0)
    ap.add_argument("--serve-e2e-requests", type=int, default=2000)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.serve:
        run_serve(args)
    elif args.batch:
        run_batch(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
