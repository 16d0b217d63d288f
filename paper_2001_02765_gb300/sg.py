"""Python binding of the C ABI in include/sg.h (argument marshalling only).

Every step of a solve runs in the CUDA library libsg.so; this module converts
arguments and checks status codes. Loading fails loudly (SgLibraryMissing) when
the library has not been built: there is no fallback implementation.

Low-level names mirror the C entry points (sg_plan_create, sg_force, ...);
``Plan`` is a small convenience wrapper that takes torch tensors (PyTorch is
used for device memory and streams only).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsg.so")

SG_OK, SG_EINVAL, SG_ENOMEM, SG_EBUDGET, SG_ECUDA, SG_ETIMEOUT, SG_EBUSY, SG_ECANCELLED, SG_ENOTFOUND = range(9)
SG_FP64, SG_FP32 = 0, 1
SG_SLOPES_NONE, SG_SLOPES_CENTRAL, SG_SLOPES_CALLER = 0, 1, 2
SG_CROSS_AUTO, SG_CROSS_DIRECT, SG_CROSS_LEVELS = 0, 1, 2
KERNEL_NAMES = ("x0", "xx", "xy", "y0", "yx", "yy", "z0", "zx", "zy")


class SgLibraryMissing(ImportError):
    pass


class SgError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        msg = "%s failed: %s (%d)" % (where, strerror(status), status)
        if detail:
            msg += ": " + detail
        super().__init__(msg)


class sg_patch(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("h", ctypes.c_double)]


class sg_geom(ctypes.Structure):
    _fields_ = [("npatches", ctypes.c_int), ("patches", ctypes.POINTER(sg_patch)),
                ("G", ctypes.c_double), ("slope_mode", ctypes.c_int), ("z", ctypes.c_double),
                ("masks", ctypes.c_void_p), ("cross_mode", ctypes.c_int)]


class sg_plan_info(ctypes.Structure):
    _fields_ = [("npatches", ctypes.c_int), ("ncells", ctypes.c_int64), ("nleaves", ctypes.c_int64),
                ("cross_pairs", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("scratch_bytes", ctypes.c_int64), ("max_pad", ctypes.c_int), ("nzones", ctypes.c_int64),
                ("launches", ctypes.c_int), ("cross_mode", ctypes.c_int)]


_I32P = ctypes.POINTER(ctypes.c_int32)
_I64P = ctypes.POINTER(ctypes.c_int64)


class sg_zones(ctypes.Structure):
    _fields_ = [("nx0", ctypes.c_int), ("ny0", ctypes.c_int), ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("h0", ctypes.c_double), ("nzones", ctypes.c_int64), ("level", _I32P), ("ix", _I32P),
                ("iy", _I32P)]


class sg_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("cancelled", ctypes.c_uint64), ("rejected", ctypes.c_uint64), ("queued", ctypes.c_int64),
                ("running", ctypes.c_int64), ("bytes_in_use", ctypes.c_int64), ("peak_bytes", ctypes.c_int64),
                ("latency_count", ctypes.c_int64), ("latency_p50_ms", ctypes.c_double),
                ("latency_p99_ms", ctypes.c_double), ("latency_mean_ms", ctypes.c_double),
                ("groups_started", ctypes.c_uint64), ("grouped_requests", ctypes.c_uint64)]


# name -> (restype, argtypes)
_VP = ctypes.c_void_p
_SIGNATURES = {
    "sg_geom_validate": (ctypes.c_int, [ctypes.POINTER(sg_geom)]),
    "sg_plan_create": (ctypes.c_int, [ctypes.POINTER(sg_geom), ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(_VP)]),
    "sg_plan_destroy": (ctypes.c_int, [_VP]),
    "sg_plan_get_info": (ctypes.c_int, [_VP, ctypes.POINTER(sg_plan_info)]),
    "sg_plan_bytes": (ctypes.c_int, [ctypes.POINTER(sg_geom), ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]),
    "sg_kernel_tables": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t]),
    "sg_force": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "sg_force_host": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "sg_force_host_async": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "sg_plan_wait": (ctypes.c_int, [_VP, _VP]),
    "sg_force3": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "sg_potential": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "sg_plan_set_timing": (ctypes.c_int, [_VP, ctypes.c_int]),
    "sg_plan_set_wait_limit": (ctypes.c_int, [_VP, ctypes.c_int]),
    "sg_plan_check_error": (ctypes.c_int, [_VP]),
    "sg_batch_check_error": (ctypes.c_int, [_VP]),
    "sg_plan_get_timing": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "sg_direct_force_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                              _VP, _VP, _VP, _VP, _VP, _VP]),
    "sg_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                       ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                       ctypes.POINTER(_VP)]),
    "sg_batch_launch": (ctypes.c_int, [_VP, _VP]),
    "sg_batch_destroy": (ctypes.c_int, [_VP]),
    "sg_batch_launches": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "sg_batch_create_mode": (ctypes.c_int, [ctypes.c_int] + [ctypes.POINTER(_VP)] * 6 + [ctypes.c_int,
                                                                                         ctypes.POINTER(_VP)]),
    "sg_batch_layout": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]),
    "sg_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(_VP)]),
    "sg_server_destroy": (ctypes.c_int, [_VP]),
    "sg_submit": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(ctypes.c_uint64)]),
    "sg_poll": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "sg_wait": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_double)]),
    "sg_cancel": (ctypes.c_int, [_VP, ctypes.c_uint64]),
    "sg_server_get_stats": (ctypes.c_int, [_VP, ctypes.POINTER(sg_server_stats), ctypes.c_int]),
    "sg_server_set_group_limit": (ctypes.c_int, [_VP, ctypes.c_int]),
    "sg_plan_autotune": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "sg_plan_direct_shape": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "sg_plan_create_zones": (ctypes.c_int, [ctypes.POINTER(sg_zones), ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(_VP)]),
    "sg_force_zones": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "sg_potential_zones": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "sg_plan_zone_slots": (ctypes.c_int, [_VP, _I64P, ctypes.c_int64]),
    "sg_zones_from_records": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                             ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, _I32P, _I32P, _I32P]),
    "sg_zones_links": (ctypes.c_int, [ctypes.POINTER(sg_zones), _I64P, ctypes.POINTER(ctypes.c_uint8), _I64P]),
    "sg_tune_get": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "sg_tune_set": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "sg_autotune": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_double)]),
    "sg_alu_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "sg_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "sg_last_error": (ctypes.c_char_p, []),
    "sg_version": (ctypes.c_int, []),
}

_lib = None


def exported_names():
    """Names of the C entry points this binding expects the library to export."""
    return sorted(_SIGNATURES)


def load(path=None):
    """Load libsg.so (once). Raises SgLibraryMissing if it is not built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise SgLibraryMissing("CUDA library %s is not built; run __graft_entry__.build() "
                               "(python -m paper_2001_02765_gb300.build)" % p)
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def strerror(status):
    try:
        return load().sg_strerror(int(status)).decode()
    except SgLibraryMissing:
        return "status %d" % status


def last_error():
    return load().sg_last_error().decode()


def _check(status, where):
    if status != SG_OK:
        raise SgError(status, where, last_error())


def make_geom(patches, G=1.0, slope_mode=SG_SLOPES_CALLER, z=0.0, masks=None, cross_mode=SG_CROSS_AUTO):
    """patches: iterable of (level, nx, ny, x0, y0, h); masks: None or one entry per
    patch (None, or an [ny, nx] array, nonzero where the cell exists).
    Returns (sg_geom, keepalive objects)."""
    patches = list(patches)
    arr = (sg_patch * len(patches))(*[sg_patch(int(p[0]), int(p[1]), int(p[2]), float(p[3]), float(p[4]), float(p[5]))
                                      for p in patches])
    keep = [arr]
    mptr = None
    if masks is not None:
        if len(masks) != len(patches):
            raise ValueError("one mask entry per patch")
        bufs = [None if m is None else np.ascontiguousarray(np.asarray(m) != 0, dtype=np.uint8).ravel() for m in masks]
        ptrs = (ctypes.c_void_p * len(bufs))(*[None if b is None else b.ctypes.data for b in bufs])
        keep += [bufs, ptrs]
        mptr = ctypes.cast(ptrs, ctypes.c_void_p)
    g = sg_geom(len(patches), ctypes.cast(arr, ctypes.POINTER(sg_patch)), float(G), int(slope_mode), float(z), mptr,
                int(cross_mode))
    return g, keep


def sg_geom_validate(patches, G=1.0, slope_mode=SG_SLOPES_CALLER, z=0.0, masks=None, cross_mode=SG_CROSS_AUTO):
    g, _keep = make_geom(patches, G, slope_mode, z, masks, cross_mode)
    return load().sg_geom_validate(ctypes.byref(g))


def sg_plan_bytes(patches, precision=SG_FP32, G=1.0, slope_mode=SG_SLOPES_CALLER, z=0.0, masks=None,
                  cross_mode=SG_CROSS_AUTO):
    g, _keep = make_geom(patches, G, slope_mode, z, masks, cross_mode)
    out = ctypes.c_int64(0)
    _check(load().sg_plan_bytes(ctypes.byref(g), int(precision), ctypes.byref(out)), "sg_plan_bytes")
    return int(out.value)


def sg_plan_create(patches, precision=SG_FP32, G=1.0, slope_mode=SG_SLOPES_CALLER, hbm_budget=0, z=0.0, masks=None,
                   cross_mode=SG_CROSS_AUTO):
    g, _keep = make_geom(patches, G, slope_mode, z, masks, cross_mode)
    h = _VP()
    _check(load().sg_plan_create(ctypes.byref(g), int(precision), int(hbm_budget), ctypes.byref(h)), "sg_plan_create")
    return h.value


def sg_plan_destroy(handle):
    if handle:
        _check(load().sg_plan_destroy(handle), "sg_plan_destroy")


def sg_plan_get_info(handle):
    info = sg_plan_info()
    _check(load().sg_plan_get_info(handle, ctypes.byref(info)), "sg_plan_get_info")
    return {k: getattr(info, k) for k, _ in sg_plan_info._fields_}


def sg_kernel_tables(handle, patch, which, nx, ny):
    n = (2 * nx - 1) * (2 * ny - 1)
    out = np.empty(n, dtype=np.float64)
    _check(load().sg_kernel_tables(handle, int(patch), int(which),
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n), "sg_kernel_tables")
    return out.reshape(2 * ny - 1, 2 * nx - 1)


def sg_force(handle, sigma_ptr, dx_ptr, dy_ptr, fx_ptr, fy_ptr, stream_ptr=0):
    """Raw device pointers (ints); enqueues one solve on the stream."""
    _check(load().sg_force(handle, sigma_ptr, dx_ptr or None, dy_ptr or None, fx_ptr, fy_ptr, stream_ptr or None),
           "sg_force")


def sg_force3(handle, sigma_ptr, dx_ptr, dy_ptr, fx_ptr, fy_ptr, fz_ptr, stream_ptr=0):
    """Raw device pointers (ints); enqueues a solve with Fz."""
    _check(load().sg_force3(handle, sigma_ptr, dx_ptr or None, dy_ptr or None, fx_ptr, fy_ptr, fz_ptr,
                            stream_ptr or None), "sg_force3")


def sg_potential(handle, sigma_ptr, dx_ptr, dy_ptr, phi_ptr, stream_ptr=0):
    """Raw device pointers (ints); enqueues the potential (builds its spectra at the first call)."""
    _check(load().sg_potential(handle, sigma_ptr, dx_ptr or None, dy_ptr or None, phi_ptr, stream_ptr or None),
           "sg_potential")


def sg_force_host(handle, sigma_ptr, dx_ptr, dy_ptr, fx_ptr, fy_ptr, stream_ptr=0):
    """Raw host pointers (ints); synchronous."""
    _check(load().sg_force_host(handle, sigma_ptr, dx_ptr or None, dy_ptr or None, fx_ptr, fy_ptr,
                                stream_ptr or None), "sg_force_host")


def sg_force_host_async(handle, sigma_ptr, dx_ptr, dy_ptr, fx_ptr, fy_ptr, stream_ptr=0):
    """Raw host pointers (ints); enqueues only: the buffers stay in use until sg_plan_wait."""
    _check(load().sg_force_host_async(handle, sigma_ptr, dx_ptr or None, dy_ptr or None, fx_ptr, fy_ptr,
                                      stream_ptr or None), "sg_force_host_async")


def sg_plan_wait(handle, stream_ptr=0):
    """Wait for the stream, then report the plan's device error word (SG_ETIMEOUT raises)."""
    _check(load().sg_plan_wait(handle, stream_ptr or None), "sg_plan_wait")


STAGE_NAMES = ("row_fwd", "col_conv", "row_inv", "corner_weights", "cross_direct", "composite")


def sg_plan_set_wait_limit(handle, tries):
    _check(load().sg_plan_set_wait_limit(handle, int(tries)), "sg_plan_set_wait_limit")


def sg_plan_check_error(handle):
    """Status of the plan's device error word (waits for the device): SG_OK or SG_ETIMEOUT."""
    return load().sg_plan_check_error(handle)


def sg_batch_check_error(batch):
    return load().sg_batch_check_error(batch)


def sg_plan_set_timing(handle, enable):
    _check(load().sg_plan_set_timing(handle, int(bool(enable))), "sg_plan_set_timing")


def sg_plan_get_timing(handle):
    ms = (ctypes.c_double * len(STAGE_NAMES))()
    _check(load().sg_plan_get_timing(handle, ms, len(STAGE_NAMES)), "sg_plan_get_timing")
    return dict(zip(STAGE_NAMES, list(ms)))


def sg_direct_force_static(nx, ny, h, G, sigma_ptr, dx_ptr, dy_ptr, fx_ptr, fy_ptr, stream_ptr=0):
    """Raw device pointers (ints) of float32 arrays; allocation-free uniform direct sum."""
    _check(load().sg_direct_force_static(int(nx), int(ny), float(h), float(G), sigma_ptr, dx_ptr or None,
                                         dy_ptr or None, fx_ptr, fy_ptr, stream_ptr or None), "sg_direct_force_static")


SG_BATCH_AUTO, SG_BATCH_PERSISTENT, SG_BATCH_GROUPED = 0, 1, 2


def sg_batch_create(plan_handles, sigma_ptrs, dx_ptrs, dy_ptrs, fx_ptrs, fy_ptrs, mode=None):
    """Bind n solves (raw device pointers; dx/dy entries 0 where unused) into one
    graph; mode None is sg_batch_create (SG_BATCH_AUTO), else sg_batch_create_mode."""
    n = len(plan_handles)
    arr = lambda v: (_VP * n)(*[x or None for x in v])
    h = _VP()
    if mode is None:
        _check(load().sg_batch_create(n, arr(plan_handles), arr(sigma_ptrs), arr(dx_ptrs), arr(dy_ptrs),
                                      arr(fx_ptrs), arr(fy_ptrs), ctypes.byref(h)), "sg_batch_create")
    else:
        _check(load().sg_batch_create_mode(n, arr(plan_handles), arr(sigma_ptrs), arr(dx_ptrs), arr(dy_ptrs),
                                           arr(fx_ptrs), arr(fy_ptrs), int(mode), ctypes.byref(h)),
               "sg_batch_create_mode")
    return h.value


def sg_batch_layout(batch):
    """(mode, ms_persistent, ms_grouped) of a batch."""
    m, a, b = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    _check(load().sg_batch_layout(batch, ctypes.byref(m), ctypes.byref(a), ctypes.byref(b)), "sg_batch_layout")
    return m.value, a.value, b.value


def sg_batch_launch(batch, stream_ptr=0):
    _check(load().sg_batch_launch(batch, stream_ptr or None), "sg_batch_launch")


def sg_batch_destroy(batch):
    if batch:
        _check(load().sg_batch_destroy(batch), "sg_batch_destroy")


def sg_batch_launches(batch):
    """Kernel launches one sg_batch_launch replays."""
    n = ctypes.c_int(0)
    _check(load().sg_batch_launches(batch, ctypes.byref(n)), "sg_batch_launches")
    return n.value


def sg_server_create(hbm_budget=0, max_inflight=8):
    h = _VP()
    _check(load().sg_server_create(int(hbm_budget), int(max_inflight), ctypes.byref(h)), "sg_server_create")
    return h.value


def sg_server_destroy(handle):
    if handle:
        _check(load().sg_server_destroy(handle), "sg_server_destroy")


def sg_submit(server, plan_handle, sigma_ptr, dx_ptr, dy_ptr, fx_ptr, fy_ptr):
    """Queue a solve (raw device pointers). Returns the ticket; raises SgError (e.g. SG_EBUDGET)."""
    t = ctypes.c_uint64(0)
    _check(load().sg_submit(server, plan_handle, sigma_ptr, dx_ptr or None, dy_ptr or None, fx_ptr, fy_ptr,
                            ctypes.byref(t)), "sg_submit")
    return int(t.value)


def sg_poll(server, ticket):
    """Returns (status, result, latency_ms): status SG_OK when finished, SG_EBUSY, or SG_ENOTFOUND."""
    res = ctypes.c_int(0)
    lat = ctypes.c_double(0.0)
    st = load().sg_poll(server, int(ticket), ctypes.byref(res), ctypes.byref(lat))
    return st, res.value, lat.value


def sg_wait(server, ticket, timeout_ms):
    """Returns (status, result, latency_ms): status SG_OK, SG_ETIMEOUT or SG_ENOTFOUND."""
    res = ctypes.c_int(0)
    lat = ctypes.c_double(0.0)
    st = load().sg_wait(server, int(ticket), float(timeout_ms), ctypes.byref(res), ctypes.byref(lat))
    return st, res.value, lat.value


def sg_cancel(server, ticket):
    return load().sg_cancel(server, int(ticket))


def sg_server_get_stats(server, reset_latencies=False):
    out = sg_server_stats()
    _check(load().sg_server_get_stats(server, ctypes.byref(out), int(bool(reset_latencies))), "sg_server_get_stats")
    return {k: getattr(out, k) for k, _ in sg_server_stats._fields_}


def sg_plan_autotune(handle, reps=5):
    """Tune a plan's cross-patch direct sum; returns the best median solve time (ms)."""
    ms = ctypes.c_double()
    _check(load().sg_plan_autotune(handle, int(reps), ctypes.byref(ms)), "sg_plan_autotune")
    return ms.value


def sg_plan_direct_shape(handle):
    """(source-tile ranges per target block, CTAs of the FP32 far-field launch)."""
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(load().sg_plan_direct_shape(handle, ctypes.byref(a), ctypes.byref(b)), "sg_plan_direct_shape")
    return a.value, b.value


def sg_server_set_group_limit(server, max_members):
    """Most requests admitted together as one group (1 admits every request alone)."""
    _check(load().sg_server_set_group_limit(server, int(max_members)), "sg_server_set_group_limit")


SG_PEAK_FP64_FMA, SG_PEAK_FP32_FMA, SG_PEAK_FP32_LG2 = 0, 1, 2


def sg_alu_peak(kind):
    """Measured pipe throughput of the current device (flop/s for the FMA kinds,
    results/s for the base-2 logarithm)."""
    out = ctypes.c_double(0.0)
    _check(load().sg_alu_peak(int(kind), ctypes.byref(out)), "sg_alu_peak")
    return float(out.value)


def sg_version():
    return int(load().sg_version())


TUNE_KNOBS = ("row_fwd", "row_inv", "col", "col_central")


def sg_tune_get(precision, pad):
    out = (ctypes.c_int * 4)()
    _check(load().sg_tune_get(int(precision), int(pad), out), "sg_tune_get")
    return dict(zip(TUNE_KNOBS, list(out)))


def sg_tune_set(precision, pad, shape):
    """shape: dict of TUNE_KNOBS (missing = default) or a 4-sequence (0 = default)."""
    vals = [int(shape.get(k, 0)) for k in TUNE_KNOBS] if isinstance(shape, dict) else [int(v) for v in shape]
    arr = (ctypes.c_int * 4)(*vals)
    _check(load().sg_tune_set(int(precision), int(pad), arr), "sg_tune_set")


def sg_autotune(precision, min_pad, max_pad, reps=5):
    """Tune the launch shapes; returns {pad: (shapes, best solve ms)}."""
    pads = []
    p = int(min_pad)
    while p <= int(max_pad):
        pads.append(p)
        p *= 2
    best = (ctypes.c_double * max(1, len(pads)))()
    _check(load().sg_autotune(int(precision), int(min_pad), int(max_pad), int(reps), best), "sg_autotune")
    return {p: (sg_tune_get(precision, p), best[i]) for i, p in enumerate(pads)}


def make_zones(nx0, ny0, x0, y0, h0, level, ix, iy):
    """sg_zones over int32 copies of the zone arrays. Returns (sg_zones, keepalive)."""
    arrs = [np.ascontiguousarray(a, dtype=np.int32).ravel() for a in (level, ix, iy)]
    if not (arrs[0].size == arrs[1].size == arrs[2].size):
        raise ValueError("level, ix, iy differ in length")
    z = sg_zones(int(nx0), int(ny0), float(x0), float(y0), float(h0), arrs[0].size,
                 *[a.ctypes.data_as(_I32P) for a in arrs])
    return z, arrs


def sg_plan_create_zones(zone_args, precision=SG_FP32, G=1.0, slope_mode=SG_SLOPES_CALLER, hbm_budget=0,
                         cross_mode=SG_CROSS_AUTO):
    """zone_args: (nx0, ny0, x0, y0, h0, level, ix, iy)."""
    z, _keep = make_zones(*zone_args)
    h = _VP()
    _check(load().sg_plan_create_zones(ctypes.byref(z), float(G), int(slope_mode), int(cross_mode), int(precision),
                                       int(hbm_budget), ctypes.byref(h)), "sg_plan_create_zones")
    return h.value


def sg_force_zones(handle, sigma_ptr, dx_ptr, dy_ptr, fx_ptr, fy_ptr, stream_ptr=0):
    """Raw device pointers (ints), zone-ordered arrays; enqueues one solve."""
    _check(load().sg_force_zones(handle, sigma_ptr, dx_ptr or None, dy_ptr or None, fx_ptr, fy_ptr,
                                 stream_ptr or None), "sg_force_zones")


def sg_potential_zones(handle, sigma_ptr, dx_ptr, dy_ptr, phi_ptr, stream_ptr=0):
    """Raw device pointers (ints), zone-ordered arrays; enqueues the potential."""
    _check(load().sg_potential_zones(handle, sigma_ptr, dx_ptr or None, dy_ptr or None, phi_ptr,
                                     stream_ptr or None), "sg_potential_zones")


def sg_plan_zone_slots(handle, nzones):
    out = np.empty(int(nzones), dtype=np.int64)
    _check(load().sg_plan_zone_slots(handle, out.ctypes.data_as(_I64P), out.size), "sg_plan_zone_slots")
    return out


def sg_zones_from_records(records, nx0, ny0, x0, y0, h0):
    """records: [n, ncols >= 6] array (ID x_c y_c L P EL ...). Returns int32 (level, ix, iy)."""
    rec = np.ascontiguousarray(records, dtype=np.float64)
    n, ncols = rec.shape
    out = [np.empty(n, dtype=np.int32) for _ in range(3)]
    _check(load().sg_zones_from_records(n, ncols, rec.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(nx0),
                                        int(ny0), float(x0), float(y0), float(h0),
                                        *[a.ctypes.data_as(_I32P) for a in out]), "sg_zones_from_records")
    return tuple(out)


def sg_zones_links(zone_args):
    """zone_args as for sg_plan_create_zones. Returns (parent [n], leaf [n] bool, neighbours [n, 4]),
    1-based indices, 0 for none."""
    z, _keep = make_zones(*zone_args)
    n = z.nzones
    parent = np.empty(n, dtype=np.int64)
    leaf = np.empty(n, dtype=np.uint8)
    nb = np.empty(4 * n, dtype=np.int64)
    _check(load().sg_zones_links(ctypes.byref(z), parent.ctypes.data_as(_I64P),
                                 leaf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), nb.ctypes.data_as(_I64P)),
           "sg_zones_links")
    return parent, leaf.astype(bool), nb.reshape(n, 4)


# ------------------------------------------------------------ convenience --

class Plan:
    """A plan for one geometry; fields are torch tensors on the current CUDA device.

    patches: list of (level, nx, ny, x0, y0, h); fields are the per-patch
    row-major arrays concatenated (length ``ncells``).
    """

    def __init__(self, patches, precision="fp32", G=1.0, slope_mode=SG_SLOPES_CALLER, hbm_budget=0, z=0.0,
                 masks=None, cross_mode=SG_CROSS_AUTO):
        self.patches = [tuple(p) for p in patches]
        self.precision = SG_FP32 if precision in ("fp32", SG_FP32) else SG_FP64
        self.slope_mode = slope_mode
        self.G = G
        self.z = z
        self.handle = sg_plan_create(self.patches, self.precision, G, slope_mode, hbm_budget, z, masks, cross_mode)
        self.info = sg_plan_get_info(self.handle)

    @property
    def ncells(self):
        return self.info["ncells"]

    @property
    def dtype_name(self):
        return "float32" if self.precision == SG_FP32 else "float64"

    def close(self):
        if self.handle:
            sg_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def kernel_table(self, patch, which):
        p = self.patches[patch]
        w = KERNEL_NAMES.index(which) if isinstance(which, str) else int(which)
        return sg_kernel_tables(self.handle, patch, w, p[1], p[2])

    def _torch_dtype(self):
        import torch
        return torch.float32 if self.precision == SG_FP32 else torch.float64

    def empty_fields(self, n=2):
        import torch
        return [torch.empty(self.ncells, dtype=self._torch_dtype(), device="cuda") for _ in range(n)]

    def force(self, sigma, dx=None, dy=None, fx=None, fy=None, stream=None):
        """Enqueue a solve on `stream` (default: torch's current stream); returns (fx, fy)."""
        import torch
        dt = self._torch_dtype()
        for t in (sigma, dx, dy, fx, fy):
            if t is not None and (t.dtype != dt or not t.is_cuda or not t.is_contiguous() or t.numel() != self.ncells):
                raise ValueError("fields must be contiguous %s CUDA tensors of %d elements" % (dt, self.ncells))
        if fx is None:
            fx = torch.empty_like(sigma)
        if fy is None:
            fy = torch.empty_like(sigma)
        st = (stream or torch.cuda.current_stream()).cuda_stream
        sg_force(self.handle, sigma.data_ptr(), dx.data_ptr() if dx is not None else 0,
                 dy.data_ptr() if dy is not None else 0, fx.data_ptr(), fy.data_ptr(), st)
        return fx, fy

    def force3(self, sigma, dx=None, dy=None, stream=None):
        """Enqueue a solve with Fz (see sg_force3); returns (fx, fy, fz)."""
        import torch
        dt = self._torch_dtype()
        for t in (sigma, dx, dy):
            if t is not None and (t.dtype != dt or not t.is_cuda or not t.is_contiguous() or t.numel() != self.ncells):
                raise ValueError("fields must be contiguous %s CUDA tensors of %d elements" % (dt, self.ncells))
        fx, fy, fz = (torch.empty_like(sigma) for _ in range(3))
        st = (stream or torch.cuda.current_stream()).cuda_stream
        sg_force3(self.handle, sigma.data_ptr(), dx.data_ptr() if dx is not None else 0,
                  dy.data_ptr() if dy is not None else 0, fx.data_ptr(), fy.data_ptr(), fz.data_ptr(), st)
        return fx, fy, fz

    def potential(self, sigma, dx=None, dy=None, phi=None, stream=None):
        """Enqueue the mid-plane potential (see sg_potential); returns phi."""
        import torch
        dt = self._torch_dtype()
        for t in (sigma, dx, dy, phi):
            if t is not None and (t.dtype != dt or not t.is_cuda or not t.is_contiguous() or t.numel() != self.ncells):
                raise ValueError("fields must be contiguous %s CUDA tensors of %d elements" % (dt, self.ncells))
        if phi is None:
            phi = torch.empty_like(sigma)
        st = (stream or torch.cuda.current_stream()).cuda_stream
        sg_potential(self.handle, sigma.data_ptr(), dx.data_ptr() if dx is not None else 0,
                     dy.data_ptr() if dy is not None else 0, phi.data_ptr(), st)
        return phi

    def force_host(self, sigma, dx=None, dy=None, fx=None, fy=None, stream=None):
        """Solve from host arrays (numpy, or pinned torch CPU tensors); returns host (fx, fy)."""
        npdt = np.float32 if self.precision == SG_FP32 else np.float64

        def host_ptr(a):
            if a is None:
                return 0, None
            if isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a, dtype=npdt).ravel()
                return a.ctypes.data, a
            return a.data_ptr(), a  # torch CPU tensor

        ps, ks = host_ptr(sigma)
        pdx, kdx = host_ptr(dx)
        pdy, kdy = host_ptr(dy)
        if fx is None:
            fx = np.empty(self.ncells, dtype=npdt)
        if fy is None:
            fy = np.empty(self.ncells, dtype=npdt)
        pfx, _ = host_ptr(fx) if not isinstance(fx, np.ndarray) else (fx.ctypes.data, fx)
        pfy, _ = host_ptr(fy) if not isinstance(fy, np.ndarray) else (fy.ctypes.data, fy)
        st = 0
        if stream is not None:
            st = stream.cuda_stream
        sg_force_host(self.handle, ps, pdx, pdy, pfx, pfy, st)
        return fx, fy

    def force_host_async(self, sigma, dx, dy, fx, fy, stream=None):
        """Enqueue a solve from pinned torch CPU tensors (sigma, dx, dy; None
        where unused) into pinned fx, fy; the tensors stay in use until wait()."""
        p = lambda a: 0 if a is None else a.data_ptr()
        sg_force_host_async(self.handle, p(sigma), p(dx), p(dy), p(fx), p(fy),
                            0 if stream is None else stream.cuda_stream)

    def wait(self, stream=None):
        """Wait for a solve enqueued by force_host_async on `stream`."""
        sg_plan_wait(self.handle, 0 if stream is None else stream.cuda_stream)

    def split(self, flat):
        """Split a flat field array into per-patch [ny, nx] views."""
        out, off = [], 0
        for p in self.patches:
            n = p[1] * p[2]
            out.append(flat[off:off + n].reshape(p[2], p[1]))
            off += n
        return out


class ZonePlan(Plan):
    """A plan for a zone-by-zone hierarchy (see sg_plan_create_zones); fields are
    zone-ordered torch tensors of ``nzones`` elements."""

    def __init__(self, nx0, ny0, x0, y0, h0, level, ix, iy, precision="fp32", G=1.0, slope_mode=SG_SLOPES_CALLER,
                 hbm_budget=0, cross_mode=SG_CROSS_AUTO):
        self.patches = []
        self.precision = SG_FP32 if precision in ("fp32", SG_FP32) else SG_FP64
        self.slope_mode = slope_mode
        self.G = G
        self.z = 0.0
        self.handle = sg_plan_create_zones((nx0, ny0, x0, y0, h0, level, ix, iy), self.precision, G, slope_mode,
                                           hbm_budget, cross_mode)
        self.info = sg_plan_get_info(self.handle)

    @property
    def nzones(self):
        return self.info["nzones"]

    def slots(self):
        return sg_plan_zone_slots(self.handle, self.nzones)

    def force_zones(self, sigma, dx=None, dy=None, fx=None, fy=None, stream=None):
        """Enqueue a solve on zone-ordered tensors; returns (fx, fy), 0 at non-leaf zones."""
        import torch
        dt = self._torch_dtype()
        for t in (sigma, dx, dy, fx, fy):
            if t is not None and (t.dtype != dt or not t.is_cuda or not t.is_contiguous() or t.numel() != self.nzones):
                raise ValueError("fields must be contiguous %s CUDA tensors of %d elements" % (dt, self.nzones))
        if fx is None:
            fx = torch.empty_like(sigma)
        if fy is None:
            fy = torch.empty_like(sigma)
        st = (stream or torch.cuda.current_stream()).cuda_stream
        sg_force_zones(self.handle, sigma.data_ptr(), dx.data_ptr() if dx is not None else 0,
                       dy.data_ptr() if dy is not None else 0, fx.data_ptr(), fy.data_ptr(), st)
        return fx, fy

    def potential_zones(self, sigma, dx=None, dy=None, phi=None, stream=None):
        """Enqueue the potential on zone-ordered tensors; returns phi, 0 at non-leaf zones."""
        import torch
        dt = self._torch_dtype()
        for t in (sigma, dx, dy, phi):
            if t is not None and (t.dtype != dt or not t.is_cuda or not t.is_contiguous() or t.numel() != self.nzones):
                raise ValueError("fields must be contiguous %s CUDA tensors of %d elements" % (dt, self.nzones))
        if phi is None:
            phi = torch.empty_like(sigma)
        st = (stream or torch.cuda.current_stream()).cuda_stream
        sg_potential_zones(self.handle, sigma.data_ptr(), dx.data_ptr() if dx is not None else 0,
                           dy.data_ptr() if dy is not None else 0, phi.data_ptr(), st)
        return phi
