"""The C-ABI library loads and exports what include/sg.h declares; host-only calls (no GPU)."""
import pytest

from paper_2001_02765_gb300 import sg
from paper_2001_02765_gb300 import workloads as W
from tests._lib import ensure_built, header_functions


@pytest.fixture(scope="module")
def lib():
    return ensure_built()


def test_header_declares_binding_names():
    assert header_functions() == sg.exported_names()


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_version_and_strerror(lib):
    assert sg.sg_version() >= 100
    assert sg.strerror(sg.SG_EINVAL) == "invalid argument"
    assert sg.strerror(99) == "unknown status"


def test_validate_uniform_and_nested(lib):
    assert sg.sg_geom_validate([(0,) + W.unit_grid(64)]) == sg.SG_OK
    pat = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(256, 3))]
    assert sg.sg_geom_validate(pat) == sg.SG_OK
    t10 = [(0, 4, 4, 0.0, 0.0, 0.25), (1, 2, 2, 0.25, 0.25, 0.125), (1, 2, 2, 0.5, 0.5, 0.125),
           (2, 2, 2, 0.25, 0.375, 0.0625), (2, 2, 2, 0.375, 0.25, 0.0625)]
    assert sg.sg_geom_validate(t10) == sg.SG_OK


@pytest.mark.parametrize("bad, why", [
    ([], "no patches"),
    ([(0, 0, 4, 0.0, 0.0, 0.1)], "empty patch"),
    ([(0, 4096, 4, 0.0, 0.0, 0.1)], "too large"),
    ([(0, 4, 4, 0.0, 0.0, -0.1)], "negative h"),
    ([(1, 4, 4, 0.0, 0.0, 0.1)], "first patch not level 0"),
    ([(0, 8, 8, 0.0, 0.0, 0.1), (1, 4, 4, 0.2, 0.2, 0.06)], "h not halved"),
    ([(0, 8, 8, 0.0, 0.0, 0.1), (1, 3, 4, 0.2, 0.2, 0.05)], "odd refined size"),
    ([(0, 8, 8, 0.0, 0.0, 0.1), (1, 4, 4, 0.25, 0.2, 0.05)], "off the parent lattice"),
    ([(0, 8, 8, 0.0, 0.0, 0.1), (1, 20, 4, 0.2, 0.2, 0.05)], "outside the parent"),
    ([(0, 8, 8, 0.0, 0.0, 0.1), (1, 4, 4, 0.2, 0.2, 0.05), (1, 4, 4, 0.3, 0.2, 0.05)], "same-level overlap"),
    ([(0, 8, 8, 0.0, 0.0, 0.1), (0, 8, 8, 0.4, 0.0, 0.1)], "level-0 overlap"),
    ([(0, 8, 8, 0.0, 0.0, 0.1), (0, 8, 8, 0.85, 0.0, 0.1)], "level-0 off lattice"),
])
def test_validate_rejects(lib, bad, why):
    assert sg.sg_geom_validate(bad) == sg.SG_EINVAL, why


def test_validate_central_slopes_on_amr(lib):
    """Central slopes are the neighbour-leaf rule on hierarchies, in the plane
    and off it."""
    pat = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(16, 2))]
    assert sg.sg_geom_validate(pat, slope_mode=sg.SG_SLOPES_CENTRAL) == sg.SG_OK
    assert sg.sg_geom_validate(pat[:1], slope_mode=sg.SG_SLOPES_CENTRAL) == sg.SG_OK
    assert sg.sg_geom_validate(pat, slope_mode=sg.SG_SLOPES_CENTRAL, z=0.1) == sg.SG_OK


def test_plan_bytes_estimate(lib):
    one = sg.sg_plan_bytes([(0,) + W.unit_grid(1024)], sg.SG_FP32)
    two = sg.sg_plan_bytes([(0,) + W.unit_grid(1024)], sg.SG_FP64)
    assert 40e6 < one < 200e6 and 1.8 < two / one < 2.2
    amr = sg.sg_plan_bytes([(lev,) + p for lev, p in enumerate(W.centred_nested_patches(256, 3))], sg.SG_FP32)
    assert amr > 0
    with pytest.raises(sg.SgError):
        sg.sg_plan_bytes([(0, 0, 0, 0.0, 0.0, 1.0)])


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(sg.SgLibraryMissing):
        sg.load(str(tmp_path / "libsg.so"))


def test_cross_mode_rules(lib):
    pat = [(lev,) + p for lev, p in enumerate(W.centred_nested_patches(64, 3))]
    assert sg.sg_geom_validate(pat, cross_mode=3) == sg.SG_EINVAL
    for m in (0, 1, 2):
        assert sg.sg_geom_validate(pat, cross_mode=m) == sg.SG_OK
    # level convolutions keep no per-patch spectra and no corner tiles; they add kernel spectra
    direct = sg.sg_plan_bytes(pat, sg.SG_FP32, cross_mode=1)
    levels = sg.sg_plan_bytes(pat, sg.SG_FP32, cross_mode=2)
    assert direct > 0 and levels > 0 and levels != direct


def test_tune_table_host_rules(lib):
    """The launch-shape table: defaults, candidates only, reset with zeros (host only)."""
    d = sg.sg_tune_get(sg.SG_FP32, 2048)
    assert d == {"row_fwd": 2, "row_inv": 4, "col": 1, "col_central": 1}
    sg.sg_tune_set(sg.SG_FP32, 2048, {"row_fwd": 1, "col": 2})
    assert sg.sg_tune_get(sg.SG_FP32, 2048)["row_fwd"] == 1 and sg.sg_tune_get(sg.SG_FP32, 2048)["col"] == 2
    with pytest.raises(sg.SgError) as e:
        sg.sg_tune_set(sg.SG_FP32, 2048, {"row_fwd": 3})
    assert e.value.status == sg.SG_EINVAL and "candidate" in str(e.value)
    with pytest.raises(sg.SgError):
        sg.sg_tune_set(sg.SG_FP32, 3000, [0, 0, 0, 0])
    sg.sg_tune_set(sg.SG_FP32, 2048, [0, 0, 0, 0])
    assert sg.sg_tune_get(sg.SG_FP32, 2048) == d
    assert sg.sg_tune_get(sg.SG_FP64, 4096)["col"] == 1


def test_host_side_argument_errors(lib):
    """Entry points reject null handles and bad arguments on the host, before
    touching the device (no GPU needed)."""
    with pytest.raises(sg.SgError) as e:
        sg.sg_server_set_group_limit(None, 4)
    assert e.value.status == sg.SG_EINVAL
    with pytest.raises(sg.SgError) as e:
        sg.sg_plan_autotune(None, 3)
    assert e.value.status == sg.SG_EINVAL
    with pytest.raises(sg.SgError) as e:
        sg.sg_plan_direct_shape(None)
    assert e.value.status == sg.SG_EINVAL
    with pytest.raises(sg.SgError) as e:
        sg.sg_plan_wait(None)
    assert e.value.status == sg.SG_EINVAL
    with pytest.raises(sg.SgError) as e:
        sg.sg_force_host_async(None, 1, 0, 0, 1, 1)
    assert e.value.status == sg.SG_EINVAL
    with pytest.raises(sg.SgError) as e:
        sg.sg_potential_zones(None, 1, 0, 0, 1)
    assert e.value.status == sg.SG_EINVAL
    with pytest.raises(sg.SgError) as e:
        sg.sg_batch_create([], [], [], [], [], [], mode=sg.SG_BATCH_PERSISTENT)
    assert e.value.status == sg.SG_EINVAL
    with pytest.raises(sg.SgError) as e:
        sg.sg_batch_layout(None)
    assert e.value.status == sg.SG_EINVAL
