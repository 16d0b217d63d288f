"""Host-only parts of zone hierarchies and masked patches (no GPU): the record
importer (Table 10), zone links, and the validation rules."""
import numpy as np
import pytest

from paper_2001_02765_gb300 import sg
from paper_2001_02765_gb300 import workloads as W
from tests._lib import ensure_built
from tests.test_oracle_pins import _load_table

# Fig. 1 / Table 10: 4 x 4 level-1 zones on [0, 1]^2
T10_GRID = (4, 4, 0.0, 0.0, 0.25)


@pytest.fixture(scope="module")
def lib():
    return ensure_built()


def _records():
    return np.array(_load_table("table10_amr_cells.txt"))


def _zone_args(level, ix, iy, grid=T10_GRID):
    return grid + (level, ix, iy)


def test_table10_records_import(lib):
    rec = _records()
    level, ix, iy = sg.sg_zones_from_records(rec, *T10_GRID)
    assert level.tolist() == (rec[:, 3] - 1).astype(int).tolist()
    h = 0.25 / 2.0 ** level
    # centres within the printed two-decimal rounding
    assert np.all(np.abs(T10_GRID[2] + (ix + 0.5) * h - rec[:, 1]) < 0.006)
    assert np.all(np.abs(T10_GRID[3] + (iy + 0.5) * h - rec[:, 2]) < 0.006)
    parent, leaf, _ = sg.sg_zones_links(_zone_args(level, ix, iy))
    assert parent.tolist() == rec[:, 4].astype(int).tolist()
    assert leaf.tolist() == (rec[:, 5] == 1).tolist() and leaf.sum() == 28


def test_table10_neighbours(lib):
    """Regenerated LN, DN, RN, UN (the printed ones contradict the printed centres)."""
    rec = _records()
    level, ix, iy = sg.sg_zones_from_records(rec, *T10_GRID)
    _, _, nb = sg.sg_zones_links(_zone_args(level, ix, iy))
    # zone 1 (corner, level 1): no left/down neighbour, right 2, up 5
    assert nb[0].tolist() == [0, 0, 2, 5]
    # zone 6 is refined; its level-1 neighbours are 5, 2, 7, 10
    assert nb[5].tolist() == [5, 2, 7, 10]
    # a level-2 zone at the edge of its parent sees the coarser zone across that edge
    k = next(i for i in range(32) if level[i] == 1 and rec[i, 0] == 18)  # zone 18 at (0.31, 0.31)
    assert nb[k][0] == 5 and nb[k][1] == 2
    # same-level neighbours are mutual
    for a in range(32):
        for s, o in ((0, 2), (1, 3), (2, 0), (3, 1)):
            b = nb[a][s] - 1
            if b >= 0 and level[b] == level[a]:
                assert nb[b][o] - 1 == a


@pytest.mark.parametrize("edit, why", [
    (lambda r: r.__setitem__((3, 0), 9), "IDs out of order"),
    (lambda r: r.__setitem__((17, 4), 11), "parent does not contain the zone"),
    (lambda r: r.__setitem__((5, 5), 1), "refined zone flagged as leaf"),
    (lambda r: r.__setitem__((0, 5), 0), "leaf flagged as refined"),
    (lambda r: r.__setitem__((2, 1), 0.5), "centre between zone centres"),
    (lambda r: r.__setitem__((4, 3), 0), "level 0 in the paper's numbering"),
])
def test_records_rejected(lib, edit, why):
    rec = _records()
    edit(rec)
    with pytest.raises(sg.SgError) as e:
        sg.sg_zones_from_records(rec, *T10_GRID)
    assert e.value.status == sg.SG_EINVAL, why
    assert "record" in str(e.value)


@pytest.mark.parametrize("zones, why", [
    (([0, 0, 1], [0, 1, 0], [0, 0, 0]), "siblings missing"),
    (([0, 1, 1, 1, 1], [0, 2, 3, 2, 3], [0, 0, 0, 1, 1]), "parent missing"),
    (([0, 0], [0, 0], [0, 0]), "listed twice"),
    (([0], [5], [0]), "outside the grid"),
    (([12], [0], [0]), "level out of range"),
])
def test_zone_lists_rejected(lib, zones, why):
    """The zone rules are checked on the host before any device work."""
    args = (2, 1, 0.0, 0.0, 1.0) + zones
    with pytest.raises(sg.SgError) as e:
        sg.sg_zones_links(args)
    assert e.value.status == sg.SG_EINVAL, why
    with pytest.raises(sg.SgError) as e:
        sg.sg_plan_create_zones(args)
    assert e.value.status == sg.SG_EINVAL, why


def test_band_hierarchy_links(lib):
    """The library's leaf flags and parents agree with the generator's hierarchy."""
    for rule, disk in (("ilr", "d2"), ("vlr", "d22")):
        hier = W.band_hierarchy(64, 3, rule, disk)
        args = (64, 64, hier["x0"], hier["y0"], hier["h0"], hier["level"], hier["ix"], hier["iy"])
        parent, leaf, nb = sg.sg_zones_links(args)
        assert np.array_equal(leaf, hier["leaf"])
        lev = hier["level"]
        p = parent[lev > 0] - 1
        assert np.all(lev[p] == lev[lev > 0] - 1)
        assert np.all(hier["ix"][p] == hier["ix"][lev > 0] // 2)
        assert np.all(nb >= 0) and np.all(nb <= lev.size)


def test_masked_patch_rules(lib):
    base = (0, 8, 8, 0.0, 0.0, 0.1)
    fine = (1, 8, 8, 0.2, 0.2, 0.05)
    ring = np.ones((8, 8), np.uint8)
    ring[2:6, 2:6] = 0  # whole 2x2 blocks
    assert sg.sg_geom_validate([base, fine], masks=[None, ring]) == sg.SG_OK
    half = ring.copy()
    half[0, 0] = 0  # breaks the block (0..1, 0..1)
    assert sg.sg_geom_validate([base, fine], masks=[None, half]) == sg.SG_EINVAL
    assert "2x2" in sg.last_error()
    hole = np.ones((8, 8), np.uint8)
    hole[2, 2] = 0  # the parent of the fine block at (0..1, 0..1) of the child is coarse cell (2, 2)
    assert sg.sg_geom_validate([base, fine], masks=[hole, None]) == sg.SG_EINVAL
    assert "absent parent" in sg.last_error()
    # central slopes on a masked patch: the neighbour-leaf rule (absent cells count as outside)
    assert sg.sg_geom_validate([base], masks=[hole], slope_mode=sg.SG_SLOPES_CENTRAL) == sg.SG_OK
    assert sg.sg_geom_validate([base], masks=[hole], z=0.1) == sg.SG_OK  # off the plane: the direct path
    assert sg.sg_geom_validate([base], masks=[np.zeros((8, 8))]) == sg.SG_EINVAL  # no leaf at all
