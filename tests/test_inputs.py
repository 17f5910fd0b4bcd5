"""The seeded input generators meet the contracts the library checks (CPU only)."""
import numpy as np

import scenes


def _boxes(grids):
    lo = np.array([np.float32(g.origin) for g in grids], np.float64)
    hi = lo + np.array([g.dims for g in grids], np.float64) * np.array(
        [float(np.float32(g.cell)) for g in grids])[:, None]
    return lo, hi


def _overlaps(lo, hi):
    o = np.argsort(lo[:, 0])
    n = 0
    for a, i in enumerate(o):
        for j in o[a + 1:]:
            if lo[j, 0] >= hi[i, 0]:
                break
            n += bool(np.all(lo[i] < hi[j]) and np.all(lo[j] < hi[i]))
    return n


def test_street_trees_fill_2000_disjoint_boxes_along_2_km():
    """2000 trees in FP32-exact 5.625 m boxes, six rows along 2 km, no two
    boxes overlapping (touching is allowed)."""
    rng = np.random.default_rng(0)
    grids = scenes.urban_trees(rng, length=2000.0, n_trees=2000, n=8, cell=0.703125)
    assert len(grids) == 2000
    lo, hi = _boxes(grids)
    assert np.allclose(hi - lo, 5.625)
    assert _overlaps(lo, hi) == 0
    assert lo[:, 0].min() >= 0.0 and hi[:, 0].max() <= 2000.0
    assert len({id(g.density) for g in grids}) <= 16          # shared templates
    n_vox = sum(int(np.prod(g.dims)) for g in grids)
    assert n_vox < 2 ** 31


def test_forest_boxes_touch_along_x_and_trees_are_sparse():
    w = scenes.voxel_forest()
    grids = w.scenes[0].grids
    lo, hi = _boxes(grids)
    assert _overlaps(lo, hi) == 0
    assert np.isclose(hi[0, 0], lo[1, 0])                      # neighbours touch
    for g in grids:
        d = g.density
        assert 0.02 < (d > 0).mean() < 0.5 and d.min() >= 0.0
