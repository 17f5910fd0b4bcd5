"""Fetch counts of the roofline's algorithmic-bytes model (GPU).

helios_fetch_counts_sample counts, per pulse, the union over its subrays of
the 4-wide BVH nodes the beam cone enters, the triangles whose box it
overlaps and the voxels the subrays march through.  The checks:

* voxels and voxel visits against the FP64 oracle's own marches (each subray
  up to its stochastic event or, in expected mode, its triangle hit, as the
  oracle's scan finds them), union and sum taken here;
* triangles against a float64 restatement of the cone-box test over every
  triangle's box, bracketed by a narrower cone on the exact boxes and a wider
  one on boxes widened beyond the FP32 test's rounding;
* a cone that holds the whole scene enters every node and every triangle;
* the structural bound of a 4-wide walk: triangles <= 3 nodes + 1.
"""
import math

import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hg():
    import __graft_entry__ as g
    g.build()
    import paper_2101_09154_gb300 as m
    return m


def _np(c):
    return {k: v.cpu().numpy() for k, v in c.items()}


def _oracle_voxels(osc, sc, leg, ref, rows, seed):
    """Distinct voxels and visits per sampled pulse from the oracle's marches."""
    q = sc.beam_sample_quality
    S = oracle.subray_count(q)
    vox, visits = [], []
    for i, k in enumerate(rows):
        o, d = oracle.pulse_ray(sc, leg, int(k), seed=seed)
        ids = []
        for s in range(S):
            ds = oracle.subray_dir(sc, q, s, d)
            t_hi = ref["subray_range"][i, s] if ref["subray_hit"][i, s] >= 0 else math.inf
            v, _, _ = osc.march(o, ds, t_hi)
            ids.append(v)
        cat = np.concatenate(ids) if ids else np.zeros(0, np.int64)
        vox.append(len(np.unique(cat)))
        visits.append(len(cat))
    return np.array(vox), np.array(visits)


@pytest.mark.parametrize("kind,mode", [("canopy", 0), ("canopy", 1), ("forest", 0), ("forest", 1)])
def test_voxel_counts_match_oracle_marches(hg, kind, mode):
    if kind == "canopy":
        w = scenes.uls_voxels(seed=6, n=48, n_pulses=2001, n_bins=512, agl=12.0, speed=1.0, prf=2000.0)
    else:
        w = scenes.voxel_forest(seed=8, n_pulses=1500, n_bins=256)
    sc, leg = w.scanners[0], w.legs[0]
    gs = hg.Scene(w.scenes[0])
    rows = np.arange(0, leg.n_pulses, 7)
    got = _np(hg.fetch_counts(gs, sc, leg, mode=mode, seed=3, first=0, stride=7, count=len(rows)))
    osc = oracle.OracleScene(w.scenes[0])
    ref = oracle.scan(osc, sc, leg, rows, mode=mode, seed=3)
    vox, visits = _oracle_voxels(osc, sc, leg, ref, rows, seed=3)
    assert (got["flags"] & ~hg.FC_LIST_OVERFLOW).max() == 0
    assert vox.sum() > 20 * len(rows)                  # the sample does cross the voxels
    # a voxel boundary within rounding of a subray's end may be counted on one
    # side only: exact on nearly every pulse, within 2 elsewhere
    for a, b in ((got["voxels"], vox), (got["voxel_visits"], visits)):
        d = np.abs(a - b)
        assert (d == 0).mean() >= 0.97 and d.max() <= 2, (np.nonzero(d)[0][:10], a[d > 0][:10], b[d > 0][:10])
    assert np.all(got["voxel_visits"] >= got["voxels"])


def _cone_box_pass(o, d, ta, lo, hi):
    """float64 form of the scan's conservative cone-box test: the box grown by
    ta times the distance from the origin to its farthest corner, against the
    pulse axis o + t d, t >= 0."""
    f = np.maximum(np.abs(lo - o), np.abs(hi - o))
    R = ta * np.sqrt((f * f).sum(axis=1))
    dd = np.where(np.abs(d) < 1e-20, np.copysign(1e-20, d), d)
    inv = 1.0 / dd
    t0 = (lo - o) * inv
    t1 = (hi - o) * inv
    grow = R[:, None] * np.abs(inv)[None, :]
    tmn = np.maximum((np.minimum(t0, t1) - grow).max(axis=1), 0.0)
    tmx = (np.maximum(t0, t1) + grow).min(axis=1)
    return tmn <= tmx


def _tri_boxes(scene):
    tris = np.concatenate([m.verts[m.faces.astype(np.int64)] for m in scene.meshes], 0)
    tris = tris.astype(np.float32).astype(np.float64)
    return tris.min(axis=1), tris.max(axis=1)


def test_triangle_counts_bracketed_by_the_cone_box_test(hg):
    w = scenes.als_terrain(seed=5, size=96, n_trees=6, n_pulses=3000, n_bins=256, agl=80.0)
    sc, leg = w.scanners[0], w.legs[0]
    gs = hg.Scene(w.scenes[0])
    rows = np.arange(0, leg.n_pulses, 13)
    got = _np(hg.fetch_counts(gs, sc, leg, mode=0, seed=1, first=0, stride=13, count=len(rows)))
    lo, hi = _tri_boxes(w.scenes[0])
    span = np.maximum(np.abs(lo), np.abs(hi))
    ta = math.tan(sc.divergence_rad / 2)
    n_in, n_out = [], []
    for k in rows:
        o, d = oracle.pulse_ray(sc, leg, int(k), seed=1)
        n_in.append(_cone_box_pass(o, d, ta * 0.99, lo, hi).sum())
        n_out.append(_cone_box_pass(o, d, ta * 1.002 + 2e-6, lo - 4e-6 * np.maximum(span, 1),
                                    hi + 4e-6 * np.maximum(span, 1)).sum())
    n_in, n_out = np.array(n_in), np.array(n_out)
    t = got["triangles"]
    assert np.all(n_in <= t) and np.all(t <= n_out), (np.nonzero((t < n_in) | (t > n_out))[0][:10])
    assert t.mean() >= 1.0
    assert np.all(got["triangles"] <= 3 * got["nodes"] + 1)
    assert np.all(got["nodes"] <= gs.info()["n_bvh4_nodes"])
    assert np.all(got["voxels"] == 0) and got["flags"].max() == 0


def test_a_cone_around_the_whole_scene_enters_every_node(hg):
    """A wide beam (0.49 rad) from 200 m above a 16 m terrain tile at nadir:
    every node and every triangle lies inside the cone."""
    w = scenes.als_terrain(seed=2, size=16, n_trees=2, n_pulses=64, n_bins=64, agl=200.0)
    w = scenes.with_scanner(w, divergence_rad=0.49, beam_sample_quality=0, scan_angle_max_rad=0.0)
    sc, leg = w.scanners[0], w.legs[0]
    gs = hg.Scene(w.scenes[0])
    info = gs.info()
    got = _np(hg.fetch_counts(gs, sc, leg, first=0, stride=1, count=leg.n_pulses))
    assert np.all(got["nodes"] == info["n_bvh4_nodes"])
    assert np.all(got["triangles"] == info["n_triangles"])


def test_sample_bounds_and_empty_sample(hg):
    w = scenes.tls_tiny(n_az=4, n_el=4)
    gs = hg.Scene(w.scenes[0])
    sc, leg = w.scanners[0], w.legs[0]
    got = hg.fetch_counts(gs, sc, leg, first=3, stride=5, count=0)
    assert got["nodes"].numel() == 0
    last = hg.fetch_counts(gs, sc, leg, first=leg.n_pulses - 1, stride=1, count=1)
    assert int(last["triangles"][0]) >= 0
    with pytest.raises(hg.HeliosError):
        hg.fetch_counts(gs, sc, leg, first=leg.n_pulses, stride=1, count=1)
