"""The allocation-free persistent scan against the allocating one (GPU).

Some callers cannot allocate device memory during a scan: processes whose
device memory belongs to another allocator (a framework's caching allocator
holding the budget), code capturing a CUDA graph into a memory pool it does
not control, and real-time loops that cannot let an allocation fail or stall.
For them helios_scan_legs_static keeps the only scratch of the persistent
scan, its work-queue counters, in a static device array instead of a
cudaMallocAsync allocation.  The array keeps the previous call's contents, so
the checks below run the entry point twice in a row and compare both results
with helios_scan_legs, within the tolerances of the other GPU tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
import scenes
from parity import compare, leg_view

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

INT_KEYS = ("window_bin", "echo_count", "echo_bin", "echo_object", "subray_hit", "pulse_flags")


@pytest.fixture(scope="module")
def hg():
    import __graft_entry__ as g
    g.build()
    import paper_2101_09154_gb300 as m
    return m


def _close(a, b, nb=None):
    a = a.detach().double().cpu().numpy()
    b = b.detach().double().cpu().numpy()
    if nb is None:                              # ranges: 1e-4 m
        return np.all(np.abs(a - b) <= 1e-4)
    W, R = a.reshape(-1, nb), b.reshape(-1, nb)  # waveform: 1e-4 |W| + 1e-7 max per pulse
    peak = np.abs(R).max(axis=1, keepdims=True)
    return np.all(np.abs(W - R) <= 1e-4 * np.abs(R) + 1e-7 * peak)


def test_static_scan_matches_allocating_scan_on_two_calls(hg):
    w = scenes.batched_legs(seed=12, n_legs=5, tile=64, block=24, n_terrain=2, n_voxel=2,
                            min_pulses=500, max_pulses=3000, n_bins=256)
    gsc = [hg.Scene(s) for s in w.scenes]
    ref, _ = hg.scan(gsc, w.scanners, w.legs, seed=9, persistent=True)
    torch.cuda.synchronize()
    for _call in range(2):
        got, _ = hg.scan_static(gsc, w.scanners, w.legs, seed=9)
        torch.cuda.synchronize()
        for k in INT_KEYS:
            assert torch.equal(got[k], ref[k]), k
        assert _close(got["waveform"], ref["waveform"], nb=256)
        for k in ("echo_range", "subray_range"):
            assert _close(got[k], ref[k]), k


def test_static_scan_rejects_too_many_legs(hg):
    w = scenes.tls_tiny(n_az=4, n_el=4)
    gsc = [hg.Scene(w.scenes[0])]
    legs = [scenes.Leg(n_pulses=16 if i == 0 else 0, leg_id=i) for i in range(2049)]
    with pytest.raises(hg.HeliosError) as e:
        hg.scan_static(gsc, w.scanners, legs)
    assert e.value.code == -1 and "2048" in str(e.value)


def test_static_scan_with_several_grids(hg):
    """A scene with nine voxel trees (one grid each): the static entry reads
    the scene's own grid descriptors, without occupancy masks."""
    w = scenes.voxel_forest(seed=8, n_pulses=1500, n_bins=256)
    gsc = [hg.Scene(s) for s in w.scenes]
    ref, _ = hg.scan(gsc, w.scanners, w.legs, seed=4, persistent=True)
    torch.cuda.synchronize()
    got, _ = hg.scan_static(gsc, w.scanners, w.legs, seed=4)
    torch.cuda.synchronize()
    for k in INT_KEYS:
        assert torch.equal(got[k], ref[k]), k
    assert _close(got["waveform"], ref["waveform"], nb=256)
    assert (ref["subray_hit"] >= gsc[0].n_triangles).float().mean() > 0.05


def _expected_pair(hg, w, seed):
    gsc = [hg.Scene(s) for s in w.scenes]
    ref, lay = hg.scan(gsc, w.scanners, w.legs, mode=hg.MODE_EXPECTED, seed=seed, persistent=True)
    torch.cuda.synchronize()
    return gsc, ref, lay


@pytest.mark.parametrize("kind", ["voxels", "mesh"])
def test_static_expected_mode_matches_allocating_scan_and_oracle(hg, kind):
    """Expected mode with a Gaussian pulse and echo objects: the static entry
    sums each waveform directly and picks echo objects from its own return
    list, the allocating one uses moment bins and a second march.  Both are
    checked against the oracle (integers exact away from flagged near-ties)
    and against each other within the waveform and range tolerances, on two
    calls in a row."""
    if kind == "voxels":
        w = scenes.uls_voxels(seed=6, n=48, n_pulses=2001, n_bins=512, agl=12.0, speed=1.0,
                              prf=2000.0)
    else:
        w = scenes.als_terrain(seed=5, size=96, n_trees=6, n_pulses=3000, n_bins=256, agl=80.0)
    sc, leg = w.scanners[0], w.legs[0]
    nb = sc.n_bins
    gsc, ref, lay = _expected_pair(hg, w, seed=2)
    S = hg.subray_count(sc.beam_sample_quality)
    rows = np.arange(leg.n_pulses)
    oref = oracle.scan(oracle.OracleScene(w.scenes[0]), sc, leg, rows, mode=1, seed=2)
    compare(leg_view(ref, lay, 0, sc, S, rows), oref, expected_mode=True)
    ok = (oref["flags"] & (oracle.F_DECISION | oracle.F_OVERFLOW)) == 0
    for _call in range(2):
        got, _ = hg.scan_static(gsc, w.scanners, w.legs, mode=hg.MODE_EXPECTED, seed=2)
        torch.cuda.synchronize()
        compare(leg_view(got, lay, 0, sc, S, rows), oref, expected_mode=True)
        assert _close(got["waveform"], ref["waveform"], nb=nb)
        assert torch.equal(got["window_bin"], ref["window_bin"])
        assert torch.equal(got["subray_hit"], ref["subray_hit"])
        assert _close(got["subray_range"], ref["subray_range"])
        K = sc.max_echoes
        for k in ("echo_count",):
            a, b = got[k].cpu().numpy(), ref[k].cpu().numpy()
            assert np.array_equal(a[ok], b[ok]), k
        for k in ("echo_bin", "echo_object"):
            a = got[k].cpu().numpy().reshape(-1, K)
            b = ref[k].cpu().numpy().reshape(-1, K)
            assert np.array_equal(a[ok], b[ok]), k


def test_static_scan_echo_widths_match_allocating_scan(hg):
    """The optional echo-width fit requested from the static entry (with the
    echo bins it reads back) gives the allocating scan's widths, twice."""
    w = scenes.als_terrain(seed=5, size=96, n_trees=6, n_pulses=3000, n_bins=256, agl=80.0)
    gsc = [hg.Scene(s) for s in w.scenes]
    ref, _ = hg.scan(gsc, w.scanners, w.legs, seed=5, persistent=True, echo_width=True)
    torch.cuda.synchronize()
    for _call in range(2):
        got, _ = hg.scan_static(gsc, w.scanners, w.legs, seed=5, echo_width=True)
        torch.cuda.synchronize()
        assert torch.equal(got["echo_bin"], ref["echo_bin"])
        a = got["echo_width"].double().cpu().numpy()
        b = ref["echo_width"].double().cpu().numpy()
        assert np.all(np.abs(a - b) <= 1e-3 * np.abs(b) + 1e-6)
        assert (b > 0).sum() > 1000
