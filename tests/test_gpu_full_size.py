"""Full-size workloads in the benchmark's launch configurations, checked on
sampled pulses against the FP64 oracle (which computes them one by one):

* the voxel canopy (256^3 voxels at 0.1 m, 1 M pulses, 19 subrays, 1024 bins),
  stochastic and expected forward, and the expected-mode adjoint;
* 128 scan legs of 10 k - 2 M pulses and 1/7/19/37 subrays over terrain tiles
  and voxel blocks, in one persistent launch with the tuned block shape;
* the urban street (20.7 M triangles, 2000 voxel trees of 128^3, 20 M pulses,
  37 subrays) in both modes.

Tolerances are those of ``tests/parity.py`` (gradients: 1e-3 relative with a
floor of 1e-6 of the largest entry).
"""
import numpy as np
import pytest

import oracle
import scenes
from parity import compare, leg_view, to_np

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def hg():
    import __graft_entry__ as g
    g.build()
    import paper_2101_09154_gb300 as m
    return m


@pytest.fixture(scope="module")
def uls():
    return scenes.uls_voxels()


@pytest.mark.parametrize("mode", [0, 1])
def test_uls_full_size_sampled(hg, uls, mode):
    """1 M pulses through the 256^3 canopy in one launch; every 997th pulse."""
    w = uls
    sc, leg = w.scanners[0], w.legs[0]
    gs = hg.Scene(w.scenes[0])
    out, lay = hg.scan([gs], [sc], [leg], mode=mode, seed=0)
    torch.cuda.synchronize()
    rows = np.arange(0, leg.n_pulses, 997)
    S = hg.subray_count(sc.beam_sample_quality)
    g = leg_view(out, lay, 0, sc, S, rows)
    del out
    torch.cuda.empty_cache()
    ref = oracle.scan(oracle.OracleScene(w.scenes[0]), sc, leg, rows, mode=mode, seed=0)
    st = compare(g, ref, expected_mode=(mode == 1))
    print(f"uls mode {mode}: {st}")
    assert st["pulses"] == len(rows) and st["echoes"] > 1500, st


def test_adjoint_full_size_sampled(hg, uls):
    """The adjoint over the whole 1 M-pulse leg with dL/dW = 2 (W - W_ref) on the
    sampled pulses (zero elsewhere, so the GPU's gradient is theirs alone),
    against the oracle's analytic gradient on the same pulses and windows."""
    w = uls
    sc, leg = w.scanners[0], w.legs[0]
    nb = sc.n_bins
    gs = hg.Scene(w.scenes[0])
    out, lay = hg.scan([gs], [sc], [leg], mode=1)
    ref_scene = scenes.Scene(meshes=w.scenes[0].meshes,
                             grids=[scenes.VoxelGrid(**{**w.scenes[0].grids[0].__dict__,
                                                       "density": scenes.perturbed_density(
                                                           w.scenes[0].grids[0].density, seed=1)})])
    out_ref, _ = hg.scan([hg.Scene(ref_scene)], [sc], [leg], mode=1, subrays=False)
    rows = np.arange(0, leg.n_pulses, 997)
    idx = torch.as_tensor(rows, device=out["waveform"].device)
    gW = torch.zeros_like(out["waveform"])
    Wv, Rv = out["waveform"].view(-1, nb), out_ref["waveform"].view(-1, nb)
    gW.view(-1, nb)[idx] = 2.0 * (Wv[idx] - Rv[idx])
    del out_ref
    grads = hg.scan_adjoint([gs], [sc], [leg], gW, out["window_bin"], out["subray_hit"])
    torch.cuda.synchronize()
    g_np = to_np(gW.view(-1, nb)[idx]).astype(np.float64)
    win = to_np(out["window_bin"])[rows]
    osc = oracle.OracleScene(w.scenes[0])
    d_refl, d_dens = oracle.adjoint(osc, sc, leg, rows, g_np, win)
    gd = to_np(grads[0]["density"][0]).ravel()
    gr = to_np(grads[0]["reflectance"][0])
    scale = np.abs(d_dens).max()
    assert scale > 0 and np.count_nonzero(d_dens) > 10000
    err = np.abs(gd - d_dens) - (1e-3 * np.abs(d_dens) + 1e-6 * scale)
    assert (err <= 0).all(), (f"density gradient: {int((err > 0).sum())} of "
                              f"{np.count_nonzero(d_dens)} entries outside tolerance")
    assert np.allclose(gr, d_refl, rtol=1e-3, atol=1e-6 * np.abs(d_refl).max())


def test_batched_legs_full_size_sampled(hg):
    """All 128 legs (42.9 M pulses) in one persistent launch with the block shape
    the autotuner picks on a GB300 (256 threads, 1536 rays per block); about 40
    evenly spaced pulses of every leg against the oracle."""
    w = scenes.batched_legs()
    gsc = [hg.Scene(s) for s in w.scenes]
    out, lay = hg.scan(gsc, w.scanners, w.legs, seed=3, persistent=True, block_threads=256,
                       rays_per_block=1536)
    torch.cuda.synchronize()
    osc = {}
    total = flagged = subrays = reruns = 0
    for l, leg in enumerate(w.legs):
        sc = w.scanners[leg.scanner_index]
        q = leg.beam_sample_quality if leg.beam_sample_quality >= 0 else sc.beam_sample_quality
        S = hg.subray_count(q)
        rows = np.unique(np.linspace(0, leg.n_pulses - 1, 40).astype(np.int64))
        g = leg_view(out, lay, l, sc, S, rows)
        if leg.scene_index not in osc:
            osc[leg.scene_index] = oracle.OracleScene(w.scenes[leg.scene_index])
        ref = oracle.scan(osc[leg.scene_index], sc, leg, rows, seed=3)
        st = compare(g, ref)
        total += st["pulses"]
        flagged += st["flagged_subrays"] * st["pulses"] * S
        subrays += st["pulses"] * S
        reruns += st["rerun_pulses"]
    print(f"batched: {total} pulses, flagged subrays {flagged / subrays:.5f}, re-run pulses {reruns}")
    assert total >= 128 * 39


@pytest.fixture(scope="module")
def urban():
    w = scenes.urban_mls()
    return w, oracle.OracleScene(w.scenes[0])


@pytest.mark.parametrize("mode", [0, 1])
def test_urban_mls_full_size_sampled(hg, urban, mode):
    """The whole urban leg (2 km street, 20.7 M triangles, 2000 voxel trees of
    128^3, 20 M pulses x 37 subrays, 512 bins) in one launch; every 4001st
    pulse against the oracle."""
    w, osc = urban
    sc, leg = w.scanners[0], w.legs[0]
    gs = hg.Scene(w.scenes[0])
    out, lay = hg.scan([gs], [sc], [leg], mode=mode, seed=6)
    torch.cuda.synchronize()
    rows = np.arange(0, leg.n_pulses, 4001)
    S = hg.subray_count(sc.beam_sample_quality)
    g = leg_view(out, lay, 0, sc, S, rows)
    del out
    torch.cuda.empty_cache()
    ref = oracle.scan(osc, sc, leg, rows, mode=mode, seed=6)
    st = compare(g, ref, expected_mode=(mode == 1))
    print(f"urban mode {mode}: {st}")
    assert st["pulses"] == len(rows) and st["echoes"] > 3000, st
