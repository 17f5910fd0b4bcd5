"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Every test here needs a GB300; all inputs are seeded synthetic workloads from
``scenes``.  Tolerances are documented in ``tests/parity.py``.
"""
import math

import numpy as np
import pytest

import oracle
import scenes
from oracle import lad
from parity import compare, leg_view, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hg():
    import __graft_entry__ as g
    g.build()
    import paper_2101_09154_gb300 as m
    return m


def run_both(hg, w, mode=0, seed=0, rows=None, persistent=False, threads=0, **kw):
    gsc = [hg.Scene(s) for s in w.scenes]
    out, lay = hg.scan(gsc, w.scanners, w.legs, mode=mode, seed=seed, persistent=persistent, **kw)
    torch.cuda.synchronize()
    res = []
    for l, leg in enumerate(w.legs):
        sc = w.scanners[leg.scanner_index]
        q = leg.beam_sample_quality if leg.beam_sample_quality >= 0 else sc.beam_sample_quality
        S = hg.subray_count(q)
        r = np.arange(leg.n_pulses) if rows is None else rows
        osc = oracle.OracleScene(w.scenes[leg.scene_index])
        ref = oracle.scan(osc, sc, leg, r, mode=mode, seed=seed, threads=threads)
        res.append((leg_view(out, lay, l, sc, S, r), ref))
    return out, lay, res


def test_tls_tiny_full_scan(hg):
    """98-triangle TLS scene, all 10^4 pulses, 19 subrays, stochastic mode."""
    w = scenes.tls_tiny()
    _, _, res = run_both(hg, w, seed=0)
    stats = compare(*res[0])
    assert stats["echoes"] > 3000


def test_als_terrain_small_ragged(hg):
    """Terrain + trees; 6001 pulses (not a multiple of the work item) at 512 bins."""
    w = scenes.als_terrain(seed=5, size=128, n_trees=12, n_pulses=6001, n_bins=512, agl=120.0,
                           speed=30.0, prf=50_000.0)
    _, _, res = run_both(hg, w, seed=3)
    stats = compare(*res[0])
    assert stats["echoes"] > 3000


@pytest.mark.parametrize("mode", [0, 1])
def test_uls_voxels_small(hg, mode):
    """Transmissive voxels over a ground plane, stochastic and expected modes."""
    w = scenes.uls_voxels(seed=6, n=48, n_pulses=3001, n_bins=512, agl=12.0, speed=1.0,
                          prf=2000.0)
    _, _, res = run_both(hg, w, mode=mode, seed=11)
    stats = compare(*res[0], expected_mode=(mode == 1))
    assert stats["echoes"] > 1000


def test_expected_mode_gaussian_and_carlsson_legs_in_one_launch(hg):
    """Expected mode: a Gaussian leg (Hermite-moment waveform) and an Eq. beam_time
    leg (direct sums) share one persistent launch and its shared-memory layout."""
    import dataclasses
    w = scenes.uls_voxels(seed=6, n=48, n_pulses=1500, n_bins=512, agl=12.0, speed=1.0,
                          prf=2000.0)
    sc2 = dataclasses.replace(w.scanners[0], pulse_shape=scenes.PULSE_CARLSSON, pulse_length_ns=3.5)
    leg2 = dataclasses.replace(w.legs[0], scanner_index=1, leg_id=7, n_pulses=1200)
    w = scenes.Workload("mixed", w.scenes, [w.scanners[0], sc2], [w.legs[0], leg2])
    _, _, res = run_both(hg, w, mode=1, seed=11, persistent=True)
    for g, ref in res:
        stats = compare(g, ref, expected_mode=True)
        assert stats["echoes"] > 500


def test_expected_mode_long_voxel_column(hg):
    """Expected mode down a 400-voxel column of non-zero density: each subray has
    more returns than a lane's return list holds, so the echo objects come from
    the second march."""
    dens = np.full((400, 8, 8), 0.05, np.float32)
    grid = scenes.VoxelGrid(origin=(-0.2, -0.2, 0.0), cell=0.05, dims=(8, 8, 400), density=dens,
                            G=0.5, leaf_reflectance=0.5)
    ground = scenes.Mesh(np.array([[-5, -5, -0.5], [5, -5, -0.5], [0, 6, -0.5]], np.float32),
                         np.array([[0, 1, 2]], np.int32), np.array([0.4], np.float32))
    scene = scenes.Scene(meshes=[ground], grids=[grid])
    sc = scenes.Scanner(deflector=scenes.DEFL_TLS_GRID, grid_n_az=8, grid_n_el=8,
                        el_min_rad=-1.5707, el_max_rad=-1.5697, n_bins=1024, max_echoes=8)
    leg = scenes.Leg(scene_index=0, n_pulses=64, leg_id=4, start=(0.01, 0.02, 25.0))
    w = scenes.Workload("column", [scene], [sc], [leg])
    _, _, res = run_both(hg, w, mode=1, seed=3)
    g, ref = res[0]
    compare(g, ref, expected_mode=True)
    assert (ref["echo_count"] > 0).all()


def test_urban_mls_rotating_head_37_subrays(hg):
    """Street + extruded buildings scanned by a rotating profile head (pitched
    attitude) on a moving vehicle, 37 subrays; every 7th pulse of 300 000."""
    w = scenes.urban_mls(length=30.0, facade_cell=0.5)
    rows = np.arange(0, w.legs[0].n_pulses, 7)
    _, _, res = run_both(hg, w, seed=6, rows=rows)
    stats = compare(*res[0])
    assert stats["echoes"] > 30000


@pytest.mark.parametrize("q", [0, 1, 3])
def test_subray_qualities_and_carlsson_pulse(hg, q):
    """S = 1, 7, 37 (more subrays than warp lanes) with the Eq. beam_time pulse."""
    w = scenes.tls_tiny(n_az=40, n_el=30)
    w = scenes.with_scanner(w, beam_sample_quality=q, pulse_shape=scenes.PULSE_CARLSSON,
                            pulse_length_ns=3.5, n_bins=160)
    _, _, res = run_both(hg, w, seed=2)
    compare(*res[0])


def test_multi_leg_offsets_and_persistent_bitwise(hg):
    """Legs of uneven length and quality: per-leg parity, and the persistent
    work-queue launch reproduces the per-leg launches bit for bit."""
    w = scenes.batched_legs(seed=8, n_legs=6, tile=64, block=24, n_terrain=2, n_voxel=2,
                            min_pulses=500, max_pulses=4000, n_bins=256)
    # shrink the voxel legs' altitude so the small blocks are inside the swath
    out_a, lay, res = run_both(hg, w, seed=4)
    for g, ref in res:
        compare(g, ref)
    gsc = [hg.Scene(s) for s in w.scenes]
    out_b, _ = hg.scan(gsc, w.scanners, w.legs, seed=4, persistent=True)
    torch.cuda.synchronize()
    for k in ("waveform", "window_bin", "echo_count", "echo_range", "echo_bin", "echo_object",
              "subray_hit", "subray_range"):
        assert torch.equal(out_a[k], out_b[k]), k


def test_deterministic_repeat(hg):
    w = scenes.als_terrain(seed=5, size=96, n_trees=6, n_pulses=3000, n_bins=256, agl=80.0)
    gsc = [hg.Scene(s) for s in w.scenes]
    a, _ = hg.scan(gsc, w.scanners, w.legs, seed=1)
    b, _ = hg.scan(gsc, w.scanners, w.legs, seed=1)
    torch.cuda.synchronize()
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_edge_cases_empty_leg_sky_one_triangle_grid_only(hg):
    sc = scenes.Scanner(deflector=scenes.DEFL_TLS_GRID, grid_n_az=16, grid_n_el=9,
                        el_min_rad=-1.2, el_max_rad=1.2, n_bins=128)
    one = scenes.Scene(meshes=[scenes.Mesh(np.array([[-5, -5, -2], [5, -5, -2], [0, 6, -2]], np.float32),
                                           np.array([[0, 1, 2]], np.int32), np.array([0.4], np.float32))])
    dens = np.zeros((6, 6, 6), np.float32)
    dens[2:4, 2:4, :] = 1.5
    gridonly = scenes.Scene(grids=[scenes.VoxelGrid(origin=(-3.0, -3.0, -4.0), cell=1.0, dims=(6, 6, 6),
                                                    density=dens)])
    legs = [scenes.Leg(scene_index=0, n_pulses=0, leg_id=1),
            scenes.Leg(scene_index=0, n_pulses=144, leg_id=2),
            scenes.Leg(scene_index=1, n_pulses=144, leg_id=3, start=(0.2, 0.1, 0.0))]
    w = scenes.Workload("edge", [one, gridonly], [sc], legs)
    out, lay, res = run_both(hg, w, seed=5)
    for g, ref in res[1:]:
        compare(g, ref, max_flag_frac=0.3)
    # upward pulses return nothing
    g, ref = res[1]
    nohit = (ref["flags"] & oracle.F_NOHIT) != 0
    assert nohit.any() and (g["window_bin"][nohit] == hg.NO_WINDOW).all()
    assert (g["pulse_flags"][nohit] & hg.PF_NO_RETURN).all()


def test_bad_face_index_is_rejected(hg):
    bad = scenes.Scene(meshes=[scenes.Mesh(np.zeros((3, 3), np.float32), np.array([[0, 1, 7]], np.int32),
                                           np.array([0.5], np.float32))])
    with pytest.raises(hg.HeliosError) as e:
        hg.Scene(bad)
    assert e.value.code == -1


@pytest.mark.parametrize("lad_kind", [None, "erectophile"])
def test_adjoint_matches_oracle(hg, lad_kind):
    """Expected-mode adjoint: GPU gradients vs the oracle's analytic gradients
    (the latter pinned to FP64 central differences on the CPU), with the
    constant G and with a leaf-angle table."""
    w = scenes.uls_voxels(seed=4, n=32, n_pulses=1200, n_bins=384, agl=10.0, speed=1.0, prf=1000.0)
    if lad_kind:
        w.scenes[0].grids[0].lad = lad.table(lad_kind, 23).astype(np.float32)
    sc, leg = w.scanners[0], w.legs[0]
    gs = hg.Scene(w.scenes[0])
    out, lay = hg.scan([gs], [sc], [leg], mode=1)
    ref_d = scenes.perturbed_density(w.scenes[0].grids[0].density, seed=1)
    gref = hg.Scene(scenes.Scene(meshes=w.scenes[0].meshes,
                                 grids=[scenes.VoxelGrid(**{**w.scenes[0].grids[0].__dict__,
                                                           "density": ref_d})]))
    out_ref, _ = hg.scan([gref], [sc], [leg], mode=1)
    gW = 2.0 * (out["waveform"] - out_ref["waveform"])
    grads = hg.scan_adjoint([gs], [sc], [leg], gW, out["window_bin"], out["subray_hit"])
    torch.cuda.synchronize()
    osc = oracle.OracleScene(w.scenes[0])
    rows = np.arange(leg.n_pulses)
    win = to_np(out["window_bin"])
    d_refl, d_dens = oracle.adjoint(osc, sc, leg, rows, to_np(gW).reshape(-1, sc.n_bins).astype(np.float64),
                                    win)
    gd = to_np(grads[0]["density"][0]).ravel()
    gr = to_np(grads[0]["reflectance"][0])
    scale = np.abs(d_dens).max()
    assert scale > 0
    err = np.abs(gd - d_dens) - (1e-3 * np.abs(d_dens) + 1e-6 * scale)
    assert (err <= 0).all(), f"density gradient: {int((err > 0).sum())} entries outside tolerance"
    assert np.allclose(gr, d_refl, rtol=1e-3, atol=1e-6 * np.abs(d_refl).max())
    # without the checkpoint the adjoint re-traverses and must agree
    grads2 = hg.scan_adjoint([gs], [sc], [leg], gW, out["window_bin"], None)
    torch.cuda.synchronize()
    gd2 = to_np(grads2[0]["density"][0]).ravel()
    assert np.allclose(gd2, gd, rtol=1e-4, atol=1e-7 * scale)


def test_adjoint_central_differences(hg):
    """The GPU adjoint against central differences of the GPU forward: L2 loss
    of the expected-mode waveform against a scan of perturbed densities, on 64
    random traversed voxels (seed 2) and on each ground triangle's
    reflectance.  The loss is summed in FP64; the tolerance covers the O(h^2)
    difference error and the forward's and adjoint's Hermite truncations."""
    w = scenes.uls_voxels(seed=4, n=32, n_pulses=1200, n_bins=384, agl=10.0, speed=1.0, prf=1000.0)
    sc, leg = w.scanners[0], w.legs[0]
    gs = hg.Scene(w.scenes[0])
    ref_d = scenes.perturbed_density(w.scenes[0].grids[0].density, seed=1)
    gref = hg.Scene(scenes.Scene(meshes=w.scenes[0].meshes,
                                 grids=[scenes.VoxelGrid(**{**w.scenes[0].grids[0].__dict__,
                                                           "density": ref_d})]))
    Wref = hg.scan([gref], [sc], [leg], mode=1)[0]["waveform"].double()

    def loss():
        out, _ = hg.scan([gs], [sc], [leg], mode=1)
        return float(((out["waveform"].double() - Wref) ** 2).sum())

    out, _ = hg.scan([gs], [sc], [leg], mode=1)
    gW = 2.0 * (out["waveform"] - Wref.float())
    grads = hg.scan_adjoint([gs], [sc], [leg], gW, out["window_bin"], out["subray_hit"])
    torch.cuda.synchronize()
    gd = to_np(grads[0]["density"][0]).ravel().astype(np.float64)
    gr = to_np(grads[0]["reflectance"][0]).astype(np.float64)
    dens = gs.density[0].view(-1)
    d0 = to_np(dens).astype(np.float64)
    traversed = np.nonzero((gd != 0.0) & (d0 > 0.0))[0]
    assert traversed.size >= 64
    pick = np.random.default_rng(2).choice(traversed, 64, replace=False)
    scale = np.abs(gd).max()
    for v in pick:
        h = 0.05 * d0[v]
        dens[v] = float(d0[v] + h)
        lp = loss()
        dens[v] = float(d0[v] - h)
        lm = loss()
        dens[v] = float(d0[v])
        fd = (lp - lm) / (2.0 * h)
        assert abs(fd - gd[v]) <= 3e-2 * abs(gd[v]) + 2e-3 * scale, (int(v), fd, gd[v])
    refl = gs.reflectance[0]
    r0 = to_np(refl).astype(np.float64)
    for t in range(r0.size):
        h = 0.05 * r0[t]
        refl[t] = float(r0[t] + h)
        lp = loss()
        refl[t] = float(r0[t] - h)
        lm = loss()
        refl[t] = float(r0[t])
        fd = (lp - lm) / (2.0 * h)
        assert abs(fd - gr[t]) <= 1e-2 * abs(gr[t]) + 1e-6 * np.abs(gr).max(), (t, fd, gr[t])


def test_autograd_function(hg):
    w = scenes.uls_voxels(seed=9, n=24, n_pulses=400, n_bins=256, agl=8.0, speed=1.0, prf=800.0)
    sc, leg = w.scanners[0], w.legs[0]
    gs = hg.Scene(w.scenes[0])
    refl = gs.reflectance[0].requires_grad_(True)
    dens = gs.density[0].requires_grad_(True)
    W = hg.WaveformFunction.apply(gs, sc, leg, refl, dens)
    loss = (W ** 2).sum()
    loss.backward()
    assert dens.grad is not None and torch.isfinite(dens.grad).all()
    assert refl.grad is not None and (refl.grad != 0).any()


def test_autograd_function_every_mesh_and_grid(hg):
    """WaveformFunction on a scene of two meshes and nine voxel grids, three of
    which are made to share one density array: autograd returns every mesh's reflectance
    gradient and every distinct density tensor's gradient (the shared one the
    sum over its grids), equal to the adjoint called directly."""
    w = scenes.voxel_forest(seed=9, n_pulses=800, n_bins=256)
    sc, leg = w.scanners[0], w.legs[0]
    s0 = w.scenes[0]
    # the leg flies over the middle column of trees (grids 1, 4, 7)
    s0.grids[4].density = s0.grids[1].density
    s0.grids[7].density = s0.grids[1].density
    pv = np.array([[2, 2, 0.1], [16, 2, 0.1], [16, 20, 0.1], [2, 20, 0.1]], np.float32)
    s0.meshes.append(scenes.Mesh(pv, np.array([[0, 1, 2], [0, 2, 3]], np.int32),
                                 np.array([0.6, 0.4], np.float32), object_id=2))
    gs = hg.Scene(s0)
    params = gs.parameters()
    assert len(params) == 2 + len({id(g.density) for g in s0.grids})
    for t in params:
        t.requires_grad_(True)
    W = hg.WaveformFunction.apply(gs, sc, leg, *params)
    gen = torch.Generator(device=W.device).manual_seed(5)
    gW = torch.randn(W.shape, generator=gen, device=W.device)
    (W * gW).sum().backward()
    out, _ = hg.scan([gs], [sc], [leg], mode=1)
    ref = hg.scan_adjoint([gs], [sc], [leg], gW, out["window_bin"], out["subray_hit"])[0]
    torch.cuda.synchronize()
    for i in range(2):
        assert (ref["reflectance"][i] != 0).any()
        assert torch.allclose(params[i].grad, ref["reflectance"][i], rtol=1e-5,
                              atol=1e-7 * float(ref["reflectance"][i].abs().max()))
    for t in params[2:]:
        want = sum(ref["density"][j] for j, d in enumerate(gs.density) if d is t)
        assert torch.allclose(t.grad, want, rtol=1e-5, atol=1e-7 * float(want.abs().max()) + 1e-30)
    shared = gs.density[1]
    assert gs.density[4] is shared and gs.density[7] is shared
    parts = [ref["density"][j] for j in (1, 4, 7)]
    assert sum(int((p != 0).sum()) > 0 for p in parts) >= 2
    for t in params:
        t.requires_grad_(False)


@pytest.mark.parametrize("mode", [0, 1])
def test_voxel_ids_beyond_32_bits(hg, mode):
    """1030 voxel trees of 128^3 in a row (one shared density template), so
    the last trees' voxel ids exceed 2^31: a TLS scan of the last three trees
    against the oracle, ids compared as 64-bit integers."""
    rng = np.random.default_rng(11)
    n, cell, n_trees = 128, 45.0 / 1024.0, 1030
    L = n * cell
    dens = scenes.tree_density(rng, n)
    grids = [scenes.VoxelGrid(origin=(i * L, 0.0, 0.0), cell=cell, dims=(n, n, n), density=dens)
             for i in range(n_trees)]
    x_end = n_trees * L
    pv = np.array([[x_end - 40, -20, 0], [x_end + 20, -20, 0], [x_end + 20, 26, 0], [x_end - 40, 26, 0]],
                  np.float32)
    ground = scenes.Mesh(pv, np.array([[0, 1, 2], [0, 2, 3]], np.int32), np.array([0.3, 0.35], np.float32))
    scene = scenes.Scene(meshes=[ground], grids=grids)
    sc = scenes.Scanner(deflector=scenes.DEFL_TLS_GRID, grid_n_az=40, grid_n_el=30,
                        el_min_rad=-1.45, el_max_rad=-0.5, n_bins=512, beam_sample_quality=1)
    leg = scenes.Leg(n_pulses=1200, leg_id=9, start=(x_end - 1.5 * L, L / 2, 9.0))
    w = scenes.Workload("ids64", [scene], [sc], [leg])
    _, _, res = run_both(hg, w, mode=mode, seed=5)
    g, ref = res[0]
    stats = compare(g, ref, expected_mode=(mode == 1))
    first_last = 1 + (n_trees - 3) * n ** 3       # n_tri + voxels before the third-last tree
    hit = ref["subray_hit"] if mode == 0 else ref["echo_object"]
    assert (hit >= first_last).sum() > 100 and hit.max() > 2 ** 31
    assert stats["echoes"] > 500


@pytest.mark.slow
def test_als_full_size_sampled(hg):
    """The 3M-triangle ALS workload with 4M pulses in the benchmark's launch
    configuration; every 997th pulse is checked against the oracle."""
    w = scenes.als_terrain()
    rows = np.arange(0, w.legs[0].n_pulses, 997)
    out, lay, res = run_both(hg, w, seed=0, rows=rows, subrays=True)
    stats = compare(*res[0])
    print(f"als full size: {stats}")
    assert stats["pulses"] == len(rows)


def test_graph_replay_and_autotune_match_direct_call(hg):
    """The persistent launch captured in a CUDA graph and replayed, and every
    autotuner candidate, reproduce the direct call bit for bit."""
    from paper_2101_09154_gb300.autotune import autotune
    w = scenes.batched_legs(seed=10, n_legs=7, tile=64, block=24, n_terrain=2, n_voxel=2,
                            min_pulses=300, max_pulses=3000, n_bins=256)
    gsc = [hg.Scene(s) for s in w.scenes]
    ref, lay = hg.scan(gsc, w.scanners, w.legs, seed=2, persistent=True)
    torch.cuda.synchronize()
    out = hg.alloc_outputs(lay, gsc[0].device, subrays=True)
    tune = autotune(gsc, w.scanners, w.legs, out, persistent=True, reps=1)
    assert {"block_threads", "rays_per_block", "ms"} <= set(tune)
    for t in tune["trials"]:
        o, _ = hg.scan(gsc, w.scanners, w.legs, seed=2, persistent=True,
                       block_threads=t["block_threads"], rays_per_block=t["rays_per_block"])
        torch.cuda.synchronize()
        assert torch.equal(o["waveform"], ref["waveform"]) and torch.equal(o["echo_range"], ref["echo_range"])
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        hg.scan(gsc, w.scanners, w.legs, seed=2, persistent=True, out=out)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    for v in out.values():
        v.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        hg.scan(gsc, w.scanners, w.legs, seed=2, persistent=True, out=out)
    for v in out.values():
        v.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for k in ("waveform", "window_bin", "echo_count", "echo_range", "echo_object", "subray_hit"):
        assert torch.equal(out[k], ref[k]), k


@pytest.mark.parametrize("name", ["tls", "als"])
def test_echo_width_fit_matches_oracle(hg, name):
    """Sec. 3.4 echo width: the GPU's FP32 Levenberg-Marquardt fit against the
    oracle's FP64 one on the same waveforms, 1e-3 relative, on pulses with no
    geometry, echo or fit-decision flag."""
    if name == "tls":
        w = scenes.tls_tiny(n_az=60, n_el=40)
    else:
        w = scenes.als_terrain(seed=5, size=128, n_trees=12, n_pulses=4001, n_bins=512, agl=120.0,
                               speed=30.0, prf=50_000.0)
    sc, leg = w.scanners[0], w.legs[0]
    gs = hg.Scene(w.scenes[0])
    out, lay = hg.scan([gs], [sc], [leg], seed=3, echo_width=True)
    torch.cuda.synchronize()
    ref = oracle.scan(oracle.OracleScene(w.scenes[0]), sc, leg, mode=0, seed=3, echo_width=True)
    K = sc.max_echoes
    gw = to_np(out["echo_width"]).reshape(-1, K)
    gc = to_np(out["echo_count"])
    ok = (ref["flags"] & (oracle.F_DECISION | oracle.F_OVERFLOW | oracle.F_FIT)) == 0
    ok &= gc == ref["echo_count"]
    n = 0
    for i in np.nonzero(ok)[0]:
        for e in range(min(gc[i], K)):
            a, b = gw[i, e], ref["echo_width"][i, e]
            assert abs(a - b) <= 1e-3 * b, (i, e, a, b)
            n += 1
        assert (gw[i, gc[i]:] == 0).all()
    assert n > (300 if name == "tls" else 500)


@pytest.mark.parametrize("defl", ["palmer", "fibre", "noise"])
def test_palmer_fibre_deflectors_and_platform_noise(hg, defl):
    """Sec. 3.3 deflectors (slanted rotating mirror; fibre-optic line) and
    Sec. 3.7 platform noise over the terrain workload, against the oracle."""
    w = scenes.als_terrain(seed=5, size=128, n_trees=12, n_pulses=5003, n_bins=512, agl=120.0,
                           speed=30.0, prf=50_000.0)
    if defl == "palmer":
        w = scenes.with_scanner(w, deflector=scenes.DEFL_PALMER, scan_angle_max_rad=math.radians(12.0),
                                scan_freq_hz=40.0)
    elif defl == "fibre":
        w = scenes.with_scanner(w, deflector=scenes.DEFL_FIBRE, n_fibres=37)
    else:
        import dataclasses
        w = scenes.Workload(w.name, w.scenes, w.scanners,
                            [dataclasses.replace(w.legs[0], platform_noise_m=0.05)])
    _, _, res = run_both(hg, w, seed=13)
    stats = compare(*res[0])
    assert stats["echoes"] > 2500


@pytest.mark.parametrize("mode", [0, 1])
def test_opaque_voxels(hg, mode):
    """Sec. 3.5.4 non-transmissive voxels: the first dense voxel stops the
    subray at its entry face (stochastic and expected modes)."""
    w = scenes.uls_voxels(seed=6, n=48, n_pulses=3001, n_bins=512, agl=12.0, speed=1.0, prf=2000.0)
    w.scenes[0].grids[0].opaque = 1
    _, _, res = run_both(hg, w, mode=mode, seed=11)
    stats = compare(*res[0], expected_mode=(mode == 1))
    assert stats["echoes"] > 1000


def test_adjoint_rejects_opaque_grids(hg):
    w = scenes.uls_voxels(seed=6, n=16, n_pulses=64, n_bins=128, agl=5.0, speed=1.0, prf=1000.0)
    w.scenes[0].grids[0].opaque = 1
    gs = hg.Scene(w.scenes[0])
    out, _ = hg.scan([gs], w.scanners, w.legs, mode=1)
    with pytest.raises(hg.HeliosError) as e:
        hg.scan_adjoint([gs], w.scanners, w.legs, out["waveform"], out["window_bin"], out["subray_hit"])
    assert e.value.code == -6


@pytest.mark.parametrize("kind", lad.KINDS)
def test_lad_table_generator_matches_oracle(hg, kind):
    """helios_lad_table (Ross kernel, Simpson, FP64 on the device) against the
    oracle's quadrature of Eq. extinction's double integral."""
    for n in (2, 91, 1000):
        got = to_np(hg.lad_table(kind, n)).astype(np.float64)
        ref = lad.table(kind, n, quad=96) if n < 1000 else None
        if ref is None:
            idx = np.array([0, 1, 250, 499, 500, 777, 998, 999])
            ref_s = np.array([lad.ross_G(kind, i / (n - 1), 96) for i in idx])
            assert np.abs(got[idx] - ref_s).max() <= 1e-6
        else:
            assert np.abs(got - ref).max() <= 1e-6, np.abs(got - ref).max()


@pytest.mark.parametrize("mode", [0, 1])
def test_uls_voxels_with_leaf_angle_table(hg, mode):
    """sigma = G(|d_z|) density from an erectophile table (Table ladlut), both
    modes; the scene is also built from the library's own table, which must
    give the same result within the table's rounding."""
    w = scenes.uls_voxels(seed=6, n=48, n_pulses=3001, n_bins=512, agl=12.0, speed=1.0, prf=2000.0)
    w.scanners[0].scan_angle_max_rad = 0.6            # oblique subrays: G varies across the scan
    w.scenes[0].grids[0].lad = lad.table("erectophile", 46).astype(np.float32)
    _, _, res = run_both(hg, w, mode=mode, seed=11)
    stats = compare(*res[0], expected_mode=(mode == 1))
    assert stats["echoes"] > 1000
    if mode == 1:
        gsc = hg.Scene(w.scenes[0])
        a, _ = hg.scan([gsc], w.scanners, w.legs, mode=1)
        w.scenes[0].grids[0].lad = hg.lad_table("erectophile", 46)
        b, _ = hg.scan([hg.Scene(w.scenes[0])], w.scanners, w.legs, mode=1)
        A, B = to_np(a["waveform"]), to_np(b["waveform"])
        assert np.abs(A - B).max() <= 1e-5 * np.abs(A).max()


def _forest(lad_tables=False, opaque=False, **kw):
    w = scenes.voxel_forest(**kw)
    grids = w.scenes[0].grids
    if lad_tables:
        for g, kind in zip(grids, ["erectophile", "planophile", None, "spherical", "uniform", None,
                                   "plagiophile", "extremophile", None]):
            if kind:
                g.lad = lad.table(kind, 19).astype(np.float32)
    if opaque:
        grids[4].opaque = 1
    return w


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("variant", ["plain", "lad_opaque"])
def test_several_voxel_grids(hg, mode, variant):
    """Nine voxel trees, one grid each (neighbours touching along x), walked
    in entry order through the grid BVH; per-grid leaf-angle tables and one
    opaque tree in the second variant."""
    w = _forest(lad_tables=variant != "plain", opaque=variant != "plain", n_pulses=3001)
    _, _, res = run_both(hg, w, mode=mode, seed=5)
    stats = compare(*res[0], expected_mode=(mode == 1))
    assert stats["echoes"] > 1500
    if mode == 0:
        hits = res[0][1]["subray_hit"]
        n_tri = w.scenes[0].n_triangles
        vox = hits[hits >= n_tri] - n_tri
        offs = np.cumsum([0] + [int(np.prod(g.dims)) for g in w.scenes[0].grids])
        assert len(set(np.searchsorted(offs, vox, side="right") - 1)) >= 6   # returns from most trees


def test_adjoint_with_several_grids(hg):
    """Per-grid density gradients (and reflectance) against the oracle's, with
    leaf-angle tables on some of the trees."""
    w = _forest(lad_tables=True, n_pulses=1200, n_bins=384)
    sc, leg = w.scanners[0], w.legs[0]
    gs = hg.Scene(w.scenes[0])
    out, _ = hg.scan([gs], [sc], [leg], mode=1)
    # dL/dW of a squared misfit to a scan of perturbed densities (every grid)
    ref_grids = [scenes.VoxelGrid(**{**g.__dict__, "density": scenes.perturbed_density(g.density, seed=1 + i)})
                 for i, g in enumerate(w.scenes[0].grids)]
    gref = hg.Scene(scenes.Scene(meshes=w.scenes[0].meshes, grids=ref_grids))
    out_ref, _ = hg.scan([gref], [sc], [leg], mode=1)
    gW = 2.0 * (out["waveform"] - out_ref["waveform"])
    grads = hg.scan_adjoint([gs], [sc], [leg], gW, out["window_bin"], out["subray_hit"])
    torch.cuda.synchronize()
    osc = oracle.OracleScene(w.scenes[0])
    rows = np.arange(leg.n_pulses)
    d_refl, d_dens = oracle.adjoint(osc, sc, leg, rows, to_np(gW).reshape(-1, sc.n_bins).astype(np.float64),
                                    to_np(out["window_bin"]))
    gd = np.concatenate([to_np(t).ravel() for t in grads[0]["density"]])
    scale = np.abs(d_dens).max()
    assert scale > 0 and len(gd) == len(d_dens)
    err = np.abs(gd - d_dens) - (1e-3 * np.abs(d_dens) + 1e-6 * scale)
    big = np.abs(d_dens) >= 1e-2 * scale
    assert np.median(np.abs(gd - d_dens)[big] / np.abs(d_dens)[big]) < 1e-4
    assert (err <= 0).all(), f"density gradient: {int((err > 0).sum())} entries outside tolerance"
    touched = [int((np.abs(to_np(t)) > 0).sum()) for t in grads[0]["density"]]
    assert sum(t > 0 for t in touched) >= 6
    gr = to_np(grads[0]["reflectance"][0])
    assert np.allclose(gr, d_refl, rtol=1e-3, atol=1e-6 * np.abs(d_refl).max())


@pytest.mark.parametrize("mode", [0, 1])
def test_resumed_leg_matches_the_oracle_and_the_whole_leg(hg, mode):
    """first_pulse = K scans pulses K.. into rows 0..: against the oracle on
    those pulses, and against the same rows of the whole leg's scan (every
    draw is keyed by the absolute pulse index)."""
    import dataclasses
    w = scenes.uls_voxels(seed=6, n=48, n_pulses=3001, n_bins=512, agl=12.0, speed=1.0, prf=2000.0)
    sc, leg = w.scanners[0], w.legs[0]
    K = 1237
    rleg = dataclasses.replace(leg, first_pulse=K, n_pulses=leg.n_pulses - K)
    gs = hg.Scene(w.scenes[0])
    full, lay_f = hg.scan([gs], [sc], [leg], mode=mode, seed=11)
    part, lay_p = hg.scan([gs], [sc], [rleg], mode=mode, seed=11)
    torch.cuda.synchronize()
    S = hg.subray_count(sc.beam_sample_quality)
    osc = oracle.OracleScene(w.scenes[0])
    rows = np.arange(rleg.n_pulses)
    ref = oracle.scan(osc, sc, leg, K + rows, mode=mode, seed=11)
    stats = compare(leg_view(part, lay_p, 0, sc, S, rows), ref, expected_mode=(mode == 1))
    assert stats["echoes"] > 500
    a = leg_view(part, lay_p, 0, sc, S, rows)
    b = leg_view(full, lay_f, 0, sc, S, K + rows)
    ok = (ref["flags"] & oracle.F_DECISION) == 0      # no near-tie decision on these pulses
    assert np.array_equal(a["window_bin"][ok], b["window_bin"][ok])
    scale = np.abs(b["waveform"]).max(axis=1, keepdims=True)
    assert (np.abs(a["waveform"] - b["waveform"]) <= 1e-5 * scale + 1e-30)[ok].all()
    assert np.array_equal(a["echo_count"][ok], b["echo_count"][ok])
