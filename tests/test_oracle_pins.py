"""Pins for the FP64 oracle: facts fixed by the paper or by mathematics,
independent of the oracle's own code (CPU only).

Each test names the passage or the closed form it relies on.  A plausible
mistake in the oracle (a dropped term, a wrong sign, a swapped axis, an
off-by-one ring) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
C_LIGHT = 299792458.0


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return np.array(rows)


# --------------------------------------------------------------------------
# counter-based generator
# --------------------------------------------------------------------------

def test_philox_matches_published_known_answers():
    """Philox4x32-10 (Salmon et al. 2011) against the generator's published
    known-answer vectors (tests/golden/philox4x32_10_kat.txt): zero, all-ones
    and digits-of-pi counters and keys."""
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [line.split() for line in f if line.strip() and not line.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_philox_counter_and_key_words_all_matter():
    """Flipping any single bit of the counter or key changes every output word
    (avalanche over ten rounds): no word of the counter layout is dropped."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        ctr = [int(x) for x in rng.integers(0, 2 ** 32, size=4, dtype=np.uint64)]
        key = [int(x) for x in rng.integers(0, 2 ** 32, size=2, dtype=np.uint64)]
        base = oracle.philox4x32_10(ctr, key)
        for w in range(6):
            for b in (0, 13, 31):
                c, k = list(ctr), list(key)
                if w < 4:
                    c[w] ^= 1 << b
                else:
                    k[w - 4] ^= 1 << b
                out = oracle.philox4x32_10(c, k)
                assert all(x != y for x, y in zip(out, base))


def test_uniform24_open_interval_and_fp32_exact():
    lib = oracle.lib()
    for w in [0, 1, 2 ** 9 - 1, 2 ** 9, 2 ** 32 - 1, 0x80000000]:
        u = lib.or_uniform24(w)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u          # identical in FP32 and FP64


# --------------------------------------------------------------------------
# subrays (Sec. 3.4)
# --------------------------------------------------------------------------

def test_subray_counts_match_paper_caption():
    for q, count in _golden("subray_counts.txt"):
        assert oracle.subray_count(int(q)) == int(count)


def test_subray_counts_small_q():
    # centre + 6 + 12 (+ 18) subrays: the 19-subray beam with rings at half and
    # full divergence radius, and the q = 3 beam of the paper's timing runs
    assert [oracle.subray_count(q) for q in range(4)] == [1, 7, 19, 37]


def test_subray_ring_geometry():
    sc = scenes.Scanner(divergence_rad=0.3e-3)
    rng = np.random.default_rng(5)
    for q in (1, 2, 3, 5):
        S = oracle.subray_count(q)
        for _ in range(5):
            d = rng.standard_normal(3)
            d /= np.linalg.norm(d)
            u, v = oracle.onb(d)
            ring_of = []
            for s in range(S):
                alpha, phi = oracle.subray_angles(q, 0.15e-3, s)
                ds = oracle.subray_dir(sc, q, s, d)
                assert abs(np.linalg.norm(ds) - 1.0) < 1e-14
                # angular offset from the pulse axis equals the ring angle
                ang = math.atan2(np.linalg.norm(np.cross(d, ds)), float(np.dot(d, ds)))
                assert abs(ang - alpha) < 1e-12
                if s > 0:
                    # azimuth in the (u, v) frame equals phi
                    az = math.atan2(float(np.dot(ds, v)), float(np.dot(ds, u))) % (2 * math.pi)
                    assert abs((az - phi + math.pi) % (2 * math.pi) - math.pi) < 1e-6
                ring_of.append(round(alpha / 0.15e-3 * q))
            # ring i holds floor(2 pi i) subrays, outermost at the full radius
            counts = np.bincount(ring_of)
            assert counts[0] == 1
            for i in range(1, q + 1):
                assert counts[i] == math.floor(2 * math.pi * i)


@pytest.mark.parametrize("n", [(0, 0, 1), (0, 0, -1), (1, 0, 0), (1, 0, -0.0), (0.6, 0.0, 0.8),
                               (-0.3, 0.9, -0.3162277660168379)])
def test_onb_is_right_handed_orthonormal(n):
    n = np.array(n, float)
    n /= np.linalg.norm(n)
    u, v = oracle.onb(n)
    M = np.stack([u, v, n])
    assert np.allclose(M @ M.T, np.eye(3), atol=1e-15)
    assert np.allclose(np.cross(u, v), n, atol=1e-15)


# --------------------------------------------------------------------------
# pulses: platform (Sec. 3.2) and deflectors (Sec. 3.3)
# --------------------------------------------------------------------------

def test_tls_grid_directions():
    sc = scenes.Scanner(deflector=scenes.DEFL_TLS_GRID, grid_n_az=8, grid_n_el=5,
                        el_min_rad=-0.5, el_max_rad=0.7)
    leg = scenes.Leg(platform=scenes.PLATFORM_STATIC, start=(1.0, 2.0, 3.0), n_pulses=40)
    for i in range(8):
        for j in range(5):
            o, d = oracle.pulse_ray(sc, leg, i * 5 + j)
            az = 2 * math.pi * i / 8
            el = -0.5 + 1.2 * j / 4
            assert np.allclose(o, [1, 2, 3])
            assert np.allclose(d, [math.cos(el) * math.cos(az), math.cos(el) * math.sin(az),
                                   math.sin(el)], atol=1e-15)


def test_linear_platform_position_heading_and_mirror():
    f = 50.0
    amax = math.radians(20)
    sc = scenes.Scanner(prf_hz=1000.0, deflector=scenes.DEFL_OSCILLATING, scan_freq_hz=f,
                        scan_angle_max_rad=amax)
    # flight along +y: heading 90 deg, the platform's left (+y) maps to world -x
    leg = scenes.Leg(platform=scenes.PLATFORM_LINEAR, start=(0, 0, 100), end=(0, 100, 100),
                     speed_mps=10.0, n_pulses=100000)
    o, d = oracle.pulse_ray(sc, leg, 0)
    assert np.allclose(o, [0, 0, 100]) and np.allclose(d, [0, 0, -1], atol=1e-15)
    k = 5  # t = 5 ms = 1/(4 f): swing at +amax
    o, d = oracle.pulse_ray(sc, leg, k)
    assert np.allclose(o, [0, 10.0 * k / 1000.0, 100])
    assert np.allclose(d, [-math.sin(amax), 0, -math.cos(amax)], atol=1e-12)
    # past the end of the leg the platform waits at the waypoint
    o, _ = oracle.pulse_ray(sc, leg, 20000)
    assert np.allclose(o, [0, 100, 100])


def _scan_angles(deflector, n=20000):
    sc = scenes.Scanner(prf_hz=n * 10.0, deflector=deflector, scan_freq_hz=10.0,
                        scan_angle_max_rad=math.radians(30))
    leg = scenes.Leg(platform=scenes.PLATFORM_STATIC, start=(0, 0, 0))
    th = []
    for k in range(n):
        _, d = oracle.pulse_ray(sc, leg, k)
        th.append(math.atan2(d[1], -d[2]))
    return np.array(th)


def test_swinging_mirror_denser_at_extrema_polygon_even():
    """Sec. 3.3: a swinging mirror yields higher point density at the extrema,
    a polygon mirror even density along parallel lines."""
    h, _ = np.histogram(_scan_angles(scenes.DEFL_OSCILLATING), bins=10)
    assert h[0] > 2 * h[5] and h[-1] > 2 * h[4]
    h, _ = np.histogram(_scan_angles(scenes.DEFL_POLYGON), bins=10)
    assert h.max() - h.min() <= 0.02 * h.mean() + 2


# --------------------------------------------------------------------------
# beam and radar equation (Eq. beamdiv, Eq. beamdiv_w, Eq. ladlut_intensity)
# --------------------------------------------------------------------------

def test_gaussian_beam_width_textbook():
    sc = scenes.Scanner(divergence_rad=0.3e-3, wavelength_m=1064e-9, focus_m=7.0)
    w0 = 1064e-9 / (math.pi * 0.15e-3)
    assert abs(w0 - 2.2578e-3) < 1e-6
    zr = math.pi * w0 ** 2 / 1064e-9
    assert abs(zr - 15.05) < 0.01
    assert abs(oracle.beam_width(sc, 7.0) - w0) < 1e-15             # waist at the focus
    assert abs(oracle.beam_width(sc, 7.0 + zr) / w0 - math.sqrt(2)) < 1e-12  # Rayleigh range
    R = 1e6
    assert abs(oracle.beam_width(sc, R) / ((R - 7.0) * 0.15e-3) - 1) < 1e-9   # far-field cone


def test_subray_intensity_one_over_e2_at_divergence_radius():
    sc = scenes.Scanner(divergence_rad=0.3e-3, peak_power_w=2.0)
    assert oracle.subray_intensity(sc, 500.0, 0.0) == 2.0
    # far field: the ring at theta_r = divergence/2 sits on the 1/e^2 contour
    assert abs(oracle.subray_intensity(sc, 1e5, 0.15e-3) / 2.0 - math.exp(-2)) < 1e-6


def test_radar_equation_with_lambertian_cross_section():
    """Eq. ladlut_intensity, P = lambda sigma P0 alpha^2 / (4 pi d^4 beta^2), with the
    extended Lambertian cross-section sigma = pi rho d^2 beta^2 cos(theta): beta cancels."""
    sc = scenes.Scanner(receiver_diam_m=0.12, eta_sys=0.8, eta_atm=0.95)
    rng = np.random.default_rng(3)
    for _ in range(20):
        I, R, rho, c = rng.uniform(0.1, 3), rng.uniform(1, 800), rng.uniform(0, 1), rng.uniform(0, 1)
        for beta in (1e-4, 3e-4, 2e-3):
            sigma = math.pi * rho * R ** 2 * beta ** 2 * c
            expect = (0.8 * 0.95) * sigma * I * 0.12 ** 2 / (4 * math.pi * R ** 4 * beta ** 2)
            got = oracle.triangle_power(sc, I, R, rho, c)
            assert abs(got - expect) <= 1e-12 * expect


def test_pulse_shapes():
    g = scenes.Scanner(pulse_shape=scenes.PULSE_GAUSSIAN, pulse_fwhm_ns=4.0)
    assert oracle.pulse_shape(g, 0.0) == 1.0
    assert abs(oracle.pulse_shape(g, 2.0) - 0.5) < 1e-15
    assert abs(oracle.pulse_shape(g, -2.0) - 0.5) < 1e-15
    # Eq. beam_time with tau = pulse length / 1.75: peak 4/e^2 at t = 2 tau, area 2 tau
    c = scenes.Scanner(pulse_shape=scenes.PULSE_CARLSSON, pulse_length_ns=3.5)
    tau = 2.0
    assert abs(oracle.pulse_shape(c, 2 * tau) - 4 * math.exp(-2)) < 1e-15
    ts = np.linspace(0, 80, 80001)
    vals = np.array([oracle.pulse_shape(c, t) for t in ts])
    assert abs(ts[np.argmax(vals)] - 2 * tau) < 1e-3
    assert abs(np.trapezoid(vals, ts) - 2 * tau) < 1e-6
    assert oracle.pulse_shape(c, -0.1) == 0.0


# --------------------------------------------------------------------------
# intersection (Sec. 5.1)
# --------------------------------------------------------------------------

def test_bvh_matches_brute_force_on_random_soups():
    rng = np.random.default_rng(11)
    for seed in range(100):
        n = int(rng.integers(1, 501))
        osc = oracle.OracleScene(scenes.triangle_soup(seed, n))
        for _ in range(50):
            o = rng.uniform(-15, 15, 3)
            d = rng.standard_normal(3)
            d /= np.linalg.norm(d)
            i, t, c, f = osc.intersect(o, d)
            j, t2, c2 = osc.intersect_brute(o, d)
            if f:
                continue
            assert i == j
            if i >= 0:
                assert t == t2 and c == c2
        osc.close()


def test_plane_range_and_incidence_closed_form():
    D = 37.5
    osc = oracle.OracleScene(scenes.flat_target(D, 0.0, half=1000.0))
    o = np.array([0.3, -0.1, 0.0])          # off the plate's shared diagonal
    for phi in np.radians([0, 5, 17, 33, 60]):
        d = np.array([0.0, math.sin(phi), -math.cos(phi)])
        i, t, c, f = osc.intersect(o, d)
        assert i >= 0 and f == 0
        assert abs(t - D / math.cos(phi)) < 1e-12 * t
        assert abs(c - math.cos(phi)) < 1e-14
    for tilt in np.radians([10, 25, 50]):
        osc = oracle.OracleScene(scenes.flat_target(D, tilt, half=16.0))
        i, t, c, f = osc.intersect(o, [0.0, 0.0, -1.0])
        # plane through (0, 0, -D) with normal (0, -sin, cos): z = -D + y tan(tilt);
        # the corners are FP32, which moves the plane by at most ~ulp(40 m)
        assert f == 0
        assert abs(t - (D - o[1] * math.tan(tilt))) < 1e-5
        assert abs(c - math.cos(tilt)) < 1e-6


def test_edge_flag_on_shared_edge():
    # the diagonal of the 2-triangle plate is shared: a ray through it is flagged
    osc = oracle.OracleScene(scenes.flat_target(10.0, 0.0, half=5.0))
    d = np.array([0.3, 0.3, -10.0])
    d /= np.linalg.norm(d)
    _, _, _, f = osc.intersect([0, 0, 0], d)
    assert f & oracle.F_EDGE
    d = np.array([0.3, -0.1, -10.0])
    d /= np.linalg.norm(d)
    _, _, _, f = osc.intersect([0, 0, 0], d)
    assert f == 0


# --------------------------------------------------------------------------
# voxels (Sec. 3.5.4, Sec. 5.2)
# --------------------------------------------------------------------------

def _grid_scene(dens, origin=(-1.0, -1.0, -1.0), cell=0.5, ground_z=None, G=0.5, refl=0.3):
    nz, ny, nx = dens.shape
    grid = scenes.VoxelGrid(origin=origin, cell=cell, dims=(nx, ny, nz),
                            density=np.ascontiguousarray(dens, np.float32), G=G,
                            leaf_reflectance=0.5)
    meshes = []
    if ground_z is not None:
        gv = np.array([[-500, -500, ground_z], [500, -500, ground_z], [500, 500, ground_z],
                       [-500, 500, ground_z]], float)
        meshes.append(scenes.Mesh(gv.astype(np.float32), np.array([[0, 1, 2], [0, 2, 3]], np.int32),
                                  np.full(2, refl, np.float32)))
    return scenes.Scene(meshes=meshes, grids=[grid])


def test_march_matches_per_voxel_slab_brute_force():
    rng = np.random.default_rng(2)
    dims = (5, 4, 3)
    dens = np.ones(dims[::-1], np.float32)
    osc = oracle.OracleScene(_grid_scene(dens, origin=(-1.0, -1.0, -1.0), cell=0.5))
    lo = np.array([-1.0, -1.0, -1.0])
    for _ in range(300):
        o = rng.uniform(-4, 4, 3)
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        vid, ti, to = osc.march(o, d)
        # brute force: every voxel box, exact slab interval, positive length, t >= 0
        ref = []
        for z in range(3):
            for y in range(4):
                for x in range(5):
                    a = lo + 0.5 * np.array([x, y, z])
                    b = a + 0.5
                    with np.errstate(divide="ignore", invalid="ignore"):
                        t1 = (a - o) / d
                        t2 = (b - o) / d
                    tin = max(0.0, np.max(np.minimum(t1, t2)))
                    tout = np.min(np.maximum(t1, t2))
                    if tout - tin > 1e-9:
                        ref.append((tin, (z * 4 + y) * 5 + x, tout))
        ref.sort()
        got = [(a, int(v), b) for a, v, b in zip(ti, vid, to) if b - a > 1e-9]
        assert [r[1] for r in ref] == [g[1] for g in got]
        for r, g in zip(ref, got):
            assert abs(r[0] - g[0]) < 1e-12 and abs(r[2] - g[2]) < 1e-12


def _f32(x):
    """The real number an FP32 input actually holds."""
    return float(np.float32(x))


def _voxel_power_unit(sc, R, alpha=0.0):
    Is = oracle.subray_intensity(sc, R, alpha)
    return oracle.triangle_power(sc, Is, R, 0.5, 1.0)


def test_expected_mode_transmittance_is_exp_minus_sigma_path():
    """Eq. intersection_dist in expectation: a slab of density d, thickness L,
    projection factor G transmits exp(-G d L) to the target behind it."""
    sc = scenes.Scanner()
    dens = np.full((4, 40, 40), 1.3, np.float32)   # 4 layers of 0.5 m, 20 x 20 m wide
    osc = oracle.OracleScene(_grid_scene(dens, origin=(-10.0, -10.0, 0.0), cell=0.5, ground_z=-2.0))
    bare = oracle.OracleScene(_grid_scene(np.zeros_like(dens), origin=(-10.0, -10.0, 0.0), cell=0.5,
                                          ground_z=-2.0))
    for phi in np.radians([0.0, 10.0, 20.0]):
        d = np.array([0.0, math.sin(phi), -math.cos(phi)])
        o = np.array([0.0, -12.0 * math.tan(phi), 10.0])
        R, P, ids, _ = oracle.trace_returns(osc, sc, o, d, mode=1)
        R0, P0, ids0, _ = oracle.trace_returns(bare, sc, o, d, mode=1)
        assert ids[-1] == ids0[-1] >= 0 and len(P0) == 1
        # path inside the slab: 2 m thick along z
        L = 2.0 / math.cos(phi)
        assert abs(P[-1] / P0[0] - math.exp(-0.5 * _f32(1.3) * L)) < 1e-12
        # voxel weights + transmitted weight = 1 (nothing is created or lost)
        w = [p / _voxel_power_unit(sc, r) for r, p in zip(R[:-1], P[:-1])]
        assert abs(sum(w) + P[-1] / P0[0] - 1.0) < 1e-12


def test_expected_mode_transmittance_multiplies_across_layers():
    sc = scenes.Scanner()
    dens = np.zeros((3, 1, 1), np.float32)
    dens[0], dens[1], dens[2] = 0.7, 0.0, 2.1        # layers 1 m each (bottom to top)
    osc = oracle.OracleScene(_grid_scene(dens, origin=(-0.5, -0.5, 0.0), cell=1.0, ground_z=-1.0))
    bare = oracle.OracleScene(_grid_scene(np.zeros_like(dens), origin=(-0.5, -0.5, 0.0), cell=1.0,
                                          ground_z=-1.0))
    d = np.array([0.0, 0.0, -1.0])
    R, P, ids, _ = oracle.trace_returns(osc, sc, [0, 0, 5.0], d, mode=1)
    R0, P0, _, _ = oracle.trace_returns(bare, sc, [0, 0, 5.0], d, mode=1)
    assert len(P) == 3   # two non-empty voxels + ground
    assert abs(P[-1] / P0[0] - math.exp(-0.5 * _f32(2.1)) * math.exp(-0.5 * _f32(0.7))) < 1e-13
    # each voxel returns at its segment midpoint
    assert abs(R[0] - 2.5) < 1e-12 and abs(R[1] - 4.5) < 1e-12


def test_stochastic_transmission_frequency_binomial():
    """Eq. intersection_dist: the probability to cross the slab is exp(-G d L)."""
    sc = scenes.Scanner()
    dens = np.full((2, 1, 1), 0.8, np.float32)
    osc = oracle.OracleScene(_grid_scene(dens, origin=(-0.5, -0.5, 0.0), cell=1.0, ground_z=-1.0))
    n = 20000
    hits_ground = 0
    depths = []
    for k in range(n):
        R, P, ids, f = oracle.trace_returns(osc, sc, [0, 0, 5.0], [0, 0, -1.0], mode=0, seed=77,
                                            leg_id=3, pulse=k, s=0)
        assert len(R) == 1
        if ids[0] < osc.n_tri:
            hits_ground += 1
        else:
            depths.append(R[0] - 3.0)
    p = math.exp(-0.5 * _f32(0.8) * 2.0)
    sd = math.sqrt(n * p * (1 - p))
    assert abs(hits_ground - n * p) < 5 * sd
    # stop depth inside the slab is exponential with rate sigma, truncated at 2 m
    sig = 0.5 * _f32(0.8)
    mean_trunc = 1 / sig - 2.0 * math.exp(-2 * sig) / (1 - math.exp(-2 * sig))
    depths = np.array(depths)
    assert abs(depths.mean() - mean_trunc) < 5 * depths.std() / math.sqrt(len(depths))


# --------------------------------------------------------------------------
# waveform and echoes (Sec. 3.4, Sec. 3.7)
# --------------------------------------------------------------------------

def _nadir_leg(n=1, el_lo=-math.pi / 2, el_hi=-math.pi / 2):
    sc = scenes.Scanner(deflector=scenes.DEFL_TLS_GRID, grid_n_az=1, grid_n_el=n,
                        el_min_rad=el_lo, el_max_rad=el_hi, n_bins=200, beam_sample_quality=0)
    leg = scenes.Leg(platform=scenes.PLATFORM_STATIC, start=(0, 0, 0), n_pulses=n)
    return sc, leg


def test_single_flat_target_waveform_area_and_echo():
    D = 23.456
    sc, leg = _nadir_leg()
    osc = oracle.OracleScene(scenes.flat_target(D, 0.0, half=100.0))
    r = oracle.scan(osc, sc, leg, mode=0, seed=1)
    assert r["echo_count"][0] == 1
    P = oracle.triangle_power(sc, sc.peak_power_w, D, 0.5, 1.0)
    W = r["waveform"][0]
    m = r["window_bin"][0]
    tau = 2 * D / C_LIGHT * 1e9
    sig = 4.0 / (2 * math.sqrt(2 * math.log(2)))
    # the bin sum is the Gaussian's integral from the window start t0, plus the
    # Euler-Maclaurin endpoint terms at t0 (the window clips the leading tail)
    dt = sc.bin_ns
    t0 = m * dt
    x0 = t0 - tau
    f0 = P * math.exp(-x0 * x0 / (2 * sig * sig))
    df0 = -f0 * x0 / (sig * sig)
    integral = P * sig * math.sqrt(2 * math.pi) * 0.5 * math.erfc(x0 / (sig * math.sqrt(2)))
    expect = integral + 0.5 * dt * f0 - dt * dt / 12.0 * df0
    assert abs(W.sum() * dt - expect) < 1e-7 * expect
    # the echo sits on the bin nearest to the delay: within half a bin in range
    b = r["echo_bin"][0, 0]
    assert abs((m + b) * sc.bin_ns - tau) <= 0.5 * sc.bin_ns + 1e-12
    assert abs(r["echo_range_clean"][0, 0] - D) <= C_LIGHT * sc.bin_ns * 1e-9 / 4 + 1e-9
    assert r["echo_object"][0, 0] in (0, 1)


def test_two_targets_in_one_footprint_give_two_echoes():
    """Sec. 3.4: parts of the footprint on different targets give separate echoes."""
    D1, D2 = 20.0, 26.0
    sc, leg = _nadir_leg()
    sc.beam_sample_quality = 2
    sc.divergence_rad = 0.3e-3
    near = np.array([[-5, 0.0005, -D1], [5, 0.0005, -D1], [5, 5, -D1], [-5, 5, -D1]], np.float32)
    far = np.array([[-50, -50, -D2], [50, -50, -D2], [50, 50, -D2], [-50, 50, -D2]], np.float32)
    F = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    scene = scenes.Scene(meshes=[scenes.Mesh(near, F, np.full(2, 0.5, np.float32)),
                                 scenes.Mesh(far, F, np.full(2, 0.5, np.float32))])
    osc = oracle.OracleScene(scene)
    r = oracle.scan(osc, sc, leg, mode=0, seed=1)
    assert r["echo_count"][0] == 2
    got = sorted(r["echo_range_clean"][0, :2])
    half_bin = C_LIGHT * sc.bin_ns * 1e-9 / 4
    assert abs(got[0] - D1) < half_bin + 1e-6 and abs(got[1] - D2) < half_bin + 2e-6
    hits = r["subray_hit"][0]
    assert set(hits[hits >= 0] // 2) == {0, 1}   # both plates are hit by some subrays


def test_range_noise_is_normal_with_scanner_sigma():
    """Sec. 3.7: each range gets a N(0, sigma) error; Box-Muller on Philox draws."""
    n = 4000
    sc, leg = _nadir_leg(n, -math.radians(89.0), -math.radians(88.0))
    osc = oracle.OracleScene(scenes.flat_target(30.0, 0.0, half=100.0))
    r = oracle.scan(osc, sc, leg, mode=0, seed=9)
    assert (r["echo_count"] == 1).all()
    e = r["echo_range"][:, 0] - r["echo_range_clean"][:, 0]
    assert abs(e.mean()) < 5 * 0.01 / math.sqrt(n)
    assert abs(e.std() / 0.01 - 1) < 0.06
    assert abs(np.mean(e ** 4) / np.mean(e ** 2) ** 2 - 3) < 0.3   # Gaussian kurtosis


def test_scan_is_deterministic_and_thread_independent():
    w = scenes.tls_tiny(n_az=30, n_el=30)
    osc = oracle.OracleScene(w.scenes[0])
    a = oracle.scan(osc, w.scanners[0], w.legs[0], threads=1, seed=5)
    b = oracle.scan(osc, w.scanners[0], w.legs[0], threads=7, seed=5)
    for k in ("waveform", "echo_range", "subray_hit", "flags", "window_bin"):
        assert np.array_equal(a[k], b[k])


# --------------------------------------------------------------------------
# adjoint (expected mode): analytic gradient vs central differences in FP64
# --------------------------------------------------------------------------

def test_adjoint_matches_central_differences():
    w = scenes.uls_voxels(seed=4, n=24, n_pulses=4000, n_bins=256, agl=8.0, speed=1.0, prf=2000.0)
    w.scanners[0].beam_sample_quality = 1
    scene = w.scenes[0]
    sc, leg = w.scanners[0], w.legs[0]
    pulses = np.arange(0, 4000, 250, dtype=np.int64)
    osc = oracle.OracleScene(scene)
    base = scene.grids[0].density.copy()
    ref_d = scenes.perturbed_density(base, seed=1)
    osc.set_density(ref_d)
    W_ref = oracle.scan(osc, sc, leg, pulses, mode=1)["waveform"]
    osc.set_density(base)
    fwd = oracle.scan(osc, sc, leg, pulses, mode=1)
    win = fwd["window_bin"]
    assert (win != oracle.NO_WINDOW).all()
    g = 2.0 * (fwd["waveform"] - W_ref)
    d_refl, d_dens = oracle.adjoint(osc, sc, leg, pulses, g, win)

    def loss(dens=None, refl=None):
        if refl is not None:
            scene.meshes[0].reflectance[:] = refl
            o2 = oracle.OracleScene(scene)
        else:
            o2 = osc
            o2.set_density(dens)
        W = oracle.scan(o2, sc, leg, pulses, mode=1, fixed_window=win)["waveform"]
        return float(((W - W_ref) ** 2).sum())

    touched = np.nonzero(d_dens)[0]
    assert len(touched) > 64
    rng = np.random.default_rng(2)
    for v in rng.choice(touched, 64, replace=False):      # 64 traversed voxels
        x = float(base.ravel()[v])
        h = 1e-4 * max(abs(x), 1e-2)
        dp = base.copy().ravel(); dp[v] = np.float32(x + h)
        dm = base.copy().ravel(); dm[v] = np.float32(x - h)
        hh = (float(dp[v]) - float(dm[v])) / 2
        fd = (loss(dens=dp.reshape(base.shape)) - loss(dens=dm.reshape(base.shape))) / (2 * hh)
        assert abs(fd - d_dens[v]) <= 1e-5 * abs(d_dens[v]) + 1e-9 * np.abs(d_dens).max()
    osc.set_density(base)
    refl0 = scene.meshes[0].reflectance.copy()
    for t in range(2):
        h = 1e-3
        rp = refl0.copy(); rp[t] += np.float32(h)
        rm = refl0.copy(); rm[t] -= np.float32(h)
        hh = (float(rp[t]) - float(rm[t])) / 2
        fd = (loss(refl=rp) - loss(refl=rm)) / (2 * hh)
        assert abs(fd - d_refl[t]) <= 1e-6 * abs(d_refl[t]) + 1e-12
    scene.meshes[0].reflectance[:] = refl0


# --------------------------------------------------------------------------
# echo width (Sec. 3.4: optional non-linear least-squares estimate)
# --------------------------------------------------------------------------

def test_echo_width_fit_recovers_an_exact_gaussian():
    """Samples of A exp(-(b - mu)^2 / (2 s^2)) are fitted back to s, from the
    standard start (the peak bin, the peak value, the emitted pulse's sigma)."""
    b = np.arange(120, dtype=np.float64)
    for A, mu, s in [(3.0, 40.3, 6.1), (0.7, 55.8, 8.9), (1.0, 60.0, 6.8), (2.5, 70.45, 5.2)]:
        W = A * np.exp(-0.5 * ((b - mu) / s) ** 2)
        got, _ = oracle.echo_width(W, int(round(mu)), 6.8)
        assert abs(got - s) < 1e-8 * s
    # a model error (wrong Jacobian, sign, or damping) shows as a miss here:
    # two overlapping Gaussians are not one, and the fit must not claim so
    W = np.exp(-0.5 * ((b - 50) / 6.8) ** 2) + 0.6 * np.exp(-0.5 * ((b - 58) / 6.8) ** 2)
    got, _ = oracle.echo_width(W, 50, 6.8)
    assert got > 7.0


def test_single_flat_target_echo_width_is_the_pulse_sigma():
    """One target at normal incidence returns the emitted pulse shape, so the
    fitted width is the pulse's sigma; a tilted target spreads the subrays'
    delays and widens the echo."""
    sc, leg = _nadir_leg()
    sig = sc.pulse_fwhm_ns / (2 * math.sqrt(2 * math.log(2)))
    osc = oracle.OracleScene(scenes.flat_target(31.7, 0.0, half=100.0))
    r = oracle.scan(osc, sc, leg, mode=0, seed=1, echo_width=True)
    assert r["echo_count"][0] == 1
    assert abs(r["echo_width"][0, 0] - sig) < 1e-6 * sig
    assert (r["echo_width"][0, 1:] == 0).all()
    widths = []
    sc.beam_sample_quality = 3
    sc.divergence_rad = 20e-3          # a wide beam: metres of range spread on a tilt
    for tilt in np.radians([0.0, 30.0, 60.0]):
        osc = oracle.OracleScene(scenes.flat_target(31.7, tilt, half=100.0))
        r = oracle.scan(osc, sc, leg, mode=0, seed=1, echo_width=True)
        widths.append(r["echo_width"][0, 0])
    assert widths[0] < widths[1] < widths[2]


# --------------------------------------------------------------------------
# deflectors (Sec. 3.3), platform noise (Sec. 3.7), opaque voxels (Sec. 3.5.4)
# --------------------------------------------------------------------------

def test_palmer_cone_and_fibre_line_directions():
    """Palmer: every pulse at the cone angle off nadir, azimuth 2 pi frac(f t);
    fibre line: pulse k leaves fibre k mod n at -max + 2 max i/(n-1) across track."""
    leg = scenes.Leg(platform=scenes.PLATFORM_STATIC, start=(1.0, -2.0, 30.0), n_pulses=500)
    amax = math.radians(15.0)
    sc = scenes.Scanner(deflector=scenes.DEFL_PALMER, scan_angle_max_rad=amax, scan_freq_hz=37.0,
                        prf_hz=10_000.0)
    for k in (0, 1, 77, 499):
        o, d = oracle.pulse_ray(sc, leg, k)
        assert np.allclose(o, leg.start)
        assert abs(math.acos(-d[2]) - amax) < 1e-12
        ph = (37.0 * k / 10_000.0) % 1.0
        az = math.atan2(d[1], d[0]) % (2 * math.pi)
        assert abs(az - 2 * math.pi * ph) < 1e-9 or abs(abs(az - 2 * math.pi * ph) - 2 * math.pi) < 1e-9
    sc = scenes.Scanner(deflector=scenes.DEFL_FIBRE, scan_angle_max_rad=amax, n_fibres=5)
    for k in range(12):
        _, d = oracle.pulse_ray(sc, leg, k)
        th = -amax + 2 * amax * (k % 5) / 4
        assert np.allclose(d, [0.0, math.sin(th), -math.cos(th)], atol=1e-15)


def test_platform_noise_moments_and_seed():
    """Per-pulse N(0, sigma) offsets of the platform on each axis, uncorrelated,
    keyed by (seed, leg, pulse); sigma 0 leaves the trajectory exact."""
    sig = 0.05
    leg = scenes.Leg(platform=scenes.PLATFORM_STATIC, start=(3.0, 4.0, 5.0), n_pulses=4000,
                     platform_noise_m=sig, leg_id=7)
    sc = scenes.Scanner(deflector=scenes.DEFL_POLYGON)
    off = np.array([oracle.pulse_ray(sc, leg, k, seed=11)[0] - leg.start for k in range(4000)])
    n = off.shape[0]
    assert np.all(np.abs(off.mean(0)) < 5 * sig / math.sqrt(n))
    assert np.all(np.abs(off.std(0) / sig - 1) < 0.06)
    c = np.corrcoef(off.T)
    assert np.all(np.abs(c[np.triu_indices(3, 1)]) < 0.06)
    o2 = oracle.pulse_ray(sc, leg, 5, seed=12)[0] - leg.start
    assert not np.allclose(o2, off[5])
    leg0 = scenes.replace(leg, platform_noise_m=0.0)
    assert np.array_equal(oracle.pulse_ray(sc, leg0, 5, seed=11)[0], np.array(leg.start))


def test_opaque_voxels_return_at_the_entry_face():
    """Non-transmissive voxels: the first voxel of non-zero density stops the
    subray where it enters, with the Lambertian cos of the face entered; an
    empty column lets it through to the ground."""
    dens = np.zeros((8, 4, 4), np.float32)          # [z][y][x], cell 0.5 m, z in [-4, 0)
    dens[2, :, :2] = 1.0                            # a layer at z in [-3, -2.5) over x < 1
    scene = _grid_scene(dens, origin=(-1.0, -1.0, -4.0), cell=0.5, ground_z=-10.0)
    scene.grids[0].opaque = 1
    osc = oracle.OracleScene(scene)
    sc, leg = _nadir_leg()
    leg = scenes.replace(leg, start=(-0.6, 0.3, 2.0))   # above the dense layer
    r = oracle.scan(osc, sc, leg, mode=0, seed=1)
    assert r["echo_count"][0] == 1
    assert abs(r["echo_range_clean"][0, 0] - (2.0 + 2.5)) < C_LIGHT * sc.bin_ns * 1e-9 / 4 + 1e-9
    hits = r["subray_hit"][0]
    assert (hits >= osc.n_tri).all()
    # the same in expected mode (deterministic), and the power is the radar
    # equation with the leaf reflectance at normal incidence
    re = oracle.scan(osc, sc, leg, mode=1, seed=1)
    assert np.allclose(re["waveform"], r["waveform"], rtol=1e-12, atol=0)
    P = oracle.triangle_power(sc, sc.peak_power_w, 4.5, 0.5, 1.0)
    assert abs(r["waveform"][0].sum() * sc.bin_ns / (P * 4.0 / 2.3548200450309493 * math.sqrt(2 * math.pi)) - 1) < 1e-3
    # over the empty half the ray reaches the ground at 12 m
    leg2 = scenes.replace(leg, start=(0.6, 0.3, 2.0))
    r2 = oracle.scan(osc, sc, leg2, mode=0, seed=1)
    assert abs(r2["echo_range_clean"][0, 0] - 12.0) < C_LIGHT * sc.bin_ns * 1e-9 / 4 + 1e-9
    # a slanted ray enters the layer through its top face (cos = |d_z|), one
    # that enters the layer's side through the x face (cos = |d_x|)
    d = np.array([0.3, 0.0, -1.0]) / math.sqrt(1.09)
    o = np.array([-2.0, 0.3, 2.0])                 # reaches z = -2.5 at x = -0.65, in the layer
    R, P, ids, _ = oracle.trace_returns(osc, sc, o, d, mode=0)
    t_top = (o[2] - (-2.5)) / -d[2]
    assert len(R) == 1 and abs(R[0] - t_top) < 1e-9
    assert abs(P[0] / oracle.triangle_power(sc, sc.peak_power_w, t_top, 0.5, abs(d[2])) - 1) < 1e-12
    d = np.array([-1.0, 0.0, -0.1]) / math.sqrt(1.01)
    o = np.array([2.0, 0.3, -2.7])
    R, P, ids, _ = oracle.trace_returns(osc, sc, o, d, mode=0)
    t_side = (o[0] - 0.0) / -d[0]                  # the layer's x = 0 face
    assert len(R) == 1 and abs(R[0] - t_side) < 1e-9
    assert abs(P[0] / oracle.triangle_power(sc, sc.peak_power_w, t_side, 0.5, abs(d[0])) - 1) < 1e-12


# --------------------------------------------------------------------------
# leaf-angle projection factor (Eq. extinction, Table ladlut)
# --------------------------------------------------------------------------

from oracle import lad  # noqa: E402

# G at a vertical and a horizontal beam, integrated by hand from de Wit's
# densities: G(0) = int f cos t dt, G(pi/2) = (2/pi) int f sin t dt.
_LAD_CLOSED = {
    "planophile": (8 / (3 * math.pi), 8 / (3 * math.pi ** 2)),
    "erectophile": (4 / (3 * math.pi), 16 / (3 * math.pi ** 2)),
    "plagiophile": (32 / (15 * math.pi), 64 / (15 * math.pi ** 2)),
    "extremophile": (28 / (15 * math.pi), 56 / (15 * math.pi ** 2)),
    "uniform": (2 / math.pi, 4 / math.pi ** 2),
    "spherical": (0.5, 0.5),
}


@pytest.mark.parametrize("kind", lad.KINDS)
def test_lad_G_vertical_and_horizontal_beam_closed_forms(kind):
    v, h = _LAD_CLOSED[kind]
    assert abs(lad.ross_G(kind, 1.0) - v) < 1e-12
    assert abs(lad.ross_G(kind, 0.0) - h) < 1e-12
    # the densities integrate to 1 (the 2 pi normalisation of g_L)
    x, w = np.polynomial.legendre.leggauss(64)
    t = (x + 1) * math.pi / 4
    assert abs(np.sum(w * lad.leaf_density(kind, t)) * math.pi / 4 - 1.0) < 1e-12


@pytest.mark.parametrize("kind", lad.KINDS)
def test_lad_G_hemispheric_mean_is_one_half(kind):
    """Ross's identity: for any leaf-normal distribution the mean of G over
    the beam directions of a hemisphere, int_0^1 G(mu) dmu, is 1/2."""
    x, w = np.polynomial.legendre.leggauss(48)
    mean = sum(0.5 * wi * lad.ross_G(kind, 0.5 * (xi + 1)) for xi, wi in zip(x, w))
    assert abs(mean - 0.5) < 1e-9


def test_lad_G_spherical_is_constant_and_inner_integral_is_ross_psi():
    """At oblique beams: spherical leaves give G = 1/2 at every angle, and the
    azimuthal integral equals Ross's closed form psi(theta, theta_L) = cos cos_L
    (1 - 2 phi/pi) + (2/pi) sin sin_L sin phi with cos phi = cot cot_L (theta +
    theta_L > pi/2), cos cos_L otherwise."""
    for mu in np.linspace(0.0, 1.0, 13):
        assert abs(lad.ross_G("spherical", mu) - 0.5) < 1e-10
    rng = np.random.default_rng(7)
    th = rng.uniform(0, math.pi / 2, 200)
    tl = rng.uniform(0, math.pi / 2, 200)
    for a, b in zip(th, tl):
        got = lad._inner(a, np.array([b]), 128)[0] / (2 * math.pi)
        c = math.cos(a) * math.cos(b)
        if a + b <= math.pi / 2:
            psi = c
        else:
            phi = math.acos(min(1.0, c / (math.sin(a) * math.sin(b))))
            psi = c * (1 - 2 * phi / math.pi) + 2 / math.pi * math.sin(a) * math.sin(b) * math.sin(phi)
        assert abs(got - psi) < 1e-12
    # quadrature converged: doubling the nodes changes nothing that matters
    for kind in lad.KINDS:
        assert abs(lad.ross_G(kind, 0.37) - lad.ross_G(kind, 0.37, n=256)) < 1e-10


def test_ladlut_printed_rows():
    """Table ladlut: the rows a labelling and one of the six densities
    reproduce agree to the printed digits (5e-6: the last row's 0.848822 is
    4e-6 below 8/(3 pi)); rows 2-3 are reproduced by neither labelling."""
    with open(os.path.join(GOLDEN, "ladlut_rows.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 5
    matched = 0
    for h, v, g, reading in rows:
        h, v, g = float(h), float(v), float(g)
        assert abs(h * h + v * v - 1.0) < 1e-5                 # a unit beam direction
        if reading == "none":
            for kind in lad.KINDS:
                assert min(abs(lad.ross_G(kind, v) - g), abs(lad.ross_G(kind, h) - g)) > 1e-4
            continue
        lab, kind = reading.split(":")
        mu = v if lab == "nat" else h
        assert abs(lad.ross_G(kind, mu) - g) < 5e-6
        matched += 1
    assert matched == 3


def _lad_slab(table):
    dens = np.full((4, 40, 40), 1.3, np.float32)
    scene = _grid_scene(dens, origin=(-10.0, -10.0, 0.0), cell=0.5, ground_z=-2.0)
    scene.grids[0].lad = None if table is None else np.asarray(table, np.float32)
    return scene


def test_lad_table_sets_sigma_from_the_vertical_component():
    """sigma = G(|d_z|) density: a table linear in mu (exact in FP32, so its
    interpolation is that line) gives exp(-(a + b cos phi) d L) through the
    slab; a constant table reproduces the constant G exactly, in both modes."""
    sc = scenes.Scanner()
    lin = [0.25, 0.375, 0.5, 0.625, 0.75]                      # 0.25 + 0.5 mu
    osc = oracle.OracleScene(_lad_slab(lin))
    bare = oracle.OracleScene(_grid_scene(np.zeros((4, 40, 40), np.float32), origin=(-10.0, -10.0, 0.0),
                                          cell=0.5, ground_z=-2.0))
    for phi in np.radians([0.0, 17.0, 41.0, 63.0]):
        d = np.array([0.0, math.sin(phi), -math.cos(phi)])
        o = np.array([0.0, -12.0 * math.tan(phi), 10.0])
        R, P, ids, _ = oracle.trace_returns(osc, sc, o, d, mode=1)
        R0, P0, _, _ = oracle.trace_returns(bare, sc, o, d, mode=1)
        L = 2.0 / math.cos(phi)
        Gmu = 0.25 + 0.5 * math.cos(phi)
        assert abs(P[-1] / P0[0] - math.exp(-Gmu * _f32(1.3) * L)) < 1e-12
    const = oracle.OracleScene(_lad_slab([0.5] * 7))
    plain = oracle.OracleScene(_lad_slab(None))
    sc2, leg = _nadir_leg(n=40, el_lo=-1.2, el_hi=-0.3)
    sc2 = scenes.replace(sc2, beam_sample_quality=2)
    leg = scenes.replace(leg, start=(0.0, 0.0, 10.0))
    for mode in (0, 1):
        a = oracle.scan(const, sc2, leg, mode=mode, seed=3)
        b = oracle.scan(plain, sc2, leg, mode=mode, seed=3)
        assert np.array_equal(a["waveform"], b["waveform"])
        assert np.array_equal(a["subray_hit"], b["subray_hit"])


def test_lad_table_stochastic_transmission_frequency():
    """Eq. intersection_dist with G from the table: the fraction of subrays
    crossing the slab at tilt phi is exp(-G(cos phi) d L) (binomial bound)."""
    sc = scenes.Scanner()
    lin = [0.25, 0.375, 0.5, 0.625, 0.75]
    osc = oracle.OracleScene(_lad_slab(lin))
    dens = 0.4
    osc.set_density(np.full((4, 40, 40), dens, np.float32))
    phi = math.radians(35.0)
    d = np.array([0.0, math.sin(phi), -math.cos(phi)])
    o = np.array([0.0, -12.0 * math.tan(phi), 10.0])
    n = 4000
    through = 0
    for k in range(n):
        R, P, ids, _ = oracle.trace_returns(osc, sc, o, d, mode=0, seed=5, pulse=k)
        through += int(ids[0] < osc.n_tri)
    p = math.exp(-(0.25 + 0.5 * math.cos(phi)) * _f32(dens) * 2.0 / math.cos(phi))
    assert abs(through / n - p) < 4.5 * math.sqrt(p * (1 - p) / n)


def test_lad_adjoint_matches_central_differences():
    """dL/ddensity = G(|d_z|) dL/dsigma with an erectophile table."""
    w = scenes.uls_voxels(seed=4, n=24, n_pulses=4000, n_bins=256, agl=8.0, speed=1.0, prf=2000.0)
    w.scanners[0].beam_sample_quality = 1
    scene = w.scenes[0]
    scene.grids[0].lad = lad.table("erectophile", 17).astype(np.float32)
    sc, leg = w.scanners[0], w.legs[0]
    pulses = np.arange(0, 4000, 250, dtype=np.int64)
    osc = oracle.OracleScene(scene)
    base = scene.grids[0].density.copy()
    osc.set_density(scenes.perturbed_density(base, seed=1))
    W_ref = oracle.scan(osc, sc, leg, pulses, mode=1)["waveform"]
    osc.set_density(base)
    fwd = oracle.scan(osc, sc, leg, pulses, mode=1)
    win = fwd["window_bin"]
    g = 2.0 * (fwd["waveform"] - W_ref)
    _, d_dens = oracle.adjoint(osc, sc, leg, pulses, g, win)

    def loss(dens):
        osc.set_density(dens)
        W = oracle.scan(osc, sc, leg, pulses, mode=1, fixed_window=win)["waveform"]
        return float(((W - W_ref) ** 2).sum())

    touched = np.nonzero(d_dens)[0]
    assert len(touched) > 20
    rng = np.random.default_rng(3)
    for v in rng.choice(touched, 8, replace=False):
        x = float(base.ravel()[v])
        h = 1e-4 * max(abs(x), 1e-2)
        dp = base.copy().ravel(); dp[v] = np.float32(x + h)
        dm = base.copy().ravel(); dm[v] = np.float32(x - h)
        hh = (float(dp[v]) - float(dm[v])) / 2
        fd = (loss(dp.reshape(base.shape)) - loss(dm.reshape(base.shape))) / (2 * hh)
        assert abs(fd - d_dens[v]) <= 1e-5 * abs(d_dens[v]) + 1e-9 * np.abs(d_dens).max()
    osc.set_density(base)


# --------------------------------------------------------------------------
# several voxel grids in one scene (boxes with disjoint interiors)
# --------------------------------------------------------------------------

def _split_grid_scene(dens, origin, cell, splits, ground_z=-30.0, order=None):
    """The grid of `dens` cut into pieces along x at the voxel indices `splits`."""
    nz, ny, nx = dens.shape
    cuts = [0] + list(splits) + [nx]
    grids = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        grids.append(scenes.VoxelGrid(origin=(origin[0] + a * cell, origin[1], origin[2]), cell=cell,
                                      dims=(b - a, ny, nz),
                                      density=np.ascontiguousarray(dens[:, :, a:b], np.float32), G=0.5,
                                      leaf_reflectance=0.5))
    if order is not None:
        grids = [grids[i] for i in order]
    scene = _grid_scene(np.zeros((1, 1, 1), np.float32), origin=(-900.0, -900.0, -900.0), cell=0.5,
                        ground_z=ground_z)
    return scenes.Scene(meshes=scene.meshes, grids=grids)


def _voxel_rows(scene, sc, leg, mode=1):
    osc = oracle.OracleScene(scene)
    return osc, oracle.scan(osc, sc, leg, mode=mode, seed=2)


def test_grids_split_into_pieces_give_the_same_waveform():
    """Cutting one grid into adjacent grids (in any listed order) changes
    voxel ids only: the expected waveform is the same (the crossing planes are
    the same numbers), and the adjoint's density gradient is the same once the
    pieces are put back together."""
    rng = np.random.default_rng(11)
    dens = np.where(rng.random((6, 8, 12)) < 0.5, rng.uniform(0.2, 1.5, (6, 8, 12)), 0.0).astype(np.float32)
    origin, cell = (-3.0, -2.0, -3.0), 0.5
    sc = scenes.Scanner(deflector=scenes.DEFL_TLS_GRID, grid_n_az=24, grid_n_el=10, el_min_rad=-1.45,
                        el_max_rad=-0.6, n_bins=400, beam_sample_quality=2)
    leg = scenes.Leg(platform=scenes.PLATFORM_STATIC, start=(0.1, 0.2, 4.0), n_pulses=240)
    one = _split_grid_scene(dens, origin, cell, [])
    o1, r1 = _voxel_rows(one, sc, leg)
    assert (_voxel_rows(one, sc, leg, mode=0)[1]["subray_hit"] >= o1.n_tri).mean() > 0.2
    for splits, order in (([5], None), ([3, 7, 10], [2, 0, 3, 1])):
        many = _split_grid_scene(dens, origin, cell, splits, order=order)
        om, rm = _voxel_rows(many, sc, leg)
        assert np.array_equal(rm["window_bin"], r1["window_bin"])
        scale = np.abs(r1["waveform"]).max()
        assert np.abs(rm["waveform"] - r1["waveform"]).max() <= 1e-12 * scale
        # the adjoint, gathered back into the one grid's layout
        pulses = np.arange(leg.n_pulses)
        g = np.sin(np.arange(r1["waveform"].size).reshape(r1["waveform"].shape))
        _, d1 = oracle.adjoint(o1, sc, leg, pulses, g, r1["window_bin"])
        _, dm = oracle.adjoint(om, sc, leg, pulses, g, rm["window_bin"])
        back = np.zeros(dens.shape)
        cuts = [0] + splits + [dens.shape[2]]
        pieces = list(zip(cuts[:-1], cuts[1:]))
        if order is not None:
            pieces = [pieces[i] for i in order]
        for i, (a, b) in enumerate(pieces):
            back[:, :, a:b] = dm[om.vox_offsets[i]:om.vox_offsets[i + 1]].reshape(dens.shape[0], dens.shape[1], b - a)
        d1 = d1.reshape(dens.shape)
        assert np.abs(back - d1).max() <= 1e-12 * np.abs(d1).max()


def test_grids_along_one_ray_multiply_transmittance_and_keep_their_own_G():
    """Two separate grids on a vertical ray: exp(-G1 d1 L1) exp(-G2 d2 L2) reaches
    the ground, with G2 from the second grid's leaf-angle table (linear in mu);
    listing the grids in either order changes nothing."""
    sc = scenes.Scanner()
    top = scenes.VoxelGrid(origin=(-1.0, -1.0, 2.0), cell=0.5, dims=(4, 4, 2),
                           density=np.full((2, 4, 4), 0.8, np.float32), G=0.5)
    low = scenes.VoxelGrid(origin=(-1.0, -1.0, -1.0), cell=0.5, dims=(4, 4, 4),
                           density=np.full((4, 4, 4), 0.3, np.float32), G=0.9,
                           lad=np.array([0.25, 0.375, 0.5, 0.625, 0.75], np.float32))
    ground = _grid_scene(np.zeros((1, 1, 1), np.float32), origin=(-900.0, -900.0, -900.0), cell=0.5,
                         ground_z=-3.0).meshes
    bare = oracle.OracleScene(scenes.Scene(meshes=ground, grids=[]))
    for phi in (0.0, 0.2):
        d = np.array([0.0, math.sin(phi), -math.cos(phi)])
        o = np.array([0.0, -6.0 * math.tan(phi), 6.0])
        ref = None
        for grids in ([top, low], [low, top]):
            osc = oracle.OracleScene(scenes.Scene(meshes=ground, grids=grids))
            R, P, ids, _ = oracle.trace_returns(osc, sc, o, d, mode=1)
            R0, P0, _, _ = oracle.trace_returns(bare, sc, o, d, mode=1)
            T = P[-1] / P0[0]
            want = (math.exp(-0.5 * _f32(0.8) * 1.0 / math.cos(phi)) *
                    math.exp(-(0.25 + 0.5 * math.cos(phi)) * _f32(0.3) * 2.0 / math.cos(phi)))
            assert abs(T - want) < 1e-12
            assert np.all(np.diff(R[:-1]) > 0)              # returns in range order across grids
            if ref is None:
                ref = (R, P)
            else:
                assert np.allclose(R, ref[0], rtol=0, atol=1e-12)
                assert np.allclose(P, ref[1], rtol=1e-13, atol=0)


def test_opaque_grid_behind_a_transmissive_one():
    """A transmissive grid above an opaque one: subrays that cross the first
    stop at the opaque grid's top face; the ids tell the grids apart."""
    sc = scenes.Scanner()
    top = scenes.VoxelGrid(origin=(-1.0, -1.0, 2.0), cell=0.5, dims=(4, 4, 2),
                           density=np.full((2, 4, 4), 0.6, np.float32), G=0.5)
    low = scenes.VoxelGrid(origin=(-1.0, -1.0, -1.0), cell=0.5, dims=(4, 4, 4),
                           density=np.full((4, 4, 4), 1.0, np.float32), G=0.5, opaque=1)
    ground = _grid_scene(np.zeros((1, 1, 1), np.float32), origin=(-900.0, -900.0, -900.0), cell=0.5,
                         ground_z=-3.0).meshes
    osc = oracle.OracleScene(scenes.Scene(meshes=ground, grids=[top, low]))
    n_top = 2 * 4 * 4
    d = np.array([0.0, 0.0, -1.0])
    o = np.array([0.1, 0.1, 6.0])
    stops, through = 0, 0
    for k in range(400):
        R, P, ids, _ = oracle.trace_returns(osc, sc, o, d, mode=0, seed=9, pulse=k)
        assert len(ids) == 1
        vid = ids[0] - osc.n_tri
        if vid < n_top:
            stops += 1
            assert 3.0 <= R[0] <= 4.0                       # inside the top grid (z in [2, 3])
        else:
            through += 1
            assert abs(R[0] - 5.0) < 1e-9                   # the opaque grid's top face at z = 1
    p = math.exp(-0.5 * _f32(0.6) * 1.0)
    assert abs(through / 400 - p) < 4.5 * math.sqrt(p * (1 - p) / 400)


def test_march_over_several_grids_matches_per_voxel_brute_force():
    """The march over three grids (two touching along x, one apart, different
    cells) lists exactly the voxels a per-voxel slab test finds, in range
    order, with ids running over the grids' voxels in their listed order."""
    rng = np.random.default_rng(5)
    specs = [((-1.0, -1.0, -1.0), 0.5, (3, 4, 2)),      # x in [-1, 0.5)
             ((0.5, -1.0, -1.0), 0.5, (2, 4, 2)),       # touches the first at x = 0.5
             ((-0.5, 1.5, -2.0), 0.25, (4, 3, 5))]      # apart
    grids = [scenes.VoxelGrid(origin=o, cell=c, dims=dm, density=np.ones(dm[::-1], np.float32))
             for o, c, dm in specs]
    osc = oracle.OracleScene(scenes.Scene(meshes=[], grids=grids))
    offs = np.cumsum([0] + [int(np.prod(dm)) for _, _, dm in specs])
    for _ in range(300):
        o = rng.uniform(-4, 4, 3)
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        vid, ti, to = osc.march(o, d)
        ref = []
        for gi, (org, c, (nx, ny, nz)) in enumerate(specs):
            for z in range(nz):
                for y in range(ny):
                    for x in range(nx):
                        a = np.array(org) + c * np.array([x, y, z])
                        b = a + c
                        with np.errstate(divide="ignore", invalid="ignore"):
                            t1 = (a - o) / d
                            t2 = (b - o) / d
                        tin = max(0.0, np.max(np.minimum(t1, t2)))
                        tout = np.min(np.maximum(t1, t2))
                        if tout - tin > 1e-9:
                            ref.append((tin, int(offs[gi] + (z * ny + y) * nx + x), tout))
        ref.sort()
        got = [(a, int(v), b) for a, v, b in zip(ti, vid, to) if b - a > 1e-9]
        assert [r[1] for r in ref] == [g[1] for g in got]
        for r, g in zip(ref, got):
            assert abs(r[0] - g[0]) < 1e-12 and abs(r[2] - g[2]) < 1e-12


def test_two_grids_stochastic_stop_frequencies():
    """Eq. intersection_dist along one ray through two separate grids (listed
    in the opposite order): it stops in the first with 1 - e^-t1, in the
    second with e^-t1 (1 - e^-t2), reaches the ground with e^-(t1 + t2)."""
    sc = scenes.Scanner()
    top = scenes.VoxelGrid(origin=(-1.0, -1.0, 2.0), cell=0.5, dims=(4, 4, 2),
                           density=np.full((2, 4, 4), 0.9, np.float32), G=0.5)
    low = scenes.VoxelGrid(origin=(-1.0, -1.0, -1.0), cell=0.5, dims=(4, 4, 4),
                           density=np.full((4, 4, 4), 0.4, np.float32), G=0.7)
    ground = _grid_scene(np.zeros((1, 1, 1), np.float32), origin=(-900.0, -900.0, -900.0), cell=0.5,
                         ground_z=-3.0).meshes
    osc = oracle.OracleScene(scenes.Scene(meshes=ground, grids=[low, top]))
    n_low = 4 * 4 * 4
    n = 8000
    counts = np.zeros(3)
    for k in range(n):
        R, P, ids, _ = oracle.trace_returns(osc, sc, [0.1, 0.1, 6.0], [0.0, 0.0, -1.0], mode=0, seed=21,
                                            pulse=k)
        vid = ids[0] - osc.n_tri
        counts[0 if vid >= n_low else (1 if vid >= 0 else 2)] += 1   # top grid, low grid, ground
    t1, t2 = 0.5 * _f32(0.9) * 1.0, 0.7 * _f32(0.4) * 2.0
    p = np.array([1 - math.exp(-t1), math.exp(-t1) * (1 - math.exp(-t2)), math.exp(-t1 - t2)])
    sd = np.sqrt(n * p * (1 - p))
    assert np.all(np.abs(counts - n * p) < 5 * sd), (counts, n * p)


def test_rotating_head_turns_at_the_head_rate_with_the_polygon_in_elevation():
    """Rotating head (the MLS/TLS head): with a flat elevation the pulse
    directions stay in the spin plane, consecutive pulses turn by
    head_rate/PRF about the spin axis and a full turn comes back; with a
    polygon mirror the elevation sweeps [-max, max] once per mirror line."""
    prf, rate = 1000.0, 2 * math.pi * 5.0          # 5 rev/s: 200 pulses per turn
    sc = scenes.Scanner(prf_hz=prf, deflector=scenes.DEFL_ROTATING_HEAD, head_rate_rad_s=rate,
                        scan_freq_hz=1.0, scan_angle_max_rad=0.0)
    leg = scenes.Leg(platform=scenes.PLATFORM_STATIC, n_pulses=400)
    ds = np.array([oracle.pulse_ray(sc, leg, k)[1] for k in range(401)])
    assert np.allclose(np.linalg.norm(ds, axis=1), 1.0, atol=1e-14)
    axis = np.cross(ds[0], ds[1])
    axis /= np.linalg.norm(axis)
    assert np.abs(ds @ axis).max() < 1e-12                         # one plane
    step = np.arccos(np.clip(np.sum(ds[1:] * ds[:-1], axis=1), -1, 1))
    assert np.allclose(step, rate / prf, atol=1e-9)
    assert np.allclose(ds[200], ds[0], atol=1e-12) and np.allclose(ds[400], ds[0], atol=1e-12)
    # polygon mirror in elevation: angle to the spin plane in [-max, max], sweeping it per line
    amax = math.radians(20.0)
    sc2 = scenes.replace(sc, scan_freq_hz=50.0, scan_angle_max_rad=amax)
    ds2 = np.array([oracle.pulse_ray(sc2, leg, k)[1] for k in range(400)])
    el = np.arcsin(np.clip(ds2 @ axis, -1, 1))
    assert np.abs(el).max() <= amax + 1e-12
    # a linear sweep sampled 20 times per line: constant steps of 2 max/20 inside a
    # line, then a jump back; the samples reach -max and max - 2 max/20
    d_el = np.diff(el)
    inside = d_el > 0
    assert np.allclose(d_el[inside], 2 * amax / 20, atol=1e-9)
    assert np.sum(~inside) == 400 // 20 - 1
    assert abs(el.min() + amax) < 1e-9 and abs(el.max() - (amax - 2 * amax / 20)) < 1e-9
    # azimuth in the spin plane still advances at the head rate
    flat = ds2 - np.outer(ds2 @ axis, axis)
    flat /= np.linalg.norm(flat, axis=1, keepdims=True)
    stepf = np.arccos(np.clip(np.sum(flat[1:] * flat[:-1], axis=1), -1, 1))
    assert np.allclose(stepf, rate / prf, atol=1e-9)


# --------------------------------------------------------------------------
# echo detection (Sec. 3.4: local maxima of the waveform above a threshold,
# the threshold 5% of the pulse's largest bin; first K echoes by bin; the
# echo's object is the return contributing most at the echo bin)
# --------------------------------------------------------------------------

def _two_peaks(a1, b1, a2, b2, nb=200, sig=6.79):
    b = np.arange(nb, dtype=np.float64)
    return a1 * np.exp(-(b - b1) ** 2 / (2 * sig * sig)) + a2 * np.exp(-(b - b2) ** 2 / (2 * sig * sig))


def test_echo_threshold_is_five_percent_of_the_waveform_maximum():
    """A second peak at 4.9% of the largest bin is not an echo, at 5.1% it is;
    exactly 5% counts (at or above).  Fails a threshold taken against the sum of
    the bins (about 17x the peak here), the first bin, the first echo, or 50%."""
    for a2, n in ((0.049, 1), (0.051, 2), (0.05, 2)):
        bins, ov, _ = oracle.echo_peaks(_two_peaks(1.0, 40, a2, 120))
        assert list(bins) == [40, 120][:n] and not ov, (a2, bins)
    # the weak peak first: the threshold is still the maximum's, not the first peak's
    for a1, n in ((0.049, 1), (0.051, 2)):
        bins, _, _ = oracle.echo_peaks(_two_peaks(a1, 40, 1.0, 120))
        assert list(bins) == ([120] if n == 1 else [40, 120]), (a1, bins)
    # a lower or higher threshold fraction moves the cut
    bins, _, _ = oracle.echo_peaks(_two_peaks(1.0, 40, 0.3, 120), thr_rel=0.5)
    assert list(bins) == [40]
    bins, _, _ = oracle.echo_peaks(_two_peaks(1.0, 40, 0.3, 120), thr_rel=0.29)
    assert list(bins) == [40, 120]


def test_echo_plateau_and_window_edges():
    """A plateau of equal bins gives one echo, on its leftmost bin (strictly
    above the left neighbour, not below the right one); outside the window the
    waveform counts as zero, so a falling first bin or a rising last bin is an
    echo."""
    W = np.zeros(20)
    W[5:11] = [0.2, 0.7, 0.7, 0.7, 0.2, 0.0]
    bins, _, near = oracle.echo_peaks(W)
    assert list(bins) == [6] and near
    W = np.zeros(20)
    W[:3] = [1.0, 0.5, 0.1]
    W[17:] = [0.1, 0.5, 0.9]
    assert list(oracle.echo_peaks(W)[0]) == [0, 19]
    W = np.zeros(20)
    W[17:] = [0.1, 0.9, 0.9]
    assert list(oracle.echo_peaks(W)[0]) == [18]
    # a constant waveform has one echo, at bin 0; an all-zero one has none
    assert list(oracle.echo_peaks(np.full(20, 0.3))[0]) == [0]
    assert len(oracle.echo_peaks(np.zeros(20))[0]) == 0


def test_echo_list_keeps_the_first_k_by_bin_and_flags_overflow():
    """Nine separated peaks with K = 8: the first eight by bin are kept even when
    the ninth is the largest, and the overflow is reported; eight peaks fit."""
    b = np.arange(200, dtype=np.float64)
    amps = [0.3, 0.5, 0.4, 0.6, 0.35, 0.45, 0.55, 0.25, 1.0]
    centres = [10 + 20 * i for i in range(9)]
    W = sum(a * np.exp(-(b - c) ** 2 / (2 * 3.0 ** 2)) for a, c in zip(amps, centres))
    bins, ov, _ = oracle.echo_peaks(W, K=8)
    assert list(bins) == centres[:8] and ov
    bins, ov, _ = oracle.echo_peaks(W, K=9)
    assert list(bins) == centres and not ov
    W8 = sum(a * np.exp(-(b - c) ** 2 / (2 * 3.0 ** 2)) for a, c in zip(amps[:8], centres[:8]))
    bins, ov, _ = oracle.echo_peaks(W8, K=8)
    assert list(bins) == centres[:8] and not ov


def test_echo_object_is_the_largest_contribution_first_on_ties():
    """The object of an echo at time tb is the return with the largest
    P p(tb - 2R/c), not the largest P, the nearest or the last; on exactly
    equal contributions the first in summation order."""
    sc = scenes.Scanner()
    sig = 4.0 / (2 * math.sqrt(2 * math.log(2)))
    R0 = 30.0
    tb = 2 * R0 / C_LIGHT * 1e9
    R_far = R0 + 2 * sig * 1e-9 * C_LIGHT / 2      # two sigma later: p = e^-2
    # a weaker return on the echo's time beats a stronger one two sigma away
    bid, near = oracle.echo_object(sc, [1.0, 1.5], [R0, R_far], [11, 22], tb)
    assert bid == 11 and not near
    bid, _ = oracle.echo_object(sc, [1.0, 1.5], [R_far, R0], [11, 22], tb)
    assert bid == 22
    # equal contributions: the first wins (and the near-tie is reported)
    bid, near = oracle.echo_object(sc, [1.0, 2.0, 2.0], [R0, R0, R0], [5, 7, 9], tb)
    assert bid == 7 and near
    bid, near = oracle.echo_object(sc, [2.0, 2.0, 1.0], [R0, R0, R0], [9, 7, 5], tb)
    assert bid == 9 and near


def _column_scene(dens_top_down, z_top, plate_z=None, plate_refl=0.5, G=0.5):
    """A 1 x 1 m voxel column under a nadir ray from the origin: voxel j (0 =
    nearest) spans depths [-z_top + j, -z_top + j + 1), densities given from the
    top down; optionally a plate at z = plate_z, whose diagonal misses the ray."""
    d = np.asarray(dens_top_down, np.float32)[::-1].reshape(-1, 1, 1)   # [z][y][x], z up
    nz = d.shape[0]
    grid = scenes.VoxelGrid(origin=(-0.5, -0.5, -z_top - nz), cell=1.0, dims=(1, 1, nz),
                            density=np.ascontiguousarray(d), G=G, leaf_reflectance=0.5)
    meshes = []
    if plate_z is not None:
        # the ray at x = y = 0 lies inside face 0 = (v0, v1, v2), 0.9 m from the diagonal
        pv = np.array([[-50, -40, plate_z], [60, -40, plate_z], [60, 50, plate_z],
                       [-50, 50, plate_z]], np.float32)
        meshes.append(scenes.Mesh(pv, np.array([[0, 1, 2], [0, 2, 3]], np.int32),
                                  np.full(2, plate_refl, np.float32)))
    return scenes.Scene(meshes=meshes, grids=[grid])


def _nadir_expected(scene, n_bins):
    sc, leg = _nadir_leg()
    sc.n_bins = n_bins
    osc = oracle.OracleScene(scene)
    return sc, oracle.scan(osc, sc, leg, mode=1, seed=1), osc


def test_scene_threshold_voxel_layer_and_plate():
    """Expected mode, one subray (I_s = I0): a voxel layer (depth 20-21 m,
    return T(1 - e^{-sigma l}) at its midpoint) and a plate 30 m down (return
    rho T).  With the radar equation's 1/R^2 the plate's peak is set to 4.9% or
    5.1% of the layer's, and then the layer's to 4.9% or 5.1% of the plate's."""
    C0 = 1.0 * 0.1 ** 2 * 0.9 * 1.0 / 4.0          # I0 Dr^2 eta_sys eta_atm / 4
    Rv, Rp = 20.5, 30.0
    for ratio, n in ((0.049, 1), (0.051, 2)):
        # strong layer (T = 1/2), weak plate
        dens = np.float32(2.0 * math.log(2.0))
        T = math.exp(-0.5 * float(dens))
        Pv = C0 * 0.5 * (1 - T) / Rv ** 2
        rho = ratio * Pv * Rp ** 2 / (C0 * T)
        sc, r, osc = _nadir_expected(_column_scene([dens], 20.0, plate_z=-30.0, plate_refl=rho), 400)
        assert r["echo_count"][0] == n, (ratio, r["echo_count"][0])
        assert r["echo_object"][0, 0] == osc.n_tri + 0          # the layer's voxel
        if n == 2:
            assert r["echo_object"][0, 1] == 0                  # the plate's face 0
        # weak layer, strong plate (rho = 0.5): solve (1-T)/T for the ratio
        x = ratio * 0.5 * Rv ** 2 / (0.5 * Rp ** 2)
        dens = np.float32(-2.0 * math.log(1.0 / (1.0 + x)))
        sc, r, osc = _nadir_expected(_column_scene([dens], 20.0, plate_z=-30.0, plate_refl=0.5), 400)
        assert r["echo_count"][0] == n, (ratio, r["echo_count"][0])
        assert r["echo_object"][0, n - 1] == 0
        dt = sc.bin_ns
        tb = (r["window_bin"][0] + r["echo_bin"][0, n - 1]) * dt
        assert abs(tb - 2 * Rp / C_LIGHT * 1e9) <= 0.5 * dt + 1e-9


def test_scene_nine_layers_keep_the_nearest_eight():
    """Nine voxel layers 4 m apart, every one an echo; the nearest is the
    weakest and the farthest among the strongest.  K = 8 keeps the eight
    nearest (by bin, not by strength) and flags the overflow."""
    dens = np.zeros(33, np.float32)
    dens[0::4] = [0.01, 0.2, 0.2, 0.2, 0.2, 0.2, 0.2, 0.2, 3.0]
    C0 = 1.0 * 0.1 ** 2 * 0.9 / 4.0
    T, P, R = 1.0, [], []
    for j in range(33):
        a = math.exp(-0.5 * float(dens[j]))
        if dens[j] > 0:
            R.append(20.0 + j + 0.5)
            P.append(C0 * 0.5 * T * (1 - a) / R[-1] ** 2)
        T *= a
    P = np.array(P)
    assert P.min() >= 0.06 * P.max() and np.argmin(P) == 0      # all echoes; the first weakest
    sc, r, osc = _nadir_expected(_column_scene(dens, 20.0), 1024)
    assert r["echo_count"][0] == 8 and (r["flags"][0] & oracle.F_OVERFLOW)
    dt = sc.bin_ns
    for e in range(8):
        tb = (r["window_bin"][0] + r["echo_bin"][0, e]) * dt
        assert abs(tb - 2 * R[e] / C_LIGHT * 1e9) <= 0.5 * dt + 1e-9
        assert r["echo_object"][0, e] == osc.n_tri + (32 - 4 * e)   # voxel z index from the bottom
    # eight layers: no overflow
    dens8 = dens.copy()
    dens8[32] = 0.0
    sc, r, _ = _nadir_expected(_column_scene(dens8, 20.0), 1024)
    assert r["echo_count"][0] == 8 and not (r["flags"][0] & oracle.F_OVERFLOW)


def test_scene_echo_object_stronger_of_two_merged_returns():
    """A voxel layer (20-20.9 m, clipped by a plate at 20.9 m) and the plate
    form one echo.  With a bright plate behind a thin layer the object is the
    plate (not the nearest, not the first return); with a dense layer in front
    of a dark plate it is the voxel (not the last return)."""
    for dens, refl, want_voxel in ((0.2, 0.9, False), (6.0, 0.1, True)):
        sc, r, osc = _nadir_expected(
            _column_scene([np.float32(dens)], 20.0, plate_z=-20.9, plate_refl=refl), 200)
        assert r["echo_count"][0] == 1
        assert r["echo_object"][0, 0] == (osc.n_tri + 0 if want_voxel else 0)


# --------------------------------------------------------------------------
# re-running a pulse with given subray events (parity support): forcing the
# oracle's own choices changes nothing; a choice an FP32 path may make on a
# flagged subray is accepted; a choice no flagged decision allows is marked
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["tls0", "tls1", "als0"])
def test_forcing_the_oracles_own_events_reproduces_the_scan(kind):
    mode = int(kind[-1])
    if kind.startswith("tls"):
        w = scenes.tls_tiny(n_az=40, n_el=40)
    else:
        w = scenes.als_terrain(seed=5, size=96, n_trees=6, n_pulses=3000, n_bins=256, agl=80.0)
    osc = oracle.OracleScene(w.scenes[0])
    r = oracle.scan(osc, w.scanners[0], w.legs[0], mode=mode, seed=3)
    flagged = (r["subray_flags"] & oracle.F_SUBRAY) != 0
    assert flagged.any()
    # every pulse's subray flags together are the pulse's subray flags
    assert np.array_equal(np.bitwise_or.reduce(r["subray_flags"], axis=1) & oracle.F_SUBRAY,
                          r["flags"] & oracle.F_SUBRAY)
    rows = np.nonzero(flagged.any(axis=1))[0]
    fh = np.where(flagged[rows], r["subray_hit"][rows], oracle.FREE_HIT).astype(np.int64)
    r2 = r["rerun"](rows, force_hit=fh)
    assert not (r2["flags"] & oracle.F_FORCED_BAD).any()
    for k in ("window_bin", "echo_count", "echo_bin", "echo_object", "subray_hit"):
        assert np.array_equal(r2[k], r[k][rows]), k
    for k in ("waveform", "echo_range", "subray_range"):
        assert np.allclose(r2[k], r[k][rows], rtol=1e-12, atol=0), k


def test_forced_events_at_an_edge_and_implausible_ones():
    """A ray through the shared diagonal may be given either triangle; a ray
    clearly inside one triangle may not be given the other, nor a miss."""
    osc = oracle.OracleScene(scenes.flat_target(10.0, 0.0, half=5.0))
    sc, leg = _nadir_leg()
    sc.n_bins = 200
    # the plate's diagonal runs through (0, 0): the nadir ray is on the edge
    r = oracle.scan(osc, sc, leg, mode=0, seed=1)
    assert r["subray_flags"][0, 0] & oracle.F_EDGE
    mine = r["subray_hit"][0, 0]
    other = 1 - mine
    r2 = r["rerun"]([0], force_hit=np.array([[other]], np.int64))
    assert not (r2["flags"][0] & oracle.F_FORCED_BAD)
    assert r2["subray_hit"][0, 0] == other
    assert abs(r2["subray_range"][0, 0] - r["subray_range"][0, 0]) < 1e-9
    assert np.allclose(r2["waveform"], r["waveform"], rtol=1e-9)
    # off the diagonal the other triangle, a miss or a voxel are not allowed
    leg2 = scenes.replace(leg, start=(0.5, -0.5, 0.0))
    r = oracle.scan(osc, sc, leg2, mode=0, seed=1)
    assert r["subray_flags"][0, 0] == 0
    for bad in (1 - r["subray_hit"][0, 0], -1, osc.n_tri + 3):
        r3 = r["rerun"]([0], force_hit=np.array([[bad]], np.int64))
        assert r3["flags"][0] & oracle.F_FORCED_BAD, bad


def test_forced_voxel_stop_and_pass():
    """Stochastic mode: a voxel the subray clearly passes may not be given as its
    stop, and a voxel it clearly stops in may not be passed (a triangle behind)."""
    dens = np.full((8, 4, 4), 0.8, np.float32)
    scene = _grid_scene(dens, origin=(-1.0, -1.0, -4.0), cell=0.5, ground_z=-10.0)
    osc = oracle.OracleScene(scene)
    sc, leg = _nadir_leg(64, -math.radians(89.5), -math.radians(88.5))
    leg = scenes.replace(leg, start=(-0.3, 0.2, 0.0))
    r = oracle.scan(osc, sc, leg, mode=0, seed=4)
    ids = r["subray_hit"][:, 0]
    stop = ids >= osc.n_tri
    assert stop.any() and (~stop).any()
    clean = (r["subray_flags"][:, 0] == 0)
    # a pulse that stopped in a voxel, forced to the ground instead
    i = np.nonzero(stop & clean)[0][0]
    r3 = r["rerun"]([i], force_hit=np.array([[0]], np.int64))
    r4 = r["rerun"]([i], force_hit=np.array([[1]], np.int64))
    assert (r3["flags"][0] | r4["flags"][0]) & oracle.F_FORCED_BAD
    # a pulse that reached the ground, forced to stop in the first voxel it crossed
    j = np.nonzero(~stop & clean)[0][0]
    o, d = oracle.pulse_ray(sc, leg, j, seed=4)
    vid, _, _ = osc.march(o, d)
    r5 = r["rerun"]([j], force_hit=np.array([[osc.n_tri + vid[0]]], np.int64))
    assert r5["flags"][0] & oracle.F_FORCED_BAD
