"""Seeded synthetic workloads shared by the FP64 oracle and the CUDA path.

This module only *generates input data*: triangle meshes, voxel densities,
instrument parameters and scan legs.  It holds none of the beam-scene
interaction arithmetic (pulse generation, subrays, intersection, radar
equation, waveform, echoes, adjoint); that lives twice, independently, in
``oracle/`` and in the CUDA library.  Both sides import this module and
nothing else in common.

Every array is produced by ``numpy.random.default_rng(seed)`` so that a
workload is fully determined by its seed and size arguments.

Workloads (the paper's surveys need data that is not available offline, so
seeded stand-ins with the same structure are used):

* ``tls_tiny``     - static tripod over a ground plane with 8 boxes (TLS, Sec. 3.2).
* ``als_terrain``  - fBm heightmap triangulated like a GeoTIFF DTM (Sec. 3.5.2)
                     plus procedural trees, flown with an oscillating mirror.
* ``uls_voxels``   - transmissive voxel canopy (Sec. 3.5.4) over a 2-triangle
                     ground, flown with a rotating polygon mirror.
* ``batched_legs`` - many legs of uneven length and subray quality over a pool
                     of terrain tiles and voxel blocks.
* ``urban_mls``    - a street with extruded building footprints scanned by a
                     rotating profile head on a vehicle (mobile laser scanning).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
import math
import numpy as np

# Deflector codes (Sec. 3.3 patterns + the two static/rotating-head TLS laws).
DEFL_POLYGON = 0       # rotating polygon mirror: sawtooth across-track angle
DEFL_OSCILLATING = 1   # swinging mirror: sinusoidal across-track angle
DEFL_TLS_GRID = 2      # static tripod: azimuth x elevation grid
DEFL_ROTATING_HEAD = 3 # 360 deg head rotation with a polygon mirror in elevation
DEFL_FIBRE = 4         # fibre-optic line scanner: fixed fibre angles across track, in turn
DEFL_PALMER = 5        # slanted rotating mirror: conical pattern at a fixed off-nadir angle

PLATFORM_STATIC = 0
PLATFORM_LINEAR = 1

PULSE_GAUSSIAN = 0
PULSE_CARLSSON = 1


@dataclass
class Scanner:
    """Instrument parameters (scanner + deflector + beam + waveform settings)."""
    prf_hz: float = 100_000.0
    divergence_rad: float = 0.3e-3        # full angle at the 1/e^2 points
    beam_sample_quality: int = 2          # number of subray rings q
    wavelength_m: float = 1064e-9
    beam_waist_m: float = 0.0             # 0: derive from divergence
    focus_m: float = 0.0
    peak_power_w: float = 1.0
    receiver_diam_m: float = 0.1
    eta_sys: float = 0.9
    eta_atm: float = 1.0
    pulse_shape: int = PULSE_GAUSSIAN
    pulse_fwhm_ns: float = 4.0
    pulse_length_ns: float = 4.0
    bin_ns: float = 0.25
    n_bins: int = 100
    max_echoes: int = 8
    echo_threshold_rel: float = 0.05
    range_noise_sigma_m: float = 0.01
    deflector: int = DEFL_OSCILLATING
    scan_freq_hz: float = 75.0
    scan_angle_max_rad: float = math.radians(30.0)
    head_rate_rad_s: float = 0.0
    grid_n_az: int = 0
    grid_n_el: int = 0
    el_min_rad: float = 0.0
    el_max_rad: float = 0.0
    n_fibres: int = 0


@dataclass
class Leg:
    """One scan leg: the platform moves from ``start`` to ``end`` (or stays)."""
    scene_index: int = 0
    scanner_index: int = 0
    platform: int = PLATFORM_STATIC
    start: tuple = (0.0, 0.0, 0.0)
    end: tuple = (0.0, 0.0, 0.0)
    speed_mps: float = 0.0
    attitude_rpy: tuple = (0.0, 0.0, 0.0)
    n_pulses: int = 0
    t0: float = 0.0
    beam_sample_quality: int = -1         # -1: use the scanner's
    leg_id: int = 0
    platform_noise_m: float = 0.0         # sigma of the per-pulse platform position noise
    first_pulse: int = 0                  # resume: scan pulses first_pulse .. first_pulse + n_pulses - 1


@dataclass
class Mesh:
    verts: np.ndarray        # float32 [V, 3]
    faces: np.ndarray        # int32 [F, 3]
    reflectance: np.ndarray  # float32 [F]
    object_id: int = 0


@dataclass
class VoxelGrid:
    origin: tuple            # (x, y, z) of the grid corner, metres
    cell: float              # voxel edge length, metres
    dims: tuple              # (nx, ny, nz)
    density: np.ndarray      # float32 [nz, ny, nx], plant area density m^2/m^3
    G: float = 0.5           # projection factor: sigma = G * density
    leaf_reflectance: float = 0.5
    object_id: int = 0
    opaque: int = 0          # 1: non-transmissive voxels
    lad: object = None       # leaf-angle table: float32 [n] of G at |d_z| = i/(n-1), or None


@dataclass
class Scene:
    meshes: list = field(default_factory=list)
    grids: list = field(default_factory=list)

    @property
    def n_triangles(self) -> int:
        return int(sum(m.faces.shape[0] for m in self.meshes))


@dataclass
class Workload:
    name: str
    scenes: list
    scanners: list
    legs: list
    note: str = ""

    @property
    def n_pulses(self) -> int:
        return int(sum(l.n_pulses for l in self.legs))


# --------------------------------------------------------------------------
# geometry helpers (pure data synthesis)
# --------------------------------------------------------------------------

def _box_mesh(center, size):
    """12-triangle axis-aligned box, outward winding."""
    cx, cy, cz = center
    sx, sy, sz = size
    x0, x1 = cx - sx / 2, cx + sx / 2
    y0, y1 = cy - sy / 2, cy + sy / 2
    z0, z1 = cz - sz / 2, cz + sz / 2
    v = np.array([[x0, y0, z0], [x1, y0, z0], [x1, y1, z0], [x0, y1, z0],
                  [x0, y0, z1], [x1, y0, z1], [x1, y1, z1], [x0, y1, z1]],
                 dtype=np.float64)
    f = np.array([[0, 2, 1], [0, 3, 2],      # bottom (-z)
                  [4, 5, 6], [4, 6, 7],      # top (+z)
                  [0, 1, 5], [0, 5, 4],      # -y
                  [2, 3, 7], [2, 7, 6],      # +y
                  [1, 2, 6], [1, 6, 5],      # +x
                  [3, 0, 4], [3, 4, 7]],     # -x
                 dtype=np.int64)
    return v, f


def _grid_mesh(nx, ny, x0, y0, dx, heights):
    """Triangulate a raster whose pixel centres are the vertices (2 triangles per cell)."""
    xs = x0 + dx * np.arange(nx)
    ys = y0 + dx * np.arange(ny)
    X, Y = np.meshgrid(xs, ys, indexing="xy")          # [ny, nx]
    verts = np.stack([X.ravel(), Y.ravel(), heights.ravel()], axis=1)
    idx = np.arange(nx * ny).reshape(ny, nx)
    a = idx[:-1, :-1].ravel()
    b = idx[:-1, 1:].ravel()
    c = idx[1:, 1:].ravel()
    d = idx[1:, :-1].ravel()
    faces = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)], 0)
    return verts, faces


def fbm_heightmap(rng, n, hurst=0.7, relief=60.0):
    """Spectral-synthesis fractional Brownian surface, n x n, range scaled to ``relief``."""
    kx = np.fft.fftfreq(n)
    ky = np.fft.rfftfreq(n)
    K = np.sqrt(kx[:, None] ** 2 + ky[None, :] ** 2)
    K[0, 0] = 1.0
    amp = K ** (-(hurst + 1.0))
    amp[0, 0] = 0.0
    phase = rng.uniform(0, 2 * np.pi, size=amp.shape)
    mag = rng.standard_normal(size=amp.shape)
    spec = amp * mag * np.exp(1j * phase)
    h = np.fft.irfft2(spec, s=(n, n))
    h = (h - h.min()) / max(h.max() - h.min(), 1e-30) * relief
    return h


def _tree_mesh(rng, base, height, n_seg=48, n_lat=32):
    """Trunk cylinder + conical or ellipsoidal crown, about 3k triangles."""
    bx, by, bz = base
    trunk_h = height * rng.uniform(0.25, 0.4)
    trunk_r = height * rng.uniform(0.015, 0.025)
    crown_r = height * rng.uniform(0.2, 0.3)
    verts = []
    faces = []
    # trunk: open cylinder from bz - 0.5 to bz + trunk_h + crown overlap
    ang = 2 * np.pi * np.arange(n_seg) / n_seg
    ring = np.stack([np.cos(ang), np.sin(ang)], 1)
    z0, z1 = bz - 0.5, bz + trunk_h + 0.2 * height
    lo = np.column_stack([bx + trunk_r * ring[:, 0], by + trunk_r * ring[:, 1], np.full(n_seg, z0)])
    hi = np.column_stack([bx + trunk_r * ring[:, 0], by + trunk_r * ring[:, 1], np.full(n_seg, z1)])
    verts.append(lo)
    verts.append(hi)
    i = np.arange(n_seg)
    j = (i + 1) % n_seg
    faces.append(np.stack([i, j, n_seg + j], 1))
    faces.append(np.stack([i, n_seg + j, n_seg + i], 1))
    off = 2 * n_seg
    cz0 = bz + trunk_h
    cz1 = bz + height
    if rng.uniform() < 0.5:
        # cone: n_lat bands from the rim to the apex, closed at the base
        ts = np.linspace(0.0, 1.0, n_lat + 1)[:-1]
        rings = []
        for t in ts:
            r = crown_r * (1.0 - t)
            rings.append(np.column_stack([bx + r * ring[:, 0], by + r * ring[:, 1],
                                          np.full(n_seg, cz0 + t * (cz1 - cz0))]))
        rv = np.concatenate(rings, 0)
        apex = np.array([[bx, by, cz1]])
        centre = np.array([[bx, by, cz0]])
        verts.extend([rv, apex, centre])
        for k in range(n_lat - 1):
            a = off + k * n_seg + i
            b = off + k * n_seg + j
            faces.append(np.stack([a, b, b + n_seg], 1))
            faces.append(np.stack([a, b + n_seg, a + n_seg], 1))
        top = off + (n_lat - 1) * n_seg
        ia = off + n_lat * n_seg
        ic = ia + 1
        faces.append(np.stack([top + i, top + j, np.full(n_seg, ia)], 1))
        faces.append(np.stack([off + j, off + i, np.full(n_seg, ic)], 1))
    else:
        # ellipsoid: latitude rings between the poles
        cz = 0.5 * (cz0 + cz1)
        hz = 0.5 * (cz1 - cz0)
        lats = np.linspace(0, np.pi, n_lat + 1)[1:-1]
        rings = []
        for th in lats:
            r = crown_r * np.sin(th)
            rings.append(np.column_stack([bx + r * ring[:, 0], by + r * ring[:, 1],
                                          np.full(n_seg, cz + hz * np.cos(th))]))
        rv = np.concatenate(rings, 0)
        north = np.array([[bx, by, cz + hz]])
        south = np.array([[bx, by, cz - hz]])
        verts.extend([rv, north, south])
        nr = len(lats)
        for k in range(nr - 1):
            a = off + k * n_seg + i
            b = off + k * n_seg + j
            faces.append(np.stack([a, a + n_seg, b + n_seg], 1))
            faces.append(np.stack([a, b + n_seg, b], 1))
        inn = off + nr * n_seg
        isn = inn + 1
        faces.append(np.stack([np.full(n_seg, inn), off + i, off + j], 1))
        last = off + (nr - 1) * n_seg
        faces.append(np.stack([np.full(n_seg, isn), last + j, last + i], 1))
    return np.concatenate(verts, 0), np.concatenate(faces, 0)


def _mesh(verts, faces, refl, object_id=0):
    return Mesh(verts=np.ascontiguousarray(verts, dtype=np.float32),
                faces=np.ascontiguousarray(faces, dtype=np.int32),
                reflectance=np.ascontiguousarray(refl, dtype=np.float32),
                object_id=object_id)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def tls_tiny(seed: int = 0, n_az: int = 100, n_el: int = 100) -> Workload:
    """Static TLS scan of a 20 x 20 m ground plus 8 seeded boxes (98 triangles)."""
    rng = np.random.default_rng(seed)
    gv = np.array([[-10, -10, 0], [10, -10, 0], [10, 10, 0], [-10, 10, 0]], dtype=np.float64)
    gf = np.array([[0, 1, 2], [0, 2, 3]])
    verts = [gv]
    faces = [gf]
    nv = 4
    for _ in range(8):
        r = rng.uniform(3.0, 9.0)
        a = rng.uniform(0.0, 2 * np.pi)
        size = rng.uniform(0.5, 2.0, size=3)
        c = (r * np.cos(a), r * np.sin(a), size[2] / 2)
        v, f = _box_mesh(c, size)
        verts.append(v)
        faces.append(f + nv)
        nv += v.shape[0]
    V = np.concatenate(verts, 0)
    F = np.concatenate(faces, 0)
    refl = rng.uniform(0.1, 0.9, size=F.shape[0])
    scene = Scene(meshes=[_mesh(V, F, refl, 1)])
    sc = Scanner(prf_hz=100_000.0, divergence_rad=0.3e-3, beam_sample_quality=2,
                 pulse_shape=PULSE_GAUSSIAN, pulse_fwhm_ns=4.0, bin_ns=0.25, n_bins=100,
                 max_echoes=8, echo_threshold_rel=0.05, range_noise_sigma_m=0.01,
                 deflector=DEFL_TLS_GRID, grid_n_az=n_az, grid_n_el=n_el,
                 el_min_rad=math.radians(-30.0), el_max_rad=math.radians(30.0))
    leg = Leg(scene_index=0, platform=PLATFORM_STATIC, start=(0.0, 0.0, 1.5),
              end=(0.0, 0.0, 1.5), n_pulses=n_az * n_el, t0=0.0, leg_id=0)
    return Workload("tls_tiny_98tri_100x100", [scene], [sc], [leg],
                    note="ground 2 tris + 8 boxes (96 tris), 100 az x 100 el, q=2 (19 subrays), N_b=100")


def terrain_scene(rng, size=1024, n_trees=300, relief=60.0, spacing=1.0, tree_extent=None):
    """fBm DTM (pixel centres -> 2 triangles per cell) plus procedural trees."""
    h = fbm_heightmap(rng, size, 0.7, relief)
    x0 = -0.5 * (size - 1) * spacing
    v, f = _grid_mesh(size, size, x0, x0, spacing, h)
    meshes = [_mesh(v, f, rng.uniform(0.2, 0.4, size=f.shape[0]), 1)]
    if n_trees > 0:
        ext = tree_extent if tree_extent is not None else 0.4 * size * spacing
        tv, tf = [], []
        nv = 0
        for _ in range(n_trees):
            px, py = rng.uniform(-ext, ext, size=2)
            ix = int(round((px - x0) / spacing))
            iy = int(round((py - x0) / spacing))
            ix = min(max(ix, 0), size - 1)
            iy = min(max(iy, 0), size - 1)
            bz = h[iy, ix]
            vv, ff = _tree_mesh(rng, (x0 + ix * spacing, x0 + iy * spacing, bz),
                                rng.uniform(8.0, 20.0))
            tv.append(vv)
            tf.append(ff + nv)
            nv += vv.shape[0]
        TV = np.concatenate(tv, 0)
        TF = np.concatenate(tf, 0)
        meshes.append(_mesh(TV, TF, rng.uniform(0.4, 0.6, size=TF.shape[0]), 2))
    return Scene(meshes=meshes), float(h.mean())


def als_terrain(seed: int = 1, size: int = 1024, n_trees: int = 300,
                n_pulses: int = 4_000_000, n_bins: int = 512, agl: float = 500.0,
                speed: float = 60.0, prf: float = 400_000.0) -> Workload:
    """ALS over a seeded fBm terrain with trees, oscillating mirror +/-30 deg at 75 Hz."""
    rng = np.random.default_rng(seed)
    scene, hmean = terrain_scene(rng, size, n_trees)
    track = speed * n_pulses / prf
    z = hmean + agl
    sc = Scanner(prf_hz=prf, divergence_rad=0.3e-3, beam_sample_quality=2,
                 pulse_shape=PULSE_GAUSSIAN, pulse_fwhm_ns=4.0, bin_ns=0.25, n_bins=n_bins,
                 max_echoes=8, echo_threshold_rel=0.05, range_noise_sigma_m=0.01,
                 deflector=DEFL_OSCILLATING, scan_freq_hz=75.0,
                 scan_angle_max_rad=math.radians(30.0))
    leg = Leg(scene_index=0, platform=PLATFORM_LINEAR, start=(-track / 2, 0.0, z),
              end=(track / 2, 0.0, z), speed_mps=speed, n_pulses=n_pulses, t0=0.0, leg_id=1)
    return Workload(f"als_terrain_{size}sq_{n_trees}trees_{n_pulses}p", [scene], [sc], [leg],
                    note=f"fBm DTM {size}^2 at 1 m (H=0.7, 60 m relief) + {n_trees} trees; "
                         f"{agl:.0f} m AGL, {speed:.0f} m/s, oscillating +/-30 deg 75 Hz, "
                         f"PRF {prf/1e3:.0f} kHz, q=2, N_b={n_bins}")


def smooth_noise_3d(rng, n, corr_cells=8.0):
    """Gaussian-filtered white noise on an n^3 lattice (spectral filter), zero mean."""
    w = rng.standard_normal((n, n, n))
    k = np.fft.fftfreq(n)
    kr = np.fft.rfftfreq(n)
    K2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + kr[None, None, :] ** 2
    filt = np.exp(-2.0 * (np.pi * corr_cells) ** 2 * K2 / 4.0)
    f = np.fft.irfftn(np.fft.rfftn(w) * filt, s=(n, n, n), axes=(0, 1, 2))
    return f


def canopy_density(rng, n=256, empty_frac=0.7, max_density=2.0, corr_cells=8.0):
    """Leaf-area density in [0, max_density] with ``empty_frac`` of voxels exactly 0."""
    f = smooth_noise_3d(rng, n, corr_cells)
    thr = np.quantile(f, empty_frac)
    top = f.max()
    d = np.clip((f - thr) / max(top - thr, 1e-30), 0.0, 1.0) * max_density
    return np.ascontiguousarray(d.astype(np.float32))


def uls_voxels(seed: int = 2, n: int = 256, n_pulses: int = 1_000_000, n_bins: int = 1024,
               cell: float = 0.1, agl: float = 50.0, speed: float = 3.0,
               prf: float = 100_000.0) -> Workload:
    """ULS over a transmissive voxel canopy (n^3 at ``cell``) above a 2-triangle ground."""
    rng = np.random.default_rng(seed)
    dens = canopy_density(rng, n)
    L = n * cell
    grid = VoxelGrid(origin=(0.0, 0.0, 0.0), cell=cell, dims=(n, n, n), density=dens,
                     G=0.5, leaf_reflectance=0.5, object_id=3)
    gv = np.array([[-10, -10, 0], [L + 10, -10, 0], [L + 10, L + 10, 0], [-10, L + 10, 0]],
                  dtype=np.float64)
    gf = np.array([[0, 1, 2], [0, 2, 3]])
    ground = _mesh(gv, gf, np.full(2, 0.3), 1)
    scene = Scene(meshes=[ground], grids=[grid])
    track = speed * n_pulses / prf
    sc = Scanner(prf_hz=prf, divergence_rad=0.3e-3, beam_sample_quality=2,
                 pulse_shape=PULSE_GAUSSIAN, pulse_fwhm_ns=4.0, bin_ns=0.25, n_bins=n_bins,
                 max_echoes=8, echo_threshold_rel=0.05, range_noise_sigma_m=0.01,
                 deflector=DEFL_POLYGON, scan_freq_hz=100.0,
                 scan_angle_max_rad=math.radians(15.0))
    c = L / 2
    leg = Leg(scene_index=0, platform=PLATFORM_LINEAR, start=(c - track / 2, c, agl),
              end=(c + track / 2, c, agl), speed_mps=speed, n_pulses=n_pulses, t0=0.0, leg_id=2)
    return Workload(f"uls_voxels_{n}cube_{n_pulses}p", [scene], [sc], [leg],
                    note=f"{n}^3 voxels at {cell} m, LAD 0..2 (70% empty), G=0.5; "
                         f"{agl:.0f} m AGL, {speed} m/s, polygon +/-15 deg 100 Hz, "
                         f"PRF {prf/1e3:.0f} kHz, q=2, N_b={n_bins}")


def tree_density(rng, n=128, max_density=2.0):
    """A voxel tree in an n^3 box (x, y centred; z from the ground): a trunk
    column of dense voxels and an ellipsoidal crown whose leaf-area density is
    smooth noise cut to zero over about half of the crown."""
    z, y, x = np.meshgrid(*(np.arange(n) + 0.5,) * 3, indexing="ij")
    c = n / 2.0
    r_tr = max(1.0, n * rng.uniform(0.02, 0.04))
    trunk = ((x - c) ** 2 + (y - c) ** 2 <= r_tr ** 2) & (z < n * rng.uniform(0.35, 0.5))
    zc, rz = n * rng.uniform(0.6, 0.7), n * rng.uniform(0.25, 0.33)
    rxy = n * rng.uniform(0.3, 0.48)
    crown = ((x - c) / rxy) ** 2 + ((y - c) / rxy) ** 2 + ((z - zc) / rz) ** 2 <= 1.0
    f = smooth_noise_3d(rng, n, max(2.0, n / 16.0))
    thr = np.quantile(f[crown], 0.5) if crown.any() else 0.0
    leaf = np.clip((f - thr) / max(f.max() - thr, 1e-30), 0.0, 1.0) * max_density
    d = np.where(crown, leaf, 0.0)
    d = np.where(trunk, 4.0 * max_density, d)
    return np.ascontiguousarray(d.astype(np.float32))


def tree_grids(rng, slots, n=128, cell=45.0 / 1024.0, n_templates=16, G=0.5):
    """Voxel trees at the given box corners (boxes n*cell wide, disjoint by
    construction of the slots).  Trees share ``n_templates`` seeded density
    arrays, so a scene with thousands of trees holds a few of them."""
    templates = [tree_density(rng, n) for _ in range(min(n_templates, len(slots)) or 1)]
    pick = rng.integers(0, len(templates), size=len(slots))
    grids = []
    for i, (x0, y0, z0) in enumerate(slots):
        grids.append(VoxelGrid(origin=(float(x0), float(y0), float(z0)), cell=cell, dims=(n, n, n),
                               density=templates[pick[i]], G=G, leaf_reflectance=0.5,
                               object_id=5))
    return grids


def voxel_forest(seed: int = 7, n_trees: int = 9, n: int = 24, cell: float = 0.25,
                 n_pulses: int = 4000, n_bins: int = 512, agl: float = 25.0, speed: float = 12.0,
                 prf: float = 2000.0) -> Workload:
    """ULS over separate voxel trees (one grid each, boxes on a 3 x 3 lattice,
    neighbours touching along x) above a 2-triangle ground."""
    rng = np.random.default_rng(seed)
    L = n * cell
    slots = []
    for k in range(n_trees):
        i, j = k % 3, k // 3
        slots.append((i * L, j * (L + 1.5), 0.0))
    grids = tree_grids(rng, slots, n=n, cell=cell, n_templates=n_trees)
    W = 3 * L
    H = (n_trees + 2) // 3 * (L + 1.5)
    gv = np.array([[-20, -20, 0], [W + 20, -20, 0], [W + 20, H + 20, 0], [-20, H + 20, 0]], dtype=np.float64)
    gf = np.array([[0, 1, 2], [0, 2, 3]])
    scene = Scene(meshes=[_mesh(gv, gf, np.full(2, 0.3), 1)], grids=grids)
    sc = Scanner(prf_hz=prf, divergence_rad=0.3e-3, beam_sample_quality=2,
                 pulse_shape=PULSE_GAUSSIAN, pulse_fwhm_ns=4.0, bin_ns=0.25, n_bins=n_bins,
                 max_echoes=8, echo_threshold_rel=0.05, range_noise_sigma_m=0.01,
                 deflector=DEFL_POLYGON, scan_freq_hz=50.0, scan_angle_max_rad=math.radians(30.0))
    track = speed * n_pulses / prf
    leg = Leg(scene_index=0, platform=PLATFORM_LINEAR, start=(W / 2 - track / 2, H / 2, agl),
              end=(W / 2 + track / 2, H / 2, agl), speed_mps=speed, n_pulses=n_pulses, t0=0.0, leg_id=6)
    return Workload(f"voxel_forest_{n_trees}x{n}cube_{n_pulses}p", [scene], [sc], [leg],
                    note=f"{n_trees} voxel trees of {n}^3 at {cell} m (one grid each) over a ground")


def _rect_mesh(p0, e1, e2, cell):
    """Planar rectangle p0 + u e1 + v e2 (u, v in [0, 1]) in square-ish cells of
    about ``cell`` metres, two triangles per cell."""
    p0, e1, e2 = (np.asarray(x, dtype=np.float64) for x in (p0, e1, e2))
    nu = max(1, int(round(np.linalg.norm(e1) / cell)))
    nv = max(1, int(round(np.linalg.norm(e2) / cell)))
    u = np.linspace(0.0, 1.0, nu + 1)
    v = np.linspace(0.0, 1.0, nv + 1)
    U, V = np.meshgrid(u, v, indexing="ij")
    verts = p0 + U[..., None] * e1 + V[..., None] * e2
    idx = np.arange((nu + 1) * (nv + 1)).reshape(nu + 1, nv + 1)
    a, b = idx[:-1, :-1].ravel(), idx[1:, :-1].ravel()
    c, d = idx[1:, 1:].ravel(), idx[:-1, 1:].ravel()
    faces = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)], 0)
    return verts.reshape(-1, 3), faces


def urban_scene(rng, length=2000.0, facade_cell=0.17, ground_cell=1.0, half_width=50.0):
    """Street planes along x plus extruded rectangular building footprints on
    both sides, facades and roofs tessellated at ``facade_cell``.  Mesh 0 is
    the street, mesh 1 the buildings; reflectance is seeded per building
    (U[0.2, 0.8]) plus per-triangle N(0, 0.05), and U[0.1, 0.3] on the street."""
    gv, gf = _rect_mesh((-30.0, -half_width, 0.0), (length + 60.0, 0.0, 0.0),
                        (0.0, 2.0 * half_width, 0.0), ground_cell)
    street = _mesh(gv, gf, rng.uniform(0.1, 0.3, size=gf.shape[0]), 1)
    verts, faces, refl, nv = [], [], [], 0
    for side in (-1.0, 1.0):
        x = -20.0
        while x < length + 20.0:
            w = rng.uniform(8.0, 25.0)
            depth = rng.uniform(8.0, 20.0)
            setback = rng.uniform(8.0, 14.0)
            h = rng.uniform(6.0, 30.0)
            base = rng.uniform(0.2, 0.8)
            y0 = setback if side > 0 else -setback - depth
            y1 = y0 + depth
            parts = [((x, y0, 0.0), (w, 0.0, 0.0), (0.0, 0.0, h)),        # facade at y0
                     ((x, y1, 0.0), (w, 0.0, 0.0), (0.0, 0.0, h)),        # facade at y1
                     ((x, y0, 0.0), (0.0, depth, 0.0), (0.0, 0.0, h)),    # gable at x
                     ((x + w, y0, 0.0), (0.0, depth, 0.0), (0.0, 0.0, h)),
                     ((x, y0, h), (w, 0.0, 0.0), (0.0, depth, 0.0))]      # roof
            for p0, e1, e2 in parts:
                v, f = _rect_mesh(p0, e1, e2, facade_cell)
                verts.append(v)
                faces.append(f + nv)
                refl.append(np.clip(base + rng.normal(0.0, 0.05, size=f.shape[0]), 0.05, 0.95))
                nv += v.shape[0]
            x += w + rng.uniform(0.0, 4.0)
    buildings = _mesh(np.concatenate(verts, 0), np.concatenate(faces, 0), np.concatenate(refl, 0), 2)
    return Scene(meshes=[street, buildings])


def urban_trees(rng, length=2000.0, n_trees=2000, n=128, cell=45.0 / 1024.0):
    """Slots for street trees: boxes n*cell wide packed end to end along x in
    six rows, one on each sidewalk (|y| in [0.75, 0.75 + n cell]) and two
    behind each side's buildings (from |y| = 34.25); ``n_trees`` of them,
    chosen at random, get a voxel tree.  The cell (45/1024 m: 128 voxels make
    a 5.625 m box) and the slot corners are exact in FP32, so neighbouring
    boxes touch without overlapping.  2000 trees of 128^3 are 4.19e9 voxels
    (primitive ids are 64-bit)."""
    L = n * cell
    per_row = int(length // L)
    rows = [(0.75, 1.0), (34.25, 1.0), (34.25 + L, 1.0), (0.75, -1.0), (34.25, -1.0), (34.25 + L, -1.0)]
    slots = []
    for y_in, side in rows:
        y0 = y_in if side > 0 else -y_in - L
        for i in range(per_row):
            slots.append((i * L, y0, 0.0))
    pick = np.sort(rng.choice(len(slots), size=min(n_trees, len(slots)), replace=False))
    return tree_grids(rng, [slots[i] for i in pick], n=n, cell=cell)


def urban_mls(seed: int = 4, length: float = 2000.0, speed: float = 10.0, prf: float = 100_000.0,
              facade_cell: float = 0.17, n_bins: int = 512, q: int = 3, n_trees: int = 2000) -> Workload:
    """Mobile laser scanning along an urban street: a profile scanner (head
    rotating 100 rev/s, its spin plane across the street) on a vehicle at
    2.5 m driving ``length`` metres at ``speed``; ``n_trees`` voxel trees
    (128^3 at 45/1024 m, one grid each) line the street."""
    rng = np.random.default_rng(seed)
    scene = urban_scene(rng, length=length, facade_cell=facade_cell)
    if n_trees > 0:
        scene.grids = urban_trees(rng, length=length, n_trees=n_trees)
    sc = Scanner(prf_hz=prf, divergence_rad=0.3e-3, beam_sample_quality=q,
                 pulse_shape=PULSE_GAUSSIAN, pulse_fwhm_ns=4.0, bin_ns=0.25, n_bins=n_bins,
                 max_echoes=8, echo_threshold_rel=0.05, range_noise_sigma_m=0.01,
                 deflector=DEFL_ROTATING_HEAD, head_rate_rad_s=2.0 * math.pi * 100.0,
                 scan_freq_hz=1.0, scan_angle_max_rad=0.0)
    n_pulses = int(round(length / speed * prf))
    leg = Leg(scene_index=0, platform=PLATFORM_LINEAR, start=(0.0, 0.0, 2.5), end=(length, 0.0, 2.5),
              speed_mps=speed, attitude_rpy=(0.0, math.pi / 2, 0.0), n_pulses=n_pulses, t0=0.0,
              leg_id=4)
    nt = len(scene.grids)
    return Workload(f"urban_mls_{scene.n_triangles}tri_{nt}trees_{n_pulses}p", [scene], [sc], [leg],
                    note=f"street + extruded buildings ({scene.n_triangles} triangles, facade cell "
                         f"{facade_cell} m), {nt} voxel trees (128^3 at 0.044 m), {length:.0f} m at "
                         f"{speed} m/s, profile head 100 rev/s, PRF {prf/1e3:.0f} kHz, q={q}, N_b={n_bins}")


def perturbed_density(density: np.ndarray, seed: int = 1, rel: float = 0.1) -> np.ndarray:
    """Reference-scan densities: non-empty voxels scaled by (1 + rel * N(0,1))."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(density.shape).astype(np.float32)
    out = np.where(density > 0, density * (1.0 + rel * z), 0.0)
    return np.ascontiguousarray(np.maximum(out, 0.0).astype(np.float32))


def batched_legs(seed: int = 3, n_legs: int = 128, min_pulses: int = 10_000,
                 max_pulses: int = 2_000_000, tile: int = 512, block: int = 128,
                 n_terrain: int = 8, n_voxel: int = 8, n_bins: int = 512) -> Workload:
    """Many independent legs of log-uniform length and random subray quality."""
    rng = np.random.default_rng(seed)
    scenes = []
    for _ in range(n_terrain):
        s, _hm = terrain_scene(rng, tile, n_trees=max(tile // 16, 1))
        scenes.append(s)
    for _ in range(n_voxel):
        dens = canopy_density(rng, block)
        L = block * 0.1
        grid = VoxelGrid(origin=(0.0, 0.0, 0.0), cell=0.1, dims=(block,) * 3, density=dens,
                         G=0.5, leaf_reflectance=0.5, object_id=3)
        gv = np.array([[-30, -30, 0], [L + 30, -30, 0], [L + 30, L + 30, 0], [-30, L + 30, 0]],
                      dtype=np.float64)
        scenes.append(Scene(meshes=[_mesh(gv, np.array([[0, 1, 2], [0, 2, 3]]), np.full(2, 0.3), 1)],
                            grids=[grid]))
    als = Scanner(prf_hz=400_000.0, divergence_rad=0.3e-3, beam_sample_quality=2,
                  n_bins=n_bins, deflector=DEFL_OSCILLATING, scan_freq_hz=75.0,
                  scan_angle_max_rad=math.radians(30.0))
    uls = Scanner(prf_hz=100_000.0, divergence_rad=0.3e-3, beam_sample_quality=2,
                  n_bins=n_bins, deflector=DEFL_POLYGON, scan_freq_hz=100.0,
                  scan_angle_max_rad=math.radians(15.0))
    legs = []
    for li in range(n_legs):
        npul = int(math.floor(math.exp(rng.uniform(math.log(min_pulses), math.log(max_pulses)))))
        q = int(rng.integers(0, 4))
        si = int(rng.integers(0, n_terrain + n_voxel))
        if si < n_terrain:
            half = 0.45 * tile
            y = rng.uniform(-0.2, 0.2) * tile
            legs.append(Leg(scene_index=si, scanner_index=0, platform=PLATFORM_LINEAR,
                            start=(-half, y, 560.0), end=(half, y, 560.0), speed_mps=60.0,
                            n_pulses=npul, t0=float(rng.uniform(0, 100)),
                            beam_sample_quality=q, leg_id=1000 + li))
        else:
            c = block * 0.05
            legs.append(Leg(scene_index=si, scanner_index=1, platform=PLATFORM_LINEAR,
                            start=(c - 15.0, c, 50.0), end=(c + 15.0, c, 50.0), speed_mps=3.0,
                            n_pulses=npul, t0=float(rng.uniform(0, 100)),
                            beam_sample_quality=q, leg_id=1000 + li))
    return Workload(f"batched_{n_legs}legs", scenes, [als, uls], legs,
                    note=f"{n_legs} legs, pulses log-uniform [{min_pulses}, {max_pulses}], "
                         f"q in 0..3, {n_terrain} terrain tiles {tile}^2 + {n_voxel} voxel blocks {block}^3")


def triangle_soup(seed: int, n: int, extent: float = 10.0, size: float = 2.0) -> Scene:
    """Random triangles in a cube, for brute-force cross-checks."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-extent, extent, size=(n, 1, 3))
    v = c + rng.uniform(-size, size, size=(n, 3, 3))
    V = v.reshape(-1, 3)
    F = np.arange(3 * n).reshape(n, 3)
    return Scene(meshes=[_mesh(V, F, rng.uniform(0.1, 0.9, size=n), 1)])


def flat_target(distance: float, tilt_rad: float = 0.0, half: float = 50.0,
                reflectance: float = 0.5) -> Scene:
    """A square plate whose centre is ``distance`` below the origin, tilted about x.

    Used for closed-form checks: a ray straight down from the origin meets the
    plate at ``distance / cos(tilt)`` with incidence angle ``tilt``.
    """
    ct, st = math.cos(tilt_rad), math.sin(tilt_rad)
    corners = []
    for (a, b) in [(-half, -half), (half, -half), (half, half), (-half, half)]:
        # plate spanned by x-axis and the tilted y-axis, through (0, 0, -distance)
        corners.append((a, b * ct, -distance + b * st))
    V = np.array(corners, dtype=np.float64)
    F = np.array([[0, 1, 2], [0, 2, 3]])
    return Scene(meshes=[_mesh(V, F, np.full(2, reflectance), 1)])


def with_scanner(w: Workload, **kw) -> Workload:
    return Workload(w.name, w.scenes, [replace(s, **kw) for s in w.scanners], w.legs, w.note)
