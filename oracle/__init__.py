"""FP64 CPU oracle for the per-pulse beam-scene interaction (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
arm of ``bench.py`` import this package.  It shares no code with the CUDA
library: its C source (``helios_oracle.c``) is compiled here with gcc and
loaded through ctypes; the only thing both sides have in common is the seeded
input module ``scenes``.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "helios_oracle.c")
_HDR = os.path.join(_HERE, "helios_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhelios_oracle.so")
_lock = threading.Lock()
_lib = None

NO_WINDOW = -(2 ** 31)
F_EDGE, F_TIE, F_VOX, F_WIN, F_ECHO, F_OBJ = 1, 2, 4, 8, 16, 32
F_OVERFLOW, F_NOHIT, F_FIT, F_FORCED_BAD = 256, 512, 1024, 2048
F_SUBRAY = F_EDGE | F_TIE | F_VOX                  # a subray's hit id / range may differ
FREE_HIT = -2                                       # force_hit entry: the oracle decides
F_GEOMETRY = F_EDGE | F_TIE | F_VOX | F_WIN        # waveform may differ
F_DECISION = F_GEOMETRY | F_ECHO | F_OBJ           # echo lists may differ


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE double, no contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-pthread", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Scanner(C.Structure):
    _fields_ = [("prf_hz", C.c_double), ("divergence_rad", C.c_double),
                ("quality", C.c_int32), ("pulse_shape", C.c_int32),
                ("wavelength_m", C.c_double), ("beam_waist_m", C.c_double), ("focus_m", C.c_double),
                ("peak_power_w", C.c_double), ("receiver_diam_m", C.c_double),
                ("eta_sys", C.c_double), ("eta_atm", C.c_double),
                ("pulse_fwhm_ns", C.c_double), ("pulse_length_ns", C.c_double), ("bin_ns", C.c_double),
                ("n_bins", C.c_int32), ("max_echoes", C.c_int32),
                ("echo_threshold_rel", C.c_double), ("range_noise_sigma_m", C.c_double),
                ("deflector", C.c_int32), ("grid_n_az", C.c_int32), ("grid_n_el", C.c_int32),
                ("n_fibres", C.c_int32),
                ("scan_freq_hz", C.c_double), ("scan_angle_max_rad", C.c_double),
                ("head_rate_rad_s", C.c_double), ("el_min_rad", C.c_double), ("el_max_rad", C.c_double)]


class Leg(C.Structure):
    _fields_ = [("platform", C.c_int32), ("quality", C.c_int32), ("leg_id", C.c_uint32),
                ("pad0", C.c_int32), ("start", C.c_double * 3), ("end", C.c_double * 3),
                ("speed_mps", C.c_double), ("attitude_rpy", C.c_double * 3), ("t0", C.c_double),
                ("n_pulses", C.c_int64), ("platform_noise_m", C.c_double)]


class GridIn(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("cell", C.c_double), ("dims", C.c_int32 * 3),
                ("opaque", C.c_int32), ("density", C.c_void_p), ("G", C.c_double),
                ("leaf_refl", C.c_double), ("lad", C.c_void_p), ("lad_n", C.c_int32), ("pad", C.c_int32)]


class SceneIn(C.Structure):
    _fields_ = [("n_tri", C.c_int64), ("tri", C.c_void_p), ("refl", C.c_void_p),
                ("n_grids", C.c_int32), ("pad0", C.c_int32), ("grids", C.c_void_p)]


class Out(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("window_bin", "waveform", "echo_count", "echo_bin",
                                            "echo_amp", "echo_range", "echo_range_clean",
                                            "echo_object", "echo_width", "subray_hit", "subray_range",
                                            "flags", "subray_flags", "echo_object_alt")]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = C.CDLL(build())
            d3 = C.POINTER(C.c_double)
            l.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
            l.or_uniform24.argtypes = [C.c_uint32]
            l.or_uniform24.restype = C.c_double
            l.or_subray_count.argtypes = [C.c_int]
            l.or_subray_angles.argtypes = [C.c_int, C.c_double, C.c_int, d3, d3]
            l.or_onb.argtypes = [d3, d3, d3]
            l.or_pulse_ray.argtypes = [C.POINTER(Scanner), C.POINTER(Leg), C.c_int64, C.c_uint64, d3, d3]
            l.or_subray_dir.argtypes = [C.POINTER(Scanner), C.c_int, C.c_int, d3, d3]
            for f in ("or_beam_width",):
                getattr(l, f).argtypes = [C.POINTER(Scanner), C.c_double]
                getattr(l, f).restype = C.c_double
            l.or_subray_intensity.argtypes = [C.POINTER(Scanner), C.c_double, C.c_double]
            l.or_echo_width.argtypes = [d3, C.c_int, C.c_int, C.c_double, C.POINTER(C.c_int)]
            l.or_echo_width.restype = C.c_double
            l.or_echo_peaks.argtypes = [d3, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_int32),
                                        C.POINTER(C.c_int), C.POINTER(C.c_int)]
            l.or_echo_peaks.restype = C.c_int
            l.or_echo_object.argtypes = [C.POINTER(Scanner), C.c_int64, d3, d3,
                                         C.POINTER(C.c_int64), C.c_double, C.POINTER(C.c_int)]
            l.or_echo_object.restype = C.c_int64
            l.or_subray_intensity.restype = C.c_double
            l.or_pulse_shape.argtypes = [C.POINTER(Scanner), C.c_double]
            l.or_pulse_shape.restype = C.c_double
            l.or_triangle_power.argtypes = [C.POINTER(Scanner)] + [C.c_double] * 4
            l.or_triangle_power.restype = C.c_double
            l.or_scene_build.argtypes = [C.POINTER(SceneIn)]
            l.or_scene_build.restype = C.c_void_p
            l.or_scene_free.argtypes = [C.c_void_p]
            l.or_scene_bvh_nodes.argtypes = [C.c_void_p]
            l.or_scene_bvh_nodes.restype = C.c_int64
            l.or_intersect.argtypes = [C.c_void_p, d3, d3, d3, d3, C.POINTER(C.c_uint32)]
            l.or_intersect.restype = C.c_int64
            l.or_intersect_brute.argtypes = [C.c_void_p, d3, d3, d3, d3]
            l.or_intersect_brute.restype = C.c_int64
            l.or_march.argtypes = [C.c_void_p, d3, d3, C.c_double, C.c_int64,
                                   C.c_void_p, C.c_void_p, C.c_void_p]
            l.or_march.restype = C.c_int64
            l.or_trace_returns.argtypes = [C.c_void_p, C.POINTER(Scanner), d3, d3, C.c_double,
                                           C.c_int, C.c_uint64, C.c_uint32, C.c_int64, C.c_int,
                                           C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.POINTER(C.c_uint32)]
            l.or_trace_returns.restype = C.c_int64
            l.or_scan.argtypes = [C.c_void_p, C.POINTER(Scanner), C.POINTER(Leg), C.c_void_p,
                                  C.c_int64, C.c_int, C.c_uint64, C.c_void_p, C.c_void_p,
                                  C.POINTER(Out), C.c_int]
            l.or_adjoint.argtypes = [C.c_void_p, C.POINTER(Scanner), C.POINTER(Leg), C.c_void_p,
                                     C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
            _lib = l
    return _lib


def _d3(x):
    return (C.c_double * 3)(*[float(v) for v in x])


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def scanner_struct(sc) -> Scanner:
    s = Scanner()
    s.prf_hz = sc.prf_hz
    s.divergence_rad = sc.divergence_rad
    s.quality = sc.beam_sample_quality
    s.pulse_shape = sc.pulse_shape
    s.wavelength_m = sc.wavelength_m
    s.beam_waist_m = sc.beam_waist_m
    s.focus_m = sc.focus_m
    s.peak_power_w = sc.peak_power_w
    s.receiver_diam_m = sc.receiver_diam_m
    s.eta_sys = sc.eta_sys
    s.eta_atm = sc.eta_atm
    s.pulse_fwhm_ns = sc.pulse_fwhm_ns
    s.pulse_length_ns = sc.pulse_length_ns
    s.bin_ns = sc.bin_ns
    s.n_bins = sc.n_bins
    s.max_echoes = sc.max_echoes
    s.echo_threshold_rel = sc.echo_threshold_rel
    s.range_noise_sigma_m = sc.range_noise_sigma_m
    s.deflector = sc.deflector
    s.grid_n_az = sc.grid_n_az
    s.grid_n_el = sc.grid_n_el
    s.n_fibres = sc.n_fibres
    s.scan_freq_hz = sc.scan_freq_hz
    s.scan_angle_max_rad = sc.scan_angle_max_rad
    s.head_rate_rad_s = sc.head_rate_rad_s
    s.el_min_rad = sc.el_min_rad
    s.el_max_rad = sc.el_max_rad
    return s


def leg_struct(lg) -> Leg:
    l = Leg()
    l.platform = lg.platform
    l.quality = lg.beam_sample_quality
    l.leg_id = lg.leg_id
    l.start = _d3(lg.start)
    l.end = _d3(lg.end)
    l.speed_mps = lg.speed_mps
    l.attitude_rpy = _d3(lg.attitude_rpy)
    l.t0 = lg.t0
    l.n_pulses = lg.n_pulses
    l.platform_noise_m = lg.platform_noise_m
    return l


class OracleScene:
    """A scene (triangles of all meshes concatenated, at most one voxel grid) in FP64."""

    def __init__(self, scene):
        tris, refl = [], []
        for m in scene.meshes:
            tris.append(m.verts[m.faces.astype(np.int64)].reshape(-1, 9))
            refl.append(m.reflectance)
        self.tri = np.ascontiguousarray(np.concatenate(tris, 0) if tris else np.zeros((0, 9)),
                                        dtype=np.float32)
        self.refl = np.ascontiguousarray(np.concatenate(refl, 0) if refl else np.zeros(0),
                                         dtype=np.float32)
        self.n_tri = self.tri.shape[0]
        self.mesh_offsets = np.cumsum([0] + [m.faces.shape[0] for m in scene.meshes])
        si = SceneIn()
        si.n_tri = self.n_tri
        si.tri = _ptr(self.tri)
        si.refl = _ptr(self.refl)
        # grids: FP32 inputs as the GPU receives them (the same real numbers)
        self.grids = list(scene.grids)
        self.grid = self.grids[0] if self.grids else None
        self._gin = (GridIn * max(len(self.grids), 1))()
        self.densities, self.lads, self.vox_offsets = [], [], [0]
        for i, g in enumerate(self.grids):
            gi = self._gin[i]
            dens = np.ascontiguousarray(g.density, dtype=np.float32)
            self.densities.append(dens)
            gi.origin = _d3(np.float32(g.origin).astype(np.float64))
            gi.cell = float(np.float32(g.cell))
            gi.dims = (C.c_int32 * 3)(*[int(x) for x in g.dims])
            gi.opaque = int(g.opaque)
            gi.density = _ptr(dens)
            gi.G = float(np.float32(g.G))
            gi.leaf_refl = float(np.float32(g.leaf_reflectance))
            lad = getattr(g, "lad", None)
            if lad is not None:
                lt = np.ascontiguousarray(lad, dtype=np.float32)
                self.lads.append(lt)
                gi.lad = _ptr(lt)
                gi.lad_n = int(lt.shape[0])
            self.vox_offsets.append(self.vox_offsets[-1] + int(np.prod(g.dims)))
        si.n_grids = len(self.grids)
        si.grids = C.cast(self._gin, C.c_void_p)
        self.density = self.densities[0] if self.densities else None
        self.n_vox = self.vox_offsets[-1]
        self._si = si
        self.handle = lib().or_scene_build(C.byref(si))

    def set_density(self, density, grid=0):
        """Point a grid at another density array (same shape)."""
        d = np.ascontiguousarray(density, dtype=np.float32)
        self.densities[grid] = d
        if grid == 0:
            self.density = d
        self._gin[grid].density = _ptr(d)
        lib().or_scene_free(self.handle)
        self.handle = lib().or_scene_build(C.byref(self._si))

    def close(self):
        if self.handle:
            lib().or_scene_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def intersect(self, o, d):
        t, c = C.c_double(), C.c_double()
        f = C.c_uint32(0)
        i = lib().or_intersect(self.handle, _d3(o), _d3(d), C.byref(t), C.byref(c), C.byref(f))
        return int(i), t.value, c.value, int(f.value)

    def intersect_brute(self, o, d):
        t, c = C.c_double(), C.c_double()
        i = lib().or_intersect_brute(self.handle, _d3(o), _d3(d), C.byref(t), C.byref(c))
        return int(i), t.value, c.value

    def march(self, o, d, t_hi=math.inf, cap=100000):
        vid = np.zeros(cap, np.int64)
        ti = np.zeros(cap)
        to = np.zeros(cap)
        n = lib().or_march(self.handle, _d3(o), _d3(d), t_hi, cap, _ptr(vid), _ptr(ti), _ptr(to))
        n = min(n, cap)
        return vid[:n], ti[:n], to[:n]


def trace_returns(oscene, scanner, o, ds, alpha=0.0, mode=0, seed=0, leg_id=0, pulse=0, s=0,
                  cap=100000):
    """Returns (R, P, id, flags) of one subray, in summation order."""
    R = np.zeros(cap)
    P = np.zeros(cap)
    ids = np.zeros(cap, np.int64)
    f = C.c_uint32(0)
    sc = scanner_struct(scanner)
    n = lib().or_trace_returns(oscene.handle, C.byref(sc), _d3(o), _d3(ds), float(alpha), int(mode),
                               int(seed) & (2 ** 64 - 1), int(leg_id), int(pulse), int(s), cap,
                               _ptr(R), _ptr(P), _ptr(ids), C.byref(f))
    n = min(n, cap)
    return R[:n], P[:n], ids[:n], int(f.value)


def subray_count(q: int) -> int:
    return int(lib().or_subray_count(q))


def subray_angles(q, theta_r, s):
    a, p = C.c_double(), C.c_double()
    lib().or_subray_angles(q, theta_r, s, C.byref(a), C.byref(p))
    return a.value, p.value


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def onb(n):
    u, v = (C.c_double * 3)(), (C.c_double * 3)()
    lib().or_onb(_d3(n), u, v)
    return np.array(u[:]), np.array(v[:])


def pulse_ray(scanner, leg, k, seed=0):
    o, d = (C.c_double * 3)(), (C.c_double * 3)()
    s, l = scanner_struct(scanner), leg_struct(leg)
    lib().or_pulse_ray(C.byref(s), C.byref(l), int(k), int(seed) & (2 ** 64 - 1), o, d)
    return np.array(o[:]), np.array(d[:])


def subray_dir(scanner, q, s, d):
    out = (C.c_double * 3)()
    sc = scanner_struct(scanner)
    lib().or_subray_dir(C.byref(sc), q, s, _d3(d), out)
    return np.array(out[:])


def beam_width(scanner, R):
    return lib().or_beam_width(C.byref(scanner_struct(scanner)), R)


def subray_intensity(scanner, R, alpha):
    return lib().or_subray_intensity(C.byref(scanner_struct(scanner)), R, alpha)


def pulse_shape(scanner, t_ns):
    return lib().or_pulse_shape(C.byref(scanner_struct(scanner)), t_ns)


def triangle_power(scanner, Is, R, refl, cos_inc):
    return lib().or_triangle_power(C.byref(scanner_struct(scanner)), Is, R, refl, cos_inc)


def echo_width(W, p, sigma_b):
    """Fitted Gaussian sigma (bins) of the echo at bin p of waveform W (Sec. 3.4
    echo width); returns (sigma, near_tie)."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    tie = C.c_int(0)
    s = lib().or_echo_width(W.ctypes.data_as(C.POINTER(C.c_double)), int(W.shape[0]), int(p),
                            float(sigma_b), C.byref(tie))
    return s, bool(tie.value)


def echo_peaks(W, thr_rel=0.05, K=8):
    """Echo bins of waveform W (Sec. 3.4): returns (bins, overflow, near)."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    bins = np.zeros(max(int(K), 1), np.int32)
    ov, near = C.c_int(0), C.c_int(0)
    n = lib().or_echo_peaks(W.ctypes.data_as(C.POINTER(C.c_double)), int(W.shape[0]),
                            float(thr_rel), int(K), bins.ctypes.data_as(C.POINTER(C.c_int32)),
                            C.byref(ov), C.byref(near))
    return bins[:n].copy(), bool(ov.value), bool(near.value)


def echo_object(scanner, P, R, ids, tb_ns):
    """Primitive with the largest contribution at time tb_ns among returns
    (P, R, id) in summation order; returns (id, near_tie)."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    near = C.c_int(0)
    sc = scanner_struct(scanner)
    b = lib().or_echo_object(C.byref(sc), int(P.shape[0]), P.ctypes.data_as(C.POINTER(C.c_double)),
                             R.ctypes.data_as(C.POINTER(C.c_double)),
                             ids.ctypes.data_as(C.POINTER(C.c_int64)), float(tb_ns), C.byref(near))
    return int(b), bool(near.value)


def scan(oscene: OracleScene, scanner, leg, pulses=None, mode=0, seed=0, fixed_window=None,
         threads=0, echo_width=False, force_hit=None):
    """Simulate the given pulse indices of one leg; returns a dict of numpy arrays
    (with ``echo_width``, the fitted echo widths in ns, Gaussian pulses only).

    ``force_hit`` ([n, S] int64, FREE_HIT where the oracle decides) gives
    subray events chosen elsewhere (an FP32 path's choices on flagged subrays);
    ``subray_flags`` in the result holds the flags each subray raised, and
    ``rerun(rows, force_hit, fixed_window)`` repeats the scan for a subset of
    the rows with the same scene, scanner, leg, mode and seed."""
    if pulses is None:
        pulses = np.arange(leg.n_pulses, dtype=np.int64)
    pulses = np.ascontiguousarray(pulses, dtype=np.int64)
    n = pulses.shape[0]
    q = leg.beam_sample_quality if leg.beam_sample_quality >= 0 else scanner.beam_sample_quality
    S = subray_count(q)
    nb, K = scanner.n_bins, scanner.max_echoes
    r = dict(window_bin=np.zeros(n, np.int32), waveform=np.zeros((n, nb)),
             echo_count=np.zeros(n, np.int32), echo_bin=np.zeros((n, K), np.int32),
             echo_amp=np.zeros((n, K)), echo_range=np.zeros((n, K)),
             echo_range_clean=np.zeros((n, K)), echo_object=np.zeros((n, K), np.int64),
             subray_hit=np.zeros((n, S), np.int64), subray_range=np.zeros((n, S)),
             flags=np.zeros(n, np.uint32), subray_flags=np.zeros((n, S), np.uint32),
             echo_object_alt=np.zeros((n, K), np.int64))
    if echo_width:
        r["echo_width"] = np.zeros((n, K))
    out = Out(**{k: _ptr(v) for k, v in r.items()})
    fw = fh = None
    if fixed_window is not None:
        fw = np.ascontiguousarray(fixed_window, dtype=np.int32)
        assert fw.shape == (n,)
    if force_hit is not None:
        fh = np.ascontiguousarray(force_hit, dtype=np.int64)
        assert fh.shape == (n, S)
    s, l = scanner_struct(scanner), leg_struct(leg)
    rc = lib().or_scan(oscene.handle, C.byref(s), C.byref(l), _ptr(pulses), n, int(mode),
                       int(seed) & (2 ** 64 - 1), _ptr(fw), _ptr(fh), C.byref(out), int(threads))
    if rc != 0:
        raise ValueError("oracle scan rejected the scanner (max_echoes outside 1..64)")
    r["pulses"] = pulses
    r["S"] = S
    r["thr_rel"] = float(scanner.echo_threshold_rel)

    def rerun(rows, force_hit=None, fixed_window=None):
        return scan(oscene, scanner, leg, pulses[np.asarray(rows, np.int64)], mode=mode, seed=seed,
                    fixed_window=fixed_window, threads=threads, echo_width=echo_width,
                    force_hit=force_hit)
    r["rerun"] = rerun
    return r


def adjoint(oscene: OracleScene, scanner, leg, pulses, g, window, threads=0):
    """dL/d(reflectance) [n_tri] and dL/d(density) [n_vox] for dL/dW = g (expected mode)."""
    pulses = np.ascontiguousarray(pulses, dtype=np.int64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    window = np.ascontiguousarray(window, dtype=np.int32)
    d_refl = np.zeros(oscene.n_tri)
    d_dens = np.zeros(max(oscene.n_vox, 1))
    s, l = scanner_struct(scanner), leg_struct(leg)
    lib().or_adjoint(oscene.handle, C.byref(s), C.byref(l), _ptr(pulses), pulses.shape[0],
                     _ptr(g), _ptr(window), _ptr(d_refl), _ptr(d_dens), int(threads))
    return d_refl, d_dens[:oscene.n_vox]
