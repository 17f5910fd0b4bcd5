"""GB300 (sm_103a) per-pulse beam-scene interaction: Python binding.

This module only marshals arguments into the C ABI of ``libhelios_gb300.so``
(declared in ``include/helios.h``): every step of the simulation runs in the
library's CUDA kernels.  PyTorch provides device memory and streams.  There is
no CPU fallback: if the library is missing or no CUDA device is present the
calls raise.

Main entry points:
    Scene(scene)                      build the BVH (and, with several voxel grids,
                                      the BVH over their boxes) on the current device
    scan(scenes, scanners, legs, ...) simulate legs -> waveforms, echoes, ...
    scan_to_host(...)                 the same with outputs in page-locked host memory
    scan_static(...)                  the same without any device allocation
    scan_adjoint(...)                 gradients of a waveform loss (per mesh, per grid)
    WaveformFunction                  torch.autograd.Function around both
    lad_table(kind, n)                leaf-angle table G(|cos zenith|) for a voxel grid
    fit.fit_reflectance(...)          adjoint-driven per-triangle reflectance fit

A leg with ``first_pulse = K`` resumes an interrupted scan at pulse K.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

__all__ = ["Scene", "scan", "scan_static", "scan_adjoint", "output_layout", "subray_count", "WaveformFunction",
           "lib", "library_path", "HeliosError"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libhelios_gb300.so")
_lock = threading.Lock()
_lib = None

OK = 0
NO_WINDOW = -(2 ** 31)
MODE_STOCHASTIC, MODE_EXPECTED = 0, 1
# leaf-angle distributions of lad_table (de Wit), codes of HELIOS_LAD_*
LAD_KINDS = {"planophile": 1, "erectophile": 2, "plagiophile": 3, "extremophile": 4,
             "uniform": 5, "spherical": 6}
PF_ECHO_OVERFLOW, PF_TRAVERSAL_CAP, PF_MARCH_CAP, PF_NO_RETURN = 1, 2, 4, 8
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "TIMEOUT", -5: "OVERFLOW",
          -6: "UNSUPPORTED"}


class HeliosError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class MeshDesc(C.Structure):
    _fields_ = [("verts", C.c_void_p), ("n_verts", C.c_int64), ("faces", C.c_void_p),
                ("n_faces", C.c_int64), ("reflectance", C.c_void_p), ("object_id", C.c_int32),
                ("reserved", C.c_int32)]


class VoxelDesc(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("cell", C.c_float), ("dims", C.c_int32 * 3),
                ("G", C.c_float), ("leaf_reflectance", C.c_float), ("object_id", C.c_int32),
                ("opaque", C.c_int32), ("density", C.c_void_p), ("lad_table", C.c_void_p),
                ("lad_n", C.c_int32), ("reserved", C.c_int32)]


class SceneDesc(C.Structure):
    _fields_ = [("meshes", C.POINTER(MeshDesc)), ("n_meshes", C.c_int32), ("n_grids", C.c_int32),
                ("grids", C.POINTER(VoxelDesc))]


class SceneInfo(C.Structure):
    _fields_ = [("n_triangles", C.c_int64), ("n_bvh_nodes", C.c_int64), ("device_bytes", C.c_int64),
                ("n_meshes", C.c_int32), ("n_grids", C.c_int32), ("n_bvh4_nodes", C.c_int64)]


class ScannerDesc(C.Structure):
    _fields_ = [("prf_hz", C.c_double), ("divergence_rad", C.c_double),
                ("beam_sample_quality", C.c_int32), ("pulse_shape", C.c_int32),
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


class LegDesc(C.Structure):
    _fields_ = [("scene_index", C.c_int32), ("scanner_index", C.c_int32), ("platform", C.c_int32),
                ("beam_sample_quality", C.c_int32), ("start", C.c_double * 3), ("end", C.c_double * 3),
                ("speed_mps", C.c_double), ("attitude_rpy", C.c_double * 3), ("t0", C.c_double),
                ("n_pulses", C.c_int64), ("leg_id", C.c_uint32), ("platform_noise_m", C.c_float),
                ("first_pulse", C.c_int64)]


class ScanOpts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("persistent", C.c_int32), ("seed", C.c_uint64),
                ("block_threads", C.c_int32), ("rays_per_block", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("reserved", C.c_int32)]


class Outputs(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("waveform", "window_bin", "echo_count", "echo_range",
                                            "echo_amp", "echo_bin", "echo_object", "pulse_flags",
                                            "subray_hit", "subray_range", "status", "echo_width")]


class Layout(C.Structure):
    _fields_ = [("total_pulses", C.c_int64), ("waveform_floats", C.c_int64),
                ("subray_elems", C.c_int64), ("echo_elems", C.c_int64)]


class FetchCounts(C.Structure):
    _fields_ = [("nodes", C.c_int64), ("triangles", C.c_int64), ("voxels", C.c_int64),
                ("voxel_visits", C.c_int64), ("flags", C.c_int32), ("reserved", C.c_int32)]


class SceneGrads(C.Structure):
    _fields_ = [("d_reflectance", C.POINTER(C.c_void_p)), ("d_density", C.POINTER(C.c_void_p))]


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Load libhelios_gb300.so; raise if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"{_LIB_PATH} is missing: build it with "
                              f"`python -c 'import __graft_entry__ as g; g.build()'`")
        l = C.CDLL(_LIB_PATH)
        st = C.c_int32
        l.helios_build_scene.argtypes = [C.POINTER(SceneDesc), C.c_void_p, C.POINTER(C.c_void_p)]
        l.helios_build_scene.restype = st
        l.helios_free_scene.argtypes = [C.c_void_p]
        l.helios_free_scene.restype = st
        l.helios_scene_get_info.argtypes = [C.c_void_p, C.POINTER(SceneInfo)]
        l.helios_scene_get_info.restype = st
        l.helios_output_layout.argtypes = [C.POINTER(ScannerDesc), C.c_int32, C.POINTER(LegDesc),
                                           C.c_int32] + [C.c_void_p] * 4 + [C.POINTER(Layout)]
        l.helios_output_layout.restype = st
        l.helios_scan_legs.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(ScannerDesc),
                                       C.c_int32, C.POINTER(LegDesc), C.c_int32,
                                       C.POINTER(ScanOpts), C.POINTER(Outputs), C.c_void_p]
        l.helios_scan_legs.restype = st
        l.helios_scan_legs_static.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(ScannerDesc),
                                              C.c_int32, C.POINTER(LegDesc), C.c_int32,
                                              C.POINTER(ScanOpts), C.POINTER(Outputs), C.c_void_p]
        l.helios_scan_legs_static.restype = st
        l.helios_scan_legs_host.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(ScannerDesc),
                                            C.c_int32, C.POINTER(LegDesc), C.c_int32,
                                            C.POINTER(ScanOpts), C.POINTER(Outputs), C.c_int64,
                                            C.c_void_p]
        l.helios_scan_legs_host.restype = st
        l.helios_scan_adjoint.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(ScannerDesc),
                                          C.c_int32, C.POINTER(LegDesc), C.c_int32,
                                          C.POINTER(ScanOpts), C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.POINTER(SceneGrads), C.c_void_p]
        l.helios_scan_adjoint.restype = st
        l.helios_lad_table.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]
        l.helios_lad_table.restype = st
        l.helios_fetch_counts_sample.argtypes = [C.c_void_p, C.POINTER(ScannerDesc), C.POINTER(LegDesc),
                                                 C.c_int32, C.c_uint64, C.c_int64, C.c_int64, C.c_int64,
                                                 C.c_void_p, C.c_void_p]
        l.helios_fetch_counts_sample.restype = st
        l.helios_subray_count.argtypes = [C.c_int32]
        l.helios_subray_count.restype = C.c_int32
        l.helios_last_error.restype = C.c_char_p
        l.helios_version.restype = C.c_char_p
        _lib = l
        return l


def _check(code):
    if code != OK:
        raise HeliosError(code, lib().helios_last_error().decode())


def subray_count(q: int) -> int:
    return int(lib().helios_subray_count(int(q)))


def _torch():
    import torch
    return torch


def lad_table(kind, n=91, device=None, stream=None):
    """Leaf-angle table on the device: G at |cos zenith| = i/(n-1), i < n
    (Eq. extinction), for a distribution name of LAD_KINDS or its code."""
    torch = _torch()
    code = LAD_KINDS[kind] if isinstance(kind, str) else int(kind)
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    out = torch.empty(int(n), dtype=torch.float32, device=dev)
    with torch.cuda.device(dev):
        _check(lib().helios_lad_table(code, int(n), C.c_void_p(out.data_ptr()), _stream_handle(stream)))
    return out


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream_handle(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def scanner_desc(sc) -> ScannerDesc:
    d = ScannerDesc()
    for name, _ in ScannerDesc._fields_:
        if name == "reserved":
            continue
        key = name
        if name == "pulse_shape":
            d.pulse_shape = int(sc.pulse_shape)
            continue
        setattr(d, name, getattr(sc, key))
    return d


def leg_desc(lg) -> LegDesc:
    d = LegDesc()
    d.scene_index = lg.scene_index
    d.scanner_index = lg.scanner_index
    d.platform = lg.platform
    d.beam_sample_quality = lg.beam_sample_quality
    d.start = (C.c_double * 3)(*[float(x) for x in lg.start])
    d.end = (C.c_double * 3)(*[float(x) for x in lg.end])
    d.speed_mps = lg.speed_mps
    d.attitude_rpy = (C.c_double * 3)(*[float(x) for x in lg.attitude_rpy])
    d.t0 = lg.t0
    d.n_pulses = int(lg.n_pulses)
    d.leg_id = int(lg.leg_id)
    d.platform_noise_m = float(lg.platform_noise_m)
    d.first_pulse = int(getattr(lg, "first_pulse", 0))
    return d


class Scene:
    """A scene resident on the current CUDA device: mesh/voxel tensors + the BVH.

    Reflectance and density tensors are referenced by the library (not
    copied), so in-place updates are seen by later scans without a rebuild.
    Grids given the same density array share one device tensor (and so see
    each other's updates); a grid's ``lad`` table (host values or a device
    tensor from ``lad_table``) is copied by the build.
    """

    def __init__(self, scene, device=None, stream=None):
        # the library reads nx*ny*nz densities per grid: check the arrays first
        for i, g in enumerate(scene.grids):
            n = int(np.prod([int(x) for x in g.dims]))
            if np.asarray(g.density).size != n:
                raise ValueError(f"grid {i}: density has {np.asarray(g.density).size} values, dims "
                                 f"{tuple(g.dims)} need {n}")
            lad = getattr(g, "lad", None)
            if lad is not None and not (2 <= int(np.prod(getattr(lad, "shape", (len(lad),)))) <= 65536):
                raise ValueError(f"grid {i}: a leaf-angle table needs 2..65536 entries")
        torch = _torch()
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.verts, self.faces, self.reflectance = [], [], []
        md = (MeshDesc * max(len(scene.meshes), 1))()
        for i, m in enumerate(scene.meshes):
            v = torch.as_tensor(np.ascontiguousarray(m.verts, np.float32)).to(dev)
            f = torch.as_tensor(np.ascontiguousarray(m.faces, np.int32)).to(dev)
            r = torch.as_tensor(np.ascontiguousarray(m.reflectance, np.float32)).to(dev)
            self.verts.append(v)
            self.faces.append(f)
            self.reflectance.append(r)
            md[i].verts = v.data_ptr()
            md[i].n_verts = v.shape[0]
            md[i].faces = f.data_ptr()
            md[i].n_faces = f.shape[0]
            md[i].reflectance = r.data_ptr()
            md[i].object_id = m.object_id
        self.density = []
        lads = []
        shared = {}      # grids that share one density array share its device copy
        gd = (VoxelDesc * max(len(scene.grids), 1))()
        for i, g in enumerate(scene.grids):
            key = id(g.density)
            if key not in shared:
                shared[key] = (g.density, torch.as_tensor(np.ascontiguousarray(g.density, np.float32)).to(dev))
            dens = shared[key][1]
            self.density.append(dens)
            lad = getattr(g, "lad", None)
            if lad is not None:
                # a device tensor (lad_table()) or host values; copied by the build
                lt = (lad.to(dev, torch.float32).contiguous() if torch.is_tensor(lad)
                      else torch.as_tensor(np.ascontiguousarray(lad, np.float32)).to(dev))
                lads.append(lt)
                gd[i].lad_table = lt.data_ptr()
                gd[i].lad_n = lt.numel()
            gd[i].origin = (C.c_float * 3)(*[float(x) for x in g.origin])
            gd[i].cell = float(g.cell)
            gd[i].dims = (C.c_int32 * 3)(*[int(x) for x in g.dims])
            gd[i].G = float(g.G)
            gd[i].leaf_reflectance = float(g.leaf_reflectance)
            gd[i].object_id = g.object_id
            gd[i].opaque = int(g.opaque)
            gd[i].density = dens.data_ptr()
        self._md, self._gd = md, gd
        desc = SceneDesc()
        desc.meshes = C.cast(md, C.POINTER(MeshDesc))
        desc.n_meshes = len(scene.meshes)
        desc.grids = C.cast(gd, C.POINTER(VoxelDesc))
        desc.n_grids = len(scene.grids)
        self.n_triangles = int(sum(f.shape[0] for f in self.faces))
        self.n_voxels = int(sum(d.numel() for d in self.density))
        h = C.c_void_p()
        with torch.cuda.device(dev):
            _check(lib().helios_build_scene(C.byref(desc), _stream_handle(stream), C.byref(h)))
        del lads
        self.handle = h

    def parameters(self) -> list:
        """The differentiable tensors: every mesh's reflectance, then every
        distinct density tensor (grids sharing an array appear once)."""
        seen, dens = set(), []
        for d in self.density:
            if id(d) not in seen:
                seen.add(id(d))
                dens.append(d)
        return list(self.reflectance) + dens

    def info(self) -> dict:
        i = SceneInfo()
        _check(lib().helios_scene_get_info(self.handle, C.byref(i)))
        return {k: getattr(i, k) for k, _ in SceneInfo._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib().helios_free_scene(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def output_layout(scanners, legs):
    n = len(legs)
    sd = (ScannerDesc * len(scanners))(*[scanner_desc(s) for s in scanners])
    ld = (LegDesc * max(n, 1))(*[leg_desc(l) for l in legs])
    offs = [np.zeros(max(n, 1), np.int64) for _ in range(4)]
    tot = Layout()
    _check(lib().helios_output_layout(sd, len(scanners), ld, n,
                                      *[o.ctypes.data_as(C.c_void_p) for o in offs], C.byref(tot)))
    return {"pulse_offset": offs[0][:n], "wave_offset": offs[1][:n], "subray_offset": offs[2][:n],
            "echo_offset": offs[3][:n], "total_pulses": tot.total_pulses,
            "waveform_floats": tot.waveform_floats, "subray_elems": tot.subray_elems,
            "echo_elems": tot.echo_elems}


def alloc_outputs(layout, device, subrays=True, status=True, echo_width=False):
    torch = _torch()
    P = int(layout["total_pulses"])
    out = {
        "waveform": torch.empty(int(layout["waveform_floats"]), dtype=torch.float32, device=device),
        "window_bin": torch.empty(P, dtype=torch.int32, device=device),
        "echo_count": torch.empty(P, dtype=torch.int32, device=device),
        "echo_range": torch.empty(int(layout["echo_elems"]), dtype=torch.float32, device=device),
        "echo_amp": torch.empty(int(layout["echo_elems"]), dtype=torch.float32, device=device),
        "echo_bin": torch.empty(int(layout["echo_elems"]), dtype=torch.int32, device=device),
        "echo_object": torch.empty(int(layout["echo_elems"]), dtype=torch.int64, device=device),
        "pulse_flags": torch.empty(P, dtype=torch.uint8, device=device),
    }
    if subrays:
        out["subray_hit"] = torch.empty(int(layout["subray_elems"]), dtype=torch.int64, device=device)
        out["subray_range"] = torch.empty(int(layout["subray_elems"]), dtype=torch.float32, device=device)
    if status:
        out["status"] = torch.zeros(1, dtype=torch.int32, device=device)
    if echo_width:
        out["echo_width"] = torch.empty(int(layout["echo_elems"]), dtype=torch.float32, device=device)
    return out


def alloc_host_outputs(layout, device, subrays=False, status=True, echo_width=False):
    """Page-locked host tensors for ``scan_to_host`` (``status`` stays on the device)."""
    torch = _torch()
    dev = alloc_outputs({"total_pulses": 0, "waveform_floats": 0, "echo_elems": 0, "subray_elems": 0},
                        "cpu", subrays=subrays, status=False, echo_width=echo_width)
    P = int(layout["total_pulses"])
    sizes = {"waveform": layout["waveform_floats"], "window_bin": P, "echo_count": P,
             "echo_range": layout["echo_elems"], "echo_amp": layout["echo_elems"],
             "echo_bin": layout["echo_elems"], "echo_object": layout["echo_elems"], "pulse_flags": P,
             "subray_hit": layout["subray_elems"], "subray_range": layout["subray_elems"],
             "echo_width": layout["echo_elems"]}
    out = {k: torch.empty(int(sizes[k]), dtype=t.dtype, pin_memory=True) for k, t in dev.items()}
    if status:
        out["status"] = torch.zeros(1, dtype=torch.int32, device=device)
    return out


def _outputs_struct(out) -> Outputs:
    o = Outputs()
    for name, _ in Outputs._fields_:
        t = out.get(name)
        setattr(o, name, t.data_ptr() if t is not None else None)
    return o


def _as_list(x):
    return list(x) if isinstance(x, (list, tuple)) else [x]


def scan(scenes, scanners, legs, mode=MODE_STOCHASTIC, seed=0, persistent=False, out=None,
         subrays=True, stream=None, block_threads=0, rays_per_block=0, blocks_per_sm=0,
         echo_width=False):
    """Run helios_scan_legs; returns (outputs dict of device tensors, layout).
    ``echo_width`` adds the fitted echo widths (an optional, costed output)."""
    scenes, scanners, legs = _as_list(scenes), _as_list(scanners), _as_list(legs)
    layout = output_layout(scanners, legs)
    dev = scenes[0].device
    if out is None:
        out = alloc_outputs(layout, dev, subrays=subrays, echo_width=echo_width)
    sh = (C.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    sd = (ScannerDesc * len(scanners))(*[scanner_desc(s) for s in scanners])
    ld = (LegDesc * max(len(legs), 1))(*[leg_desc(l) for l in legs])
    opts = ScanOpts(mode=int(mode), persistent=int(bool(persistent)), seed=int(seed) & (2 ** 64 - 1),
                    block_threads=int(block_threads), rays_per_block=int(rays_per_block),
                    blocks_per_sm=int(blocks_per_sm))
    o = _outputs_struct(out)
    _check(lib().helios_scan_legs(sh, len(scenes), sd, len(scanners), ld, len(legs), C.byref(opts),
                                  C.byref(o), _stream_handle(stream)))
    return out, layout


def scan_to_host(scenes, scanners, legs, mode=MODE_STOCHASTIC, seed=0, persistent=False,
                 host_out=None, subrays=False, chunk_pulses=1 << 18, stream=None, block_threads=0,
                 rays_per_block=0, blocks_per_sm=0):
    """helios_scan_legs_host: the scan with its outputs in (page-locked) host memory.

    Chunks of about ``chunk_pulses`` pulses are scanned into device staging
    buffers while the previous chunk is copied to the host on a second
    stream.  Returns (host outputs dict, layout); the host tensors are
    complete once ``stream`` (default: the current stream) is synchronised.
    """
    scenes, scanners, legs = _as_list(scenes), _as_list(scanners), _as_list(legs)
    layout = output_layout(scanners, legs)
    if host_out is None:
        host_out = alloc_host_outputs(layout, scenes[0].device, subrays=subrays)
    sh = (C.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    sd = (ScannerDesc * len(scanners))(*[scanner_desc(s) for s in scanners])
    ld = (LegDesc * max(len(legs), 1))(*[leg_desc(l) for l in legs])
    opts = ScanOpts(mode=int(mode), persistent=int(bool(persistent)), seed=int(seed) & (2 ** 64 - 1),
                    block_threads=int(block_threads), rays_per_block=int(rays_per_block),
                    blocks_per_sm=int(blocks_per_sm))
    o = _outputs_struct(host_out)
    _check(lib().helios_scan_legs_host(sh, len(scenes), sd, len(scanners), ld, len(legs), C.byref(opts),
                                       C.byref(o), int(chunk_pulses), _stream_handle(stream)))
    return host_out, layout


def scan_static(scenes, scanners, legs, mode=MODE_STOCHASTIC, seed=0, out=None, subrays=True,
                stream=None, block_threads=0, rays_per_block=0, blocks_per_sm=0, echo_width=False):
    """helios_scan_legs_static: the persistent scan with no device allocation.

    For callers that cannot allocate device memory mid-scan (another
    allocator owns the budget, a graph capture into a pool they do not
    control, real-time loops).  The work-queue counters live in a static
    device array shared by all calls, so calls must not overlap on the GPU;
    at most 2048 legs per call.  Outputs are those of ``scan``; ``echo_width``
    adds the fitted echo widths (read back from the stored echo bins).
    """
    scenes, scanners, legs = _as_list(scenes), _as_list(scanners), _as_list(legs)
    layout = output_layout(scanners, legs)
    if out is None:
        out = alloc_outputs(layout, scenes[0].device, subrays=subrays, echo_width=echo_width)
    sh = (C.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    sd = (ScannerDesc * len(scanners))(*[scanner_desc(s) for s in scanners])
    ld = (LegDesc * max(len(legs), 1))(*[leg_desc(l) for l in legs])
    opts = ScanOpts(mode=int(mode), persistent=1, seed=int(seed) & (2 ** 64 - 1),
                    block_threads=int(block_threads), rays_per_block=int(rays_per_block),
                    blocks_per_sm=int(blocks_per_sm))
    o = _outputs_struct(out)
    _check(lib().helios_scan_legs_static(sh, len(scenes), sd, len(scanners), ld, len(legs),
                                         C.byref(opts), C.byref(o), _stream_handle(stream)))
    return out, layout


def scan_adjoint(scenes, scanners, legs, d_waveform, window_bin, subray_hit=None, grads=None,
                 stream=None, block_threads=0, rays_per_block=0):
    """Accumulate dL/d(reflectance), dL/d(density) for dL/dW = d_waveform (expected mode).

    Returns a list (one per scene) of dicts {"reflectance": [...], "density": [...]}.
    """
    torch = _torch()
    if subray_hit is not None and subray_hit.dtype != torch.int64:
        raise TypeError("subray_hit must be the forward's int64 primitive ids")
    scenes, scanners, legs = _as_list(scenes), _as_list(scanners), _as_list(legs)
    if grads is None:
        grads = [{"reflectance": [torch.zeros_like(r) for r in s.reflectance],
                  "density": [torch.zeros_like(d) for d in s.density]} for s in scenes]
    gs = (SceneGrads * len(scenes))()
    keep = []
    for i, g in enumerate(grads):
        rp = (C.c_void_p * max(len(g["reflectance"]), 1))(*[t.data_ptr() if t is not None else None
                                                            for t in g["reflectance"]])
        dp = (C.c_void_p * max(len(g["density"]), 1))(*[t.data_ptr() if t is not None else None
                                                        for t in g["density"]])
        keep += [rp, dp]
        gs[i].d_reflectance = C.cast(rp, C.POINTER(C.c_void_p))
        gs[i].d_density = C.cast(dp, C.POINTER(C.c_void_p))
    sh = (C.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    sd = (ScannerDesc * len(scanners))(*[scanner_desc(s) for s in scanners])
    ld = (LegDesc * max(len(legs), 1))(*[leg_desc(l) for l in legs])
    opts = ScanOpts(mode=MODE_EXPECTED, block_threads=int(block_threads), rays_per_block=int(rays_per_block))
    d_waveform = d_waveform.contiguous()
    _check(lib().helios_scan_adjoint(sh, len(scenes), sd, len(scanners), ld, len(legs),
                                     C.byref(opts), _ptr(d_waveform), _ptr(window_bin),
                                     _ptr(subray_hit), gs, _stream_handle(stream)))
    return grads


# helios_fetch_counts: bytes of one fetch of each kind, and the flag bits
NODE4_BYTES, TRIANGLE_BYTES, VOXEL_BYTES = 128, 48, 4
FC_STACK, FC_LIST_OVERFLOW, FC_SET_FULL, FC_MARCH_CAP = 0x01, 0x02, 0x04, 0x08


def fetch_counts(scene, scanner, leg, mode=MODE_STOCHASTIC, seed=0, first=0, stride=1, count=None,
                 stream=None):
    """What pulses first + i * stride of one leg need from memory, each as a
    union over its subrays (helios_fetch_counts_sample): a dict of int64
    tensors on the scene's device, keys nodes, triangles, voxels,
    voxel_visits and flags (FC_* bits).  count defaults to every such pulse
    of the leg."""
    torch = _torch()
    if count is None:
        count = max(0, -(-(int(leg.n_pulses) - int(first)) // int(stride)))
    assert C.sizeof(FetchCounts) == 5 * 8       # one row of five int64 per pulse
    raw = torch.zeros((int(count), 5), dtype=torch.int64, device=scene.device)
    with torch.cuda.device(scene.device):
        _check(lib().helios_fetch_counts_sample(scene.handle, C.byref(scanner_desc(scanner)),
                                                C.byref(leg_desc(leg)), int(mode),
                                                int(seed) & (2 ** 64 - 1), int(first), int(stride),
                                                int(count), _ptr(raw), _stream_handle(stream)))
    return {"nodes": raw[:, 0], "triangles": raw[:, 1], "voxels": raw[:, 2],
            "voxel_visits": raw[:, 3], "flags": raw[:, 4] & 0xFFFFFFFF}


def fetch_bytes(counts):
    """Scene bytes per pulse of fetch_counts: 128 per 4-wide node, 48 per
    triangle, 4 per voxel (an int64 tensor)."""
    return (NODE4_BYTES * counts["nodes"] + TRIANGLE_BYTES * counts["triangles"]
            + VOXEL_BYTES * counts["voxels"])


class WaveformFunction:
    """Differentiable expected-mode waveform: W = scan(reflectances, densities).

    ``apply(scene, scanners, legs, *tensors)`` returns the flat waveform tensor
    of the legs (one scene).  ``tensors`` are tensors the scene references:
    any of ``scene.reflectance`` (one per mesh) and ``scene.density`` (one per
    distinct density array; grids built from the same array share it); by
    default all of them (``scene.parameters()``).  The kernels read their
    current values, and the gradient of every one of them comes back from the
    hand-written adjoint kernel: a density tensor shared by several grids
    receives the sum of their gradients.  ``scanners`` and ``legs`` may be
    single objects or lists.
    """

    @staticmethod
    def apply(scene, scanners, legs, *tensors):
        torch = _torch()
        scanners, legs = _as_list(scanners), _as_list(legs)
        if not tensors:
            tensors = tuple(scene.parameters())
        routes = []
        for t in tensors:
            r_idx = [i for i, r in enumerate(scene.reflectance) if r is t]
            d_idx = [j for j, d in enumerate(scene.density) if d is t]
            if not r_idx and not d_idx:
                raise ValueError("WaveformFunction: a tensor that the scene does not reference")
            routes.append((r_idx, d_idx))

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, *ts):
                out, _ = scan([scene], scanners, legs, mode=MODE_EXPECTED, subrays=True)
                ctx.save_for_backward(out["window_bin"], out["subray_hit"])
                return out["waveform"]

            @staticmethod
            def backward(ctx, gW):
                window, hits = ctx.saved_tensors
                g = scan_adjoint([scene], scanners, legs, gW.contiguous(), window, hits)[0]
                res = []
                for r_idx, d_idx in routes:
                    parts = [g["reflectance"][i] for i in r_idx] + [g["density"][j] for j in d_idx]
                    acc = parts[0]
                    for q in parts[1:]:
                        acc = acc + q
                    res.append(acc)
                return tuple(res)

        return _Fn.apply(*tensors)
