"""The C-ABI library loads and exports every function include/helios.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "helios.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(helios_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    import paper_2101_09154_gb300 as hg
    return hg.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("helios_build_scene", "helios_scan_legs", "helios_scan_adjoint",
                     "helios_free_scene", "helios_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    import paper_2101_09154_gb300 as hg
    import scenes
    assert [hg.subray_count(q) for q in range(4)] == [1, 7, 19, 37]
    assert hg.subray_count(-1) == -1
    assert lib.helios_version().startswith(b"helios_gb300")
    w = scenes.batched_legs(n_legs=5, tile=16, block=8, n_terrain=1, n_voxel=1,
                            min_pulses=100, max_pulses=1000)
    lay = hg.output_layout(w.scanners, w.legs)
    S = [hg.subray_count(l.beam_sample_quality) for l in w.legs]
    n = [l.n_pulses for l in w.legs]
    assert lay["total_pulses"] == sum(n)
    assert list(lay["pulse_offset"]) == [sum(n[:i]) for i in range(5)]
    assert list(lay["subray_offset"]) == [sum(a * b for a, b in zip(n[:i], S[:i])) for i in range(5)]
    nb = [w.scanners[l.scanner_index].n_bins for l in w.legs]
    assert list(lay["wave_offset"]) == [sum(a * b for a, b in zip(n[:i], nb[:i])) for i in range(5)]


def test_invalid_arguments_return_codes_without_a_gpu(lib):
    import paper_2101_09154_gb300 as hg
    import scenes
    sc = scenes.Scanner(n_bins=2)          # below the 4-bin minimum
    leg = scenes.Leg(n_pulses=10)
    with pytest.raises(hg.HeliosError) as e:
        hg.output_layout([sc], [leg])
    assert e.value.code == -1 and "n_bins" in str(e.value)
    sc = scenes.Scanner(beam_sample_quality=12)
    with pytest.raises(hg.HeliosError):
        hg.output_layout([sc], [leg])
    sc = scenes.Scanner()
    with pytest.raises(hg.HeliosError):
        hg.output_layout([sc], [scenes.Leg(scanner_index=3, n_pulses=1)])
    # NULL scene list is rejected before anything touches a device
    opts = hg.ScanOpts()
    outs = hg.Outputs()
    code = lib.helios_scan_legs(None, 0, None, 0, None, 0, ctypes.byref(opts), ctypes.byref(outs), None)
    assert code == -1
    assert b"n_scenes" in lib.helios_last_error()
    code = lib.helios_scan_legs_host(None, 0, None, 0, None, 0, ctypes.byref(opts), ctypes.byref(outs),
                                     1024, None)
    assert code == -1
    assert b"n_scenes" in lib.helios_last_error()
    # fetch counts: a NULL scene or a sample outside the leg is refused on the host
    sd, ld = hg.scanner_desc(scenes.Scanner()), hg.leg_desc(scenes.Leg(n_pulses=10))
    assert lib.helios_fetch_counts_sample(None, ctypes.byref(sd), ctypes.byref(ld), 0, 0, 0, 1, 4,
                                          ctypes.c_void_p(16), None) == -1
    assert b"NULL" in lib.helios_last_error()
    assert lib.helios_fetch_counts_sample(ctypes.c_void_p(16), ctypes.byref(sd), ctypes.byref(ld), 0, 0,
                                          4, 3, 3, ctypes.c_void_p(16), None) == -1
    assert b"inside the leg" in lib.helios_last_error()
    assert lib.helios_fetch_counts_sample(ctypes.c_void_p(16), ctypes.byref(sd), ctypes.byref(ld), 0, 0,
                                          0, 0, 3, ctypes.c_void_p(16), None) == -1
    # leaf-angle tables: bad requests are refused before any launch
    assert lib.helios_lad_table(0, 91, ctypes.c_void_p(16), None) == -1
    assert lib.helios_lad_table(7, 91, ctypes.c_void_p(16), None) == -1
    assert lib.helios_lad_table(2, 1, ctypes.c_void_p(16), None) == -1
    assert lib.helios_lad_table(2, 65537, ctypes.c_void_p(16), None) == -1
    assert lib.helios_lad_table(2, 91, None, None) == -1
    assert b"NULL" in lib.helios_last_error()


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors have the C structs' sizes and field offsets."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    import paper_2101_09154_gb300 as hg
    structs = {"helios_voxel_desc": hg.VoxelDesc, "helios_mesh_desc": hg.MeshDesc,
               "helios_scanner_desc": hg.ScannerDesc, "helios_leg_desc": hg.LegDesc,
               "helios_outputs": hg.Outputs, "helios_scan_opts": hg.ScanOpts,
               "helios_fetch_counts": hg.FetchCounts, "helios_scene_info": hg.SceneInfo}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "helios.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for line in filter(None, out):
        cname, field, val = line.split()
        py = structs[cname]
        got = ctypes.sizeof(py) if field == "size" else getattr(py, field).offset
        assert got == int(val), (cname, field, got, int(val))


def test_scene_build_rejects_overlapping_grids_before_any_device_call(lib):
    """Grid boxes must have disjoint interiors (touching is fine) and hold fewer
    than 2^40 voxels in all; the checks run on the host before anything
    touches a device (the density pointers here are never dereferenced)."""
    import paper_2101_09154_gb300 as hg

    def grid(x0, n=4, cell=0.5):
        g = hg.VoxelDesc()
        g.origin = (ctypes.c_float * 3)(x0, 0.0, 0.0)
        g.cell = cell
        g.dims = (ctypes.c_int32 * 3)(n, n, n)
        g.G = 0.5
        g.leaf_reflectance = 0.5
        g.density = 16
        return g

    for xs, ok in (((0.0, 1.5), False), ((0.0, 2.0, 4.0, 1.9), False)):
        gd = (hg.VoxelDesc * len(xs))(*[grid(x) for x in xs])
        desc = hg.SceneDesc()
        desc.n_meshes = 0
        desc.n_grids = len(xs)
        desc.grids = ctypes.cast(gd, ctypes.POINTER(hg.VoxelDesc))
        h = ctypes.c_void_p()
        code = lib.helios_build_scene(ctypes.byref(desc), None, ctypes.byref(h))
        assert code == -1 and b"overlap" in lib.helios_last_error()
    # more than 2^40 - 1 voxels in all (the draws' counter holds 40 bits of voxel id):
    # 513 grids of 1024 x 1024 x 2047 voxels, each below the per-grid 2^31 limit
    gd = (hg.VoxelDesc * 513)(*[grid(3000.0 * i, 1024, 1.0) for i in range(513)])
    for g in gd:
        g.dims = (ctypes.c_int32 * 3)(1024, 1024, 2047)
    desc = hg.SceneDesc()
    desc.n_meshes = 0
    desc.n_grids = 513
    desc.grids = ctypes.cast(gd, ctypes.POINTER(hg.VoxelDesc))
    h = ctypes.c_void_p()
    assert lib.helios_build_scene(ctypes.byref(desc), None, ctypes.byref(h)) == -6
    assert b"2^40" in lib.helios_last_error()
    # too many grids
    desc = hg.SceneDesc()
    desc.n_grids = 4097
    gd = (hg.VoxelDesc * 1)()
    desc.grids = ctypes.cast(gd, ctypes.POINTER(hg.VoxelDesc))
    h = ctypes.c_void_p()
    assert lib.helios_build_scene(ctypes.byref(desc), None, ctypes.byref(h)) == -6


def test_scene_build_takes_rounding_thin_overlaps_as_touching(lib):
    """Boxes whose FP32 corners overlap by rounding (1e-7 of their size) pass
    the host check; what happens next needs a device (no-device builds stop
    with a CUDA error)."""
    import paper_2101_09154_gb300 as hg
    gd = (hg.VoxelDesc * 2)()
    for i, x0 in enumerate((0.0, 1.9999998)):
        gd[i].origin = (ctypes.c_float * 3)(x0, 0.0, 0.0)
        gd[i].cell = 0.5
        gd[i].dims = (ctypes.c_int32 * 3)(4, 4, 4)
        gd[i].G = 0.5
        gd[i].density = 16
    desc = hg.SceneDesc()
    desc.n_grids = 2
    desc.grids = ctypes.cast(gd, ctypes.POINTER(hg.VoxelDesc))
    h = ctypes.c_void_p()
    code = lib.helios_build_scene(ctypes.byref(desc), None, ctypes.byref(h))
    assert b"overlap" not in lib.helios_last_error()
    assert code in (0, -3)
    if code == 0:
        lib.helios_free_scene(h)


def test_host_side_fault_injection(lib, monkeypatch):
    """HELIOS_FAULT=badarg fails every call at entry; HELIOS_FAULT=oom fails a
    call where it would first allocate device memory (the scene build's first
    buffer here: no device is touched before it)."""
    import paper_2101_09154_gb300 as hg
    import scenes
    sc, leg = scenes.Scanner(), scenes.Leg(n_pulses=10)
    monkeypatch.setenv("HELIOS_FAULT", "badarg")
    with pytest.raises(hg.HeliosError) as e:
        hg.output_layout([sc], [leg])
    assert e.value.code == -1 and "injected" in str(e.value)
    monkeypatch.setenv("HELIOS_FAULT", "oom")
    assert hg.output_layout([sc], [leg])["total_pulses"] == 10     # allocates nothing
    verts = (ctypes.c_float * 9)(0, 0, 0, 1, 0, 0, 0, 1, 0)
    m = hg.MeshDesc()
    m.verts = ctypes.cast(verts, ctypes.c_void_p)     # never read before the failing allocation
    m.n_verts = 3
    m.faces = 16
    m.n_faces = 2
    m.reflectance = 16
    md = (hg.MeshDesc * 1)(m)
    desc = hg.SceneDesc()
    desc.meshes = ctypes.cast(md, ctypes.POINTER(hg.MeshDesc))
    desc.n_meshes = 1
    h = ctypes.c_void_p()
    assert lib.helios_build_scene(ctypes.byref(desc), None, ctypes.byref(h)) == -2
    assert b"memory" in lib.helios_last_error().lower()
    monkeypatch.delenv("HELIOS_FAULT")


def test_first_pulse_resume_layout_and_validation(lib):
    """A resumed leg (first_pulse = K) has n_pulses rows like any other; a
    negative first_pulse, or one whose last pulse reaches 2^44, is refused."""
    import paper_2101_09154_gb300 as hg
    import scenes
    sc = scenes.Scanner(n_bins=64)
    a = hg.output_layout([sc], [scenes.Leg(n_pulses=100), scenes.Leg(n_pulses=50, leg_id=1)])
    b = hg.output_layout([sc], [scenes.Leg(n_pulses=100, first_pulse=12345),
                                scenes.Leg(n_pulses=50, leg_id=1, first_pulse=7)])
    for k in ("pulse_offset", "wave_offset", "subray_offset", "echo_offset"):
        assert list(a[k]) == list(b[k])
    assert a["total_pulses"] == b["total_pulses"] == 150
    with pytest.raises(hg.HeliosError) as e:
        hg.output_layout([sc], [scenes.Leg(n_pulses=5, first_pulse=-1)])
    assert e.value.code == -1 and "first_pulse" in str(e.value)
    # the draws' counter holds pulse indices below 2^44
    hg.output_layout([sc], [scenes.Leg(n_pulses=5, first_pulse=2 ** 44 - 5)])
    with pytest.raises(hg.HeliosError) as e:
        hg.output_layout([sc], [scenes.Leg(n_pulses=5, first_pulse=2 ** 44 - 4)])
    assert e.value.code == -1 and "2^44" in str(e.value)


def test_scene_wrapper_checks_density_sizes_before_any_upload():
    import numpy as np
    import paper_2101_09154_gb300 as hg
    import scenes
    g = scenes.VoxelGrid(origin=(0, 0, 0), cell=1.0, dims=(4, 4, 4), density=np.zeros((4, 4, 3), np.float32))
    with pytest.raises(ValueError, match="need 64"):
        hg.Scene(scenes.Scene(meshes=[], grids=[g]))
    g = scenes.VoxelGrid(origin=(0, 0, 0), cell=1.0, dims=(2, 2, 2), density=np.zeros((2, 2, 2), np.float32),
                         lad=np.ones(1, np.float32))
    with pytest.raises(ValueError, match="2..65536"):
        hg.Scene(scenes.Scene(meshes=[], grids=[g]))
