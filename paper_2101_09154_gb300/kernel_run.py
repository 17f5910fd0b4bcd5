"""Run one kernel of the path on a seeded workload, for profiling and timing.

    python -m paper_2101_09154_gb300.kernel_run --workload uls --pulses 200000 \
        --kernel adjoint --repeat 3

Kernels: ``stochastic`` (the scan in stochastic mode), ``expected`` (the
expected-mode scan that the adjoint differentiates) and ``adjoint`` (the
reverse pass, dL/dW from an L2 loss against a scan of perturbed densities).
The forward scans the adjoint needs run before the timed repeats.  Workloads
are the seeded generators of ``scenes`` at their stated sizes, with the leg cut
to ``--pulses`` pulses (centred on the scene as in the full leg).  Prints one
JSON line with the mean device time per call (CUDA events).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _workload(name, pulses):
    import scenes
    if name == "uls":
        return scenes.uls_voxels(n_pulses=pulses) if pulses else scenes.uls_voxels()
    if name == "forest":
        return scenes.voxel_forest(n_pulses=pulses) if pulses else scenes.voxel_forest()
    if name == "als":
        return scenes.als_terrain(n_pulses=pulses) if pulses else scenes.als_terrain()
    if name == "mls":
        w = scenes.urban_mls()
        if pulses:
            w.legs[0].n_pulses = pulses
        return w
    raise ValueError(name)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="uls", choices=["uls", "forest", "als", "mls"])
    ap.add_argument("--pulses", type=int, default=0)
    ap.add_argument("--kernel", default="stochastic", choices=["stochastic", "expected", "adjoint"])
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--block-threads", type=int, default=0, help="0: the library's default")
    ap.add_argument("--rays-per-block", type=int, default=0, help="subrays per work item, 0: the library's default")
    a = ap.parse_args(argv)

    import torch
    import scenes
    import paper_2101_09154_gb300 as hg
    from paper_2101_09154_gb300 import build as _b

    _b.build()
    w = _workload(a.workload, a.pulses)
    gsc = [hg.Scene(s) for s in w.scenes]
    lay = hg.output_layout(w.scanners, w.legs)
    dev = gsc[0].device
    mode = hg.MODE_STOCHASTIC if a.kernel == "stochastic" else hg.MODE_EXPECTED
    out = hg.alloc_outputs(lay, dev, subrays=True)

    def scan():
        hg.scan(gsc, w.scanners, w.legs, mode=mode, out=out, block_threads=a.block_threads,
                rays_per_block=a.rays_per_block)

    fn = scan
    if a.kernel == "adjoint":
        # reference waveform from perturbed densities, then dL/dW = 2 (W - W_ref)
        ref_scenes = []
        for s in w.scenes:
            grids = [scenes.VoxelGrid(**{**g.__dict__, "density": scenes.perturbed_density(g.density, seed=1)})
                     for g in s.grids]
            ref_scenes.append(hg.Scene(scenes.Scene(meshes=s.meshes, grids=grids)))
        out_ref, _ = hg.scan(ref_scenes, w.scanners, w.legs, mode=mode, subrays=False)
        scan()
        gW = 2.0 * (out["waveform"] - out_ref["waveform"])
        del out_ref, ref_scenes
        grads = [{"reflectance": [torch.zeros_like(r) for r in s.reflectance],
                  "density": [torch.zeros_like(d) for d in s.density]} for s in gsc]

        def fn():
            hg.scan_adjoint(gsc, w.scanners, w.legs, gW, out["window_bin"], out["subray_hit"],
                            grads=grads, block_threads=a.block_threads,
                            rays_per_block=a.rays_per_block)
    for _ in range(a.warmup):
        fn()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(a.repeat):
        fn()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(a.repeat, 1)
    print(json.dumps({"workload": w.name, "kernel": a.kernel, "pulses": int(w.n_pulses),
                      "block_threads": a.block_threads, "rays_per_block": a.rays_per_block,
                      "repeat": a.repeat, "ms_per_call": ms,
                      "pulses_per_s": w.n_pulses / (ms / 1e3)}), flush=True)


if __name__ == "__main__":
    main()
