"""Benchmark: simulated pulses per second of the fused GB300 pulse kernel.

Default workload (N=1): seeded ALS over terrain -- 1024^2 fBm DTM at 1 m plus
300 procedural trees (3.03 M triangles), 4 M pulses, 19 subrays per pulse,
512-bin full waveform, echoes, range noise.  One step = one helios_scan_legs
call over the whole leg (pulse pose -> subrays -> BVH -> power -> waveform ->
echoes).  The scene (BVH 0.35 GB) and the step's outputs (8.7 GB) are both
larger than the 129 MB L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
(the reference arm) on a bounded sample of the same workload instead.
Multi-GPU (torchrun, --gpus N): the leg does not shard here, so each rank runs
an independent replica (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="als", choices=["als", "uls", "tls", "batched", "mls"])
    p.add_argument("--no-extras", action="store_true", help="skip adjoint ratio, e2e and CPU baseline")
    p.add_argument("--cpu-sample-s", type=float, default=15.0, help="target seconds of oracle work")
    p.add_argument("--small", action="store_true", help="tiny sizes (tests only)")
    p.add_argument("--pulses", type=int, default=0, help="override the leg's pulse count (profiling)")
    return p.parse_args()


# --------------------------------------------------------------------------
# distributed plumbing (barrier + max over ranks only)
# --------------------------------------------------------------------------
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
def workload(name, small=False):
    import scenes
    if name == "als":
        if small:
            return scenes.als_terrain(size=128, n_trees=8, n_pulses=20000, agl=120.0)
        return scenes.als_terrain()
    if name == "uls":
        if small:
            return scenes.uls_voxels(n=48, n_pulses=20000, agl=12.0, speed=1.0, prf=2000.0)
        return scenes.uls_voxels()
    if name == "tls":
        return scenes.tls_tiny()
    if name == "mls":
        if small:
            return scenes.urban_mls(length=30.0, facade_cell=0.5)
        return scenes.urban_mls()
    if small:
        return scenes.batched_legs(n_legs=8, tile=64, block=24, n_terrain=2, n_voxel=2,
                                   min_pulses=1000, max_pulses=20000)
    return scenes.batched_legs()


def workload_config(w, name, subray_count, world=1):
    """The workload's description, the same for both arms (each passes its own
    subray-count function: the library's, or the oracle's for the reference arm)."""
    sc = w.scanners[0]
    S = [subray_count(l.beam_sample_quality if l.beam_sample_quality >= 0
                      else w.scanners[l.scanner_index].beam_sample_quality) for l in w.legs]
    return {"workload": w.name, "description": w.note, "pulses": w.n_pulses,
            "subrays_per_pulse": S[0] if len(set(S)) == 1 else "mixed",
            "triangles": int(sum(s.n_triangles for s in w.scenes)),
            "voxels": int(sum(int(np.prod(g.dims)) for s in w.scenes for g in s.grids)),
            "n_bins": sc.n_bins, "legs": len(w.legs),
            "l2": "inputs larger than L2 (BVH + triangles > 129 MB, outputs > 1 GB); no flush",
            "parallelism": f"replicas x{world}"}


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# roofline helpers
# --------------------------------------------------------------------------
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("hg_device.cuh", "scan.cu"):
        with open(os.path.join(ROOT, "paper_2101_09154_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload_name, pulses):
    """DRAM bytes per launch from the committed ncu summary, if it is for this kernel source."""
    p = os.path.join(ROOT, "profiles", "scan_kernel_als_terrain.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m_src = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", txt)
    m_b = re.search(r"dram_bytes_per_pulse:\s*([0-9.eE+]+)", txt)
    if not m_src or not m_b or m_src.group(1) != kernel_source_hash():
        return None
    return float(m_b.group(1)) * pulses


def output_bytes(layout, subray_outputs=False):
    """Bytes one scan launch writes: waveform rows, window, count, flags and K
    echo slots (range, amplitude, bin, 8-byte object) per pulse."""
    P = layout["total_pulses"]
    out = layout["waveform_floats"] * 4 + P * (4 + 4 + 1) + layout["echo_elems"] * (4 + 4 + 4 + 8)
    if subray_outputs:
        out += layout["subray_elems"] * 12
    return int(out)


def scene_bytes_once(w):
    """Every scene byte read once: BVH nodes, packed triangles, reflectance, voxels."""
    scene = 0
    for s in w.scenes:
        n = s.n_triangles
        scene += max(n - 1, 0) * 64 + n * 48 + n * 4
        # grids that share one density array read it once
        scene += sum(int(np.prod(g.dims)) * 4 for g in {id(g.density): g for g in s.grids}.values())
    return int(scene)


def algorithmic_bytes(w, layout, subray_outputs=False):
    """Compulsory traffic of one scan launch: every output byte written once,
    every scene byte read once."""
    return output_bytes(layout, subray_outputs) + scene_bytes_once(w)


def fetch_model(hg, w, gsc, mode, seed, per_leg=65536):
    """What the pulses need from memory (helios_fetch_counts_sample on an
    evenly spaced sample of at most per_leg pulses of each leg): means per
    pulse, weighted by the legs' pulse counts, of the 4-wide nodes (128 B),
    triangles (48 B) and distinct voxels (4 B) of each pulse's subrays, and
    the resulting scene bytes per pulse."""
    import torch
    keys = ("nodes", "triangles", "voxels", "voxel_visits")
    acc = {k: 0.0 for k in keys}
    acc["fetch_bytes"] = 0.0
    P = sampled = flagged = 0
    for l in w.legs:
        if l.n_pulses == 0:
            continue
        stride = max(1, -(-l.n_pulses // per_leg))
        count = -(-l.n_pulses // stride)
        c = hg.fetch_counts(gsc[l.scene_index], w.scanners[l.scanner_index], l, mode=mode, seed=seed,
                            first=0, stride=stride, count=count)
        fb = hg.fetch_bytes(c)
        for k in keys:
            acc[k] += float(c[k].double().mean()) * l.n_pulses
        acc["fetch_bytes"] += float(fb.double().mean()) * l.n_pulses
        flagged += int((c["flags"] != 0).sum())
        P += l.n_pulses
        sampled += count
    torch.cuda.synchronize()
    res = {k: v / max(P, 1) for k, v in acc.items()}
    res.update(sampled_pulses=sampled, flagged_pulses=flagged,
               coherence=res["voxel_visits"] / res["voxels"] if res["voxels"] > 0 else None)
    return res


BYTES_MODEL = ("per pulse: its output row (waveform 4*N_b, window, count, flags, K echo slots of "
               "20 B) written once, plus what it needs from the scene as a union over its subrays, "
               "counted by helios_fetch_counts_sample on a sample of the leg: 128 B per 4-wide BVH "
               "node the beam cone enters, 48 B per triangle whose box the cone overlaps (each read "
               "once per pulse however many subrays test it), 4 B per distinct voxel the subrays "
               "march through; reuse across pulses (L1/L2) is not subtracted")


# --------------------------------------------------------------------------
# the GPU arm
# --------------------------------------------------------------------------
def run_ours(args, D):
    import torch
    import paper_2101_09154_gb300 as hg
    from paper_2101_09154_gb300 import build as _b

    _b.build()
    assert torch.cuda.is_available(), "bench.py needs a CUDA device for --impl ours"
    torch.cuda.set_device(D.local)
    dev = torch.device("cuda", D.local)
    w = workload(args.workload, args.small)
    if args.pulses > 0:
        for l in w.legs:
            l.n_pulses = args.pulses
        w.name += f"_first{args.pulses}p"
    t0 = time.time()
    gsc = [hg.Scene(s, device=dev) for s in w.scenes]
    torch.cuda.synchronize()
    build_s = time.time() - t0
    persistent = args.workload == "batched"
    mode = 0
    layout = hg.output_layout(w.scanners, w.legs)
    out = hg.alloc_outputs(layout, dev, subrays=False, status=True)
    stream = torch.cuda.current_stream()

    def step():
        hg.scan(gsc, w.scanners, w.legs, mode=mode, seed=12345, persistent=persistent, out=out,
                subrays=False)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    clk = Clocks(D.local)
    clk.start()
    time.sleep(0.3)
    D.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for i in range(args.steps):
        step()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    D.barrier()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    clocks = clk.stop()
    ms = float(np.mean(per))
    ms_max = D.max(ms)
    P = w.n_pulses
    n_launch = len(w.legs) if not persistent else math.ceil(len(w.legs) / 128)
    S = workload_config(w, args.workload, hg.subray_count)["subrays_per_pulse"]
    subrays_total = sum(l.n_pulses * hg.subray_count(l.beam_sample_quality if l.beam_sample_quality >= 0
                                                     else w.scanners[l.scanner_index].beam_sample_quality)
                        for l in w.legs)
    value = D.world * P / (ms_max / 1e3)
    st = int(out["status"].item())
    res = {"metric": f"pulses/s ({S} subrays, waveform on)", "value": value, "unit": "pulses/s",
           "n_gpus": D.world, "steps": args.steps, "warmup": max(args.warmup, 3),
           "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": workload_config(w, args.workload, hg.subray_count, D.world),
           "bvh_build_s": round(build_s, 3),
           "precision": "fp32 traversal/waveform, fp64 pose and hit range",
           "subrays_per_s": D.world * subrays_total / (ms_max / 1e3),
           "gpu_launches": n_launch * args.steps,
           "device_status": st,
           "step_ms_all": [round(x, 4) for x in per]}
    # roofline of the (single) kernel per step
    peaks, kind = measured_peaks()
    fm = fetch_model(hg, w, gsc, mode, 12345, per_leg=4096 if persistent else 65536)
    alg = output_bytes(layout) + int(round(fm["fetch_bytes"] * P))
    comp = algorithmic_bytes(w, layout)
    achieved = alg / (ms / 1e3) / 1e9
    traffic = ncu_traffic(args.workload, P) if args.workload == "als" and not args.small else None
    gk = max((2 if len(s.grids) > 1 else len(s.grids)) for s in w.scenes)
    kern = "hg::scan_kernel<0,%d,%d>" % (gk, 128 if persistent else 1)
    res["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                       "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                       "algorithmic_bytes_per_launch": alg, "peak_source": kind, "kernel": kern,
                       "bytes_model": BYTES_MODEL,
                       "fetch_counts_per_pulse": {k: (round(v, 3) if isinstance(v, float) else v)
                                                  for k, v in fm.items()},
                       "compulsory_bytes_per_launch": comp,
                       "frac_compulsory": comp / (ms / 1e3) / 1e9 / peaks["hbm_gbs"]}
    res["clocks"] = clocks
    if not args.no_extras:
        res["e2e"] = e2e(w, gsc, layout, out, args, stream, D)
        if D.rank == 0 and D.world == 1:
            res["adjoint"] = adjoint_ratio(args)
            res["adjoint_forward_ratio"] = res["adjoint"]["adjoint_forward_ratio"]
            if args.workload == "als":
                res["batched"] = batched_compare(args)
                res["echo_width_fit"] = echo_width_cost(w, gsc, layout, args)
                res["mls"] = mls_step(args)
            if args.workload == "mls":
                res["reflectance_fit"] = reflectance_fit(args)
    return res, w


def mls_step(args):
    """The urban MLS workload at full size (2 km street of extruded buildings,
    20.7 M triangles, 2000 voxel trees of 128^3, rotating profile head, 20 M
    pulses, 37 subrays, 512 bins): device time of one stochastic scan step
    (2 warm-up steps, mean of 2)."""
    import torch
    import paper_2101_09154_gb300 as hg
    w = workload("mls", args.small)
    t0 = time.time()
    gsc = [hg.Scene(s) for s in w.scenes]
    torch.cuda.synchronize()
    build_s = time.time() - t0
    lay = hg.output_layout(w.scanners, w.legs)
    out = hg.alloc_outputs(lay, gsc[0].device, subrays=False)
    ms = _timed(lambda: hg.scan(gsc, w.scanners, w.legs, seed=12345, out=out, subrays=False), 2, 2)
    P = w.n_pulses
    S = hg.subray_count(w.scanners[0].beam_sample_quality)
    fm = fetch_model(hg, w, gsc, 0, 12345, per_leg=50_000)
    alg = output_bytes(lay) + P * fm["fetch_bytes"]
    peaks, _ = measured_peaks()
    res = {"workload": w.name, "description": w.note, "pulses": P, "subrays_per_pulse": S,
           "triangles": int(sum(s.n_triangles for s in w.scenes)),
           "voxel_trees": int(sum(len(s.grids) for s in w.scenes)),
           "voxels": int(sum(int(np.prod(g.dims)) for s in w.scenes for g in s.grids)),
           "scene_build_s": round(build_s, 3), "ms_per_step": ms,
           "pulses_per_s": P / (ms / 1e3), "subrays_per_s": P * S / (ms / 1e3),
           "roofline": {"bytes_per_pulse": round(alg / P, 1), "achieved_gbs": alg / (ms / 1e3) / 1e9,
                        "frac": alg / (ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                        "fetch_counts_per_pulse": {k: (round(v, 3) if isinstance(v, float) else v)
                                                   for k, v in fm.items()}}}
    del out, gsc
    torch.cuda.empty_cache()
    return res


def echo_width_cost(w, gsc, layout, args):
    """The same scan with the optional echo-width fit on (Sec. 3.4: the paper
    prices it at x1.3 of the run time): device time and ratio."""
    import torch
    import paper_2101_09154_gb300 as hg
    dev = gsc[0].device
    o0 = hg.alloc_outputs(layout, dev, subrays=False)
    o1 = hg.alloc_outputs(layout, dev, subrays=False, echo_width=True)
    t0 = _timed(lambda: hg.scan(gsc, w.scanners, w.legs, seed=12345, out=o0, subrays=False), 3, 2)
    t1 = _timed(lambda: hg.scan(gsc, w.scanners, w.legs, seed=12345, out=o1, subrays=False), 3, 2)
    ne = int(o1["echo_count"].clamp(max=w.scanners[0].max_echoes).sum())
    return {"ms_without": t0, "ms_with": t1, "ratio": t1 / t0, "echoes_fitted": ne}


def reflectance_fit(args):
    """50 adjoint-driven SIRT iterations of per-triangle reflectance over the
    whole urban MLS leg (2 km, 20 M pulses, 37 subrays, 2000 trees of 128^3;
    pieces of 4 M pulses): time, loss drop and RMSE against the seeded ground
    truth over the triangles the scan sees."""
    import torch
    import scenes
    import paper_2101_09154_gb300 as hg
    from paper_2101_09154_gb300.fit import fit_reflectance
    w = scenes.urban_mls(length=30.0, facade_cell=0.5) if args.small else scenes.urban_mls()
    sc, leg = w.scanners[0], w.legs[0]
    chunk = 0 if args.small else 4_000_000
    gs = hg.Scene(w.scenes[0])
    truth = [r.clone() for r in gs.reflectance]
    # the target: the expected-mode scan of the seeded reflectances, piece by piece
    nb = sc.n_bins
    target = torch.empty(leg.n_pulses * nb, dtype=torch.float32, device=gs.device)
    from paper_2101_09154_gb300.fit import _chunks
    for k0, piece in _chunks(leg, chunk):
        o, _ = hg.scan([gs], [sc], [piece], mode=1, subrays=False)
        target[k0 * nb:(k0 + piece.n_pulses) * nb] = o["waveform"]
        del o
    fit_reflectance(gs, sc, leg, target, iters=1, chunk_pulses=chunk)          # warm-up
    for r, t in zip(gs.reflectance, truth):
        r.copy_(t)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    res = fit_reflectance(gs, sc, leg, target, iters=50, chunk_pulses=chunk)
    e1.record()
    torch.cuda.synchronize()
    sq, n, sq_w, n_w = 0.0, 0, 0.0, 0
    for m, t in enumerate(truth):
        cw = res["column_weight"][m].cpu().numpy()
        err = (gs.reflectance[m] - t).cpu().numpy().astype(np.float64)
        seen = cw > 0
        well = seen & (cw >= np.percentile(cw[seen], 25)) if seen.any() else seen
        sq, n = sq + float((err[seen] ** 2).sum()), n + int(seen.sum())
        sq_w, n_w = sq_w + float((err[well] ** 2).sum()), n_w + int(well.sum())
    return {"workload": w.name, "pulses": w.n_pulses, "triangles": w.scenes[0].n_triangles,
            "iterations": 50, "fit_ms": e0.elapsed_time(e1), "chunk_pulses": chunk,
            "loss_first": res["loss"][0], "loss_last": res["loss"][-1],
            "triangles_seen": n, "rmse_seen": (sq / max(n, 1)) ** 0.5,
            "rmse_well_observed": (sq_w / max(n_w, 1)) ** 0.5}


def e2e(w, gsc, layout, out, args, stream, D):
    """Same metric through the public API with host buffers: each step uploads
    the per-step input (the meshes' reflectance) from pinned host memory and
    runs helios_scan_legs_host, which returns the whole result (waveform +
    echoes + window) in pinned host memory, copying each chunk of pulses to the
    host while the next one is scanned."""
    import torch
    import paper_2101_09154_gb300 as hg
    host_refl = [[r.cpu().pin_memory() for r in s.reflectance] for s in gsc]
    host_out = hg.alloc_host_outputs(layout, gsc[0].device, subrays=False)
    h2d = sum(t.numel() * t.element_size() for s in host_refl for t in s)
    d2h = sum(t.numel() * t.element_size() for k, t in host_out.items() if k != "status")
    persistent = args.workload == "batched"

    def step():
        for s, hs in zip(gsc, host_refl):
            for r, h in zip(s.reflectance, hs):
                r.copy_(h, non_blocking=True)
        hg.scan_to_host(gsc, w.scanners, w.legs, seed=12345, persistent=persistent, host_out=host_out,
                        chunk_pulses=1 << 18)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    n = max(2, min(args.steps, 5))
    D.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = D.max(e0.elapsed_time(e1) / n)
    # this box's device-to-host rate into the same pinned buffers (one plain
    # copy of the waveform, after the timed steps): the bound the step meets
    src, dst = out["waveform"], host_out["waveform"]
    torch.cuda.synchronize()
    e0.record(stream)
    dst.copy_(src, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    link = src.numel() * src.element_size() / (e0.elapsed_time(e1) / 1e3) / 1e9
    return {"value": D.world * w.n_pulses / (ms / 1e3), "unit": "pulses/s", "ms_per_step": ms,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": n,
            "d2h_link_gbs": link, "link_bound_ms": d2h / (link * 1e9) * 1e3}


def _timed(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def batched_compare(args):
    """Many legs of uneven length and subray quality (1, 7, 19, 37 subrays) over
    terrain tiles and voxel blocks: one launch per leg vs one persistent launch
    fed by a work queue vs that launch replayed from a CUDA graph, all with the
    autotuned launch parameters."""
    import torch
    import paper_2101_09154_gb300 as hg
    from paper_2101_09154_gb300.autotune import autotune
    w = workload("batched", args.small)
    gsc = [hg.Scene(s) for s in w.scenes]
    lay = hg.output_layout(w.scanners, w.legs)
    out = hg.alloc_outputs(lay, gsc[0].device, subrays=False)
    cache = os.path.join(ROOT, "paper_2101_09154_gb300", "_build", "autotune.json")
    tune = autotune(gsc, w.scanners, w.legs, out, persistent=True, cache_path=cache)
    kw = dict(block_threads=tune["block_threads"], rays_per_block=tune["rays_per_block"])
    steps, warm = max(2, min(args.steps, 5)), 2
    per_leg_ms = _timed(lambda: hg.scan(gsc, w.scanners, w.legs, persistent=False, out=out, **kw),
                        steps, warm)
    pers_ms = _timed(lambda: hg.scan(gsc, w.scanners, w.legs, persistent=True, out=out, **kw),
                     steps, warm)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        hg.scan(gsc, w.scanners, w.legs, persistent=True, out=out, **kw)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        hg.scan(gsc, w.scanners, w.legs, persistent=True, out=out, **kw)
    graph_ms = _timed(graph.replay, steps, warm)
    P = w.n_pulses
    res = {"workload": w.name, "description": w.note, "legs": len(w.legs), "pulses": P,
           "autotune": {k: tune[k] for k in ("block_threads", "rays_per_block")},
           "autotune_trials_ms": {f"{t['block_threads']}x{t['rays_per_block']}": round(t["ms"], 3)
                                  for t in tune["trials"]},
           "per_leg_ms": per_leg_ms, "per_leg_launches": len(w.legs),
           "persistent_ms": pers_ms, "persistent_launches": math.ceil(len(w.legs) / 128),
           "graph_ms": graph_ms,
           "speedup_persistent_vs_per_leg": per_leg_ms / pers_ms,
           "speedup_graph_vs_per_leg": per_leg_ms / graph_ms,
           "pulses_per_s_graph": P / (graph_ms / 1e3),
           "pulses_per_s_per_leg": P / (per_leg_ms / 1e3)}
    del out, graph
    torch.cuda.empty_cache()
    return res


def adjoint_ratio(args):
    """Expected-mode forward and adjoint on the voxel-canopy workload (1 M pulses,
    256^3 voxels, 19 subrays, 1024 bins): time of the adjoint / time of the forward."""
    import torch
    import paper_2101_09154_gb300 as hg
    import scenes
    w = workload("uls", args.small)
    sc, leg = w.scanners[0], w.legs[0]
    gs = hg.Scene(w.scenes[0])
    lay = hg.output_layout([sc], [leg])
    out = hg.alloc_outputs(lay, gs.device, subrays=True)
    ref_scene = scenes.Scene(meshes=w.scenes[0].meshes,
                             grids=[scenes.VoxelGrid(**{**w.scenes[0].grids[0].__dict__,
                                                       "density": scenes.perturbed_density(
                                                           w.scenes[0].grids[0].density, seed=1)})])
    gref = hg.Scene(ref_scene)
    out_ref, _ = hg.scan([gref], [sc], [leg], mode=1, subrays=False)
    grads = [{"reflectance": [torch.zeros_like(r) for r in gs.reflectance],
              "density": [torch.zeros_like(d) for d in gs.density]}]

    def fwd():
        hg.scan([gs], [sc], [leg], mode=1, out=out)

    def bwd(gW):
        hg.scan_adjoint([gs], [sc], [leg], gW, out["window_bin"], out["subray_hit"], grads=grads)

    fwd()
    gW = 2.0 * (out["waveform"] - out_ref["waveform"])
    bwd(gW)
    fs = [hg.scan([gs], [sc], [leg], mode=0, out=out) for _ in range(2)]
    del fs
    torch.cuda.synchronize()

    def timed(fn, n=5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s = torch.cuda.current_stream()
        e0.record(s)
        for _ in range(n):
            fn()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    f_ms = timed(fwd)
    b_ms = timed(lambda: bwd(gW))
    s_ms = timed(lambda: hg.scan([gs], [sc], [leg], mode=0, out=out))
    # algorithmic bytes per kernel: the per-pulse fetch model of each mode
    # (the forwards also write the subray hit/range checkpoint); the adjoint
    # reads dL/dW, the window and the checkpoint, needs the expected mode's
    # fetches and updates a gradient (read + write, 8 B) per distinct voxel
    P = leg.n_pulses
    S = hg.subray_count(sc.beam_sample_quality)
    peaks, kind = measured_peaks()
    fm = {m: fetch_model(hg, w, [gs], m, 12345 if m == 0 else 0) for m in (0, 1)}
    outb = output_bytes(lay, subray_outputs=True)
    per_kernel = {
        "stochastic_forward": (outb + P * fm[0]["fetch_bytes"], s_ms),
        "expected_forward": (outb + P * fm[1]["fetch_bytes"], f_ms),
        "adjoint": (P * (4 * sc.n_bins + 4 + 8 * S + fm[1]["fetch_bytes"] + 8 * fm[1]["voxels"]), b_ms),
    }
    roof = {k: {"bytes_per_pulse": round(b / P, 1), "achieved_gbs": b / (t / 1e3) / 1e9,
                "frac": b / (t / 1e3) / 1e9 / peaks["hbm_gbs"]} for k, (b, t) in per_kernel.items()}
    return {"workload": w.name, "pulses": leg.n_pulses, "expected_forward_ms": f_ms,
            "adjoint_ms": b_ms, "adjoint_forward_ratio": b_ms / f_ms,
            "stochastic_forward_ms": s_ms,
            "stochastic_pulses_per_s": leg.n_pulses / (s_ms / 1e3),
            "expected_pulses_per_s": leg.n_pulses / (f_ms / 1e3),
            "roofline": roof, "peak_source": kind,
            "fetch_counts_per_pulse": {("stochastic", "expected")[m]: {k: (round(v, 3) if isinstance(v, float) else v)
                                                                      for k, v in fm[m].items()}
                                       for m in (0, 1)}}


# --------------------------------------------------------------------------
# the oracle on the host cores
# --------------------------------------------------------------------------
def oracle_rate(w, target_s, pulses_cap=None, one_core=False):
    """Time the FP64 oracle (as it stands) on an evenly strided pulse sample."""
    import oracle
    osc = oracle.OracleScene(w.scenes[w.legs[0].scene_index])
    sc, leg = w.scanners[w.legs[0].scanner_index], w.legs[0]
    cores = os.cpu_count() or 1
    # calibrate on a small sample, then size the timed sample to ~target_s
    probe = np.arange(0, leg.n_pulses, max(leg.n_pulses // 2000, 1))[:2000]
    t0 = time.time()
    oracle.scan(osc, sc, leg, probe, threads=cores)
    dt = max(time.time() - t0, 1e-3)
    n = int(min(leg.n_pulses, max(len(probe), target_s * len(probe) / dt)))
    if pulses_cap:
        n = min(n, pulses_cap)
    rows = np.unique(np.linspace(0, leg.n_pulses - 1, n).astype(np.int64))
    t0 = time.time()
    oracle.scan(osc, sc, leg, rows, threads=cores)
    dt = time.time() - t0
    q = leg.beam_sample_quality if leg.beam_sample_quality >= 0 else sc.beam_sample_quality
    res = {"value": len(rows) / dt, "unit": "pulses/s", "cores": cores, "kind": "oracle",
           "elapsed_s": dt, "sample_pulses": int(len(rows)),
           "sample": f"{len(rows)} evenly spaced pulses of the {leg.n_pulses}-pulse leg "
                     f"({oracle.subray_count(q)} subrays each), {dt:.1f} s of FP64 CPU work "
                     f"on {cores} threads"}
    if one_core and cores > 1:
        # the same oracle on one thread, on every (10 x cores)-th pulse of the
        # sample (about a tenth of the multi-thread run's wall time)
        r1 = rows[:: cores * 10] if len(rows) > 100 else rows
        t0 = time.time()
        oracle.scan(osc, sc, leg, r1, threads=1)
        res["value_1core"] = len(r1) / (time.time() - t0)
    return res


def run_reference(args, D):
    if D.rank != 0:
        return None
    w = workload(args.workload, args.small)
    import oracle
    oracle.build()
    # each step: one bounded, evenly strided sample of the leg's pulses (about
    # cpu_sample_s / steps seconds of FP64 work), timed on the wall clock
    n_done, t_done, step_ms = 0, 0.0, []
    per_step_target = max(1.0, args.cpu_sample_s / max(args.steps, 1))
    info = None
    for i in range(args.warmup + args.steps):
        r = oracle_rate(w, per_step_target)
        if i >= args.warmup:
            n_done += r["sample_pulses"]
            t_done += r["elapsed_s"]
            step_ms.append(1e3 * r["elapsed_s"])
            info = r
    value = n_done / t_done
    return {"impl": "reference", "metric": "pulses/s (19 subrays, waveform on)", "value": value,
            "unit": "pulses/s", "n_gpus": D.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, args.workload, oracle.subray_count, D.world),
            "step_pulses": n_done // max(args.steps, 1),
            "cpu_baseline": {**info, "value": value,
                             "sample": f"per step: {info['sample']}"},
            "e2e": {"value": value, "unit": "pulses/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}


def main():
    args = parse()
    D = Dist()
    try:
        if args.impl == "reference":
            res = run_reference(args, D)
            if res is not None:
                print(json.dumps(res), flush=True)
            return
        res, w = run_ours(args, D)
        if D.rank == 0:
            if not args.no_extras and D.world == 1:
                res["cpu_baseline"] = oracle_rate(w, args.cpu_sample_s, one_core=True)
            print(json.dumps(res), flush=True)
    finally:
        D.close()


if __name__ == "__main__":
    main()
