"""Launch-parameter autotuner for the scan kernel.

Candidates are (threads per block, target subrays per work item).  The work
item size decides pulses per block iteration (subrays / S) and therefore the
shared-memory footprint and occupancy; results do not depend on it (each
pulse is computed by one warp in a fixed order), only the time does.  The
choice is cached per workload signature in a JSON file.
"""
from __future__ import annotations

import hashlib
import json
import os

CANDIDATES = [(256, 768), (256, 384), (256, 1536), (128, 384), (128, 768), (192, 576)]


def _signature(scanners, legs, mode, persistent, device_name):
    h = hashlib.sha256()
    for s in scanners:
        h.update(repr((s.n_bins, s.beam_sample_quality, s.deflector, s.pulse_shape)).encode())
    for l in legs:
        h.update(repr((l.scene_index, l.scanner_index, l.beam_sample_quality, l.n_pulses)).encode())
    h.update(repr((mode, persistent, device_name)).encode())
    return h.hexdigest()[:20]


def autotune(scenes, scanners, legs, out, mode=0, persistent=True, cache_path=None, reps=2,
             candidates=CANDIDATES):
    """Return {"block_threads", "rays_per_block", "ms", "trials"} for this workload."""
    import torch
    from . import scan

    key = _signature(scanners, legs, mode, persistent, torch.cuda.get_device_name())
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return cache[key]
    trials = []
    for bt, rpb in candidates:
        scan(scenes, scanners, legs, mode=mode, persistent=persistent, out=out,
             block_threads=bt, rays_per_block=rpb)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            scan(scenes, scanners, legs, mode=mode, persistent=persistent, out=out,
                 block_threads=bt, rays_per_block=rpb)
        e1.record()
        torch.cuda.synchronize()
        trials.append({"block_threads": bt, "rays_per_block": rpb, "ms": e0.elapsed_time(e1) / reps})
    best = min(trials, key=lambda t: t["ms"])
    res = {**best, "trials": trials}
    if cache_path:
        cache[key] = res
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return res
