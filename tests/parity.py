"""Comparison helpers: CUDA outputs vs the FP64 oracle on the same seeded inputs.

Tolerances (stated once, used by every GPU parity test):
  * integers (window start, hit / echo / object ids, echo counts): exact, on
    pulses the oracle does not flag (flags mark rays within 1e-6 R of a triangle
    edge, near-equal hits, transmission draws within rounding of the segment
    length, window starts within 1e-6 of a bin boundary, echo decisions within
    the waveform tolerance);
  * ranges: |dR| <= 1e-4 m;
  * waveform samples: |dW| <= 1e-4 |W| + 1e-7 max_b |W| per pulse (FP32 samples
    underflow or are cut where the pulse shape is below 2^-30 of its peak,
    hence the floor relative to the pulse's maximum).
"""
import numpy as np

import oracle

RANGE_TOL = 1e-4
W_REL = 1e-4
W_FLOOR = 1e-7


def to_np(t):
    return t.detach().cpu().numpy()


def leg_view(out, lay, l, scanner, S, rows):
    """Slice the concatenated outputs of leg l at the given pulse rows."""
    po = int(lay["pulse_offset"][l])
    wo = int(lay["wave_offset"][l])
    so = int(lay["subray_offset"][l])
    eo = int(lay["echo_offset"][l])
    nb, K = scanner.n_bins, scanner.max_echoes
    rows = np.asarray(rows, np.int64)
    v = {}
    v["window_bin"] = to_np(out["window_bin"])[po + rows]
    v["echo_count"] = to_np(out["echo_count"])[po + rows]
    W = to_np(out["waveform"])
    v["waveform"] = W[wo + rows[:, None] * nb + np.arange(nb)[None, :]]
    for k in ("echo_range", "echo_amp", "echo_bin", "echo_object"):
        a = to_np(out[k])
        v[k] = a[eo + rows[:, None] * K + np.arange(K)[None, :]]
    if "subray_hit" in out:
        for k in ("subray_hit", "subray_range"):
            a = to_np(out[k])
            v[k] = a[so + rows[:, None] * S + np.arange(S)[None, :]]
    v["pulse_flags"] = to_np(out["pulse_flags"])[po + rows]
    return v


def compare(g, ref, max_flag_frac=0.2, check_subrays=True, expected_mode=False):
    """Assert parity of one leg's GPU view `g` against oracle result `ref`."""
    f = ref["flags"]
    geo = (f & oracle.F_GEOMETRY) == 0
    dec = (f & (oracle.F_DECISION | oracle.F_OVERFLOW)) == 0
    n = len(f)
    assert (~geo).mean() <= max_flag_frac, f"too many flagged pulses: {(~geo).mean():.3f}"
    # window start
    bad = np.nonzero(geo & (g["window_bin"] != ref["window_bin"]))[0]
    assert bad.size == 0, f"window_bin differs on {bad.size} unflagged pulses, e.g. {bad[:5]}"
    # subray events
    if check_subrays and "subray_hit" in g:
        hit_ok = g["subray_hit"] == ref["subray_hit"]
        bad = np.nonzero(geo[:, None] & ~hit_ok)
        assert bad[0].size == 0, (f"subray hit ids differ on {bad[0].size} unflagged subrays, "
                                  f"e.g. pulse rows {bad[0][:5]}: gpu {g['subray_hit'][bad][:5]} "
                                  f"oracle {ref['subray_hit'][bad][:5]}")
        m = geo[:, None] & (ref["subray_hit"] >= 0)
        dr = np.abs(g["subray_range"] - ref["subray_range"])[m]
        assert dr.size == 0 or dr.max() <= RANGE_TOL, f"subray range error {dr.max():.3e} m"
    # waveform
    W, R = g["waveform"].astype(np.float64), ref["waveform"]
    peak = np.abs(R).max(axis=1, keepdims=True)
    excess = np.abs(W - R) - (W_REL * np.abs(R) + W_FLOOR * peak)
    rows = np.nonzero(geo & (excess > 0).any(axis=1))[0]
    assert rows.size == 0, (f"waveform outside tolerance on {rows.size} unflagged pulses, e.g. row "
                            f"{rows[0]}: max rel err "
                            f"{(np.abs(W - R) / np.maximum(np.abs(R), 1e-300))[rows[0]].max():.3e}")
    # echoes
    bad = np.nonzero(dec & (g["echo_count"] != ref["echo_count"]))[0]
    assert bad.size == 0, (f"echo counts differ on {bad.size} unflagged pulses, e.g. {bad[:5]}: "
                           f"gpu {g['echo_count'][bad[:5]]} oracle {ref['echo_count'][bad[:5]]}")
    K = ref["echo_bin"].shape[1]
    valid = dec[:, None] & (np.arange(K)[None, :] < ref["echo_count"][:, None])
    assert np.array_equal(g["echo_bin"][valid], ref["echo_bin"][valid]), "echo bins differ"
    assert np.array_equal(g["echo_object"][valid], ref["echo_object"][valid]), "echo objects differ"
    de = np.abs(g["echo_range"] - ref["echo_range"])[valid]
    assert de.size == 0 or de.max() <= RANGE_TOL, f"echo range error {de.max():.3e} m"
    amp_tol = W_REL * np.abs(ref["echo_amp"]) + W_FLOOR * peak
    assert (np.abs(g["echo_amp"] - ref["echo_amp"]) <= amp_tol)[valid].all(), "echo amplitudes differ"
    return {"pulses": n, "flagged_geometry": float((~geo).mean()),
            "flagged_decision": float((~dec).mean()), "echoes": int(ref["echo_count"][dec].sum())}
