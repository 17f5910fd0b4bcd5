"""The parity comparison itself, on the CPU: a stand-in for a GPU result is
made from the oracle (so no GPU is needed), with the other legitimate choice on
flagged subrays; the comparison must accept it and must reject planted
mistakes on unflagged subrays and pulses."""
import math
import os
import sys

import numpy as np
import pytest

import oracle
import scenes

sys.path.insert(0, os.path.dirname(__file__))
from parity import compare  # noqa: E402


def _as_gpu(r, S):
    """An oracle result in the GPU's output types (one leg, all rows)."""
    g = {"window_bin": r["window_bin"].copy(), "echo_count": r["echo_count"].copy(),
         "waveform": r["waveform"].astype(np.float32),
         "echo_range": r["echo_range"].astype(np.float32), "echo_amp": r["echo_amp"].astype(np.float32),
         "echo_bin": r["echo_bin"].copy(), "echo_object": r["echo_object"].copy(),
         "subray_hit": r["subray_hit"].copy(), "subray_range": r["subray_range"].astype(np.float32),
         "pulse_flags": np.zeros(len(r["flags"]), np.uint8)}
    return g


def _diagonal_scan():
    # a plate whose diagonal runs under the scanner: pulses at azimuth 45 deg
    # cross it, and their subrays near it are flagged
    osc = oracle.OracleScene(scenes.flat_target(10.0, 0.0, half=20.0))
    sc = scenes.Scanner(deflector=scenes.DEFL_TLS_GRID, grid_n_az=8, grid_n_el=24,
                        el_min_rad=-math.radians(85), el_max_rad=-math.radians(40), n_bins=200,
                        beam_sample_quality=2, divergence_rad=2e-3)
    leg = scenes.Leg(n_pulses=8 * 24)
    r = oracle.scan(osc, sc, leg, mode=0, seed=3)
    return osc, sc, leg, r


def test_other_choice_on_flagged_subrays_is_accepted():
    osc, sc, leg, r = _diagonal_scan()
    S = r["S"]
    flagged = (r["subray_flags"] & oracle.F_SUBRAY) != 0
    assert flagged.sum() >= 3
    # the GPU stand-in took the other triangle of the diagonal on flagged subrays
    other = np.where(flagged, 1 - r["subray_hit"], oracle.FREE_HIT).astype(np.int64)
    rows = np.nonzero(flagged.any(axis=1))[0]
    alt = r["rerun"](rows, force_hit=other[rows])
    assert not (alt["flags"] & oracle.F_FORCED_BAD).any()
    gr = dict(r)
    for k in ("waveform", "echo_range", "echo_amp", "echo_bin", "echo_object", "echo_count",
              "window_bin", "subray_hit", "subray_range"):
        a = r[k].copy()
        a[rows] = alt[k]
        gr[k] = a
    g = _as_gpu(gr, S)
    assert (g["subray_hit"] != r["subray_hit"]).any()
    st = compare(g, r)
    assert st["rerun_pulses"] == rows.size and st["excluded_pulses"] == 0.0
    assert 0 < st["flagged_subrays"] < 0.05


@pytest.mark.parametrize("plant", ["hit", "echo_bin", "waveform", "window"])
def test_planted_mistakes_are_rejected(plant):
    osc, sc, leg, r = _diagonal_scan()
    g = _as_gpu(r, r["S"])
    clean = np.nonzero(((r["subray_flags"] & oracle.F_SUBRAY) == 0).all(axis=1)
                       & ((r["flags"] & oracle.F_DECISION) == 0) & (r["echo_count"] > 0))[0]
    i = clean[len(clean) // 2]
    if plant == "hit":
        g["subray_hit"][i, 0] = 1 - g["subray_hit"][i, 0]
    elif plant == "echo_bin":
        g["echo_bin"][i, 0] += 1
    elif plant == "waveform":
        b = int(np.argmax(g["waveform"][i]))
        g["waveform"][i, b] *= np.float32(1.001)
    else:
        g["window_bin"][i] += 1
    with pytest.raises(AssertionError):
        compare(g, r)


def test_unforceable_choice_is_rejected():
    """A flagged subray given an event no flagged decision allows (a miss on a
    plate that the subray's neighbours clearly hit)."""
    osc, sc, leg, r = _diagonal_scan()
    g = _as_gpu(r, r["S"])
    flagged = (r["subray_flags"] & oracle.F_SUBRAY) != 0
    p, s = np.argwhere(flagged)[0]
    g["subray_hit"][p, s] = -1
    with pytest.raises(AssertionError, match="no flagged decision allows"):
        compare(g, r)
