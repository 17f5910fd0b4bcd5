"""helios_scan_legs_host (outputs in host memory, chunked and overlapped with
the copies) against helios_scan_legs on the same inputs: bit for bit (GPU)."""
import numpy as np
import pytest

import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("waveform", "window_bin", "echo_count", "echo_range", "echo_amp", "echo_bin", "echo_object",
        "pulse_flags", "subray_hit", "subray_range", "echo_width")


@pytest.fixture(scope="module")
def hg():
    import __graft_entry__ as g
    g.build()
    import paper_2101_09154_gb300 as m
    return m


@pytest.mark.parametrize("mode,persistent,chunk", [(0, False, 1000), (0, True, 777), (1, True, 2000),
                                                   (0, False, 1 << 30)])
def test_host_scan_equals_device_scan(hg, mode, persistent, chunk):
    """Legs of uneven length and quality over terrain tiles and voxel blocks;
    chunk boundaries fall inside legs, and with more than two chunks the
    staging slots are reused."""
    w = scenes.batched_legs(seed=21, n_legs=6, tile=64, block=24, n_terrain=2, n_voxel=2,
                            min_pulses=300, max_pulses=3000, n_bins=256)
    gsc = [hg.Scene(s) for s in w.scenes]
    ref, lay = hg.scan(gsc, w.scanners, w.legs, mode=mode, seed=5, persistent=persistent,
                       echo_width=True)
    host = hg.alloc_host_outputs(lay, gsc[0].device, subrays=True, echo_width=True)
    host, lay2 = hg.scan_to_host(gsc, w.scanners, w.legs, mode=mode, seed=5, persistent=persistent,
                                 host_out=host, chunk_pulses=chunk)
    torch.cuda.synchronize()
    assert lay2["total_pulses"] == lay["total_pulses"]
    if chunk < lay["total_pulses"]:
        assert lay["total_pulses"] > 2 * chunk
    for k in KEYS:
        a, b = ref[k].cpu(), host[k]
        assert a.dtype == b.dtype and a.shape == b.shape, k
        assert torch.equal(a, b), (k, int((a != b).sum()))


def test_host_scan_rejects_bad_chunk(hg):
    w = scenes.tls_tiny(n_az=4, n_el=4)
    gsc = [hg.Scene(w.scenes[0])]
    with pytest.raises(hg.HeliosError) as e:
        hg.scan_to_host(gsc, w.scanners, w.legs, chunk_pulses=0)
    assert e.value.code == -1 and "chunk_pulses" in str(e.value)


def test_host_scan_of_a_resumed_leg(hg):
    """The host-memory scan honours first_pulse in every chunk."""
    import dataclasses
    w = scenes.als_terrain(seed=5, size=96, n_trees=6, n_pulses=5000, n_bins=256, agl=120.0,
                           speed=30.0, prf=50_000.0)
    leg = dataclasses.replace(w.legs[0], first_pulse=1900, n_pulses=3100)
    gsc = [hg.Scene(s) for s in w.scenes]
    dev, lay = hg.scan(gsc, w.scanners, [leg], seed=3, subrays=False)
    host, lay2 = hg.scan_to_host(gsc, w.scanners, [leg], seed=3, chunk_pulses=1000)
    torch.cuda.synchronize()
    for k in ("waveform", "window_bin", "echo_count", "echo_range", "echo_bin"):
        assert np.array_equal(dev[k].cpu().numpy(), host[k].numpy()), k
