"""Per-triangle reflectance fit driven by the adjoint.

The expected-mode waveform is affine in the reflectances: W = J rho + W(0),
where J (pulse bins x triangles, non-negative) holds each triangle's return
power at unit reflectance times the transmittance of the voxels before it,
spread by the pulse shape (Eq. beamdiv, Eq. ladlut_intensity with a
Lambertian cross-section, Sec. 3.4), and W(0) is the voxels' own returns.
The forward scan evaluates J rho and helios_scan_adjoint evaluates J^T g, so
the least-squares fit of rho to a target waveform y can be run without ever
forming J.  The iteration is the simultaneous one used for non-negative
tomographic systems (SIRT):

    rho <- clip(rho - (J^T (W(rho) - y)) / (J^T J 1), 0, 1)

where J^T J 1 is one adjoint of J 1 = W(1) - W(0).
For non-negative J that diagonal bounds every row sum of J^T J, so each step
lowers the residual.  Triangles no pulse sees (J^T J 1 = 0) keep their value.

The scans and adjoints run in the library's kernels; this module only holds
the loop and the element-wise update of the reflectance tensors.
"""
from __future__ import annotations

import torch

from . import MODE_EXPECTED, scan, scan_adjoint


def _chunks(leg, chunk_pulses):
    """The leg as consecutive pieces of at most chunk_pulses pulses (a piece
    resumes the leg at its first pulse, so every draw is the whole leg's)."""
    from dataclasses import replace
    if not chunk_pulses or chunk_pulses >= leg.n_pulses:
        return [(0, leg)]
    out = []
    for k0 in range(0, leg.n_pulses, int(chunk_pulses)):
        n = min(int(chunk_pulses), leg.n_pulses - k0)
        out.append((k0, replace(leg, first_pulse=leg.first_pulse + k0, n_pulses=n)))
    return out


def fit_reflectance(scene, scanner, leg, target, iters=50, rho0=0.5, block_threads=0,
                    rays_per_block=0, chunk_pulses=0):
    """Fit ``scene.reflectance`` (updated in place) to the waveform ``target``.

    ``scene`` is a :class:`Scene` whose meshes' reflectance tensors are the
    unknowns (voxel grids, if any, are held fixed: their returns do not depend
    on rho, so the model is affine, W = J rho + W(0)); ``target`` is a device
    waveform with the layout of ``scan``'s output for (scanner, leg).  With
    ``chunk_pulses`` the leg is scanned and differentiated in pieces of that
    many pulses (the sums over pieces are the whole leg's), so that device
    memory holds the target and one piece's buffers.  Returns a dict with the
    loss (sum of squared residuals) before each iteration and after the last,
    and the column weights J^T J 1 per mesh.
    """
    opts = dict(mode=MODE_EXPECTED, block_threads=block_threads, rays_per_block=rays_per_block)
    refl = scene.reflectance
    nb = scanner.n_bins
    pieces = _chunks(leg, chunk_pulses)
    tgt = target.view(-1, nb)
    bufs = {}       # output buffers by piece length (all pieces but the last share one)

    def scan_piece(i, piece):
        out, _ = scan([scene], [scanner], [piece], out=bufs.get(piece.n_pulses), **opts)
        bufs[piece.n_pulses] = out
        return out

    def adjoint(g, win, hits, piece, grads):
        # reflectance gradients only: the grids' densities are held fixed
        return scan_adjoint([scene], [scanner], [piece], g, win, hits, grads=grads)[0]

    def zero_grads():
        return [{"reflectance": [torch.zeros_like(r) for r in refl],
                 "density": [None] * len(scene.density)}]

    # voxel returns do not depend on rho: W = J rho + W(0), so J 1 = W(1) - W(0)
    cg = zero_grads()
    for i, (k0, piece) in enumerate(pieces):
        for r in refl:
            r.fill_(0.0)
        w0 = scan_piece(i, piece)["waveform"].clone()
        for r in refl:
            r.fill_(1.0)
        out = scan_piece(i, piece)
        adjoint(out["waveform"] - w0, out["window_bin"], out["subray_hit"], piece, cg)
        del w0
    colw = cg[0]["reflectance"]
    for r in refl:
        r.fill_(float(rho0))
    hist = []

    def residuals(grads):
        loss = 0.0
        for i, (k0, piece) in enumerate(pieces):
            out = scan_piece(i, piece)
            resid = out["waveform"] - tgt[k0:k0 + piece.n_pulses].reshape(-1)
            loss += float(torch.sum(resid.double() ** 2))
            if grads is not None:
                adjoint(resid, out["window_bin"], out["subray_hit"], piece, grads)
        return loss

    for _ in range(int(iters)):
        g = zero_grads()
        hist.append(residuals(g))
        for r, gr, cw in zip(refl, g[0]["reflectance"], colw):
            seen = cw > 0
            step = torch.where(seen, gr / torch.where(seen, cw, torch.ones_like(cw)), torch.zeros_like(gr))
            r.sub_(step).clamp_(0.0, 1.0)
    hist.append(residuals(None))
    return {"loss": hist, "column_weight": colw}
