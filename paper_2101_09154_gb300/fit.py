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


def fit_reflectance(scene, scanner, leg, target, iters=50, rho0=0.5, block_threads=0,
                    rays_per_block=0):
    """Fit ``scene.reflectance`` (updated in place) to the waveform ``target``.

    ``scene`` is a :class:`Scene` whose meshes' reflectance tensors are the
    unknowns (voxel grids, if any, are held fixed: their returns do not depend
    on rho, so the model is affine, W = J rho + W(0)); ``target`` is a device
    waveform with
    the layout of ``scan``'s output for (scanner, leg).  Returns a dict with the
    loss (sum of squared residuals) before each iteration and after the last,
    and the column weights J^T J 1 per mesh.
    """
    opts = dict(mode=MODE_EXPECTED, block_threads=block_threads, rays_per_block=rays_per_block)
    refl = scene.reflectance
    torch = __import__("torch")

    def adjoint(g, win, hits):
        # reflectance gradients only: the grids' densities are held fixed
        grads = [{"reflectance": [torch.zeros_like(r) for r in refl],
                  "density": [None] * len(scene.density)}]
        return scan_adjoint([scene], [scanner], [leg], g, win, hits, grads=grads)[0]

    # voxel returns do not depend on rho: W = J rho + W(0), so J 1 = W(1) - W(0)
    for r in refl:
        r.fill_(0.0)
    out0, _ = scan([scene], [scanner], [leg], **opts)
    w0 = out0["waveform"].clone()
    for r in refl:
        r.fill_(1.0)
    out, _ = scan([scene], [scanner], [leg], **opts)
    colw = adjoint(out["waveform"] - w0, out["window_bin"], out["subray_hit"])["reflectance"]
    for r in refl:
        r.fill_(float(rho0))
    hist = []
    for _ in range(int(iters)):
        out, _ = scan([scene], [scanner], [leg], out=out, **opts)
        resid = out["waveform"] - target
        hist.append(float(torch.sum(resid.double() ** 2)))
        g = adjoint(resid, out["window_bin"], out["subray_hit"])
        for r, gr, cw in zip(refl, g["reflectance"], colw):
            seen = cw > 0
            step = torch.where(seen, gr / torch.where(seen, cw, torch.ones_like(cw)), torch.zeros_like(gr))
            r.sub_(step).clamp_(0.0, 1.0)
    out, _ = scan([scene], [scanner], [leg], out=out, **opts)
    hist.append(float(torch.sum((out["waveform"] - target).double() ** 2)))
    return {"loss": hist, "column_weight": colw}
