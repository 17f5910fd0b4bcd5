"""Leaf-angle projection factor G of Eq. extinction, in FP64 (test infrastructure).

Like the rest of ``oracle/``, this module is imported only by the tests,
``__graft_entry__.smoke()`` and the CPU arm of ``bench.py``; it shares no code
with the CUDA library, which builds its own tables (``helios_lad_table``).

Eq. extinction (Sec. 3.5.4) gives the extinction coefficient of a voxel as
sigma = mu_L * G(Omega') with

    G(Omega') = 1/(2 pi) * integral over the hemisphere of leaf normals Omega_L
                of g_L(Omega_L) |Omega' . Omega_L| dOmega_L,

g_L normalised so that its hemispheric integral is 2 pi (the caption of Table
ladlut: "normalised over 2 pi").  Leaves are taken azimuthally uniform with
inclination density f(theta_L) on [0, pi/2] (integral 1); then
g_L = f(theta_L) / sin(theta_L) and

    G(theta) = 1/(2 pi) int_0^{pi/2} f(theta_L) int_0^{2 pi}
               |cos theta cos theta_L + sin theta sin theta_L cos phi| dphi dtheta_L,

theta the zenith angle of the beam.  This module evaluates that double integral
as written, by Gauss-Legendre quadrature on the pieces where the integrand is
smooth: the absolute value changes sign at cos phi = -cot theta cot theta_L,
and that point exists only for theta_L > pi/2 - theta, so both integrals are
split there.  No closed form of the inner integral is used.

The six inclination densities the paper names (Sec. 3.5.4) are de Wit's:
planophile (2/pi)(1 + cos 2t), erectophile (2/pi)(1 - cos 2t), plagiophile
(2/pi)(1 - cos 4t), extremophile (2/pi)(1 + cos 4t), uniform 2/pi and
spherical sin t.

Table ladlut indexes G by the beam's horizontal and vertical components; the
table built here holds G at mu_i = i/(n-1), mu = |vertical component| =
|cos theta|, and the scan interpolates it linearly in mu.
"""
from __future__ import annotations

import math

import numpy as np

KINDS = ("planophile", "erectophile", "plagiophile", "extremophile", "uniform", "spherical")


def leaf_density(kind: str, t):
    """de Wit's leaf-inclination density f(theta_L) (integral 1 on [0, pi/2]);
    ``kind`` may also be a callable f."""
    t = np.asarray(t, dtype=np.float64)
    if callable(kind):
        return np.asarray(kind(t), dtype=np.float64)
    c = 2.0 / math.pi
    if kind == "planophile":
        return c * (1.0 + np.cos(2.0 * t))
    if kind == "erectophile":
        return c * (1.0 - np.cos(2.0 * t))
    if kind == "plagiophile":
        return c * (1.0 - np.cos(4.0 * t))
    if kind == "extremophile":
        return c * (1.0 + np.cos(4.0 * t))
    if kind == "uniform":
        return np.full_like(t, c)
    if kind == "spherical":
        return np.sin(t)
    raise ValueError(f"unknown leaf angle distribution {kind!r}")


def _gl(a, b, n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def _inner(theta, tl, n):
    """int_0^{2 pi} |cos th cos tl + sin th sin tl cos phi| dphi for each tl (array)."""
    a = math.cos(theta) * np.cos(tl)
    b = math.sin(theta) * np.sin(tl)
    # the integrand is even in phi: twice the integral over [0, pi], split at
    # the sign change phi* = arccos(-a/b) when b > a
    with np.errstate(divide="ignore", invalid="ignore"):
        ps = np.where(b > a, np.arccos(np.clip(-a / np.where(b > 0, b, 1.0), -1.0, 1.0)), math.pi)
    x, w = np.polynomial.legendre.leggauss(n)
    tot = np.zeros_like(tl)
    for lo, hi in ((np.zeros_like(ps), ps), (ps, np.full_like(ps, math.pi))):
        h = 0.5 * (hi - lo)
        phi = h[:, None] * x[None, :] + (0.5 * (hi + lo))[:, None]
        val = np.abs(a[:, None] + b[:, None] * np.cos(phi))
        tot += h * (val * w[None, :]).sum(axis=1)
    return 2.0 * tot


def ross_G(kind: str, mu: float, n: int = 128) -> float:
    """G at a beam with |cos zenith| = mu, by quadrature of Eq. extinction."""
    mu = min(max(float(mu), 0.0), 1.0)
    theta = math.acos(mu)
    split = 0.5 * math.pi - theta
    tot = 0.0
    for a, b in ((0.0, split), (split, 0.5 * math.pi)):
        if b - a <= 0.0:
            continue
        tl, wl = _gl(a, b, n)
        tot += float(np.sum(wl * leaf_density(kind, tl) * _inner(theta, tl, n)))
    return tot / (2.0 * math.pi)


def table(kind: str, n: int = 91, quad: int = 128) -> np.ndarray:
    """G at mu_i = i/(n-1), i = 0..n-1 (FP64)."""
    if n < 2:
        raise ValueError("a table needs at least 2 entries")
    return np.array([ross_G(kind, i / (n - 1), quad) for i in range(n)])

