"""Diagnostics of a two-phase DUGKS state -- TEST INFRASTRUCTURE ONLY.

Same rules as the rest of ``oracle/``: only tests, the smoke check and the
benchmark's CPU leg use it.  Plain numpy in FP64 over the fields that the
oracle's ``moments`` and ``derivatives`` return.

Definitions, each from the paper's test section it serves:

* Laplace pressure (Sec. 3.1, Laplace's law): P = p0 - kappa phi lap(phi)
  + kappa |grad phi|^2 / 2 + p with the equation of state p0 = phi psi'(phi)
  - psi(phi) and the double-well bulk energy psi = beta (phi - phiA)^2
  (phi - phiB)^2 (Sec. 2.1).  The sign of the gradient term is the printed
  one; it makes P the pressure normal to a flat interface, which is constant
  across a flat interface at equilibrium (pinned in the tests).
* Droplet mass (Sec. 3.1, Table A1): the total volume of the cells whose
  order parameter lies strictly on the A side of the median level
  (phiA + phiB) / 2.  With unit cells this is a cell count; it reproduces the
  initial masses printed in Table A1 exactly.
* Centroid and mean velocity of that region (Sec. 3.3, the rising bubble),
  volume-weighted, in the mesh's coordinates (low faces at 0, no unwrapping
  across periodic boundaries).
* Bulk pressures: the volume-weighted mean of P over the cells with
  c = (phi - phiB) / (phiA - phiB) > 0.9 (bulk A) and c < 0.1 (bulk B); their
  difference is the Laplace jump Delta P of Sec. 3.1.
* Front and tip (Sec. 3.4, Rayleigh-Taylor): every pair of vertically
  adjacent cells of a column with c < 1/2 below and c >= 1/2 above holds one
  crossing of the median level, placed by linear interpolation between the
  two cell centres.  With fluid A on top, the highest crossing is the bubble
  front and the lowest the spike tip.  Pairs across a periodic y boundary are
  not counted.
"""
from __future__ import annotations

import numpy as np


def laplace_pressure(phi, p, gphix, gphiy, lapphi, phiA, phiB, beta, kappa):
    """Sec. 3.1: P = phi psi' - psi - kappa phi lap(phi) + kappa |grad phi|^2 / 2 + p."""
    psi = beta * (phi - phiA) ** 2 * (phi - phiB) ** 2
    dpsi = 2.0 * beta * (phi - phiA) * (phi - phiB) * ((phi - phiA) + (phi - phiB))
    p0 = phi * dpsi - psi
    return p0 - kappa * phi * lapphi + 0.5 * kappa * (gphix ** 2 + gphiy ** 2) + p


def region_stats(mesh, phi, ux, uy, P, phiA, phiB):
    """Droplet mass, centroid, mean velocity and bulk pressures (definitions above)."""
    xc, yc = mesh.centres()
    X, Y = np.meshgrid(xc, yc)
    vol = np.outer(mesh.dy, mesh.dx)
    c = (phi - phiB) / (phiA - phiB)
    a = c > 0.5
    mass = float(vol[a].sum())
    out = {"mass": mass}
    if mass > 0:
        out["xc"] = float((vol * X)[a].sum() / mass)
        out["yc"] = float((vol * Y)[a].sum() / mass)
        out["ux"] = float((vol * ux)[a].sum() / mass)
        out["uy"] = float((vol * uy)[a].sum() / mass)
    else:
        out.update(xc=np.nan, yc=np.nan, ux=np.nan, uy=np.nan)
    for key, sel in (("p_bulk_A", c > 0.9), ("p_bulk_B", c < 0.1)):
        v = float(vol[sel].sum())
        out[key] = float((vol * P)[sel].sum() / v) if v > 0 else np.nan
    return out


def crossings(mesh, phi, phiA, phiB):
    """Heights of the upward crossings of the median level (definition above)."""
    _, yc = mesh.centres()
    c = (phi - phiB) / (phiA - phiB)
    lo, hi = c[:-1, :], c[1:, :]
    j, i = np.nonzero((lo < 0.5) & (hi >= 0.5))
    t = (0.5 - lo[j, i]) / (hi[j, i] - lo[j, i])
    return yc[j] + t * (yc[j + 1] - yc[j])


def front_and_tip(mesh, phi, phiA, phiB):
    y = crossings(mesh, phi, phiA, phiB)
    if y.size == 0:
        return np.nan, np.nan
    return float(y.max()), float(y.min())


def diagnostics(o, mesh, params):
    """All diagnostics of the oracle ``o``'s current state, and the P field."""
    m = o.moments()
    gx, gy, lap = o.derivatives(m["phi"])
    P = laplace_pressure(m["phi"], m["p"], gx, gy, lap, params.phiA, params.phiB, params.beta, params.kappa)
    d = region_stats(mesh, m["phi"], m["ux"], m["uy"], P, params.phiA, params.phiB)
    d["front_y"], d["tip_y"] = front_and_tip(mesh, m["phi"], params.phiA, params.phiB)
    return d, P
