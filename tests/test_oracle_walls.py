"""Pins of the oracle's no-slip wall treatment (reading of Sec. 3.2's
"no-slip" and Sec. 3.4's "bounce-back" walls): what a wall face carries
besides its bar distributions.

A y-invariant order-parameter field phi(x) at rest, whose pressure balances
the capillary force -phi dmu/dx, stays at rest in the continuum (the force is
a gradient along x that the pressure takes up), so a no-slip wall at rest
exerts no shear on it at the start (Stokes' first problem: the wall shear of
a fluid at rest is zero).  Two consequences are checked after the first step,
against the same state on a mesh without walls (periodic in y), where every
y face carries the y-mirror image of its distributions:

* the distributions that enter each wall row through the wall (bounced back
  from the outgoing ones) equal those that cross the same face without the
  wall, up to a small fraction of the distributions' x-asymmetry
  |phi_5 - phi_6|, the scale on which a wall shear would show;
* the wall row's velocity is the bulk velocity of its column times one no-slip
  factor in (0.8, 1], the same for every column: the wall only retards the
  flow, by an amount set by nu t / dy^2 and not by the local force.

At a wall face the reading keeps the wall cell's tangential gradients of mu,
p and phi (zero normal gradients).  A wall face that drops the tangential
grad mu (the capillary force along the wall) or the tangential grad p makes
the bounced-back distributions carry a shear of 5e-3 to 9e-2 of that scale
and breaks the column-independent factor; the current reading stays below
2e-3.  The tangential grad phi enters only through u_b . grad rho and
s_i(u_b) c_s^2 grad rho (Eqs. P, F), both zero with the wall velocity u_b = 0,
so its reading cannot change a wall flux.
"""
import numpy as np
import pytest

import oracle
from paper_1802_02868_gb300 import inputs as I

CASES = [
    # (amplitude, rhoA, rhoB, nu, mobility)
    (0.3, 1.0, 1.0, 0.1, 0.1),
    (0.2, 3.0, 1.0, 0.5, 0.5),
]
NX, NY = 32, 8


def _state(amp, rhoA, rhoB, nu, lam):
    beta, kappa = I.params_from_sigma_width(1e-3, 4.0)
    prm = I.Params(rhoA=rhoA, rhoB=rhoB, nuA=nu, nuB=nu, mobility=lam, beta=beta, kappa=kappa,
                   rho_ref=0.5 * (rhoA + rhoB))
    x = np.arange(NX) + 0.5
    phi = np.repeat((0.5 + amp * np.cos(2 * np.pi * x / NX))[None, :], NY, axis=0)
    # pressure that balances F_x = -phi dmu/dx column by column (trapezoidal
    # integral of the oracle's own cell force), periodic with zero mean
    o = oracle.Oracle(I.Mesh(np.ones(NX), np.ones(NY)), prm).init(phi)
    o.moments()
    Fx = -phi[0] * o.aux()["gmux"][0]
    P = np.concatenate([[0.0], np.cumsum(0.5 * (Fx[1:] + Fx[:-1]))])
    P -= P.mean()
    return prm, phi, np.repeat(P[None, :], NY, axis=0)


def _one_step(prm, phi, p0, bc_y):
    o = oracle.Oracle(I.Mesh(np.ones(NX), np.ones(NY), I.PERIODIC, bc_y), prm).init(phi, p=p0)
    o.step(1)
    f, g = o.state()
    return f, g, o.moments()


@pytest.mark.parametrize("case", CASES)
def test_wall_exerts_no_shear_on_a_force_balanced_fluid_at_rest(case):
    prm, phi, p0 = _state(*case)
    fw, gw, mw = _one_step(prm, phi, p0, I.WALL)
    fp, gp, mp = _one_step(prm, phi, p0, I.PERIODIC)
    # without walls the state keeps its y-mirror symmetry exactly
    assert np.abs(mp["uy"]).max() < 1e-15
    for wall, ref in ((fw, fp), (gw, gp)):
        scale = np.abs(ref[5, 0] - ref[6, 0]).max()
        assert scale > 1e-8
        # incoming directions at the bottom wall (4, 7, 8) and at the top wall (2, 5, 6)
        low = max(np.abs(wall[q, 0] - ref[q, 0]).max() for q in (4, 7, 8))
        high = max(np.abs(wall[q, -1] - ref[q, -1]).max() for q in (2, 5, 6))
        assert low < 0.01 * scale and high < 0.01 * scale, (low / scale, high / scale)
    # the wall row moves like the bulk of its column, retarded by one factor
    bulk = mp["ux"][0]
    sel = np.abs(bulk) > 0.3 * np.abs(bulk).max()
    for row in (0, NY - 1):
        r = mw["ux"][row][sel] / bulk[sel]
        assert 0.8 < r.min() and r.max() <= 1.0 and r.max() - r.min() < 0.05, (r.min(), r.max())
