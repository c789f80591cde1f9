"""The single-phase limit (phi = phiA everywhere, so mu = 0 and the g
distributions stay at equilibrium): DUGKS for one fluid, the scheme the paper
extends (Sec. 1, 2).  Closed forms on the GPU: shear-wave and Taylor-Green
decay at the rates nu k^2 and 2 nu k^2 with nu = c_s^2 tau_f (Eq.
kineticandmobility), and the body-force channel's parabolic profile between
bounce-back walls; plus parity with the oracle on the same inputs."""
import math

import numpy as np
import pytest

import oracle
from paper_1802_02868_gb300 import dugks
from paper_1802_02868_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _params(nu, **kw):
    beta, kappa = I.params_from_sigma_width(1e-3, 4.0)
    return I.Params(rhoA=1.0, rhoB=1.0, nuA=nu, nuB=nu, beta=beta, kappa=kappa, **kw)


def _rate(ts, amps):
    return -math.log(amps[-1] / amps[0]) / (ts[-1] - ts[0])


@pytest.mark.parametrize("prec", [dugks.FP64, dugks.FP32])
def test_shear_wave_decay_rate(prec):
    nx, ny, nu = 64, 96, 0.05
    mesh = I.uniform_mesh(nx, ny)
    _, yc = mesh.centres()
    k = 2 * math.pi / ny
    ux = 1e-3 * np.repeat(np.sin(k * yc)[:, None], nx, axis=1)
    s = dugks.Sim(mesh, _params(nu), prec).init(np.ones((ny, nx)), ux=ux)
    ts, amps = [], []
    for n in range(1, 7):
        s.step(200)
        u = s.moments()["ux"]
        amps.append(2 / ny * np.mean(np.sum(u * np.sin(k * yc)[:, None], axis=0)))
        ts.append(n * 200 * s.dt())
    assert _rate(ts[1:], amps[1:]) == pytest.approx(nu * k * k, rel=0.015)


@pytest.mark.parametrize("prec", [dugks.FP64, dugks.FP32])
def test_taylor_green_decay_rate(prec):
    """u = U sin(kx) cos(ky), v = -U cos(kx) sin(ky) on a periodic square: the
    kinetic energy's amplitude decays at 2 nu k^2."""
    n, nu, U = 64, 0.02, 1e-3
    mesh = I.uniform_mesh(n, n)
    xc, yc = mesh.centres()
    X, Y = np.meshgrid(xc, yc)
    k = 2 * math.pi / n
    ux, uy = U * np.sin(k * X) * np.cos(k * Y), -U * np.cos(k * X) * np.sin(k * Y)
    p = 0.25 * U * U * (np.cos(2 * k * X) + np.cos(2 * k * Y))   # the vortex's pressure (rho = 1)
    s = dugks.Sim(mesh, _params(nu), prec).init(np.ones((n, n)), ux=ux, uy=uy, p=p)
    ts, amps = [], []
    for m in range(1, 6):
        s.step(300)
        u = s.moments()["ux"]
        amps.append(np.sum(u * np.sin(k * X) * np.cos(k * Y)) / np.sum((np.sin(k * X) * np.cos(k * Y)) ** 2))
        ts.append(m * 300 * s.dt())
    assert _rate(ts[1:], amps[1:]) == pytest.approx(2 * nu * k * k, rel=0.02)


@pytest.mark.parametrize("prec", [dugks.FP64, dugks.FP32])
def test_body_force_channel_profile(prec):
    """Walls at y = 0 and H (bounce-back), x periodic, force G: the steady
    profile G y (H - y) / (2 nu), held from the analytic start on a tanh-refined
    mesh."""
    nx, ny, H, G, nu = 4, 64, 64.0, 1e-6, 0.1
    mesh = I.Mesh(np.ones(nx), I.tanh_channel_heights(ny, H, 2.5), I.PERIODIC, I.WALL)
    _, yc = mesh.centres()
    ua = G * yc * (H - yc) / (2 * nu)
    s = dugks.Sim(mesh, _params(nu, gx=G), prec)
    s.init(np.ones((ny, nx)), ux=np.repeat(ua[:, None], nx, axis=1)).step(20000)
    u = s.moments()["ux"][:, 0]
    assert np.linalg.norm(u - ua) / np.linalg.norm(ua) < 5e-3
    s.close()
    # and a channel started from rest approaches it: after five viscous times
    # (H^2 / (pi^2 nu) each; nu = 0.5 to keep the run short) the centre-line
    # speed is within 2 %
    nu2 = 0.5
    s = dugks.Sim(mesh, _params(nu2, gx=G), prec).init(np.ones((ny, nx)))
    s.step(int(round(5 * H * H / (math.pi ** 2 * nu2) / s.dt())))
    u = s.moments()["ux"][:, 0]
    assert u[ny // 2] == pytest.approx(ua[ny // 2] * nu / nu2, rel=0.02)
    s.close()


def test_single_phase_parity_with_oracle():
    """FP64, one step from the oracle's state after 50 steps of a Taylor-Green
    vortex on a non-uniform periodic mesh."""
    rng = np.random.default_rng(9)
    mesh = I.Mesh(0.8 + 0.4 * rng.random(40), 0.8 + 0.4 * rng.random(24))
    xc, yc = mesh.centres()
    X, Y = np.meshgrid(xc, yc)
    Lx, Ly = mesh.dx.sum(), mesh.dy.sum()
    ux = 1e-3 * np.sin(2 * math.pi * X / Lx) * np.cos(2 * math.pi * Y / Ly)
    prm = _params(0.03)
    o = oracle.Oracle(mesh, prm).init(np.ones_like(X), ux=ux)
    o.step(50)
    f, g = o.state()
    s = dugks.Sim(mesh, prm, dugks.FP64).init(np.ones_like(X), ux=ux)
    s.set_state(f, g)
    o.step(1)
    s.step(1)
    fo, go = o.state()
    fs, gs = s.state()
    assert np.max(np.abs(fs - fo)) <= 1e-12 * np.max(np.abs(fo))
    assert np.max(np.abs(gs - go)) <= 1e-12 * np.max(np.abs(go))
