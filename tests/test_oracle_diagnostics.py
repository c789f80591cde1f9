"""Pins of the oracle's diagnostics (oracle/diagnostics.py) against values the
paper prints and closed forms: Table A1's initial droplet masses, the flat
equilibrium interface for the Laplace pressure's sign, exact crossings of
linear columns, and symmetric centroids."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import diagnostics as D
from paper_1802_02868_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_table_a1_initial_droplet_masses():
    """Sec. 3.1, Table A1: droplets of radius R0 = 20..36 on a 100 x 100 periodic
    mesh, W = 4, centred on a cell centre.  The droplet mass is the volume on the
    A side of the median level; the printed initial masses are reproduced
    exactly, both from the field and from the oracle's state after its
    initialisation (Sec. 2.2, step 1)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "table_a1_mass.txt"))
    beta, kappa = I.params_from_sigma_width(1e-3, 4.0)
    for R0, m_ini, _, _ in rows:
        mesh = I.uniform_mesh(100, 100)
        phi = I.drop_field(mesh, R0, (50.5, 50.5), 4.0)
        zeros = np.zeros_like(phi)
        d = D.region_stats(mesh, phi, zeros, zeros, zeros, 1.0, 0.0)
        assert d["mass"] == m_ini
        p = I.Params(rhoA=1.0, rhoB=0.2, beta=beta, kappa=kappa, cfl=0.4)
        o = oracle.Oracle(mesh, p).init(phi)
        assert D.diagnostics(o, mesh, p)[0]["mass"] == m_ini
        o.close()


def test_table_a1_relative_errors_follow_from_the_printed_masses():
    """The printed relative errors are (M_ini - M_ter) / M_ini in percent, to the
    printed two decimals (one of them truncated rather than rounded)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "table_a1_mass.txt"))
    for _, m_ini, m_ter, err in rows:
        assert 100.0 * (m_ini - m_ter) / m_ini == pytest.approx(err, abs=0.0095)


def _flat_interface(dy, width=4.0, ny=None):
    ny = ny or int(round(64 / dy))
    mesh = I.Mesh(np.ones(4), np.full(ny, dy), I.PERIODIC, I.WALL)
    beta, kappa = I.params_from_sigma_width(1e-3, width)
    p = I.Params(beta=beta, kappa=kappa)
    _, yc = mesh.centres()
    Y = np.broadcast_to(yc[:, None], (ny, 4))
    H = 0.5 * ny * dy
    # fluid A below, the equilibrium profile of the double well: W^2 = 8 kappa / beta
    phi = 0.5 + 0.5 * np.tanh(2.0 * (H - Y) / width)
    return mesh, p, phi


def test_laplace_pressure_is_constant_across_a_flat_equilibrium_interface():
    """Sec. 3.1's P with the printed + kappa |grad phi|^2 / 2: across a flat
    equilibrium profile psi' = kappa phi'' and kappa phi'^2 / 2 = psi, so
    P - p vanishes (with the opposite sign it would reach 2 psi = beta / 8).
    With the oracle's own derivatives the residual is the stencils' truncation
    error: a few percent of max psi, falling four-fold per halving of dy."""
    res = []
    for dy in (0.5, 0.25):
        mesh, p, phi = _flat_interface(dy)
        o = oracle.Oracle(mesh, p)
        gx, gy, lap = o.derivatives(phi)
        o.close()
        zero = np.zeros_like(phi)
        dP = D.laplace_pressure(phi, zero, gx, gy, lap, p.phiA, p.phiB, p.beta, p.kappa)
        psi_max = p.beta / 16.0
        res.append(np.max(np.abs(dP)) / psi_max)
        # the gradient term alone is of the size of psi: the sign is decisive
        assert np.max(0.5 * p.kappa * gy ** 2) > 0.9 * psi_max
    assert res[1] < 0.025
    assert 3.5 < res[0] / res[1] < 4.5


def test_laplace_pressure_terms_on_a_quadratic_field():
    """Each term in its place: on a quadratic phi the three-point derivatives of
    Eqs. (nonphi), (nonphi2) are exact on any spacing, so P equals the closed
    form away from the walls (mirror ghosts there)."""
    rng = np.random.default_rng(11)
    ny = 24
    mesh = I.Mesh(np.ones(3), 0.6 + 0.8 * rng.random(ny), I.PERIODIC, I.WALL)
    beta, kappa = 0.7, 0.3
    p = I.Params(beta=beta, kappa=kappa)
    _, yc = mesh.centres()
    Y = np.broadcast_to(yc[:, None], (ny, 3))
    a, b, c = 0.2, 0.03, 0.002
    phi = a + b * Y + c * Y ** 2
    pp = np.sin(Y)
    o = oracle.Oracle(mesh, p)
    gx, gy, lap = o.derivatives(phi)
    o.close()
    P = D.laplace_pressure(phi, pp, gx, gy, lap, 1.0, 0.0, beta, kappa)
    d1, d2 = b + 2 * c * Y, 2 * c
    psi = beta * phi ** 2 * (phi - 1) ** 2
    dpsi = 2 * beta * phi * (phi - 1) * (2 * phi - 1)
    expect = phi * dpsi - psi - kappa * phi * d2 + 0.5 * kappa * d1 ** 2 + pp
    inner = slice(1, ny - 1)
    assert np.allclose(P[inner], expect[inner], rtol=1e-12, atol=1e-15)


def test_front_and_tip_of_linear_columns_are_exact():
    """Sec. 3.4's front and tip: with phi linear in y in each column (A above),
    linear interpolation puts each crossing exactly at the column's level."""
    rng = np.random.default_rng(5)
    nx, ny = 7, 40
    mesh = I.Mesh(np.ones(nx), 0.5 + rng.random(ny), I.PERIODIC, I.WALL)
    _, yc = mesh.centres()
    H = yc[3] + (yc[-4] - yc[3]) * rng.random(nx)
    phi = 0.5 + (yc[:, None] - H[None, :]) / 50.0
    phi[:, 2] = 0.2                                # a column without a crossing
    front, tip = D.front_and_tip(mesh, phi, 1.0, 0.0)
    keep = np.delete(H, 2)
    assert front == pytest.approx(keep.max(), rel=1e-13)
    assert tip == pytest.approx(keep.min(), rel=1e-13)
    assert all(np.isnan(v) for v in D.front_and_tip(mesh, np.full((ny, nx), 0.2), 1.0, 0.0))


def test_front_and_tip_of_a_cosine_interface():
    """A single-mode Rayleigh-Taylor interface y0 + a cos(2 pi x / L) (Sec. 3.4):
    the front and tip sit at y0 +- a times the extreme cosine at the cell
    centres, to within the interpolation error of the tanh profile."""
    L, a, y0 = 64, 6.4, 128.0
    mesh = I.Mesh(np.ones(L), np.ones(4 * L), I.PERIODIC, I.WALL)
    phi = I.rt_field(mesh, L, y0, [a], 4.0)
    xc, _ = mesh.centres()
    cs = np.cos(2 * math.pi * xc / L)
    front, tip = D.front_and_tip(mesh, phi, 1.0, 0.0)
    assert front == pytest.approx(y0 + a * cs.max(), abs=0.02)
    assert tip == pytest.approx(y0 + a * cs.min(), abs=0.02)


def test_centroid_and_mean_velocity():
    """A drop centred on a mirror-symmetric mesh has its centroid at the centre;
    the region's mean velocity of a uniform flow is that flow."""
    dx = np.concatenate([np.linspace(1.5, 0.5, 20), np.linspace(0.5, 1.5, 20)])
    mesh = I.Mesh(dx, dx.copy())
    xc, _ = mesh.centres()
    ctr = float(dx.sum() / 2)
    phi = I.drop_field(mesh, 7.0, (ctr, ctr), 3.0)
    ux, uy = np.full_like(phi, 0.3), np.full_like(phi, -0.2)
    d = D.region_stats(mesh, phi, ux, uy, np.zeros_like(phi), 1.0, 0.0)
    assert d["xc"] == pytest.approx(ctr, rel=1e-13) and d["yc"] == pytest.approx(ctr, rel=1e-13)
    assert d["ux"] == pytest.approx(0.3, rel=1e-13) and d["uy"] == pytest.approx(-0.2, rel=1e-13)
    vol = np.outer(mesh.dy, mesh.dx)
    assert d["mass"] == pytest.approx(vol[phi > 0.5].sum(), rel=1e-15)
    assert 0 < d["mass"] < math.pi * 7.0 ** 2 * 1.1
