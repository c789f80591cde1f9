"""Pins of the CPU oracle's building blocks against what the paper fixes exactly:
moment identities of the equilibria and sources (Appendix A), the defining
auxiliary transformations (Eqs. auxf, auxfbar) behind the shortcut relations,
the parameter closed forms (Eqs. thickness, sigma), printed caption values and
the non-uniform difference formulas (Eqs. nonphi, nonphi2, Appendix B)."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1802_02868_gb300 import inputs as I

XI = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], float)
CS2 = 1.0 / 3.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_point(rng):
    return dict(p=rng.normal() * 1e-2, rho=rng.uniform(0.2, 3.0), ux=rng.normal() * 0.05,
                uy=rng.normal() * 0.05, phi=rng.uniform(-0.1, 1.1), mu=rng.normal() * 1e-3,
                eta=rng.uniform(0.1, 5.0), Fx=rng.normal() * 1e-4, Fy=rng.normal() * 1e-4,
                grx=rng.normal() * 0.1, gry=rng.normal() * 0.1, gamma=rng.normal(),
                lam=rng.uniform(0.01, 1.0), lap_mu=rng.normal() * 1e-4, gpx=rng.normal() * 1e-4,
                gpy=rng.normal() * 1e-4)


def test_feq_moments():
    """Eq. (sum f cf) and Eq. (sum cccf): zeroth to third moments of f^eq."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        s = _rand_point(rng)
        f = oracle.feq(s["p"], s["rho"], s["ux"], s["uy"])
        u = np.array([s["ux"], s["uy"]])
        assert abs(f.sum() - s["p"]) < 1e-15
        np.testing.assert_allclose(XI.T @ f, CS2 * s["rho"] * u, atol=1e-15)
        m2 = np.einsum("ia,ib,i->ab", XI, XI, f)
        np.testing.assert_allclose(m2, CS2 * s["p"] * np.eye(2) + CS2 * s["rho"] * np.outer(u, u), atol=1e-15)
        m3 = np.einsum("ia,ib,ic,i->abc", XI, XI, XI, f)
        d = np.eye(2)
        ref = CS2 * CS2 * s["rho"] * (np.einsum("a,bc->abc", u, d) + np.einsum("b,ac->abc", u, d)
                                      + np.einsum("c,ab->abc", u, d))
        np.testing.assert_allclose(m3, ref, atol=1e-15)


def test_geq_moments():
    """Eq. (sum g cg): sum g^eq = phi, sum xi g^eq = phi u, sum xi xi g^eq = c_s^2 eta mu I + phi u u."""
    rng = np.random.default_rng(2)
    for _ in range(50):
        s = _rand_point(rng)
        g = oracle.geq(s["phi"], s["mu"], s["eta"], s["ux"], s["uy"])
        u = np.array([s["ux"], s["uy"]])
        assert abs(g.sum() - s["phi"]) < 1e-15
        np.testing.assert_allclose(XI.T @ g, s["phi"] * u, atol=1e-15)
        m2 = np.einsum("ia,ib,i->ab", XI, XI, g)
        np.testing.assert_allclose(m2, CS2 * s["eta"] * s["mu"] * np.eye(2) + s["phi"] * np.outer(u, u),
                                   atol=1e-15)
        # the rest-particle weight: H_0 = phi - (1 - omega_0) eta mu (Eq. Hi)
        g0 = oracle.geq(s["phi"], s["mu"], s["eta"], 0.0, 0.0)
        assert abs(g0[0] - (s["phi"] - 5.0 / 9.0 * s["eta"] * s["mu"])) < 1e-15


def test_source_moments():
    """Eqs. (sumF), (sumcF) and (sumG): sum F^f = c_s^2 u.grad rho - c_s^2 rho gamma div(lambda grad mu),
    sum xi F^f = c_s^2 F; sum F^g = 0, sum xi F^g = phi/rho (F - grad p)."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        s = _rand_point(rng)
        Ff = oracle.src_f(s["ux"], s["uy"], s["Fx"], s["Fy"], s["grx"], s["gry"], s["rho"], s["gamma"],
                          s["lam"], s["lap_mu"])
        zero = CS2 * (s["ux"] * s["grx"] + s["uy"] * s["gry"]) - CS2 * s["rho"] * s["gamma"] * s["lam"] * s["lap_mu"]
        assert abs(Ff.sum() - zero) < 1e-16
        np.testing.assert_allclose(XI.T @ Ff, CS2 * np.array([s["Fx"], s["Fy"]]), atol=1e-18)
        Fg = oracle.src_g(s["phi"], s["rho"], s["ux"], s["uy"], s["Fx"], s["Fy"], s["gpx"], s["gpy"])
        assert abs(Fg.sum()) < 1e-17
        G = np.array([s["Fx"] - s["gpx"], s["Fy"] - s["gpy"]])
        np.testing.assert_allclose(XI.T @ Fg, s["phi"] / s["rho"] * G, atol=1e-18)


def test_relations_follow_from_auxiliary_definitions():
    """Eq. (relations1)/(relations2) against the route through the definitions:
    original phi from Eq. (auxf a) inverted, then Eq. (auxfbar a) and (b) with h = dt/2
    for bar-plus and Eq. (auxf b) for tilde-plus; Eq. (original-function) inverts (auxfbar a)."""
    rng = np.random.default_rng(4)
    for _ in range(200):
        tau = rng.uniform(0.01, 50.0)
        dt = rng.uniform(0.01, 2.0)
        h = dt / 2
        tilde, eq, src = rng.normal(size=3)
        # invert auxf(a): tilde = (2tau+dt)/(2tau) phi - dt/(2tau) eq - dt/2 src
        phi = (tilde + dt / (2 * tau) * eq + dt / 2 * src) * 2 * tau / (2 * tau + dt)
        # auxfbar(a), (b) at the cell centre (t_n), bar-plus
        bar = (2 * tau + h) / (2 * tau) * phi - h / (2 * tau) * eq - h / 2 * src
        bar_plus = (2 * tau - h) / (2 * tau + h) * bar + 2 * h / (2 * tau + h) * eq + 2 * tau * h / (2 * tau + h) * src
        # auxf(b)
        tilde_plus = (2 * tau - dt) / (2 * tau + dt) * tilde + 2 * dt / (2 * tau + dt) * eq + 2 * tau * dt / (2 * tau + dt) * src
        scale = 1.0 + abs(tilde) + abs(eq) + abs(src) * (1 + tau)
        assert abs(oracle.bar_plus(tilde, eq, src, tau, dt) - bar_plus) < 1e-13 * scale
        assert abs(oracle.tilde_plus(oracle.bar_plus(tilde, eq, src, tau, dt), tilde) - tilde_plus) < 1e-13 * scale
        # original-function inverts auxfbar(a)
        assert abs(oracle.original(bar, eq, src, tau, h) - phi) < 1e-13 * scale


def test_width_and_sigma_closed_forms():
    """Eqs. (thickness), (sigma); with phiA - phiB = 1, beta = 12 sigma / W and kappa = 3 sigma W / 2."""
    for sigma, W in ((1e-3, 4.0), (5e-5, 4.0), (0.01, 5.0)):
        beta, kappa = I.params_from_sigma_width(sigma, W)
        assert abs(beta - 12 * sigma / W) < 1e-18 and abs(kappa - 1.5 * sigma * W) < 1e-18
        W2, s2 = oracle.width_sigma(beta, kappa)
        assert abs(W2 - W) < 1e-12 * W and abs(s2 - sigma) < 1e-12 * sigma
    # a non-unit phase contrast
    beta, kappa = I.params_from_sigma_width(2e-3, 3.0, phiA=1.0, phiB=-1.0)
    W2, s2 = oracle.width_sigma(beta, kappa, 1.0, -1.0)
    assert abs(W2 - 3.0) < 1e-12 and abs(s2 - 2e-3) < 1e-15


def test_rising_bubble_caption_numbers():
    """Eo, Mo, Re printed in the rising-bubble caption (Sec. 3.3)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "rising_bubble_caption.txt"))
    for ratio, rhoB, Eo, Mo, Re in rows:
        rhoA = rhoB / ratio
        muB = rhoB / 6.0
        e, m, r = I.rising_bubble_numbers(1e-5, 1e-3, 64.0, rhoA, rhoB, muB)
        assert round(e, 2) == pytest.approx(Eo) and round(m, 2) == pytest.approx(Mo)
        assert round(r, 2) == pytest.approx(Re)


def test_tanh_mesh_nodes():
    """Refined-channel generator of Sec. 3.2: nodes span [-1, 1], hit 0 at the centre,
    are symmetric, and cluster toward the walls and the centre (eps = 2.5)."""
    xi = I.tanh_nodes(16)
    assert xi[0] == pytest.approx(-1.0) and xi[-1] == pytest.approx(1.0) and xi[16] == 0.0
    np.testing.assert_allclose(xi, -xi[::-1], atol=1e-15)
    w = np.diff(xi)
    assert w.min() == pytest.approx(w[0]) and w[0] < w[8] and w[15] < w[8]
    dy = I.tanh_channel_heights(64, 64.0)
    assert dy.sum() == pytest.approx(64.0) and dy.min() > 0


def _tanh_mesh(nx, ny, bcx, bcy):
    dx = 1.0 + 0.6 * np.sin(np.linspace(0, 3, nx)) ** 2
    dy = I.tanh_channel_heights(ny, float(ny))
    return I.Mesh(dx, dy, bcx, bcy)


def test_nonuniform_differences_exact_for_quadratics():
    """Eqs. (nonphi), (nonphi2) are exact for quadratics on any 3-point stencil (Appendix B)."""
    mesh = _tanh_mesh(12, 16, I.WALL, I.WALL)
    o = oracle.Oracle(mesh, I.Params(beta=0.003, kappa=0.006))
    xc, yc = mesh.centres()
    X, Y = np.meshgrid(xc, yc)
    F = 0.3 * X ** 2 - 0.2 * X * Y + 0.7 * Y ** 2 + 2 * X - Y
    dx, dy, lap = o.derivatives(F)
    inner = (slice(1, -1), slice(1, -1))
    np.testing.assert_allclose(dx[inner], (0.6 * X - 0.2 * Y + 2)[inner], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(dy[inner], (-0.2 * X + 1.4 * Y - 1)[inner], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(lap[inner], 0.6 + 1.4, rtol=1e-10)


def test_uniform_differences_are_central():
    """On a uniform periodic mesh the formulas reduce to central differences."""
    rng = np.random.default_rng(5)
    mesh = I.uniform_mesh(7, 5, dx=0.5, dy=0.5)
    o = oracle.Oracle(mesh, I.Params(beta=0.003, kappa=0.006))
    F = rng.normal(size=(5, 7))
    dx, dy, lap = o.derivatives(F)
    cdx = (np.roll(F, -1, 1) - np.roll(F, 1, 1)) / (2 * 0.5)
    cdy = (np.roll(F, -1, 0) - np.roll(F, 1, 0)) / (2 * 0.5)
    clap = (np.roll(F, -1, 1) + np.roll(F, 1, 1) + np.roll(F, -1, 0) + np.roll(F, 1, 0) - 4 * F) / 0.25
    np.testing.assert_allclose(dx, cdx, atol=1e-13)
    np.testing.assert_allclose(dy, cdy, atol=1e-13)
    np.testing.assert_allclose(lap, clap, atol=1e-12)


def test_wall_mirror_ghost_gives_zero_normal_flux_of_gradient():
    """Mirror ghosts at walls: a field constant in y has zero y-derivative everywhere and a
    linear-in-y field has the damped one-sided value at the wall rows."""
    mesh = I.uniform_mesh(4, 6, I.PERIODIC, I.WALL)
    o = oracle.Oracle(mesh, I.Params(beta=0.003, kappa=0.006))
    xc, yc = mesh.centres()
    F = np.broadcast_to(yc[:, None], (6, 4)).copy()
    _, dy, lap = o.derivatives(F)
    np.testing.assert_allclose(dy[1:-1], 1.0, atol=1e-14)
    # ghost at distance 1 with the same value: (1*F1 + 2*0*F0 - 1*F0)/(1*1*2) = 0.5
    np.testing.assert_allclose(dy[0], 0.5, atol=1e-14)
    np.testing.assert_allclose(dy[-1], 0.5, atol=1e-14)


def test_derived_parameters():
    """dt = CFL dx_min / sqrt(6 RT) (Eq. cfl, Sec. 3), eta = lambda/(c_s^2 tau_g)
    (Eq. kineticandmobility), gamma = (rho_r - 1)/(phiA - phiB rho_r) (Eq. Gama)."""
    mesh = I.Mesh(np.array([1.0, 0.5, 2.0]), np.array([0.8, 1.2]), I.PERIODIC, I.WALL)
    prm = I.Params(rhoA=3.0, rhoB=1.0, nuA=0.1, nuB=0.2, mobility=0.2, tau_g=0.4, beta=0.003,
                   kappa=0.006, cfl=0.4)
    d = oracle.Oracle(mesh, prm).derived()
    assert d["dt"] == pytest.approx(0.4 * 0.5 / math.sqrt(2.0), rel=1e-15)
    assert d["h"] == pytest.approx(d["dt"] / 2)
    assert d["eta"] == pytest.approx(0.2 / (0.4 / 3.0), rel=1e-15)
    assert d["gamma"] == pytest.approx((3.0 - 1.0) / (1.0 - 0.0), rel=1e-15)
    assert d["muA"] == pytest.approx(0.3) and d["muB"] == pytest.approx(0.2)


def test_complex_step_build_matches_real_build_and_central_differences():
    """The double-complex oracle (complex step) reproduces the real oracle's values
    exactly and its derivatives agree with central differences of the real oracle."""
    mesh = I.Mesh(1.0 + 0.2 * np.sin(np.arange(12)), np.ones(10), I.PERIODIC, I.WALL)
    beta, kappa = I.params_from_sigma_width(1e-2, 3.0)
    prm = I.Params(rhoA=2.0, rhoB=1.0, nuA=0.1, nuB=0.2, mobility=0.3, beta=beta, kappa=kappa, gy=-1e-4, rho_ref=1.5)
    phi0 = I.drop_field(mesh, 3.0, (6.0, 5.0), 3.0)
    steps = 6
    target = np.full(phi0.shape, 0.3)
    o = oracle.Oracle(mesh, prm).init(phi0)
    o.step(steps)
    cs = oracle.OracleCS(mesh, prm.as_list()).init(phi0).step(steps)
    np.testing.assert_array_equal(cs.phi().real, o.moments()["phi"])

    def L(p, phi):
        r = oracle.Oracle(mesh, p).init(phi)
        r.step(steps)
        d = r.moments()["phi"] - target
        return np.sum(d * d)

    rng = np.random.default_rng(9)
    v = rng.standard_normal(phi0.shape)
    g = oracle.complex_step_gradient(mesh, prm, phi0, steps, target, direction_phi0=v, which=("kappa", "mobility"))
    for name in ("kappa", "mobility"):
        eps = 1e-5 * getattr(prm, name)
        pp, pm = I.Params(**vars(prm)), I.Params(**vars(prm))
        setattr(pp, name, getattr(prm, name) + eps)
        setattr(pm, name, getattr(prm, name) - eps)
        fd = (L(pp, phi0) - L(pm, phi0)) / (2 * eps)
        assert g[name] == pytest.approx(fd, rel=1e-5)
    eps = 1e-6
    fd = (L(prm, phi0 + eps * v) - L(prm, phi0 - eps * v)) / (2 * eps)
    assert g["phi0_dir"] == pytest.approx(fd, rel=1e-6)
