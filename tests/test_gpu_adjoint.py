"""GPU adjoint (dugks_adjoint) against the oracle's exact FP64 derivatives by
the complex step, for L = sum_cells (phi_T - phi*)^2 with respect to kappa, the
mobility lambda and the initial phi field (random directional derivatives), on
periodic and walled meshes; checkpoint spacing must not change the gradient."""
import numpy as np
import pytest

import oracle
from paper_1802_02868_gb300 import dugks
from paper_1802_02868_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _cases():
    beta, kappa = I.params_from_sigma_width(1e-2, 3.0)
    out = []
    m = I.Mesh(1.0 + 0.2 * np.sin(np.arange(12)), np.ones(10), I.PERIODIC, I.WALL)
    p = I.Params(rhoA=2.0, rhoB=1.0, nuA=0.1, nuB=0.2, mobility=0.3, beta=beta, kappa=kappa, gy=-1e-4, rho_ref=1.5)
    out.append(("rt_walls_y", m, p, I.drop_field(m, 3.0, (6.0, 5.0), 3.0)))
    m = I.uniform_mesh(10, 9)
    p = I.Params(rhoA=3.0, rhoB=1.0, nuA=0.05, nuB=0.15, mobility=0.2, tau_g=0.7, beta=beta, kappa=kappa, gx=2e-5,
                 rho_ref=1.0, cfl=0.6)
    out.append(("drop_periodic", m, p, I.drop_field(m, 2.5, (5.0, 4.5), 3.0)))
    rng = np.random.default_rng(3)
    m = I.Mesh(0.8 + 0.4 * rng.random(9), 0.8 + 0.4 * rng.random(8), I.WALL, I.WALL)
    p = I.Params(rhoA=1.5, rhoB=1.0, nuA=0.2, nuB=0.1, mobility=0.25, beta=beta, kappa=kappa, gx=1e-4, gy=-2e-4,
                 rho_ref=1.2, cfl=0.7)
    out.append(("box_walls_xy", m, p, I.drop_field(m, 2.5, (4.0, 3.5), 3.0)))
    return out


CASES = _cases()
STEPS = 12


@pytest.mark.parametrize("name,mesh,prm,phi0", CASES, ids=[c[0] for c in CASES])
def test_fp64_adjoint_matches_complex_step_oracle(name, mesh, prm, phi0):
    rng = np.random.default_rng(11)
    target = 0.5 + 0.1 * rng.standard_normal(phi0.shape)
    sim = dugks.Sim(mesh, prm, dugks.FP64).init(phi0)
    got = sim.adjoint(STEPS, target, ckpt_every=5)
    v = rng.standard_normal(phi0.shape)
    ref = oracle.complex_step_gradient(mesh, prm, phi0, STEPS, target, direction_phi0=v, which=("kappa", "mobility"))
    o = oracle.Oracle(mesh, prm).init(phi0)
    o.step(STEPS)
    d = o.moments()["phi"] - target
    assert got["loss"] == pytest.approx(np.sum(d * d), rel=1e-11)
    assert got["dkappa"] == pytest.approx(ref["kappa"], rel=1e-8)
    assert got["dlambda"] == pytest.approx(ref["mobility"], rel=1e-8)
    assert np.sum(got["dphi0"] * v) == pytest.approx(ref["phi0_dir"], rel=1e-8)


def test_checkpoint_spacing_does_not_change_the_gradient():
    name, mesh, prm, phi0 = CASES[0]
    target = np.full(phi0.shape, 0.4)
    sim = dugks.Sim(mesh, prm, dugks.FP64).init(phi0)
    a = sim.adjoint(STEPS, target, ckpt_every=1)
    b = sim.adjoint(STEPS, target, ckpt_every=STEPS)
    c = sim.adjoint(STEPS, target, ckpt_every=5)
    # the recomputed forward is bit-identical; the adjoint's scatter uses FP64
    # atomics, whose summation order varies, so agreement is to rounding
    for k in ("loss", "dkappa", "dlambda"):
        assert b[k] == pytest.approx(a[k], rel=1e-12) and c[k] == pytest.approx(a[k], rel=1e-12)
    scale = np.abs(a["dphi0"]).max()
    assert np.abs(a["dphi0"] - b["dphi0"]).max() <= 1e-12 * scale
    assert np.abs(a["dphi0"] - c["dphi0"]).max() <= 1e-12 * scale
    # and the simulation is left at the final forward state
    ref = dugks.Sim(mesh, prm, dugks.FP64).init(phi0)
    ref.step(STEPS)
    np.testing.assert_array_equal(sim.state()[1], ref.state()[1])


def test_fp32_adjoint_close_to_fp64():
    name, mesh, prm, phi0 = CASES[1]
    target = np.full(phi0.shape, 0.3)
    a = dugks.Sim(mesh, prm, dugks.FP64).init(phi0).adjoint(STEPS, target, ckpt_every=4)
    b = dugks.Sim(mesh, prm, dugks.FP32).init(phi0).adjoint(STEPS, target, ckpt_every=4)
    assert b["dkappa"] == pytest.approx(a["dkappa"], rel=2e-3)
    assert b["dlambda"] == pytest.approx(a["dlambda"], rel=2e-3)
    assert np.abs(b["dphi0"] - a["dphi0"]).max() <= 2e-3 * np.abs(a["dphi0"]).max()


def test_batch_adjoint_is_per_instance():
    sims = [c for c in CASES[:2]]
    targets = [np.full(c[3].shape, 0.45) for c in sims]
    batch = dugks.Sim([c[1] for c in sims], [c[2] for c in sims], dugks.FP64).init([c[3] for c in sims])
    got = batch.adjoint(STEPS, targets, ckpt_every=6)
    for k, (name, mesh, prm, phi0) in enumerate(sims):
        one = dugks.Sim(mesh, prm, dugks.FP64).init(phi0).adjoint(STEPS, targets[k], ckpt_every=6)
        assert got["loss"][k] == pytest.approx(one["loss"], rel=1e-12)
        assert got["dkappa"][k] == pytest.approx(one["dkappa"], rel=1e-10)
        assert got["dlambda"][k] == pytest.approx(one["dlambda"], rel=1e-10)
        np.testing.assert_allclose(got["dphi0"][k], one["dphi0"], rtol=1e-10, atol=1e-14)
