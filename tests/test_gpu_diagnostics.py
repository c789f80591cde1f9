"""GPU diagnostics (dugks_diagnostics, dugks_laplace_pressure) against the
oracle's (oracle/diagnostics.py) on the same states, and against Table A1's
printed initial droplet masses; at full size on the Rayleigh-Taylor mesh and a
sample of the 512-instance ensemble."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import diagnostics as D
from paper_1802_02868_gb300 import dugks
from paper_1802_02868_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KEYS = ("mass", "xc", "yc", "ux", "uy", "p_bulk_A", "p_bulk_B", "front_y", "tip_y")


def _cases():
    rng = np.random.default_rng(3)
    out = [I.stationary_drop(n=64, radius=16.0), I.rayleigh_taylor(nx=32, ny=96, amplitudes=[3.2])]
    m = I.Mesh(1.0 + 0.5 * rng.random(37), 0.7 + 0.6 * rng.random(29), I.WALL, I.WALL)
    beta, kappa = I.params_from_sigma_width(2e-3, 4.0)
    p = I.Params(rhoA=3.0, rhoB=1.0, nuA=0.2, nuB=0.05, mobility=0.2, tau_g=0.7, beta=beta, kappa=kappa,
                 gx=2e-6, gy=-1e-5, rho_ref=2.0, cfl=0.7)
    out.append(I.Case("ragged", m, p, I.drop_field(m, 8.0, (20.0, 12.0), 4.0)))
    return out


CASES = _cases()


def _ambiguous_volume(mesh, phi, params, eps=1e-9):
    """Volume of the cells whose side of the median level rounding may decide."""
    c = (phi - params.phiB) / (params.phiA - params.phiB)
    return float(np.outer(mesh.dy, mesh.dx)[np.abs(c - 0.5) < eps].sum())


def _compare(dg, do, Pg, Po, mesh, m, params, rtol, ptol, eps=1e-9, ufloor=1e-16, mtol=0.0):
    """m: the oracle's moments; velocities are compared on the scale of the
    largest velocity of the mesh.  mtol: relative rounding of the volume sum
    (FP32 sims sum single-precision cell volumes within a strip); in any
    precision the two sides add the same FP64 volumes in different orders,
    which moves an n-term sum by at most about n units of 2^-53 relative."""
    mtol = max(mtol, mesh.ncells * 2.0 ** -53)
    assert abs(dg["mass"] - do["mass"]) <= _ambiguous_volume(mesh, m["phi"], params, eps) + mtol * do["mass"]
    scale_u = max(np.max(np.abs(m["ux"])), np.max(np.abs(m["uy"])), 1e-300)
    for k in KEYS[1:]:
        a, b = dg[k], do[k]
        if math.isnan(b):
            assert math.isnan(a), k
            continue
        # velocities: on the mesh's velocity scale, with a floor at the rounding
        # level of a state at rest
        tol = rtol * scale_u + ufloor if k in ("ux", "uy") else rtol * max(abs(b), 1.0)
        assert abs(a - b) <= tol, (k, a, b)
    assert np.max(np.abs(Pg - Po)) <= ptol * max(np.max(np.abs(Po)), 1e-300)


@pytest.mark.parametrize("steps", [0, 60])
def test_fp64_diagnostics_match_oracle(steps):
    """Each case and all three as one batch: P field, mass, centroid, mean
    velocity, bulk pressures, front and tip against the oracle's on the
    oracle's state (loaded into the GPU)."""
    states, refs = [], []
    for c in CASES:
        o = oracle.Oracle(c.mesh, c.params).init(c.phi0)
        o.step(steps)
        d, P = D.diagnostics(o, c.mesh, c.params)
        states.append(o.state())
        refs.append((d, P, o.moments()))
        o.close()
    for k, c in enumerate(CASES):
        s = dugks.Sim(c.mesh, c.params, dugks.FP64)
        s.init(c.phi0)
        s.set_state(*states[k])
        _compare(s.diagnostics(), refs[k][0], s.laplace_pressure(), refs[k][1], c.mesh, refs[k][2], c.params,
                 1e-10, 1e-11)
        s.close()
    b = dugks.Sim([c.mesh for c in CASES], [c.params for c in CASES], dugks.FP64)
    b.init([c.phi0 for c in CASES])
    b.set_state(np.concatenate([st[0].reshape(9, -1) for st in states], axis=1),
                np.concatenate([st[1].reshape(9, -1) for st in states], axis=1))
    ds, Ps = b.diagnostics(), b.laplace_pressure()
    for k, c in enumerate(CASES):
        _compare(ds[k], refs[k][0], Ps[k], refs[k][1], c.mesh, refs[k][2], c.params, 1e-10, 1e-11)
    b.close()


def test_fp32_diagnostics_after_init_match_oracle():
    """FP32 storage: the same quantities after the initialisation of step 1, to
    the single-precision rounding of p and u."""
    for c in CASES:
        o = oracle.Oracle(c.mesh, c.params).init(c.phi0)
        d, P = D.diagnostics(o, c.mesh, c.params)
        m = o.moments()
        o.close()
        s = dugks.Sim(c.mesh, c.params, dugks.FP32).init(c.phi0)
        _compare(s.diagnostics(), d, s.laplace_pressure(), P, c.mesh, m, c.params, 2e-5, 2e-5, eps=1e-6,
                 ufloor=1e-12, mtol=1e-6)
        s.close()


@pytest.mark.parametrize("prec", [dugks.FP64, dugks.FP32])
def test_table_a1_initial_masses_on_the_gpu(prec):
    """Sec. 3.1, Table A1: the printed initial droplet masses, as a batch of the
    five droplets on 100 x 100 periodic meshes."""
    rows = np.loadtxt(os.path.join(GOLDEN, "table_a1_mass.txt"))
    beta, kappa = I.params_from_sigma_width(1e-3, 4.0)
    mesh = I.uniform_mesh(100, 100)
    p = I.Params(rhoA=1.0, rhoB=0.2, beta=beta, kappa=kappa, cfl=0.4)
    phis = [I.drop_field(mesh, R0, (50.5, 50.5), 4.0) for R0 in rows[:, 0]]
    s = dugks.Sim([mesh] * len(rows), [p] * len(rows), prec).init(phis)
    ds = s.diagnostics()
    assert [d["mass"] for d in ds] == list(rows[:, 1])
    for d in ds:   # centred drops at rest
        assert d["xc"] == pytest.approx(50.5, abs=1e-9) and d["yc"] == pytest.approx(50.5, abs=1e-9)
    s.close()


def test_rayleigh_taylor_full_mesh_diagnostics():
    """The 256 x 1024 Rayleigh-Taylor mesh (FP32, the benchmark's storage) after
    initialisation and after 20 steps of both: front and tip against the oracle."""
    c = I.rayleigh_taylor()
    o = oracle.Oracle(c.mesh, c.params).init(c.phi0)
    s = dugks.Sim(c.mesh, c.params, dugks.FP32).init(c.phi0)
    for steps in (0, 20):
        if steps:
            o.step(steps)
            s.step(steps)
        d, P = D.diagnostics(o, c.mesh, c.params)
        dg = s.diagnostics()
        assert abs(dg["mass"] - d["mass"]) <= _ambiguous_volume(c.mesh, o.moments()["phi"], c.params, 1e-6)
        assert dg["front_y"] == pytest.approx(d["front_y"], abs=1e-4)
        assert dg["tip_y"] == pytest.approx(d["tip_y"], abs=1e-4)
        assert dg["p_bulk_A"] == pytest.approx(d["p_bulk_A"], rel=1e-4, abs=1e-9)
        assert np.max(np.abs(s.laplace_pressure() - P)) <= 1e-4 * np.max(np.abs(P))
    o.close()
    s.close()


def test_ensemble_diagnostics_sampled():
    """All 512 ensemble instances at once (FP32): the smallest instance of each
    kind against the oracle after initialisation; every bubble's region lies
    about its seeded centre."""
    cases = I.batched_ensemble(512)
    s = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], dugks.FP32)
    s.init([c.phi0 for c in cases])
    ds = s.diagnostics()
    order = sorted(range(len(cases)), key=lambda k: cases[k].mesh.ncells)
    for kind in ("bubble", "drop"):
        k = next(k for k in order if cases[k].name.startswith(kind))
        c = cases[k]
        o = oracle.Oracle(c.mesh, c.params).init(c.phi0)
        d, _ = D.diagnostics(o, c.mesh, c.params)
        o.close()
        assert ds[k]["mass"] == d["mass"]
        assert ds[k]["xc"] == pytest.approx(d["xc"], rel=1e-9)
        assert ds[k]["yc"] == pytest.approx(d["yc"], rel=1e-9)
    for c, d in zip(cases, ds):
        side = c.mesh.nx
        cy = side / 3.0 if c.name.startswith("bubble") else side / 2.0
        assert d["xc"] == pytest.approx(side / 2.0, abs=0.5) and d["yc"] == pytest.approx(cy, abs=0.5)
    s.close()
