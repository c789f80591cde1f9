"""Parameter sweeps run as batches (Sec. 3.1 mobility and CFL sweeps, Sec. 3.2
viscosity-ratio sweep), and the pause / per-instance step counts that let
instances with different time steps reach the same time."""
import math

import numpy as np
import pytest

from paper_1802_02868_gb300 import dugks
from paper_1802_02868_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _slices(cases):
    off = np.cumsum([0] + [c.mesh.ncells for c in cases])
    return [slice(off[k], off[k + 1]) for k in range(len(cases))]


@pytest.mark.parametrize("shape", range(dugks.NUM_TILE_SHAPES))
@pytest.mark.parametrize("prec", [dugks.FP64, dugks.FP32])
def test_step_each_equals_separate_runs(prec, shape):
    """dugks_batch_step_each: every instance ends bit for bit where a run of its
    own count ends; an instance paused beforehand does not move and stays
    paused.  Every fused-step shape (tiles and strips) passes a paused
    instance's state through."""
    cases = I.mobility_sweep(mobilities=(0.01, 0.1, 1.0, 0.3), n=48, radius=12.0)
    counts = [7, 0, 12, 5]
    b = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], prec).init([c.phi0 for c in cases])
    b.set_tile_shape(shape)
    f0, g0 = b.state()
    b.set_paused([False, False, False, True])
    b.step_each(counts)
    fb, gb = b.state()
    sl = _slices(cases)
    for k, (c, n) in enumerate(zip(cases, counts)):
        s = dugks.Sim(c.mesh, c.params, prec).init(c.phi0)
        if n and k != 3:
            s.step(n)
        f, g = s.state()
        assert np.array_equal(fb[:, sl[k]], f.reshape(9, -1)) and np.array_equal(gb[:, sl[k]], g.reshape(9, -1)), k
        s.close()
    assert np.array_equal(fb[:, sl[3]], f0[:, sl[3]]) and np.array_equal(gb[:, sl[3]], g0[:, sl[3]])
    b.step(2)                                       # still paused
    assert np.array_equal(b.state()[0][:, sl[3]], f0[:, sl[3]])
    assert b.status() == [0, 0, 0, 0]
    b.close()


def test_paused_instance_reports_and_init_resumes():
    """A paused instance still has moments, conservation sums and diagnostics;
    dugks_init resumes it."""
    cases = I.mobility_sweep(mobilities=(0.1, 0.1), n=48, radius=12.0)
    s = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], dugks.FP32).init([c.phi0 for c in cases])
    s.set_paused([True, False]).step(20)
    m = s.moments()
    d = s.diagnostics()
    sp, _ = s.conservation()
    assert np.max(np.abs(m["phi"][0] - cases[0].phi0)) < 1e-12    # held still
    assert np.all(np.isfinite(m["p"][0])) and not math.isnan(d[0]["mass"])
    assert sp[0] == pytest.approx(float(np.sum(cases[0].phi0)), rel=1e-12)
    assert not np.array_equal(m["phi"][0], m["phi"][1])   # the other one moved
    s.init([c.phi0 for c in cases]).step(20)
    m = s.moments()
    assert np.array_equal(m["phi"][0], m["phi"][1])        # both moved alike after init
    s.close()


def _profile_deviation(s, cases, radius=25.0):
    """Largest deviation of the density from the drop's analytic tanh profile
    (Sec. 3.1, with the drop's own rhoA, rhoB and W = 4)."""
    rho = s.moments()["rho"]
    out = []
    for k, c in enumerate(cases):
        xc, yc = c.mesh.centres()
        X, Y = np.meshgrid(xc, yc)
        ctr = 0.5 * c.mesh.nx + 0.5
        r = np.hypot(X - ctr, Y - ctr)
        pa, pb = c.params.rhoA, c.params.rhoB
        ana = 0.5 * (pa + pb) + 0.5 * (pa - pb) * np.tanh(2.0 * (radius - r) / 4.0)
        out.append(float(np.max(np.abs(rho[k] - ana))))
    return out


def test_mobility_sweep_deviation_grows_with_mobility():
    """Sec. 3.1: the density profile departs further from the analytic shape as
    the mobility grows (lambda = 0.01, 0.1, 1, one batch, t = 2000); the
    pressure jump keeps Laplace's law."""
    cases = I.mobility_sweep(mobilities=(0.01, 0.1, 1.0))
    s = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], dugks.FP64).init([c.phi0 for c in cases])
    s.step(int(round(2000.0 / s.dt(0))))
    dev = _profile_deviation(s, cases)
    assert dev[0] < dev[1] < dev[2]
    for d in s.diagnostics():
        assert (d["p_bulk_A"] - d["p_bulk_B"]) * 25.0 / 1e-3 == pytest.approx(1.0, abs=0.1)
    s.close()


def test_cfl_sweep_reaches_one_time_and_smaller_cfl_is_closer():
    """Sec. 3.1: CFL = 0.1 ... 0.8 at lambda = 0.1, each brought to t = 500 with
    its own step count; the smaller the CFL (time step), the closer the
    density profile to the analytic shape."""
    cases = I.cfl_sweep()
    s = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], dugks.FP64).init([c.phi0 for c in cases])
    counts = [int(round(500.0 / s.dt(k))) for k in range(len(cases))]
    for k in range(len(cases)):
        assert abs(counts[k] * s.dt(k) - 500.0) <= s.dt(k)
    s.step_each(counts)
    dev = _profile_deviation(s, cases)
    assert all(a < b for a, b in zip(dev, dev[1:]))
    s.close()


def _two_layer(y, H, G, muA, muB):
    Hp = H / 2
    Y = Hp - y
    r = (muA - muB) / (muA + muB)
    uA = G * Hp ** 2 / (2 * muA) * (-(Y / Hp) ** 2 - (Y / Hp) * r + 2 * muA / (muA + muB))
    uB = G * Hp ** 2 / (2 * muB) * (-(Y / Hp) ** 2 - (Y / Hp) * r + 2 * muB / (muA + muB))
    return np.where(Y >= 0, uA, uB)


@pytest.mark.parametrize("prec", [dugks.FP64, dugks.FP32])
def test_viscosity_ratio_sweep_keeps_the_two_layer_profiles(prec):
    """Sec. 3.2: the layered channel at viscosity ratios 3, 10, 100 and 1000 as
    one batch, held 1e4 steps from the analytic two-layer profiles: every
    profile within 2% (L2), the error growing with the ratio."""
    cases = I.viscosity_ratio_sweep()
    uas, ux0 = [], []
    for c in cases:
        _, yc = c.mesh.centres()
        ua = _two_layer(yc, 256.0, 1e-6, c.params.nuA, c.params.nuB)
        uas.append(ua)
        ux0.append(np.repeat(ua[:, None], c.mesh.nx, axis=1))
    s = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], prec)
    s.init([c.phi0 for c in cases], ux=ux0).step(10000)
    u = s.moments()["ux"]
    errs = [np.linalg.norm(u[k][:, 0] - uas[k]) / np.linalg.norm(uas[k]) for k in range(len(cases))]
    assert max(errs) < 0.02
    assert all(a < b for a, b in zip(errs, errs[1:]))
    assert s.status() == [0] * len(cases)
    s.close()


@pytest.mark.parametrize("prec", [dugks.FP64, dugks.FP32])
def test_cfl_sweep_instances_match_oracle_runs_of_their_own_counts(prec):
    """Sec. 3.1's CFL sweep as one batch: dugks_batch_step_each brings the
    instances at CFL 0.2, 0.4 and 0.8 to the same time t = 40 (283, 141 and 71
    steps), and each instance matches an oracle run of its own step count:
    in FP64 the distributions element by element to 1e-10 normwise, in FP32
    phi to 1e-5 (L-infinity) and u to 1e-4 (L2-relative)."""
    import oracle
    cases = I.cfl_sweep(cfls=(0.2, 0.4, 0.8), n=64, radius=16.0)
    b = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], prec).init([c.phi0 for c in cases])
    counts = [int(round(40.0 / b.dt(k))) for k in range(len(cases))]
    assert counts == [283, 141, 71]
    b.step_each(counts)
    fb, gb = b.state()
    mb = b.moments()
    sl = _slices(cases)
    for k, (c, n) in enumerate(zip(cases, counts)):
        o = oracle.Oracle(c.mesh, c.params).init(c.phi0)
        o.step(n)
        if prec == dugks.FP64:
            fo, go = o.state()
            for got, ref in ((fb[:, sl[k]], fo.reshape(9, -1)), (gb[:, sl[k]], go.reshape(9, -1))):
                assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-10, (k, n)
        else:
            mo = o.moments()
            u, uo = np.stack([mb["ux"][k], mb["uy"][k]]), np.stack([mo["ux"], mo["uy"]])
            assert np.max(np.abs(mb["phi"][k] - mo["phi"])) < 1e-5, (k, n)
            assert np.linalg.norm(u - uo) / np.linalg.norm(uo) < 1e-4, (k, n)
    b.close()
