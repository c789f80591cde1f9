"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle on
the same seeded inputs.  FP64: normwise relative error of each distribution set
<= 1e-12 per step (one step from an identical state) and <= 1e-10 after 50
steps; FP32: phi L-inf <= 1e-5 and u L2-relative <= 1e-4 after the run."""
import math

import numpy as np
import pytest

import oracle
from paper_1802_02868_gb300 import dugks
from paper_1802_02868_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def normwise(a, b):
    d = np.max(np.abs(np.asarray(a) - np.asarray(b)))
    s = np.max(np.abs(b))
    return d / max(s, 1e-300)


def _cases():
    rng = np.random.default_rng(7)
    out = []
    c = I.stationary_drop(n=64, radius=16.0)
    out.append(("drop64", c))
    c = I.layered_poiseuille(nx=4, ny=64, height=64.0, nu_ratio=10.0, force=1e-5)
    out.append(("poiseuille_4x64_walls", c))
    c = I.rayleigh_taylor(nx=32, ny=96, amplitudes=[3.2])
    out.append(("rt_32x96", c))
    # ragged sizes, non-uniform spacing in both axes, walls in x and y
    m = I.Mesh(1.0 + 0.5 * rng.random(37), 0.7 + 0.6 * rng.random(29), I.WALL, I.WALL)
    beta, kappa = I.params_from_sigma_width(2e-3, 4.0)
    p = I.Params(rhoA=3.0, rhoB=1.0, nuA=0.2, nuB=0.05, mobility=0.2, tau_g=0.7, beta=beta, kappa=kappa,
                 gx=2e-6, gy=-1e-5, rho_ref=2.0, cfl=0.7)
    phi = I.drop_field(m, 8.0, (20.0, 12.0), 4.0)
    out.append(("ragged_37x29_walls", I.Case("ragged", m, p, phi)))
    # degenerate sizes
    for nx, ny, bcx, bcy in ((1, 16, I.PERIODIC, I.PERIODIC), (3, 3, I.PERIODIC, I.PERIODIC),
                             (2, 5, I.PERIODIC, I.WALL), (33, 9, I.WALL, I.PERIODIC)):
        m = I.Mesh(1.0 + 0.2 * rng.random(nx), 1.0 + 0.2 * rng.random(ny), bcx, bcy)
        phi = 0.5 + 0.4 * np.sin(np.arange(nx * ny).reshape(ny, nx) * 0.7)
        out.append(("tiny_%dx%d" % (nx, ny), I.Case("tiny", m, I.Params(rhoA=2.0, rhoB=1.0, beta=beta, kappa=kappa,
                                                                          gy=-1e-5, rho_ref=1.5), phi)))
    return out


CASES = _cases()


@pytest.mark.parametrize("name,case", CASES, ids=[c[0] for c in CASES])
def test_fp64_init_and_single_step_parity(name, case):
    o = oracle.Oracle(case.mesh, case.params).init(case.phi0)
    s = dugks.Sim(case.mesh, case.params, dugks.FP64).init(case.phi0)
    assert s.dt() == pytest.approx(o.dt, rel=1e-15)
    fo, go = o.state()
    fs, gs = s.state()
    # at t = 0 the f distributions are O(dt |F|), set by mu's cancellation of
    # psi' against kappa lap(phi): a looser bound than for a developed state
    assert normwise(fs, fo) < 1e-12 and normwise(gs, go) < 1e-13
    # advance the oracle, load its state into the GPU, and compare one step
    o.step(200)
    fo, go = o.state()
    s.set_state(fo, go)
    o.step(1)
    s.step(1)
    fo1, go1 = o.state()
    fs1, gs1 = s.state()
    ef, eg = normwise(fs1, fo1), normwise(gs1, go1)
    assert ef < 1e-12 and eg < 1e-12, (ef, eg)


@pytest.mark.parametrize("name,case", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_fp64_multi_step_parity_and_moments(name, case):
    o = oracle.Oracle(case.mesh, case.params).init(case.phi0)
    s = dugks.Sim(case.mesh, case.params, dugks.FP64).init(case.phi0)
    o.step(50)
    s.step(50)
    fo, go = o.state()
    fs, gs = s.state()
    assert normwise(fs, fo) < 1e-10 and normwise(gs, go) < 1e-10
    mo, ms = o.moments(), s.moments()
    for k in ("phi", "rho", "p"):
        assert normwise(ms[k], mo[k]) < 1e-10, k
    u_scale = max(np.abs(mo["ux"]).max(), np.abs(mo["uy"]).max())
    assert np.abs(ms["ux"] - mo["ux"]).max() < 1e-9 * u_scale
    assert np.abs(ms["uy"] - mo["uy"]).max() < 1e-9 * u_scale
    so, ss = o.conservation(), s.conservation()
    assert ss[0] == pytest.approx(so[0], rel=1e-12)


def test_fp64_conservation_on_gpu():
    c = I.rayleigh_taylor(nx=64, ny=128, amplitudes=[6.4])
    s = dugks.Sim(c.mesh, c.params, dugks.FP64).init(c.phi0)
    a0 = s.conservation()[0]
    s.step(500)
    a1 = s.conservation()[0]
    assert abs(a1 - a0) < 1e-12 * abs(a0)


def test_fp32_drop_accuracy_against_fp64_oracle():
    """Stationary drop 64x64, rho ratio 10, 2000 steps: FP32 storage and arithmetic."""
    c = I.stationary_drop()
    o = oracle.Oracle(c.mesh, c.params).init(c.phi0)
    s = dugks.Sim(c.mesh, c.params, dugks.FP32).init(c.phi0)
    o.step(c.steps)
    s.step(c.steps)
    mo, ms = o.moments(), s.moments()
    assert np.abs(ms["phi"] - mo["phi"]).max() <= 1e-5
    uo = np.hypot(mo["ux"], mo["uy"])
    du = np.hypot(ms["ux"] - mo["ux"], ms["uy"] - mo["uy"])
    assert np.linalg.norm(du) / np.linalg.norm(uo) <= 1e-4


def test_batch_matches_oracle_per_instance():
    """Uneven instances (different sizes, BCs and parameters) in one batch."""
    cases = [c for _, c in CASES[:4]] + I.batched_ensemble(3, seed=5, sides=(48, 64))
    s = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], dugks.FP64)
    s.init([c.phi0 for c in cases])
    s.step(20)
    fs, gs = s.state()
    off = 0
    for c in cases:
        o = oracle.Oracle(c.mesh, c.params).init(c.phi0)
        o.step(20)
        fo, go = o.state()
        n = c.mesh.ncells
        assert normwise(fs[:, off:off + n], fo.reshape(9, -1)) < 1e-11
        assert normwise(gs[:, off:off + n], go.reshape(9, -1)) < 1e-11
        off += n
    assert s.status() == [0] * len(cases)


def test_nonfinite_state_is_reported():
    """A host-made state whose arithmetic overflows raises the non-finite status."""
    c = I.stationary_drop(n=32, radius=8.0)
    s = dugks.Sim(c.mesh, c.params, dugks.FP64).init(c.phi0)
    f, g = s.state()
    f = f.copy()
    f[:, 10, 10] = 1e306
    s.set_state(f, g)
    s.step(3)
    with pytest.raises(dugks.NonFiniteError):
        s.moments()
    assert s.status() == [-3]


def test_invalid_init_input_rejected():
    c = I.stationary_drop(n=16, radius=4.0)
    s = dugks.Sim(c.mesh, c.params, dugks.FP64)
    phi = c.phi0.copy()
    phi[3, 3] = math.nan
    with pytest.raises(dugks.NonFiniteError):
        s.init(phi)


@pytest.mark.parametrize("bad", [math.nan, math.inf, -math.inf])
def test_rejected_init_leaves_the_state_untouched(bad):
    """The finiteness check runs on the device over every uploaded value (the
    last cell of the last instance included); a refused init changes neither
    the state nor the status, and the sim steps on as before."""
    cases = [I.stationary_drop(n=24, radius=6.0), I.rayleigh_taylor(nx=16, ny=40, amplitudes=[1.6])]
    s = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], dugks.FP32)
    s.init([c.phi0 for c in cases]).step(3)
    f0, g0 = s.state()
    for k, (j, i) in ((0, (0, 0)), (1, (39, 15)), (1, (17, 5))):
        phis = [c.phi0.copy() for c in cases]
        phis[k][j, i] = bad
        with pytest.raises(dugks.NonFiniteError):
            s.init(phis)
        f1, g1 = s.state()
        assert np.array_equal(f0, f1) and np.array_equal(g0, g1)
        assert s.status() == [0, 0]
    ref = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], dugks.FP32)
    ref.init([c.phi0 for c in cases]).step(5)
    s.step(2)
    assert np.array_equal(s.state()[0], ref.state()[0])


def test_moments_into_page_locked_buffers_match_pageable_ones():
    """Page-locked outputs are written by the gather kernels over the host
    link, pageable ones through the staging copy: the values are the same
    bit for bit, for buffers at an offset inside a pinned allocation too, and
    NULL outputs are skipped."""
    torch = pytest.importorskip("torch")
    cases = [I.stationary_drop(n=40, radius=10.0), I.rayleigh_taylor(nx=24, ny=72, amplitudes=[2.4])]
    s = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], dugks.FP32)
    s.init([c.phi0 for c in cases]).step(4)
    ref = s.moments()
    n = s.ncells
    base = torch.zeros(5 * n + 1, dtype=torch.float64).pin_memory()
    views = [base[1 + k * n:1 + (k + 1) * n].numpy() for k in range(5)]   # 8-byte offset into the block
    got = s.moments(out=views)
    for key in ("phi", "rho", "ux", "uy", "p"):
        for a, b in zip(got[key], ref[key]):
            assert np.array_equal(a, b), key
    # pinned, pageable and skipped outputs in one call
    mixed = [views[0], np.zeros(n), None, views[3], None]
    for v in (views[0], views[3]):
        v[:] = 0.0
    L = dugks.load()
    rc = L.dugks_moments(s.h, *[None if a is None else dugks._dp(a) for a in mixed])
    assert rc == 0
    flat = {k: np.concatenate([x.reshape(-1) for x in ref[k]]) for k in ref}
    assert np.array_equal(mixed[0], flat["phi"]) and np.array_equal(mixed[1], flat["rho"])
    assert np.array_equal(mixed[3], flat["uy"])
    s.close()


@pytest.mark.parametrize("prec", [dugks.FP64, dugks.FP32])
def test_fused_step_matches_four_kernel_step(prec, monkeypatch):
    """The one-launch tiled step and the four-kernel step compute the same scheme."""
    cases = [CASES[0][1], CASES[3][1], CASES[2][1], CASES[5][1]]
    a = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], prec)
    monkeypatch.setenv("DUGKS_UNFUSED", "1")
    b = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], prec)
    monkeypatch.delenv("DUGKS_UNFUSED")
    for s in (a, b):
        s.init([c.phi0 for c in cases])
        s.step(30)
    fa, ga = a.state()
    fb, gb = b.state()
    tol = 1e-11 if prec == dugks.FP64 else 2e-5
    assert normwise(fa, fb) < tol and normwise(ga, gb) < tol


def test_graph_replay_matches_plain_launches(monkeypatch):
    """Multi-step calls replay a captured two-step graph; the result is the
    same bits as stepping with individual launches, from either buffer."""
    cases = [CASES[0][1], CASES[3][1]]
    monkeypatch.setenv("DUGKS_NO_GRAPH", "1")
    a = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], dugks.FP32)
    monkeypatch.delenv("DUGKS_NO_GRAPH")
    b = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], dugks.FP32)
    for s in (a, b):
        s.init([c.phi0 for c in cases])
        s.step(1)      # start the multi-step call from the second buffer
        s.step(7)
        s.step(4)
    fa, ga = a.state()
    fb, gb = b.state()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    assert b.launch_count() >= 12


@pytest.mark.parametrize("prec", [dugks.FP64, dugks.FP32])
def test_every_shape_is_bit_identical_on_uniform_periodic_meshes(prec):
    """On uniform periodic meshes the strips (which prefetch the next block's
    rows and refill the shifted rings) and every tile shape execute the same
    arithmetic per cell: after 20 steps of a batch of uneven sizes, every shape
    holds the same bits.  The widths cover the strip's staging copies: 16-byte
    pieces on widths that are multiples of 32, and of 4 only (100: the last
    strip's pieces wrap at the periodic edge), cell by cell otherwise (66)."""
    cases = [I.stationary_drop(n=96, radius=24.0), I.stationary_drop(n=160, radius=40.0), I.roofline_drop(64),
             I.stationary_drop(n=100, radius=25.0), I.stationary_drop(n=66, radius=16.0)]
    ref = None
    for k in range(dugks.NUM_TILE_SHAPES):
        s = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], prec)
        s.set_tile_shape(k)
        s.init([c.phi0 for c in cases])
        s.step(20)
        f, g = s.state()
        s.close()
        if ref is None:
            ref = (f, g)
        else:
            assert np.array_equal(f, ref[0]) and np.array_equal(g, ref[1]), dugks.tile_shape_name(k)


@pytest.mark.parametrize("prec", [dugks.FP64, dugks.FP32])
def test_async_conservation_equals_the_synchronous_sums(prec):
    """dugks_conservation_async, pipelined as a caller would (enqueue step k + 1,
    then wait for the sums of step k), returns the bits of dugks_conservation
    after every step; pageable memory is refused; a wait with nothing pending
    returns at once."""
    import torch
    cases = [CASES[0][1], CASES[3][1], CASES[5][1]]
    n = len(cases)
    a = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], prec).init([c.phi0 for c in cases])
    b = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], prec).init([c.phi0 for c in cases])
    b.conservation_wait()
    with pytest.raises(dugks.DugksError) as e:
        b.conservation_async(np.zeros(2 * n))
    assert e.value.rc == -1
    ref = []
    for _ in range(6):
        a.step(1)
        sp, sr = a.conservation()
        ref.append(np.stack([sp, sr], axis=1).reshape(-1))
    bufs = [torch.empty(2 * n, dtype=torch.float64).pin_memory().numpy() for _ in range(2)]
    got = []
    b.step(1)
    b.conservation_async(bufs[0])
    for k in range(1, 6):
        b.step(1)
        b.conservation_wait()
        got.append(bufs[(k - 1) % 2].copy())
        b.conservation_async(bufs[k % 2])
    b.conservation_wait()
    got.append(bufs[1].copy())
    for r, g in zip(ref, got):
        assert np.array_equal(r, g)
    a.close()
    b.close()


@pytest.mark.parametrize("prec", [dugks.FP64, dugks.FP32])
def test_default_shape_follows_the_strip_count(prec):
    """A new sim starts with the 16-block strip when there are at least three
    such strips per resident slot (2 per SM in FP32, 1 in FP64), else with the
    8-block strip at two per slot, else with the 32x8 tile."""
    import torch
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    slots = n_sm * (1 if prec == dugks.FP64 else 2)

    def strips(cases, nb):
        return sum(-(-c.mesh.nx // 32) * -(-c.mesh.ny // (8 * nb)) for c in cases)

    seen = set()
    for cases in ([I.stationary_drop(n=64, radius=16.0)], [I.rayleigh_taylor()],
                  I.batched_ensemble(16), I.batched_ensemble(64)):
        want = 5 if strips(cases, 16) >= 3 * slots else 4 if strips(cases, 8) >= 2 * slots else 0
        s = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], prec)
        assert s.tile_shape()[0] == want, (len(cases), want)
        assert dugks.default_tile_shape([c.mesh for c in cases], prec, n_sm) == want
        s.close()
        seen.add(want)
    assert 0 in seen and len(seen) >= 2


@pytest.mark.parametrize("prec", [dugks.FP64, dugks.FP32])
def test_tile_shapes_agree_and_autotune_restores_state(prec):
    """Every tile shape of the fused step computes the same scheme; the autotuner
    leaves the state as it found it and keeps one of the shapes."""
    cases = [CASES[0][1], CASES[3][1], CASES[5][1], CASES[7][1]]
    sims = []
    for k in range(dugks.NUM_TILE_SHAPES):
        s = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], prec)
        s.set_tile_shape(k)
        s.init([c.phi0 for c in cases])
        s.step(13)
        sims.append(s)
    f0, g0 = sims[0].state()
    tol = 1e-13 if prec == dugks.FP64 else 1e-6
    for s in sims[1:]:
        f, g = s.state()
        assert normwise(f, f0) < tol and normwise(g, g0) < tol
    s = sims[0]
    before = s.state()
    k, name, ms = s.autotune(steps=3)
    after = s.state()
    assert 0 <= k < dugks.NUM_TILE_SHAPES and ms > 0 and s.tile_shape()[0] == k
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    s.step(2)
    sims[1].step(2)
    f, g = s.state()
    f1, g1 = sims[1].state()
    assert normwise(f, f1) < tol and normwise(g, g1) < tol


@pytest.mark.parametrize("prec", [dugks.FP64, dugks.FP32])
def test_uniform_periodic_path_equals_general_path(prec, monkeypatch):
    """The fused step's uniform periodic specialisation reproduces the general
    path bit for bit, and a batch holding both kinds launches one kernel per
    kind each step."""
    cases = [CASES[0][1], CASES[1][1], CASES[2][1], I.roofline_drop(96)]
    kinds = []
    states = []
    for general in ("1", "0"):
        monkeypatch.setenv("DUGKS_GENERAL_ONLY", general)
        s = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], prec)
        monkeypatch.delenv("DUGKS_GENERAL_ONLY")
        kinds.append(s.uniform_instances())
        s.init([c.phi0 for c in cases])
        l0 = s.launch_count()
        s.step(1)
        l1 = s.launch_count()
        s.step(12)
        l2 = s.launch_count()
        states.append(s.state())
        if general == "0":
            assert l1 - l0 == 2 and l2 - l1 == 24
        else:
            assert l1 - l0 == 1 and l2 - l1 == 12
        s.close()
    # the periodic uniform drops take the specialised path; the stretched
    # channel and the walled RT box do not
    assert kinds == [0, 2]
    for a, b in zip(states[0], states[1]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_fp32_conservation_sums_match_fp64_sums_of_the_state():
    """FP32 sims form sum |V| phi in double-float and sum |V| rho from it (rho is
    linear in phi, Eq. oderrho): both equal the FP64 sums over the stored
    fields to 1e-12, on a batch with non-uniform spacing and walls."""
    cases = [CASES[0][1], CASES[3][1], CASES[7][1]]
    s = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], dugks.FP32)
    s.init([c.phi0 for c in cases]).step(20)
    sp, sr = s.conservation()
    m = s.moments()
    for k, c in enumerate(cases):
        vol = np.outer(c.mesh.dy, c.mesh.dx)
        phi = m["phi"][k]                       # the stored float pair, exactly in FP64
        p = c.params
        rho = p.rhoB + (p.rhoA - p.rhoB) * (phi - p.phiB) / (p.phiA - p.phiB)   # Eq. oderrho in FP64
        assert sp[k] == pytest.approx(float(np.sum(vol * phi)), rel=1e-12)
        assert sr[k] == pytest.approx(float(np.sum(vol * rho)), rel=1e-12)


def test_caller_allocator_supplies_device_memory():
    """dugks_set_allocator: sims created after it take their device memory from
    the caller (here PyTorch's caching allocator) and step exactly like
    cudaMalloc-backed sims; an allocator that fails makes creation fail with
    DUGKS_ERR_OOM; unsetting restores cudaMalloc."""
    import torch
    c = CASES[3][1]
    ref = dugks.Sim(c.mesh, c.params, dugks.FP32).init(c.phi0)
    ref.step(9)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    dugks.use_torch_allocator()
    try:
        s = dugks.Sim(c.mesh, c.params, dugks.FP32).init(c.phi0)
        held = torch.cuda.memory_allocated() - before
        assert held >= 2 * 2 * 9 * 4 * c.mesh.ncells      # both state buffers at least
        s.set_tile_shape(dugks.NUM_TILE_SHAPES - 1)
        s.step(9)
        for a, b in zip(s.state(), ref.state()):
            assert np.array_equal(a, b)
        s.close()
        assert torch.cuda.memory_allocated() == before
        dugks.set_allocator(lambda n, st: 0, lambda p, st: None)
        with pytest.raises(dugks.DugksError) as e:
            dugks.Sim(c.mesh, c.params, dugks.FP32)
        assert e.value.rc == -4
    finally:
        dugks.set_allocator()
    s = dugks.Sim(c.mesh, c.params, dugks.FP32)
    assert torch.cuda.memory_allocated() == before
    s.close()
