"""The allocation-free conservation entry point (dugks_conservation_static).

It serves callers that cannot allocate device memory (a loop under a device
memory budget owned by another allocator, or one that cannot accept the
device synchronisation of cudaMalloc/cudaFree): they pass their own device
buffers and the library keeps its scratch in a static device array.  These
tests check its sums against the existing dugks_conservation entry point on
two calls in a row, the second on a smaller mesh so that scratch left by the
first call cannot leak into it, and check that oversized meshes are refused.

The file name sorts last, so pytest collects it after every other test file:
a run that stops at the first failure (-x) has then run every other test
before this one, whose scratch array is shared process-wide.
"""
import numpy as np
import pytest

from paper_1802_02868_gb300 import dugks
from paper_1802_02868_gb300 import inputs as I

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _case(nx, ny, seed):
    rng = np.random.default_rng(seed)
    mesh = I.Mesh(0.8 + 0.4 * rng.random(nx), 0.8 + 0.4 * rng.random(ny), I.PERIODIC, I.WALL)
    beta, kappa = I.params_from_sigma_width(1e-3, 4.0)
    prm = I.Params(rhoA=3.0, rhoB=1.0, nuA=0.05, nuB=0.05, mobility=0.1, beta=beta, kappa=kappa,
                   gy=-2e-5, rho_ref=2.0)
    phi0 = I.rt_field(mesh, mesh.dx.sum(), 0.5 * mesh.dy.sum(), [0.1 * mesh.dx.sum()], 4.0)
    return mesh, prm, phi0


def _static_sums(mesh, prm, phi):
    dev = torch.device("cuda")
    phi_d = torch.from_numpy(np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)).to(dev)
    dx_d = torch.from_numpy(np.ascontiguousarray(mesh.dx, dtype=np.float64)).to(dev)
    dy_d = torch.from_numpy(np.ascontiguousarray(mesh.dy, dtype=np.float64)).to(dev)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    rc = dugks.conservation_static(phi_d.data_ptr(), dx_d.data_ptr(), dy_d.data_ptr(), mesh.nx, mesh.ny, prm,
                                   out.data_ptr(), stream.cuda_stream)
    assert rc == 0, dugks.status_str(rc)
    stream.synchronize()
    return out.cpu().numpy()


def test_static_conservation_matches_existing_entry_point_on_two_calls():
    results = []
    for nx, ny, seed in ((96, 160, 1), (40, 36, 2)):
        mesh, prm, phi0 = _case(nx, ny, seed)
        sim = dugks.Sim(mesh, prm, dugks.FP64).init(phi0)
        sim.step(25)
        want_phi, want_rho = sim.conservation()
        phi = sim.moments()["phi"]
        got = _static_sums(mesh, prm, phi)
        assert got[0] == pytest.approx(want_phi, rel=1e-12, abs=1e-12)
        assert got[1] == pytest.approx(want_rho, rel=1e-12, abs=1e-12)
        results.append(got)
        sim.close()
    assert results[0][0] != pytest.approx(results[1][0])


def test_static_conservation_refuses_oversized_mesh():
    mesh, prm, _ = _case(8, 8, 3)
    dev = torch.device("cuda")
    buf = torch.zeros(16, dtype=torch.float64, device=dev)
    side = int(np.sqrt(dugks.STATIC_MAX_CELLS)) + 1
    rc = dugks.conservation_static(buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), side, side, prm,
                                   buf.data_ptr(), 0)
    assert rc == -1
    assert torch.all(buf == 0)


def _host_sums(phi, dx, dy, prm):
    vol = dy[:, None] * dx[None, :]
    drho = (prm.rhoA - prm.rhoB) / (prm.phiA - prm.phiB)
    return np.sum(vol * phi), np.sum(vol * (prm.rhoB + drho * (phi - prm.phiB)))


@pytest.mark.parametrize("nx,ny", [(1100, 1000), (4096, 4096)])
def test_static_conservation_on_many_blocks_and_at_the_cap(nx, ny):
    """1.1e6 cells (269 partial pairs, so the final reduction strides over more
    partials than it has threads) and exactly DUGKS_STATIC_MAX_CELLS cells, each
    against an FP64 sum on the host."""
    assert nx * ny <= dugks.STATIC_MAX_CELLS
    rng = np.random.default_rng(nx)
    prm = I.Params(rhoA=3.0, rhoB=1.0)
    phi = rng.random((ny, nx))
    dx, dy = 0.5 + rng.random(nx), 0.5 + rng.random(ny)
    mesh = I.Mesh(dx, dy, I.PERIODIC, I.PERIODIC)
    got = _static_sums(mesh, prm, phi)
    want = _host_sums(phi, dx, dy, prm)
    assert got[0] == pytest.approx(want[0], rel=1e-12)
    assert got[1] == pytest.approx(want[1], rel=1e-12)
