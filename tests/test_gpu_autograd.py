"""torch.autograd interface: gradients of the DUGKS loss with respect to
Fourier amplitudes of the initial interface, kappa and the mobility, against
central finite differences of the GPU FP64 forward run, on a small
Rayleigh-Taylor mesh and at the full 256x512 adjoint workload size."""
import math

import numpy as np
import pytest

from paper_1802_02868_gb300 import dugks
from paper_1802_02868_gb300 import inputs as I

torch = pytest.importorskip("torch")
from paper_1802_02868_gb300.autograd import DugksLoss, Problem, interface_field  # noqa: E402

pytestmark = pytest.mark.gpu


def _problem(nx, ny, steps, seed):
    c = I.rayleigh_taylor(nx=nx, ny=ny, amplitudes=[0.1 * nx], sigma=1e-3, sqrt_gl=0.04)
    rng = np.random.default_rng(seed)
    amps = np.concatenate([[0.1 * nx], rng.normal(0.0, 0.01 * nx, 7)])
    target_amps = amps + rng.normal(0.0, 0.01 * nx, 8)
    tgt = I.rt_field(c.mesh, float(nx), 0.5 * ny, target_amps, 4.0)
    return c, amps, Problem(c.mesh, c.params, tgt, steps, ckpt_every=max(1, steps // 4), precision=dugks.FP64)


def _loss(prob, amps, kappa, mobility):
    prm = I.Params(**{**vars(prob.params), "kappa": kappa, "mobility": mobility})
    phi0 = I.rt_field(prob.mesh, float(prob.mesh.nx), 0.5 * prob.mesh.ny, amps, 4.0)
    s = dugks.Sim(prob.mesh, prm, dugks.FP64).init(phi0)
    s.step(prob.steps)
    d = s.moments()["phi"] - prob.phi_target
    return float(np.sum(d * d))


@pytest.mark.parametrize("nx,ny,steps", [(16, 48, 40), (256, 512, 120)])
def test_gradients_through_autograd_match_finite_differences(nx, ny, steps):
    c, amps, prob = _problem(nx, ny, steps, seed=nx)
    a = torch.tensor(amps, dtype=torch.float64, requires_grad=True)
    kap = torch.tensor(c.params.kappa, dtype=torch.float64, requires_grad=True)
    mob = torch.tensor(c.params.mobility, dtype=torch.float64, requires_grad=True)
    phi0 = interface_field(a, c.mesh, 0.5 * ny, float(nx), 4.0)
    L = DugksLoss.apply(phi0, kap, mob, prob)
    L.backward()
    assert float(L.detach()) == pytest.approx(_loss(prob, amps, c.params.kappa, c.params.mobility), rel=1e-12)
    # a random direction in amplitude space, and each scalar parameter
    rng = np.random.default_rng(5)
    v = rng.standard_normal(8)
    e = 1e-4 * nx * 0.01
    fd = (_loss(prob, amps + e * v, c.params.kappa, c.params.mobility)
          - _loss(prob, amps - e * v, c.params.kappa, c.params.mobility)) / (2 * e)
    assert float(a.grad @ torch.tensor(v)) == pytest.approx(fd, rel=2e-5)
    for name, t in (("kappa", kap), ("mobility", mob)):
        base = getattr(c.params, name)
        h = 1e-5 * base
        kw = {"kappa": c.params.kappa, "mobility": c.params.mobility}
        kp, km = dict(kw), dict(kw)
        kp[name] = base + h
        km[name] = base - h
        fd = (_loss(prob, amps, **kp) - _loss(prob, amps, **km)) / (2 * h)
        assert float(t.grad) == pytest.approx(fd, rel=2e-5)


def test_gradients_land_on_the_devices_of_their_inputs():
    """phi0 built on the GPU, kappa and the mobility on the CPU: each gradient
    arrives on its own input's device and equals the all-CPU result."""
    c, amps, prob = _problem(16, 48, 10, seed=3)
    grads = {}
    for dev_phi, dev_par in (("cpu", "cpu"), ("cuda", "cpu"), ("cpu", "cuda")):
        a = torch.tensor(amps, dtype=torch.float64, device=dev_phi, requires_grad=True)
        kap = torch.tensor(c.params.kappa, dtype=torch.float64, device=dev_par, requires_grad=True)
        mob = torch.tensor(c.params.mobility, dtype=torch.float64, device=dev_par, requires_grad=True)
        L = DugksLoss.apply(interface_field(a, c.mesh, 24.0, 16.0, 4.0), kap, mob, prob)
        L.backward()
        assert a.grad.device.type == dev_phi
        assert kap.grad.device.type == dev_par and mob.grad.device.type == dev_par
        grads[(dev_phi, dev_par)] = [t.grad.cpu().numpy() for t in (a, kap, mob)]
    ref = grads[("cpu", "cpu")]
    for k, g in grads.items():
        for x, y in zip(g, ref):
            np.testing.assert_allclose(x, y, rtol=1e-12, atol=0)
