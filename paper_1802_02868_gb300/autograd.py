"""``torch.autograd`` interface to the library's adjoint.

``DugksLoss.apply(phi0, kappa, mobility, problem)`` returns the loss
L = sum_cells (phi_T - phi_target)^2 of a DUGKS run of ``problem.steps`` steps
from the initial order parameter ``phi0`` (a float64 tensor shaped like the
mesh) with the free-energy coefficient ``kappa`` and the mobility ``mobility``
(0-d tensors).  The forward call runs the library's checkpointed forward and
reverse sweeps (``dugks_adjoint``) at once; backward scales the stored
gradients.  Anything upstream of ``phi0`` (for instance an interface built from
Fourier amplitudes) is differentiated by PyTorch as usual.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

from . import dugks
from . import inputs as I


@dataclasses.dataclass
class Problem:
    mesh: I.Mesh
    params: I.Params           # kappa and mobility are overridden by the tensors
    phi_target: np.ndarray
    steps: int
    ckpt_every: int = 100
    precision: int = dugks.FP32


class DugksLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi0, kappa, mobility, problem: Problem):
        prm = dataclasses.replace(problem.params, kappa=float(kappa), mobility=float(mobility))
        sim = dugks.Sim(problem.mesh, prm, problem.precision)
        try:
            sim.init(phi0.detach().cpu().numpy().astype(np.float64))
            r = sim.adjoint(problem.steps, problem.phi_target, ckpt_every=problem.ckpt_every)
        finally:
            sim.close()
        # each gradient lives on the device (and in the dtype) of its own input
        ctx.save_for_backward(torch.as_tensor(r["dphi0"], dtype=phi0.dtype, device=phi0.device),
                              torch.tensor(r["dkappa"], dtype=torch.float64, device=kappa.device),
                              torch.tensor(r["dlambda"], dtype=torch.float64, device=mobility.device))
        ctx.dtypes = (kappa.dtype, mobility.dtype)
        return torch.tensor(r["loss"], dtype=torch.float64, device=phi0.device)

    @staticmethod
    def backward(ctx, grad):
        dphi0, dk, dl = ctx.saved_tensors
        g = grad.to(torch.float64)
        return (g.to(dphi0.device) * dphi0, (g.to(dk.device) * dk).to(ctx.dtypes[0]),
                (g.to(dl.device) * dl).to(ctx.dtypes[1]), None)


def interface_field(amplitudes, mesh, y0, wavelength, width, phiA=1.0, phiB=0.0):
    """Differentiable initial order parameter of a perturbed flat interface,
    heavy fluid A above y = y0 + sum_k a_k cos(2 pi k x / L) (as
    ``inputs.rt_field``), built with torch so that gradients reach the
    amplitudes."""
    xc, yc = mesh.centres()
    x = torch.as_tensor(xc, dtype=torch.float64, device=amplitudes.device)
    y = torch.as_tensor(yc, dtype=torch.float64, device=amplitudes.device)
    k = torch.arange(1, amplitudes.numel() + 1, dtype=torch.float64, device=amplitudes.device)
    eta = y0 + (amplitudes.to(torch.float64)[:, None] * torch.cos(2.0 * math.pi * k[:, None] * x[None, :] / wavelength)).sum(0)
    return 0.5 * (phiA + phiB) + 0.5 * (phiA - phiB) * torch.tanh(2.0 * (y[:, None] - eta[None, :]) / width)
