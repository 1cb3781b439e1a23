"""The coupled phi-mu LBM trajectory as a differentiable torch operation.

``LbpfTrajectory.apply(phi0, c0, theta, model, nsteps, precision, checkpoint_every,
mass_every)`` runs ``nsteps`` coupled steps (Sec. 3) from the initial fields in the
library's CUDA kernels and returns the final ``(phi, c)`` as CUDA float64 tensors.
Its backward calls ``lbpf_adjoint_step``: the hand-written discrete adjoint
replayed segment by segment from checkpoints taken every ``checkpoint_every``
steps.  ``theta`` = (D_l, tau_g, tau_h, lambda) as a float64 tensor; the
kinetic coefficient M_phi = tau_g / 3, so gradients with respect to M_phi are
3 dL/dtau_g (plus 3 dL/dtau_h when tau_h is tied to it).  Every other parameter
(W, D_s, a of the anti-trapping current, ...) is taken from ``model`` and held
fixed.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import lbpf as L

THETA_NAMES = ("D_l", "tau_g", "tau_h", "lam")


class LbpfTrajectory(torch.autograd.Function):
    @staticmethod
    def forward(fctx, phi0, c0, theta, model, nsteps, precision="fp32", checkpoint_every=100, mass_every=0):
        th = [float(v) for v in theta.detach().cpu().tolist()]
        m = dataclasses.replace(model, **dict(zip(THETA_NAMES, th)))
        dev = phi0.device
        phi0_d = phi0.detach().to(device=dev, dtype=torch.float64).contiguous()
        c0_d = c0.detach().to(device=dev, dtype=torch.float64).contiguous()
        stream = torch.cuda.current_stream(dev).cuda_stream
        sim = L.Simulation(m, phi0_d, c0_d, precision=precision, stream=stream, mass_every=mass_every,
                           checkpoint_every=checkpoint_every)
        sim.step(int(nsteps))
        phi = torch.empty(m.shape, dtype=torch.float64, device=dev)
        c = torch.empty(m.shape, dtype=torch.float64, device=dev)
        L.lbpf_get_fields(sim.ctx, phi, c, None, 1)
        fctx.sim = sim
        fctx.theta_dtype = theta.dtype
        fctx.theta_device = theta.device
        return phi, c

    @staticmethod
    def backward(fctx, gphi, gc):
        sim = fctx.sim
        dev = gphi.device if gphi is not None else gc.device
        gphi = None if gphi is None else gphi.to(torch.float64).contiguous()
        gc = None if gc is None else gc.to(torch.float64).contiguous()
        dphi0 = torch.empty(sim.shape, dtype=torch.float64, device=dev)
        dc0 = torch.empty(sim.shape, dtype=torch.float64, device=dev)
        pv = L.lbpf_adjoint_step(sim.ctx, gphi, gc, dphi0, dc0, 1)
        sim.close()
        fctx.sim = None
        # the gradient lives where theta does (the autograd engine checks it)
        dtheta = torch.tensor(np.asarray(pv[:4]), dtype=fctx.theta_dtype, device=fctx.theta_device)
        return dphi0, dc0, dtheta, None, None, None, None, None


def trajectory(phi0, c0, theta, model, nsteps, precision="fp32", checkpoint_every=100, mass_every=0):
    """Final (phi, c) after nsteps steps; differentiable in phi0, c0 and theta."""
    return LbpfTrajectory.apply(phi0, c0, theta, model, nsteps, precision, checkpoint_every, mass_every)
