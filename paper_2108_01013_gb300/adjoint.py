"""Differentiable rollouts: the library's reverse sweep (dss_adjoint) behind a
``torch.autograd.Function``.

``rollout_stress(x0, theta, ...)`` returns J = sum_n sum_q W[n, q] sigma^{n+1}_q
of a rollout that starts from positions x0 (velocities u0, w0 given; initial
accelerations from a force evaluation, as ``dss_set_state`` computes them)
with model constants theta = (k_n, k_t, gamma_n, mu, delta_lub), and carries
dJ/dx0 and dJ/dtheta back through autograd.  Every derivative is computed by
the CUDA kernels of libdss (the pair vector-Jacobian products, the reverse
integrator, checkpointed replay); this module only marshals tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from .suspension import Suspension, default_params

PARAM_NAMES = ("kn", "kt", "gamma_n", "mu", "delta_lub")


def viscosity_weights(nsteps: int, eta0: float = 1.0, shear_rate: float = 1.0) -> np.ndarray:
    """Weights that make J the time-averaged relative viscosity
    eta_r = sigma_xy / (eta0 gdot) over the steps."""
    W = np.zeros((nsteps, 9))
    W[:, 1] = 1.0 / (nsteps * eta0 * shear_rate)
    return W


class _RolloutStress(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, theta, a, box, u0, w0, nsteps, weights, ckpt_every, kw):
        t = theta.detach().cpu().double().numpy()
        p = default_params(box, kn=float(t[0]), kt=float(t[1]), gamma_n=float(t[2]), mu=float(t[3]),
                           delta_lub=float(t[4]), **kw)
        s = Suspension(x0.detach(), a, box, p, u=u0, w=w0)
        r = s.adjoint(nsteps, weights, ckpt_every=ckpt_every, initial_forces=True)
        s.close()
        ctx.save_for_backward(torch.as_tensor(r["x0"], dtype=torch.float64, device=x0.device),
                              torch.as_tensor(r["params"], dtype=torch.float64, device=theta.device))
        return torch.tensor(r["J"], dtype=torch.float64, device=x0.device)

    @staticmethod
    def backward(ctx, gJ):
        gx, gp = ctx.saved_tensors
        return gJ * gx, gJ * gp, None, None, None, None, None, None, None, None


def rollout_stress(x0, theta, a, box, u0, w0, nsteps, weights, *, ckpt_every=20, **kw):
    """J of the rollout as a differentiable function of x0 (3, n) and theta (5,)."""
    return _RolloutStress.apply(x0, theta, a, np.asarray(box, dtype=np.float64), u0, w0, int(nsteps),
                                np.asarray(weights, dtype=np.float64), int(ckpt_every), kw)
