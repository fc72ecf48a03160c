"""Differentiable witness field for PyTorch.

``witness_field(driver, profile, cfg, nsteps, witness)`` runs the wake
simulation on the GPU and returns J, the accelerating field E_z at one slot
after ``nsteps`` steps (Sec. 6 setup), as a 0-d tensor; its backward pass is
the library's discrete adjoint (lbpwfa_record / lbpwfa_adjoint_step), which
gives dJ/d(alpha, sigma_z, sigma_r) for the Gaussian driver of Eq.
(bunch-density) and dJ/d(profile samples) for a sampled profile.  Only
argument marshalling happens here; the forward steps and the reverse sweep
run in the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbpwfa as lb


class WitnessField(torch.autograd.Function):
    @staticmethod
    def forward(ctx, driver, profile, cfg, nsteps, witness, precision, checkpoint_every):
        c = dict(cfg)
        alpha, sigma_z, sigma_r = (float(v) for v in driver.detach().to("cpu", torch.float64).tolist())
        c.update(alpha=alpha, sigma_z=sigma_z, sigma_r=sigma_r)
        has_profile = profile is not None and profile.numel() > 0
        if has_profile:
            c["profile"] = profile.detach().to("cpu", torch.float64).numpy().copy()
        else:
            c.pop("profile", None)
        run = lb.Run(c, precision)
        run.record(int(nsteps), int(checkpoint_every))
        run.step(int(nsteps))
        ez = run.fields(lb.F_EZ)[0]
        nz = run.cfg["n"][0]
        w = list(witness) + [0, 0]
        J = float(ez[int(w[0]) + nz * int(w[1])]) if run.cfg["dim"] >= 2 else float(ez[int(w[0])])
        ctx.run = run
        ctx.witness = tuple(int(v) for v in w[:3])
        ctx.has_profile = has_profile
        ctx.driver_device = driver.device
        ctx.profile_device = profile.device if has_profile else None
        return torch.tensor(J, dtype=torch.float64, device=driver.device)

    @staticmethod
    def backward(ctx, gJ):
        run = ctx.run
        _, g3, gp = run.adjoint(ctx.witness, seed=float(gJ.detach().cpu()))
        run.close()
        ctx.run = None
        gd = torch.as_tensor(np.asarray(g3), dtype=torch.float64, device=ctx.driver_device)
        gpr = None
        if ctx.has_profile:
            gpr = torch.as_tensor(np.asarray(gp), dtype=torch.float64, device=ctx.profile_device)
        return gd, gpr, None, None, None, None, None


def witness_field(driver, profile, cfg, nsteps, witness, precision="fp32", checkpoint_every=50):
    """J = E_z at the witness node's slot after nsteps (differentiable in
    driver = (alpha, sigma_z, sigma_r) and in profile, when given)."""
    if profile is None:
        profile = torch.zeros(0, dtype=torch.float64)
    return WitnessField.apply(driver, profile, cfg, nsteps, witness, precision, checkpoint_every)
