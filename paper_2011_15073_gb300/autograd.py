"""``torch.autograd`` entry to the discrete adjoint (``lbm_adjoint_nu``).

:func:`hot_wall_nusselt` returns the hot-wall average Nusselt number J after
``steps`` time steps from the rest state of a cavity with a per-node Darcy
field, as a tensor that carries its gradient with respect to the Darcy field
Da(x), the power-law index n and the Rayleigh number Ra.  The forward call
runs the library's forward sweep and its hand-written reverse sweep
(checkpoints every ``ckpt_every`` steps, recomputation in between) in one
C call; ``backward`` only scales the stored gradients by the incoming one.
Argument marshalling only: every step runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbm


class _HotWallNusselt(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Da, n, Ra, spec):
        nx, ny, Pr, porosity, steps, ckpt_every, opts = spec
        Da_h = Da.detach().to("cpu", torch.float64).numpy()
        if Da_h.shape != (ny, nx):
            raise ValueError(f"Da must be [{ny}][{nx}], got {tuple(Da_h.shape)}")
        with lbm.Cavity(nx, ny, float(n), float(np.mean(Da_h)), float(Ra), Pr, porosity, **opts) as cav:
            cav.set_darcy_field(Da_h)
            J, dDa, dn, dRa, _ = cav.adjoint_nu(steps, ckpt_every=ckpt_every, from_rest=True)
        ctx.save_for_backward(torch.from_numpy(dDa).to(Da.device, Da.dtype),
                              torch.tensor(dn, dtype=torch.float64, device=n.device),
                              torch.tensor(dRa, dtype=torch.float64, device=Ra.device))
        return torch.tensor(J, dtype=torch.float64, device=Da.device)

    @staticmethod
    def backward(ctx, gJ):
        dDa, dn, dRa = ctx.saved_tensors
        return (gJ.to(dDa.dtype) * dDa, (gJ.to(dn.device) * dn).to(dn.dtype),
                (gJ.to(dRa.device) * dRa).to(dRa.dtype), None)


def hot_wall_nusselt(Da: torch.Tensor, n: torch.Tensor, Ra: torch.Tensor, *, Pr: float, porosity: float = 0.6,
                     steps: int, ckpt_every: int = 500, **opts) -> torch.Tensor:
    """J = hot-wall average Nu after ``steps`` steps from rest (a 0-d FP64
    tensor), differentiable in ``Da`` ([ny][nx] Darcy numbers), ``n`` and
    ``Ra`` (0-d tensors).  ``opts`` are ``lbm_opts`` fields (e.g.
    ``prec="f32"``, ``clamp_mode=1``); the grid is Da's shape."""
    ny, nx = Da.shape
    return _HotWallNusselt.apply(Da, n, Ra, (nx, ny, float(Pr), float(porosity), int(steps), int(ckpt_every), opts))
