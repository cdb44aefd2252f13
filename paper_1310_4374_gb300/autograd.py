"""torch.autograd.Function for the periodic Coulomb energy E = 1/2 sum_i q_i phi(x_i).

Forward calls psum_eval, psum_energy and psum_coeffs_device (the fitted coefficients of
this evaluation, kept with the saved tensors); backward calls psum_energy_backward_c with
those coefficients, which returns the exact derivatives of the method's discrete energy
with respect to the positions and the charges.  Several forwards through one module may
therefore share one backward pass.  torch only allocates the tensors; every arithmetic
step runs in libpsum.so.
"""
from __future__ import annotations

import torch

from . import binding as B


class _EnergyFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, q, module):
        x = x.detach().contiguous()
        q = q.detach().contiguous()
        N = q.numel()
        phi = torch.empty(N, dtype=torch.float64, device=x.device)
        grad = torch.empty((N, 3), dtype=torch.float64, device=x.device)
        B.psum_eval(module.plan, x, q, phi, grad, check=module.check)
        E = torch.empty(1, dtype=torch.float64, device=x.device)
        B.psum_energy(module.plan, q, phi, E)
        C = torch.empty(module.P, dtype=torch.float64, device=x.device)
        B.psum_coeffs_device(module.plan, C)
        ctx.module = module
        ctx.save_for_backward(x, q, phi, grad, C)
        return E[0]

    @staticmethod
    def backward(ctx, gE):
        x, q, phi, grad, C = ctx.saved_tensors
        m = ctx.module
        gE = gE.detach().to(torch.float64).reshape(1).contiguous()
        dEdq = torch.empty_like(q) if ctx.needs_input_grad[1] else None
        dEdx = torch.empty_like(x) if ctx.needs_input_grad[0] else None
        if dEdq is None and dEdx is None:
            return None, None, None
        B.psum_energy_backward_c(m.plan, x, q, phi, grad, C, gE, dEdq, dEdx)
        return dEdx, dEdq, None


class PeriodicCoulombEnergy(torch.nn.Module):
    """E(x, q) = 1/2 sum_i q_i phi(x_i) for the periodic Coulomb sum of a fixed box.

    Each forward keeps the fitted coefficients of its own evaluation for its backward, so
    any number of forwards (other positions or charges) may come before one backward.
    """

    def __init__(self, d, p: int, M: int, precision: str = "fp32c", mean: str = "zero", K=(1, 1, 1),
                 check: bool = True, terms: str = "fast"):
        super().__init__()
        self.plan = B.psum_plan_create_ex(d, p, M, precision, mean, K, terms=terms)
        self.P = B.psum_plan_info(self.plan)["P"]
        self.check = check

    def forward(self, x, q):
        return _EnergyFn.apply(x, q, self)

    def close(self):
        if self.plan:
            B.psum_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
