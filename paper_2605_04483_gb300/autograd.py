"""torch.autograd binding of the CDFCI ground-state energy (argument
marshalling only; the solve, the RDMs and the derivatives run in libcdfci).

E(h, g) is the converged Rayleigh quotient of CDFCI (Alg. 1, m = 1) or mCDFCI
(Alg. 2, m > 1).  At convergence the energy is variational, so its derivative
with respect to the integrals is the expectation value of the derivative of H
(Hellmann-Feynman): dE/dh = gamma and dE/dg = 1/2 Gamma (symmetrised over the
8-fold symmetry of (pq|rs)), with the spin-summed RDMs of Sec. "Optimal Orbital
Selections"; the orbital-rotation gradient dE/dkappa = 2 (F - F^T) is what an
orbital-optimisation outer loop consumes.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import api


def _solve(h: torch.Tensor, g: torch.Tensor, N: int, n_alpha: int, n_beta: int, n_iter: int,
           params: Optional[dict]) -> api.Solver:
    s = api.Solver(h.detach().to(torch.float64).contiguous(), g.detach().to(torch.float64).contiguous(), N,
                   n_alpha, n_beta, **(params or {}))
    s.step(int(n_iter))
    return s


class CDFCIEnergy(torch.autograd.Function):
    """E = CDFCIEnergy.apply(h, g, N, n_alpha, n_beta, n_iter, params); h (N, N),
    g (N, N, N, N) float64, host or device.  params: cdfci_params fields."""

    @staticmethod
    def forward(ctx, h, g, N, n_alpha, n_beta, n_iter, params=None):
        s = _solve(h, g, N, n_alpha, n_beta, n_iter, params)
        try:
            E = s.energy(1)
            dh, dg, _ = s.gradient()
        finally:
            s.close()
        ctx.save_for_backward(torch.from_numpy(dh).to(h.device), torch.from_numpy(dg).to(g.device))
        return torch.tensor(E, dtype=torch.float64, device=h.device)

    @staticmethod
    def backward(ctx, grad_E):
        dh, dg = ctx.saved_tensors
        return grad_E * dh, grad_E * dg, None, None, None, None, None


def dE_dkappa(solver: api.Solver) -> torch.Tensor:
    """dE/dkappa (N, N, antisymmetric) of the solver's current vector for the
    orbitals rotated by U = exp(kappa): dE = 1/2 sum_pq G_pq dkappa_pq."""
    return torch.from_numpy(solver.gradient()[2])
