"""VMCForces: the VMC energy of fixed walker configurations as a differentiable function of
the nuclear positions R and the frozen orbital coefficients C (a torch.autograd.Function).

Forward: E(R, C) = mean of E_L over the walkers, evaluated by libvmcf (the positions stay
fixed; the wavefunction is rebuilt for the given R and C).
Backward: dE/dR = -F with F the Hellmann-Feynman + Pulay force in covariance form (Eqs. hf,
pulay). On fixed walkers this is exactly the derivative of the correlated-sampling
(reweighted) energy, so it matches central finite differences of that functional.
dE/dC^s = B^s = 2 (<E_L O> - E <O>), the paper's orbital gradient (App. A, Eq. fc-vmc-eval,
read as dE/dC): the derivative of the reweighted energy minus <dE_L/dC>, a term whose
expectation is zero.

Every number comes out of libvmcf's kernels and its estimator finish; torch only carries the
tensors.
"""
from __future__ import annotations

import copy

import numpy as np
import torch

from . import vmcf


class VMCForces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, R, C_up, C_dn, template, pos, precision=vmcf.FP64, nblocks=16):
        """R (K, 3), C_up (M, n_up), C_dn (M, n_dn): float64 tensors (any device).
        template: a systems.System giving the basis, charges and Jastrow.
        pos: (W, Ne, 3) float64 CUDA tensor of fixed walker positions."""
        sysx = copy.copy(template)
        sysx.R = np.ascontiguousarray(R.detach().cpu().numpy(), dtype=np.float64)
        sysx.C_up = np.ascontiguousarray(C_up.detach().cpu().numpy(), dtype=np.float64)
        sysx.C_dn = np.ascontiguousarray(C_dn.detach().cpu().numpy(), dtype=np.float64)
        g = vmcf.System(sysx, precision)
        wk = vmcf.Walkers(g, pos, nblocks=nblocks)
        wk.reset_accumulators(0.0)
        wk.measure()
        est = wk.reduce_estimators()
        M, nu = g.M, g.n_up
        ctx.save_for_backward(torch.as_tensor(-est["F"], dtype=R.dtype, device=R.device),
                              torch.as_tensor(est["dEdC"][:M * nu].reshape(M, nu), dtype=C_up.dtype,
                                              device=C_up.device),
                              torch.as_tensor(est["dEdC"][M * nu:].reshape(M, -1), dtype=C_dn.dtype,
                                              device=C_dn.device))
        ctx.estimates = est
        return torch.as_tensor(est["E"], dtype=R.dtype, device=R.device)

    @staticmethod
    def backward(ctx, gE):
        dR, dCu, dCd = ctx.saved_tensors
        return gE * dR, gE * dCu, gE * dCd, None, None, None, None


def vmc_energy(R, C_up, C_dn, template, pos, precision=vmcf.FP64, nblocks=16):
    return VMCForces.apply(R, C_up, C_dn, template, pos, precision, nblocks)
