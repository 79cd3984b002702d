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
tensors. The library objects are kept between calls for the same template, precision, block count and
walker count: each call moves the system to the given R and C (vmcf_system_set_geometry) and re-inverts
the walker set at the given positions instead of building both again.
"""
from __future__ import annotations

from collections import OrderedDict

import numpy as np
import torch

from . import vmcf

_STATE: "OrderedDict[tuple, tuple]" = OrderedDict()  # (id(template), precision, nblocks, W) -> (template, System, Walkers)
_STATE_MAX = 4


def _state(template, precision, nblocks, pos):
    key = (id(template), precision, nblocks, int(pos.shape[0]))
    ent = _STATE.get(key)
    if ent is None or ent[0] is not template:
        g = vmcf.System(template, precision)
        ent = (template, g, vmcf.Walkers(g, pos, nblocks=nblocks))
        _STATE[key] = ent
        while len(_STATE) > _STATE_MAX:
            _STATE.popitem(last=False)
    else:
        _STATE.move_to_end(key)
    return ent[1], ent[2]


class VMCForces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, R, C_up, C_dn, template, pos, precision=vmcf.FP64, nblocks=16):
        """R (K, 3), C_up (M, n_up), C_dn (M, n_dn): float64 tensors (any device).
        template: a systems.System giving the basis, charges and Jastrow.
        pos: (W, Ne, 3) float64 CUDA tensor of fixed walker positions."""
        g, wk = _state(template, precision, nblocks, pos)
        g.set_geometry(R.detach().cpu().numpy(), C_up.detach().cpu().numpy(), C_dn.detach().cpu().numpy())
        wk.set_positions(pos)  # re-inverts at the new geometry
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
