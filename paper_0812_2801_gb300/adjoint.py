"""torch.autograd.Function over libemd's adjoint propagation.

``ObservableGrad.apply(R, field, sysin, n_steps, dt, mu, ckpt_every, kind[, V])``
returns the final-state observable (dipole along z, or E_KS plus the ions'
kinetic energy when they move) of a trajectory started from ``sysin``'s
orbitals at ion positions ``R`` under the per-step field amplitudes
``field``: fixed ions when ``V`` is omitted or None, otherwise ions moving by
velocity Verlet from velocities ``V`` (held constant for the gradient).  Its
backward pass returns the gradients libemd computes by adjoint propagation.  Marshalling only: the forward and
backward sweeps run in the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import emd

KINDS = {"energy": emd.EMD_OBS_ENERGY, "dipole": emd.EMD_OBS_DIPOLE_Z}


class ObservableGrad(torch.autograd.Function):
    @staticmethod
    def forward(ctx, R, field, sysin, n_steps, dt, mu, ckpt_every, kind, V=None):
        h = emd.emd_init_system(emd.config_for(sysin, emd.EMD_FP64))
        try:
            Rn = R.detach().cpu().numpy().astype(np.float64)
            if V is None:
                emd.emd_set_option(h, emd.EMD_OPT_FROZEN_IONS, 1)
                Vn = np.zeros_like(Rn)
            else:
                Vn = np.asarray(V.detach().cpu().numpy() if torch.is_tensor(V) else V,
                                dtype=np.float64)
            emd.emd_set_ions(h, Rn, Vn)
            emd.emd_set_orbitals(h, sysin.psi)
            L, dR, df = emd.emd_propagate_adjoint(
                h, n_steps, dt, mu, field.detach().cpu().numpy(), ckpt_every,
                KINDS[kind], sysin.n_atoms)
        finally:
            emd.emd_destroy(h)
        ctx.save_for_backward(torch.as_tensor(dR, dtype=R.dtype),
                              torch.as_tensor(df, dtype=field.dtype))
        return torch.tensor(L, dtype=torch.float64)

    @staticmethod
    def backward(ctx, g):
        dR, df = ctx.saved_tensors
        return g * dR, g * df, None, None, None, None, None, None, None
