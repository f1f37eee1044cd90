"""Misfit gradients for structure estimation, exposed to PyTorch.

``ElementShearMisfit`` is a ``torch.autograd.Function``: its input is one
shear modulus G_e per element of a workload (each element keeps the bulk
modulus and density of its material; ``vfe_set_shear_moduli``), its output
the receiver misfit J = 1/2 sum |u^{n+1}(r) - d^n(r)|^2 of a run from rest,
and its backward pass returns dJ/dG_e.  ``ShearModulusMisfit`` is the same
with one G per material (the per-element gradient summed over the material's
elements).  Both directions run through the C ABI (``vfe_misfit_gradient``):
the forward simulation with checkpoints, the adjoint leapfrog backward in
time and the per-element accumulation of mu . (dK_e/dG) u.

The time step must be given: the critical step depends on G, so a step chosen
from the moduli would change the forward map with its own input.
"""
from __future__ import annotations

import numpy as np

from . import vfe


def with_shear_moduli(workload, G):
    """Copy of ``workload`` whose material m has shear modulus G[m] with its
    bulk modulus and density unchanged."""
    tab = np.array(workload["material_table"], dtype=np.float64)
    vp, vs, rho = tab[:, 0], tab[:, 1], tab[:, 2]
    kappa = rho * (vp * vp - 4.0 / 3.0 * vs * vs)
    G = np.asarray(G, dtype=np.float64)
    new = np.stack([np.sqrt((kappa + 4.0 / 3.0 * G) / rho), np.sqrt(G / rho), rho], axis=1)
    return dict(workload, material_table=new)


def shear_moduli(workload):
    tab = np.array(workload["material_table"], dtype=np.float64)
    return tab[:, 2] * tab[:, 1] ** 2


def _need_dt(dt):
    if dt is None or not dt > 0:
        raise ValueError("the misfit needs a fixed time step dt > 0 (the critical step "
                         "depends on the moduli being differentiated)")
    return float(dt)


def misfit_and_gradient(workload, data, path=vfe.VFE_PATH_TC, checkpoint_every=100, dt=None,
                        element_G=None):
    """(J, dJ/dG per element, dJ/dG per material) for the workload's run,
    with per-element shear moduli element_G if given."""
    dt = _need_dt(dt)
    with vfe.Mesh(workload, path=path, dt=dt) as m:
        if element_G is not None:
            vfe.vfe_set_shear_moduli(m.handle, element_G)
        grad_e, J = vfe.vfe_misfit_gradient(m.handle, data, checkpoint_every)
    mat = np.asarray(workload["material_ids"])
    solid = mat >= 0
    grad_m = np.bincount(mat[solid], weights=grad_e[solid],
                         minlength=len(workload["material_table"]))
    return J, grad_e, grad_m


try:
    import torch

    class ElementShearMisfit(torch.autograd.Function):
        """J(G) with dJ/dG from the adjoint run; G: one shear modulus per
        element (float64 tensor of nx*ny*nz; void cells' entries unused)."""

        @staticmethod
        def forward(ctx, G, workload, data, dt, path=vfe.VFE_PATH_TC, checkpoint_every=100):
            J, grad_e, _ = misfit_and_gradient(workload, data, path, checkpoint_every, dt,
                                               element_G=G.detach().cpu().numpy())
            ctx.save_for_backward(torch.as_tensor(grad_e, dtype=G.dtype, device=G.device))
            return torch.as_tensor(J, dtype=G.dtype, device=G.device)

        @staticmethod
        def backward(ctx, gout):
            (grad_e,) = ctx.saved_tensors
            return gout * grad_e, None, None, None, None, None

    class ShearModulusMisfit(torch.autograd.Function):
        """J(G) with dJ/dG from the adjoint run (G: one value per material)."""

        @staticmethod
        def forward(ctx, G, workload, data, path=vfe.VFE_PATH_TC, checkpoint_every=100,
                    dt=None):
            w = with_shear_moduli(workload, G.detach().cpu().numpy())
            J, _, grad_m = misfit_and_gradient(w, data, path, checkpoint_every, _need_dt(dt))
            ctx.save_for_backward(torch.as_tensor(grad_m, dtype=G.dtype))
            return torch.as_tensor(J, dtype=G.dtype)

        @staticmethod
        def backward(ctx, gout):
            (grad_m,) = ctx.saved_tensors
            return gout * grad_m, None, None, None, None, None
except ImportError:  # pragma: no cover - torch is always present in this project
    ShearModulusMisfit = ElementShearMisfit = None
