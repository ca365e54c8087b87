"""The ensemble-mean energy as a differentiable torch function.

``EnsembleEnergy.apply(nu, nu_m, eps_u, eps_B, solver, shape, nsteps,
checkpoint_every)`` sets the member viscosities and the initial fields
u0_j = eps_u[j] * shape, B0_j = eps_B[j] * shape (shape: [n2, 2] P2 nodal
values), runs ``nsteps`` steps of the ensemble scheme on ``solver`` (whose
Dirichlet and forcing data the caller has set) and returns
L = E_h = 1/2(||<v_h>||^2 + ||<w_h>||^2) at the last step.  The backward pass
returns the gradient that the library's discrete adjoint computed in the same
call (mhde_energy_adjoint): dL/d nu_j, dL/d nu_m,j and, contracted with
``shape``, dL/d eps_u,j and dL/d eps_B,j.  The context is left at the last
step.
"""
import numpy as np
import torch


class EnsembleEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, nu, nu_m, eps_u, eps_B, solver, shape, nsteps, checkpoint_every=5):
        shape = np.asarray(shape, dtype=np.float64)
        solver.set_viscosity(nu.detach().cpu().double().numpy(), nu_m.detach().cpu().double().numpy())
        eu = eps_u.detach().cpu().double().numpy()
        eB = eps_B.detach().cpu().double().numpy()
        solver.set_initial(eu[:, None, None] * shape[None], eB[:, None, None] * shape[None])
        res = solver.energy_adjoint(int(nsteps), int(checkpoint_every))
        g_eu = np.einsum("jnd,nd->j", res["grad_u0"], shape)
        g_eB = np.einsum("jnd,nd->j", res["grad_B0"], shape)
        dev, dt = nu.device, torch.float64
        ctx.save_for_backward(torch.as_tensor(res["grad_nu"], dtype=dt, device=dev),
                              torch.as_tensor(res["grad_nu_m"], dtype=dt, device=dev),
                              torch.as_tensor(g_eu, dtype=dt, device=dev),
                              torch.as_tensor(g_eB, dtype=dt, device=dev))
        return torch.tensor(res["loss"], dtype=dt, device=dev)

    @staticmethod
    def backward(ctx, grad_out):
        g_nu, g_nu_m, g_eu, g_eB = ctx.saved_tensors
        return grad_out * g_nu, grad_out * g_nu_m, grad_out * g_eu, grad_out * g_eB, None, None, None, None
