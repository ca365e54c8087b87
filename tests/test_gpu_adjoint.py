"""The library's discrete adjoint (mhde_energy_adjoint) against the oracle's
adjoint (itself pinned by central differences in test_oracle_adjoint.py) and
against central differences of the library's own forward run; the torch
autograd wrapper against the raw call."""
import dataclasses

import numpy as np
import pytest

from oracle.adjoint import energy_gradient
from paper_2108_05110_gb300 import PREC_FP64, PREC_MIXED, ensemble_io
from workloads.ensembles import sensitivity

pytestmark = pytest.mark.gpu


def _solver(ens, **opts):
    sol = ensemble_io.solver_for(ens, **opts)
    ensemble_io.feed_initial(sol, ens)
    ensemble_io.feed_step_data(sol, ens, ens.dt)        # the cavity data are constant in time
    return sol


def _amp_grads(ens, sol, res):
    psi = ens.info["perturbation_shape"](sol._nodes)
    return (np.einsum("jnd,nd->j", res["grad_u0"], psi), np.einsum("jnd,nd->j", res["grad_B0"], psi))


def _oracle_amp_grads(ens, du0, dB0):
    from oracle.fe import P2Space
    psi = ens.info["perturbation_shape"](P2Space(ens.mesh).node_xy)
    return np.einsum("jnd,nd->j", du0, psi), np.einsum("jnd,nd->j", dB0, psi)


@pytest.mark.parametrize("precision,tol", [(PREC_FP64, 1e-8), (PREC_MIXED, 1e-6)])
def test_adjoint_matches_oracle_adjoint(precision, tol):
    """8x8 mesh, J = 3, s = 0.5, 4 steps, a checkpoint every 3 steps (two
    segments): loss and every gradient entry against the oracle's adjoint."""
    ens = sensitivity(N=8, J=3, s=0.5, nsteps=4)
    K = 4
    L0, gnu0, gnum0, du0, dB0 = energy_gradient(ens, K)
    sol = _solver(ens, precision=precision, rtol=1e-13 if precision == PREC_FP64 else 1e-12)
    res = sol.energy_adjoint(K, checkpoint_every=3)
    assert abs(res["loss"] - L0) <= 1e-10 * abs(L0)
    for got, want in ((res["grad_nu"], gnu0), (res["grad_nu_m"], gnum0)):
        assert np.abs(got - want).max() <= tol * np.abs(want).max(), (got, want)
    # initial-field gradients, nodal and contracted with the perturbation shape
    for got, want in ((res["grad_u0"], du0), (res["grad_B0"], dB0)):
        assert np.abs(got - want).max() <= tol * np.abs(want).max()
    gu, gB = _amp_grads(ens, sol, res)
    ou, oB = _oracle_amp_grads(ens, du0, dB0)
    assert np.abs(gu - ou).max() <= tol * np.abs(ou).max()
    assert np.abs(gB - oB).max() <= tol * np.abs(oB).max()
    # the context is left at the final step with the forward run's state
    assert sol.stats().steps == K
    assert abs(sol.energy() - L0) <= 1e-10 * abs(L0)
    sol.close()


def _gpu_loss(ens, K, **opts):
    sol = _solver(ens, **opts)
    sol.advance(K)
    L = sol.energy()
    sol.close()
    return L


def test_adjoint_matches_central_differences_sensitivity_workload():
    """The differentiation workload (64x64, J = 8, s = 0.5, dt = 0.01, 40
    steps, a checkpoint every 5 steps), FP64 path: the adjoint gradient in
    nu_0, nu_m,0 and both perturbation amplitudes of member 0 against central
    differences of the library's forward run with h = 1e-6."""
    ens = sensitivity(N=64, J=8, s=0.5, nsteps=40)
    K = 40
    opts = dict(precision=PREC_FP64, rtol=1e-13)
    sol = _solver(ens, **opts)
    res = sol.energy_adjoint(K, checkpoint_every=5)
    gu, gB = _amp_grads(ens, sol, res)
    sol.close()
    h = 1e-6
    checks = {"nu": res["grad_nu"][0], "nu_m": res["grad_nu_m"][0], "eps_u": gu[0], "eps_B": gB[0]}
    scales = {"nu": np.abs(res["grad_nu"]).max(), "nu_m": np.abs(res["grad_nu_m"]).max(),
              "eps_u": np.abs(gu).max(), "eps_B": np.abs(gB).max()}
    for name, g in checks.items():
        vals = []
        for sgn in (1.0, -1.0):
            if name in ("nu", "nu_m"):
                arr = getattr(ens, name).copy()
                arr[0] += sgn * h
                vals.append(_gpu_loss(dataclasses.replace(ens, **{name: arr}), K, **opts))
            else:
                amp = ens.info[name]
                old = amp[0]
                amp[0] = old + sgn * h
                try:
                    vals.append(_gpu_loss(ens, K, **opts))
                finally:
                    amp[0] = old
        fd = (vals[0] - vals[1]) / (2 * h)
        # the central difference carries the forward runs' own error: each
        # solve stops at a relative residual of 1e-13, which leaves the loss
        # (0.59 here, set by the lid flow) uncertain by about 1e-13 |L|, and
        # the difference divides that by 2h
        noise = 2e-13 * abs(vals[0]) / h
        assert abs(fd - g) <= 1e-5 * scales[name] + noise, (name, fd, g)


def test_autograd_function_returns_the_adjoint_gradient():
    import torch
    from paper_2108_05110_gb300 import energy_function
    ens = sensitivity(N=8, J=3, s=0.5, nsteps=3)
    sol = _solver(ens, precision=PREC_FP64, rtol=1e-13)
    shape = ens.info["perturbation_shape"](sol._nodes)
    nu = torch.tensor(ens.nu, requires_grad=True)
    nu_m = torch.tensor(ens.nu_m, requires_grad=True)
    eu = torch.tensor(ens.info["eps_u"], requires_grad=True)
    eB = torch.tensor(ens.info["eps_B"], requires_grad=True)
    L = energy_function().apply(nu, nu_m, eu, eB, sol, shape, 3, 2)
    (2.0 * L).backward()
    ref = _solver(ens, precision=PREC_FP64, rtol=1e-13).energy_adjoint(3, 2)
    assert abs(L.item() - ref["loss"]) <= 1e-12 * abs(ref["loss"])
    assert np.allclose(nu.grad.numpy(), 2.0 * ref["grad_nu"], rtol=1e-10, atol=0)
    assert np.allclose(nu_m.grad.numpy(), 2.0 * ref["grad_nu_m"], rtol=1e-10, atol=0)
    psi = shape
    assert np.allclose(eu.grad.numpy(), 2.0 * np.einsum("jnd,nd->j", ref["grad_u0"], psi), rtol=1e-10, atol=0)
    assert np.allclose(eB.grad.numpy(), 2.0 * np.einsum("jnd,nd->j", ref["grad_B0"], psi), rtol=1e-10, atol=0)
    sol.close()
