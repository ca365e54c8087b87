"""Pins of the oracle's discrete adjoint (oracle/adjoint.py) against the plain
definition of the derivative: central finite differences of the oracle's own
forward run (Algorithm 1) in the parameters nu_j, nu_m,j and the initial
perturbation amplitudes, and the closed form of the zero-step case."""
import dataclasses

import numpy as np
import pytest

from oracle.adjoint import energy_gradient
from oracle.scheme import OracleRun
from workloads.ensembles import sensitivity


def _loss(ens, nsteps, form="skew", element="TH"):
    run = OracleRun(ens, form=form, element=element)
    for _ in range(nsteps):
        run.step()
    return run.energy()


def _amplitude_grads(ens, du0, dB0):
    """dL/d eps_u,j = psi . dL/du0_j and dL/d eps_B,j = psi . dL/dB0_j with
    psi the perturbation shape at the P2 nodes."""
    from oracle.fe import P2Space
    xy = P2Space(ens.mesh).node_xy
    psi = ens.info["perturbation_shape"](xy)
    return np.einsum("jnd,nd->j", du0, psi), np.einsum("jnd,nd->j", dB0, psi)


def _fd(ens, nsteps, which, k, h, form="skew", element="TH"):
    """Central difference of L in one parameter (h absolute, FP64)."""
    vals = []
    for sgn in (+1.0, -1.0):
        if which in ("nu", "nu_m"):
            arr = getattr(ens, which).copy()
            arr[k] += sgn * h
            e = dataclasses.replace(ens, **{which: arr})
            vals.append(_loss(e, nsteps, form, element))
        else:
            amp = ens.info[which]
            old = amp[k]
            amp[k] = old + sgn * h
            try:
                vals.append(_loss(ens, nsteps, form, element))
            finally:
                amp[k] = old
    return (vals[0] - vals[1]) / (2.0 * h)


def test_zero_steps_is_the_energy_gradient():
    """K = 0: L = 1/2(<v>^T M <v> + <w>^T M <w>) with v = u + sqrt(s) B,
    w = u - sqrt(s) B, so dL/d eps_u,j = psi^T M (<v> + <w>)/J and
    dL/d eps_B,j = sqrt(s) psi^T M (<v> - <w>)/J; checked by differencing."""
    ens = sensitivity(N=4, J=3, s=0.5, nsteps=0)
    L, gnu, gnum, du0, dB0 = energy_gradient(ens, 0)
    assert np.all(gnu == 0.0) and np.all(gnum == 0.0)
    gu, gB = _amplitude_grads(ens, du0, dB0)
    for k in range(3):
        assert abs(_fd(ens, 0, "eps_u", k, 1e-6) - gu[k]) <= 1e-8 * max(1e-30, np.abs(gu).max())
        assert abs(_fd(ens, 0, "eps_B", k, 1e-6) - gB[k]) <= 1e-8 * max(1e-30, np.abs(gB).max())


@pytest.mark.parametrize("form", ["skew", "standard"])
def test_adjoint_matches_central_differences(form):
    """Every parameter of a 3-step, 3-member run on a 4x4 mesh (s = 0.5,
    nu_j, nu_m,j = 0.005(1 + delta), independent): the adjoint gradient
    equals the central difference (h = 1e-6) to 1e-6 of the largest entry."""
    ens = sensitivity(N=4, J=3, s=0.5, nsteps=3)
    K = 3
    L, gnu, gnum, du0, dB0 = energy_gradient(ens, K, form=form)
    assert np.isclose(L, _loss(ens, K, form), rtol=1e-13)
    gu, gB = _amplitude_grads(ens, du0, dB0)
    for name, g in (("nu", gnu), ("nu_m", gnum), ("eps_u", gu), ("eps_B", gB)):
        scale = np.abs(g).max()
        assert scale > 0.0
        for k in range(3):
            fd = _fd(ens, K, name, k, 1e-6, form)
            assert abs(fd - g[k]) <= 1e-6 * scale, (name, k, fd, g[k])


def test_adjoint_matches_central_differences_scott_vogelius():
    """The same check with the discontinuous pressure on the barycenter
    refinement of a 3x3 mesh (2 steps, 2 members)."""
    from workloads.mesh import barycentric_refine
    base = sensitivity(N=3, J=2, s=0.5, nsteps=2)
    ens = dataclasses.replace(base, mesh=barycentric_refine(base.mesh))
    K = 2
    L, gnu, gnum, du0, dB0 = energy_gradient(ens, K, element="SV")
    assert np.isclose(L, _loss(ens, K, element="SV"), rtol=1e-13)
    gu, gB = _amplitude_grads(ens, du0, dB0)
    for name, g in (("nu", gnu), ("nu_m", gnum), ("eps_u", gu), ("eps_B", gB)):
        scale = np.abs(g).max()
        assert scale > 0.0
        for k in range(2):
            fd = _fd(ens, K, name, k, 1e-6, element="SV")
            assert abs(fd - g[k]) <= 1e-6 * scale, (name, k, fd, g[k])


def test_planted_sign_error_is_caught():
    """A dropped factor in the nu chain (here: the mean-diffusivity term
    c1 = (nubar + nubar_m)/2 counted twice) must break the agreement, so
    the comparison above is sensitive to the terms it pins."""
    import oracle.adjoint as adj
    ens = sensitivity(N=4, J=3, s=0.5, nsteps=2)
    orig = adj.reverse_step

    def planted(*a, **kw):
        lv, lw, gn, gm = orig(*a, **kw)
        return lv, lw, 2.0 * gn, gm

    adj.reverse_step = planted
    try:
        _, gnu, _, _, _ = adj.energy_gradient(ens, 2)
    finally:
        adj.reverse_step = orig
    fd = _fd(ens, 2, "nu", 0, 1e-6)
    assert abs(fd - gnu[0]) > 1e-3 * abs(fd)
