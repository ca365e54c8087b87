"""Discrete adjoint of Algorithm 1 for the ensemble-mean energy (oracle; test
infrastructure only).

Loss: L = E_h^K = 1/2 (||<v_h>^K||^2 + ||<w_h>^K||^2) (the energy of
Section 4.2 at the final step), as a function of the member parameters
nu_j, nu_m,j and of the initial fields u^0_j, B^0_j.  Reverse-mode
differentiation of the fully discrete step (Algorithm 1, eq. weaknew1 /
weaknew2), written out term by term:

For subproblem z (z = v with other field y = w, and the mirror), member j,
the step solves A_z(<y>, l_z^2) x_j = b_j(z_j, y_j, y'_j) with
  F_z = M/dt + N(<y>) + c1 K + K_T(2 mu dt l_z^2),  c1 = (nubar + nubar_m)/2,
  l_z^2(x_q) = max_k |y'_k(x_q)|^2,
  b_j = M f_j + M z_j/dt - N(y'_j) z_j - (cross_j/2) K y_j - (same_j/2) K z_j,
  cross_j = nu_j - nu_m,j,  same_j = nu'_j + nu'_m,j.
Given the seed mu_j on the new velocity x_j, the adjoint solve is
A_z^T y_j = mu_j with the Dirichlet velocity rows of mu set to zero (those
values are data) and zero pressure rows; only the unconstrained components of
y_j enter the contractions (Dirichlet rows of A and b are constant).  With
yh_j that interior velocity part, dL/d(state, parameters) receives
  yh_j^T (d b_j - d F_z x_j)   summed over members,
which gives, per term:
  z_j:   M yh_j/dt - N(y'_j)^T yh_j - (same_j/2) K yh_j
  y_j:   -(cross_j/2) K yh_j, and through y'_j = y_j - <y>:
         -G(z_j, yh_j) on y_j, +G(z_j, yh_j)/J on every y_k
  <y>:   -G(x_j, yh_j)/J on every y_k       (matrix convection N(<y>))
  l_z^2: -2 mu dt sum_j grad yh_j : grad x_j at each quadrature point, times
         d l^2 = 2 y'_{k*} . d y'_{k*} with k* the member attaining the max
  same_j: -(1/2) yh_j^T K z_j,  cross_j: -(1/2) yh_j^T K y_j,
  c1: -sum_j yh_j^T K x_j,
where G(u, y) = d/da [y^T N(a) u] (the convecting field enters linearly).
The chain to nu_k, nu_m,k uses d same_j/d nu_k = delta_jk - 1/J,
d cross_j/d nu_k = +-delta_jk, d c1/d nu_k = 1/(2J).  At the final step
dL/dz_j = M <z>/J; at the start z^0 = u^0 +- sqrt(s) B^0.

Checked in ``tests/test_oracle_adjoint.py`` against central finite
differences of :class:`oracle.scheme.OracleRun` and against the closed form
of the K = 0 case.
"""
import numpy as np
from scipy.sparse.linalg import splu

from .scheme import OracleRun, ensemble_mean, mixing_length_sq


def trilinear_grad(space, u, y, form="skew"):
    """G(u, y)[b, d] = d/d a_{b,d} of y^T N(a) u, for P2 fields u, y [n2, 2]:
    skew form 1/2[(phi_b e_d . grad u, y) - (phi_b e_d . grad y, u)],
    standard form (phi_b e_d . grad u, y).  Returns [n2, 2]."""
    uq, yq = space.at_quad(u), space.at_quad(y)               # [nt, nq, 2]
    gu, gy = space.grad_at_quad(u), space.grad_at_quad(y)     # [nt, nq, comp, dir]
    g = np.einsum("tqcd,tqc->tqd", gu, yq)
    if form == "skew":
        g = 0.5 * (g - np.einsum("tqcd,tqc->tqd", gy, uq))
    loc = np.einsum("tq,qa,tqd->tad", space.wq, space.phi, g)
    out = np.zeros((space.n2, 2))
    np.add.at(out, space.dofs.ravel(), loc.reshape(-1, 2))
    return out


def _scatter_quad(space, coef):
    """sum_q w_q coef(x_q) phi_b(x_q) per node b, coef [nt, nq, 2] -> [n2, 2]."""
    loc = np.einsum("tq,qa,tqd->tad", space.wq, space.phi, coef)
    out = np.zeros((space.n2, 2))
    np.add.at(out, space.dofs.ravel(), loc.reshape(-1, 2))
    return out


def _apply(Mat, z):
    return np.stack([Mat @ z[:, 0], Mat @ z[:, 1]], axis=1)


def _dot(Mat, a, b):
    return float(sum(a[:, d] @ (Mat @ b[:, d]) for d in range(2)))


def reverse_step(run, Vn, Wn, Xv, Xw, seed_v, seed_w):
    """One reverse step: seeds [J, n2, 2] on the step's new velocities
    (Xv, Xw) -> seeds on its inputs (Vn, Wn) and the step's contribution to
    dL/d nu, dL/d nu_m."""
    S, J, form = run.S, run.J, run.form
    n2 = S.n2
    mv, mw = ensemble_mean(Vn), ensemble_mean(Wn)
    Vp, Wp = Vn - mv, Wn - mw
    l2v, l2w = mixing_length_sq(S, Vp), mixing_length_sq(S, Wp)
    same = run.nu_p + run.nu_m_p
    cross = run.nu - run.nu_m
    lamV, lamW = np.zeros_like(Vn), np.zeros_like(Wn)
    g_same, g_cross, g_c1 = np.zeros(J), np.zeros(J), 0.0
    subproblems = (
        (Vn, Wn, Wp, mw, l2w, Xv, seed_v, lamV, lamW),      # v: convected by <w>, eddy from w'
        (Wn, Vn, Vp, mv, l2v, Xw, seed_w, lamW, lamV),      # w: the mirror
    )
    for Z, Y, Yp, mean_y, l2, X, seed, lamZ, lamY in subproblems:
        A = run.saddle(run.shared_matrix(mean_y, l2))
        luT = splu(A.T.tocsc())
        H = np.zeros((S.nt, S.nq))
        for j in range(J):
            rhs = np.zeros(A.shape[0])
            mu = seed[j].copy()
            mu[S.boundary] = 0.0
            rhs[:n2], rhs[n2:2 * n2] = mu[:, 0], mu[:, 1]
            y = luT.solve(rhs)
            yh = np.stack([y[:n2], y[n2:2 * n2]], axis=1)
            yh[S.boundary] = 0.0
            Nj = S.convection(Yp[j], form)
            lamZ[j] += _apply(run.M, yh) / run.dt - _apply(Nj.T, yh) - 0.5 * same[j] * _apply(run.K, yh)
            G = trilinear_grad(S, Z[j], yh, form)
            lamY[j] -= G
            lamY += G / J
            lamY[j] -= 0.5 * cross[j] * _apply(run.K, yh)
            g_same[j] += -0.5 * _dot(run.K, yh, Z[j])
            g_cross[j] += -0.5 * _dot(run.K, yh, Y[j])
            g_c1 += -_dot(run.K, yh, X[j])
            lamY -= trilinear_grad(S, X[j], yh, form) / J
            H += np.einsum("tqcd,tqcd->tq", S.grad_at_quad(yh), S.grad_at_quad(X[j]))
        # eddy term: l^2 = max_k |y'_k|^2 at each quadrature point
        Ypq = S.at_quad(Yp)                                   # [J, nt, nq, 2]
        kstar = np.argmax(np.sum(Ypq * Ypq, axis=-1), axis=0)  # [nt, nq]
        coef = -2.0 * run.mu * run.dt * H                     # dL/d l^2 per quadrature point (weight in scatter)
        total = np.zeros((n2, 2))
        for k in range(J):
            sel = (kstar == k)[..., None]
            Pk = _scatter_quad(S, np.where(sel, coef[..., None] * 2.0 * Ypq[k], 0.0))
            lamY[k] += Pk
            total += Pk
        lamY -= total / J
    mean_same = g_same.sum() / J
    g_nu = g_same - mean_same + g_cross + g_c1 / (2.0 * J)
    g_nu_m = g_same - mean_same - g_cross + g_c1 / (2.0 * J)
    return lamV, lamW, g_nu, g_nu_m


def energy_gradient(ens, nsteps, form="skew", element="TH"):
    """L = E_h^K after ``nsteps`` steps of Algorithm 1 and its gradient:
    returns (L, dL/d nu [J], dL/d nu_m [J], dL/d u0 [J, n2, 2], dL/d B0 [J, n2, 2])
    with u0, B0 the nodal initial fields; ``element`` as in OracleRun."""
    run = OracleRun(ens, form=form, element=element)
    states = [(run.V.copy(), run.W.copy())]
    for _ in range(nsteps):
        run.step()
        states.append((run.V.copy(), run.W.copy()))
    J = run.J
    L = run.energy()
    VK, WK = states[-1]
    seed_v = np.repeat((_apply(run.M, ensemble_mean(VK)) / J)[None], J, axis=0)
    seed_w = np.repeat((_apply(run.M, ensemble_mean(WK)) / J)[None], J, axis=0)
    g_nu, g_nu_m = np.zeros(J), np.zeros(J)
    for n in range(nsteps - 1, -1, -1):
        Vn, Wn = states[n]
        Xv, Xw = states[n + 1]
        seed_v, seed_w, a, b = reverse_step(run, Vn, Wn, Xv, Xw, seed_v, seed_w)
        g_nu += a
        g_nu_m += b
    du0 = seed_v + seed_w
    dB0 = run.rs * (seed_v - seed_w)
    return L, g_nu, g_nu_m, du0, dB0
