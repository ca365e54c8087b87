"""Algorithm 1 (fully discrete decoupled ensemble scheme, eq. weaknew1 and
weaknew2) as a plain FP64 CPU program (oracle; test infrastructure only).

Per step n -> n+1, in the order of Section 1 (eq. scheme1-incom2) and
Algorithm 1:
 1. ensemble means <v>^n, <w>^n and fluctuations v'_j, w'_j (Section 1,
    definition of the ensemble mean and fluctuation);
 2. the mixing-length quantity l^2 = max_j |z'_j|^2 at every quadrature point
    (Section 1, eddy viscosity nu_T = mu dt l^2);
 3. the shared matrices
      F_v = M/dt + N(<w>) + (nubar+nubar_m)/2 K + K_T(2 mu dt l_w^2)
      F_w = M/dt + N(<v>) + (nubar+nubar_m)/2 K + K_T(2 mu dt l_v^2)
    (left-hand sides of eq. weaknew1 / weaknew2) inside the saddle-point
    matrix [[F, 0, Bx^T], [0, F, By^T], [Bx, By, 0]] with identity rows for
    Dirichlet velocity nodes and pressure dof 0 pinned (P1 pressure:
    continuous, Taylor-Hood, or discontinuous, Scott-Vogelius);
 4. for every member j the right-hand side of eq. weaknew1
      M f1_j + M v_j^n / dt - N(w'_j) v_j^n - (nu_j - nu_m,j)/2 K w_j^n
        - (nu'_j + nu'_m,j)/2 K v_j^n
    and its mirror for eq. weaknew2 (v <-> w, f1 -> f2), Dirichlet values
    g_{v,j}(t^{n+1}) on boundary rows, zeros on pressure rows;
 5. a direct sparse LU solve (SuperLU) per member, or one factorisation per
    step shared by all members (Section 1: every member has the same matrix);
 6. pressures shifted to mean zero on output (Q = L^2_0, Section 2).

The time loop runs n = 0, ..., M-1 with forcing and boundary data at t^{n+1}.
"""
import time

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import splu

from .fe import P2Space


def ensemble_mean(Z):
    """<z> = (1/J) sum_j z_j over the member axis 0 (Section 1)."""
    return Z.sum(axis=0) / Z.shape[0]


def mixing_length_sq(space, Zp):
    """l^2(x_q) = max_j |z'_j(x_q)|^2 at every quadrature point -> [nt, nq]."""
    zq = space.at_quad(Zp)                       # [J, nt, nq, 2]
    return np.max(np.sum(zq * zq, axis=-1), axis=0)


def skew_action(space, a_nodal, u_nodal, form="skew"):
    """Vector of b*(a, u, phi_a) over all scalar test functions, per component:
    skew form 1/2[(a.grad u, phi) - (a.grad phi, u)], standard form
    (a.grad u, phi).  a_nodal, u_nodal: [n2, 2]. Returns [n2, 2]."""
    aq = space.at_quad(a_nodal)                  # [nt, nq, 2]
    uq = space.at_quad(u_nodal)                  # [nt, nq, 2]
    gu = space.grad_at_quad(u_nodal)             # [nt, nq, comp, dir]
    a_grad_u = np.einsum("tqx,tqcx->tqc", aq, gu)             # [nt, nq, comp]
    t1 = np.einsum("tq,tqc,qa->tac", space.wq, a_grad_u, space.phi)
    if form == "skew":
        a_grad_phi = np.einsum("tqx,tqax->tqa", aq, space.gphi)  # [nt, nq, 6]
        t2 = np.einsum("tq,tqa,tqc->tac", space.wq, a_grad_phi, uq)
        loc = 0.5 * (t1 - t2)
    else:
        loc = t1
    out = np.zeros((space.n2, 2))
    np.add.at(out, space.dofs.ravel(), loc.reshape(-1, 2))
    return out


class OracleRun:
    """State and one-step update of Algorithm 1 for an ``workloads.Ensemble``."""

    def __init__(self, ens, form="skew", lu_per_member=False, mu=None, element="TH"):
        """``element``: "TH" (Taylor-Hood P2/P1) or "SV" (Scott-Vogelius
        P2/P1disc, for barycenter-refined meshes; Section 2 and Section 4)."""
        if element not in ("TH", "SV"):
            raise ValueError(element)
        self.ens = ens
        self.form = form
        self.lu_per_member = lu_per_member
        self.mu = ens.mu if mu is None else mu
        self.element = element
        self.S = P2Space(ens.mesh, pressure="P1" if element == "TH" else "P1disc")
        S = self.S
        self.M = S.mass()
        self.K = S.stiffness()
        self.Bx, self.By = S.divergence()
        self.Mp = S.pressure_mass()
        self.J = ens.J
        self.nu = np.asarray(ens.nu, dtype=np.float64)
        self.nu_m = np.asarray(ens.nu_m, dtype=np.float64)
        self.nubar = self.nu.sum() / self.J
        self.nubar_m = self.nu_m.sum() / self.J
        self.nu_p = self.nu - self.nubar            # nu'_j
        self.nu_m_p = self.nu_m - self.nubar_m      # nu'_{m,j}
        self.rs = np.sqrt(ens.s)
        xy = S.node_xy
        u0, B0 = ens.u0(xy), ens.B0(xy)
        self.V = u0 + self.rs * B0                   # [J, n2, 2]
        self.W = u0 - self.rs * B0
        self.Q = np.zeros((self.J, S.np_))
        self.R = np.zeros((self.J, S.np_))
        self.n = 0
        self.dt = ens.dt
        self.timing = {"assemble": 0.0, "factor": 0.0, "solve": 0.0}
        self.last = {}

    # ---------------------------------------------------------------- pieces
    def alpha(self):
        """alpha_j = nubar + nubar_m - |nu_j - nu_m,j| - |nu'_j + nu'_m,j| (Section 3.1)."""
        return (self.nubar + self.nubar_m - np.abs(self.nu - self.nu_m)
                - np.abs(self.nu_p + self.nu_m_p))

    def shared_matrix(self, mean_conv, l2):
        """F = M/dt + N(mean_conv) + (nubar+nubar_m)/2 K + K_T(2 mu dt l^2)."""
        S = self.S
        F = (self.M / self.dt + S.convection(mean_conv, self.form)
             + 0.5 * (self.nubar + self.nubar_m) * self.K
             + S.eddy_stiffness(2.0 * self.mu * self.dt * l2))
        return F.tocsr()

    def saddle(self, F):
        """[[F, 0, Bx^T], [0, F, By^T], [Bx, By, 0]] with identity rows on
        Dirichlet velocity nodes and pressure row 0 replaced by p_0 = 0."""
        S = self.S
        keep = sp.diags((~S.is_boundary).astype(np.float64))
        bnd = sp.diags(S.is_boundary.astype(np.float64))
        Fb = keep @ F + bnd
        BxT = keep @ self.Bx.T
        ByT = keep @ self.By.T
        rows = np.ones(S.np_)
        rows[0] = 0.0
        pin = sp.diags(rows)
        e0 = sp.csr_matrix(([1.0], ([0], [0])), shape=(S.np_, S.np_))
        A = sp.bmat([[Fb, None, BxT], [None, Fb, ByT], [pin @ self.Bx, pin @ self.By, e0]])
        return A.tocsc()

    def member_data(self, t):
        """Elsaesser forcing and Dirichlet data at time t (Section 1):
        f1 = f + sqrt(s) curl g, f2 = f - sqrt(s) curl g, g_v = u + sqrt(s) B,
        g_w = u - sqrt(s) B, all at P2 nodes [J, n2, 2]."""
        ens, xy = self.ens, self.S.node_xy
        shape = (self.J, self.S.n2, 2)
        f = ens.f(xy, t) if ens.f is not None else np.zeros(shape)
        cg = ens.curl_g(xy, t) if ens.curl_g is not None else np.zeros(shape)
        ub, Bb = ens.u_bc(xy, t), ens.B_bc(xy, t)
        return (f + self.rs * cg, f - self.rs * cg, ub + self.rs * Bb, ub - self.rs * Bb)

    def rhs(self, Z, Y, Yp, f, g, j, diff_same, diff_cross):
        """Right-hand side of eq. weaknew1 for member j of subproblem z
        (z = v: Y = W, Yp = W', diff_same = nu'+nu'_m, diff_cross = nu-nu_m)."""
        S = self.S
        out = np.empty((S.n2, 2))
        conv = skew_action(S, Yp[j], Z[j], self.form)
        for d in range(2):
            out[:, d] = (self.M @ f[j][:, d] + (self.M @ Z[j][:, d]) / self.dt - conv[:, d]
                         - 0.5 * diff_cross[j] * (self.K @ Y[j][:, d])
                         - 0.5 * diff_same[j] * (self.K @ Z[j][:, d]))
        out[S.boundary] = g[j][S.boundary]
        b = np.concatenate([out[:, 0], out[:, 1], np.zeros(S.np_)])
        return b

    def solve_members(self, A, rhs_list):
        t0 = time.perf_counter()
        xs = []
        if self.lu_per_member:
            for b in rhs_list:
                lu = splu(A)
                xs.append(lu.solve(b))
        else:
            lu = splu(A)
            for b in rhs_list:
                xs.append(lu.solve(b))
        self.timing["solve"] += time.perf_counter() - t0
        return xs

    # ---------------------------------------------------------------- step
    def step(self, keep=False):
        S, J = self.S, self.J
        t1 = (self.n + 1) * self.dt
        t0 = time.perf_counter()
        mv, mw = ensemble_mean(self.V), ensemble_mean(self.W)
        Vp, Wp = self.V - mv, self.W - mw
        l2v, l2w = mixing_length_sq(S, Vp), mixing_length_sq(S, Wp)
        Fv = self.shared_matrix(mw, l2w)
        Fw = self.shared_matrix(mv, l2v)
        Av, Aw = self.saddle(Fv), self.saddle(Fw)
        f1, f2, gv, gw = self.member_data(t1)
        cross = self.nu - self.nu_m
        same = self.nu_p + self.nu_m_p
        bv = [self.rhs(self.V, self.W, Wp, f1, gv, j, same, cross) for j in range(J)]
        bw = [self.rhs(self.W, self.V, Vp, f2, gw, j, same, cross) for j in range(J)]
        self.timing["assemble"] += time.perf_counter() - t0
        xv = self.solve_members(Av, bv)
        xw = self.solve_members(Aw, bw)
        if keep:
            self.last = dict(mean_v=mv, mean_w=mw, l2_v=l2v, l2_w=l2w, Fv=Fv, Fw=Fw, Av=Av, Aw=Aw,
                             bv=np.array(bv), bw=np.array(bw), V=self.V.copy(), W=self.W.copy())
        n2 = S.n2
        Vn = np.stack([np.stack([x[:n2], x[n2:2 * n2]], axis=1) for x in xv])
        Wn = np.stack([np.stack([x[:n2], x[n2:2 * n2]], axis=1) for x in xw])
        self.Q = np.stack([x[2 * n2:] for x in xv])
        self.R = np.stack([x[2 * n2:] for x in xw])
        self.V, self.W = Vn, Wn
        self.n += 1

    # ---------------------------------------------------------------- read-out
    def zero_mean(self, P):
        """Shift pressures [J, np] to mean zero: p - (int p)/|Omega|."""
        m = np.asarray(self.Mp.sum(axis=1)).ravel()
        return P - (P @ m)[:, None] / m.sum()

    def primitive_mean(self):
        """<u> = (<v>+<w>)/2 and <B> = (<v>-<w>)/(2 sqrt s) (Section 1)."""
        mv, mw = ensemble_mean(self.V), ensemble_mean(self.W)
        u = 0.5 * (mv + mw)
        B = 0.5 * (mv - mw) / self.rs if self.rs > 0 else None
        return u, B

    def energy(self):
        """E_h^n = 1/2 (||<v_h>||^2 + ||<w_h>||^2) (Section 4.2)."""
        mv, mw = ensemble_mean(self.V), ensemble_mean(self.W)
        return 0.5 * (self.S.l2_sq(self.M, mv) + self.S.l2_sq(self.M, mw))


def run_ensemble(ens, nsteps=None, callback=None, **kw):
    run = OracleRun(ens, **kw)
    for _ in range(ens.nsteps if nsteps is None else nsteps):
        run.step()
        if callback is not None:
            callback(run)
    return run
