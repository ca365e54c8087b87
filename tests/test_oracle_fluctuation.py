"""Pins of the oracle's two fluctuation terms against closed forms.

Algorithm 1 (eq. weaknew1 / weaknew2) carries the ensemble fluctuations in
two places:
* the eddy-viscosity term (2 nu_T(w'_h, t^n) grad v, grad chi) on the left of
  eq. weaknew1, with nu_T(z', t^n) = mu dt (l_z^n)^2 and l_z^n = max_j |z'_j^n|
  the pointwise length of the largest fluctuation (Section 1, definition of
  the eddy viscosity), and its mirror with v' in eq. weaknew2;
* the explicit fluctuation convection -b(w'_j^n, v_j^n, chi) on the right of
  eq. weaknew1, and -b(v'_j^n, w_j^n, chi) on the right of eq. weaknew2.

Every expected value below is fixed by the mathematics, not by the oracle's
own formulas: fluctuation fields that are linear (so the P2 interpolant is
exact and max_j |z'_j|^2 is a known polynomial), quadratic forms u^T F u of
fields u whose integrals over the unit square are written out by hand, and
trilinear forms of global polynomials integrated exactly by sympy over the
unit square.  Each pin is a function of the oracle pieces it checks; the
``*_catches_*`` tests plant plausible mistakes in copies of those pieces
(a dropped square, a mean for the max, a dropped factor 2 or mu, a flipped
sign, the full field for its fluctuation, the wrong subproblem's field) and
require the pin to fail on each.
"""
import numpy as np
import pytest
import sympy as sym

import oracle.scheme as scheme
from oracle.fe import P2Space
from oracle.quadrature import triangle_rule_deg5
from oracle.scheme import OracleRun, mixing_length_sq, skew_action
from workloads.ensembles import Ensemble
from workloads.mesh import unit_square

N_MESH = 4


def _mesh_quad_points(mesh):
    """Physical quadrature points [nt, nq, 2] from the barycentric rule and the
    triangle vertices (independent of the P2 space's own tables)."""
    _, lam, _ = triangle_rule_deg5()
    return np.einsum("qk,tkd->tqd", lam, mesh.xy[mesh.tri])


def _linear_fluctuations(xy):
    """Three fluctuations summing to zero: (x, 0), (0, y), -(x, y).  Their
    squared lengths are x^2, y^2 and x^2 + y^2, so the pointwise maximum is
    x^2 + y^2 and the member mean is 2 (x^2 + y^2) / 3."""
    x, y = xy[:, 0], xy[:, 1]
    z = np.zeros_like(x)
    return np.stack([np.stack([x, z], 1), np.stack([z, y], 1), -np.stack([x, y], 1)])


# --------------------------------------------------------------------------- l^2 = max_j |z'_j|^2
def check_mixing_length(fn):
    mesh = unit_square(N_MESH)
    S = P2Space(mesh)
    q = _mesh_quad_points(mesh)
    # (1) z'_1 = -z'_2 = c (a constant vector): l^2 = |c|^2 everywhere
    c = np.array([0.3, -0.5])
    Zp = np.stack([np.broadcast_to(c, (S.n2, 2)), np.broadcast_to(-c, (S.n2, 2))])
    l2 = fn(S, Zp)
    assert l2.shape == (S.nt, S.nq)
    assert np.allclose(l2, 0.34, rtol=0, atol=1e-15)
    # (2) linear fluctuations: l^2 = x^2 + y^2 at every quadrature point
    l2 = fn(S, _linear_fluctuations(S.node_xy))
    assert np.allclose(l2, q[..., 0] ** 2 + q[..., 1] ** 2, rtol=0, atol=1e-14)


def test_mixing_length_closed_forms():
    check_mixing_length(mixing_length_sq)


def _l2_no_square(S, Zp):
    zq = S.at_quad(Zp)
    return np.max(np.sqrt(np.sum(zq * zq, axis=-1)), axis=0)


def _l2_mean(S, Zp):
    zq = S.at_quad(Zp)
    return np.mean(np.sum(zq * zq, axis=-1), axis=0)


def _l2_first_component(S, Zp):
    zq = S.at_quad(Zp)
    return np.max(zq[..., 0] ** 2, axis=0)


@pytest.mark.parametrize("mutant", [_l2_no_square, _l2_mean, _l2_first_component])
def test_mixing_length_pin_catches_planted_mistakes(mutant):
    with pytest.raises(AssertionError):
        check_mixing_length(mutant)


# --------------------------------------------------------------------------- shared matrix eddy term
def _plain_ensemble(mesh, J=3, nu=0.01, nu_m=0.02, dt=0.05, mu=0.75, s=1.0):
    zero = lambda p, t=0.0: np.zeros((J, p.shape[0], 2))
    return Ensemble("pin", mesh, np.full(J, nu), np.full(J, nu_m), s, dt, 1, u0=zero, B0=zero,
                    u_bc=zero, B_bc=zero, mu=mu)


def _quadratic_forms(F, xy):
    """u^T F u for the nodal interpolants of u = x, y and x + 2y (exact in P2)."""
    x, y = xy[:, 0], xy[:, 1]
    return np.array([u @ (F @ u) for u in (x, y, x + 2 * y)])


def _expected_forms(dt, nu_hat, mu, eddy, conv_std=0.0):
    """Closed forms on the unit square for l^2 = x^2 + y^2 (eddy = True) or 0:
      int x^2 = int y^2 = 1/3, int (x+2y)^2 = 8/3, |grad u|^2 = 1, 1, 5,
      int (x^2+y^2) = 2/3,
    so u^T F u = int u^2 / dt + nu_hat int |grad u|^2 + 2 mu dt int l^2 |grad u|^2
    (+ the convection form, 0 for the skew form)."""
    mass = np.array([1 / 3, 1 / 3, 8 / 3])
    grad = np.array([1.0, 1.0, 5.0])
    out = mass / dt + nu_hat * grad
    if eddy:
        out = out + 2.0 * mu * dt * (2.0 / 3.0) * grad
    return out + conv_std


def check_shared_matrix(shared_matrix, form="skew"):
    mesh = unit_square(N_MESH)
    ens = _plain_ensemble(mesh)
    run = OracleRun(ens, form=form)
    S = run.S
    l2 = mixing_length_sq(S, _linear_fluctuations(S.node_xy))
    nu_hat = 0.5 * (run.nubar + run.nubar_m)
    if form == "skew":
        # any mean field: the skew form adds nothing to u^T N u
        rng = np.random.default_rng(7)
        mean = rng.standard_normal((S.n2, 2))
        conv = 0.0
    else:
        # mean (1, 0): int (d_x u) u = 1/2 int_0^1 [u^2(1, y) - u^2(0, y)] dy
        #   = 1/2, 1/2 * 0, and 1/2 int (1 + 4y) dy = 3/2 for u = x, y, x + 2y
        mean = np.broadcast_to(np.array([1.0, 0.0]), (S.n2, 2)).copy()
        conv = np.array([0.5, 0.0, 1.5])
    got = _quadratic_forms(shared_matrix(run, mean, l2), S.node_xy)
    want = _expected_forms(ens.dt, nu_hat, ens.mu, True, conv)
    assert np.allclose(got, want, rtol=1e-13, atol=0)
    got0 = _quadratic_forms(shared_matrix(run, mean, np.zeros_like(l2)), S.node_xy)
    assert np.allclose(got0, _expected_forms(ens.dt, nu_hat, ens.mu, False, conv), rtol=1e-13, atol=0)


@pytest.mark.parametrize("form", ["skew", "standard"])
def test_shared_matrix_eddy_term_closed_form(form):
    check_shared_matrix(OracleRun.shared_matrix, form)


def _F_without_factor_two(run, mean, l2):
    S = run.S
    return (run.M / run.dt + S.convection(mean, run.form) + 0.5 * (run.nubar + run.nubar_m) * run.K
            + S.eddy_stiffness(run.mu * run.dt * l2)).tocsr()


def _F_without_mu(run, mean, l2):
    S = run.S
    return (run.M / run.dt + S.convection(mean, run.form) + 0.5 * (run.nubar + run.nubar_m) * run.K
            + S.eddy_stiffness(2.0 * run.dt * l2)).tocsr()


def _F_eddy_sign(run, mean, l2):
    S = run.S
    return (run.M / run.dt + S.convection(mean, run.form) + 0.5 * (run.nubar + run.nubar_m) * run.K
            - S.eddy_stiffness(2.0 * run.mu * run.dt * l2)).tocsr()


@pytest.mark.parametrize("mutant", [_F_without_factor_two, _F_without_mu, _F_eddy_sign])
def test_shared_matrix_pin_catches_planted_mistakes(mutant):
    with pytest.raises(AssertionError):
        check_shared_matrix(mutant)


# --------------------------------------------------------------------------- b*(a, u, chi)
X, Y = sym.symbols("x y")
A_SYM = (Y + sym.Rational(3, 10), -X + sym.Rational(1, 5))       # linear advecting field
U_SYM = (X ** 2, X * Y)                                          # quadratic field
CHI_SYM = (Y ** 2, X + Y)                                        # quadratic test field


def _sympy_trilinear(a, u, chi, form):
    """b(a, u, chi) = (a . grad u, chi), skew form 1/2[b(a, u, chi) - b(a, chi, u)],
    integrated exactly over the unit square (Section 2, trilinear form b)."""
    def b(a_, u_, c_):
        return sum((a_[0] * sym.diff(u_[k], X) + a_[1] * sym.diff(u_[k], Y)) * c_[k] for k in range(2))
    expr = b(a, u, chi) if form == "standard" else sym.Rational(1, 2) * (b(a, u, chi) - b(a, chi, u))
    return float(sym.integrate(sym.integrate(sym.expand(expr), (X, 0, 1)), (Y, 0, 1)))


def _nodal(field, xy):
    f = sym.lambdify((X, Y), list(field), "numpy")
    vals = f(xy[:, 0], xy[:, 1])
    return np.stack([np.broadcast_to(np.asarray(v, dtype=np.float64), xy[:, 0].shape) for v in vals], 1)


def check_skew_action(fn):
    """chi^T fn(a, u) = b*(a, u, chi) for global polynomials (the integrand
    has degree 5, exact with the degree-5 rule), both forms."""
    S = P2Space(unit_square(N_MESH))
    xy = S.node_xy
    a, u, chi = _nodal(A_SYM, xy), _nodal(U_SYM, xy), _nodal(CHI_SYM, xy)
    for form in ("skew", "standard"):
        got = float(np.sum(chi * fn(S, a, u, form)))
        want = _sympy_trilinear(A_SYM, U_SYM, CHI_SYM, form)
        assert abs(got - want) <= 1e-13 * max(1.0, abs(want)), (form, got, want)


def test_skew_action_equals_exact_trilinear_form():
    check_skew_action(skew_action)


def test_skew_action_matches_convection_matrix():
    """The vector of b*(a, u, phi_i) equals the convection matrix (pinned
    element by element against sympy) applied to u, per component."""
    S = P2Space(unit_square(N_MESH))
    rng = np.random.default_rng(3)
    a, u = rng.standard_normal((S.n2, 2)), rng.standard_normal((S.n2, 2))
    for form in ("skew", "standard"):
        N = S.convection(a, form)
        out = skew_action(S, a, u, form)
        for d in range(2):
            assert np.allclose(out[:, d], N @ u[:, d], rtol=0, atol=1e-13 * np.abs(out).max())


def _skew_flipped(S, a, u, form="skew"):
    return -skew_action(S, a, u, form)


def _skew_transposed(S, a, u, form="skew"):
    # (a . grad phi, u) alone: the second half of the skew form without the first
    out = skew_action(S, a, u, "standard")
    return out - 2.0 * skew_action(S, a, u, "skew") if form == "skew" else out


@pytest.mark.parametrize("mutant", [_skew_flipped, _skew_transposed])
def test_skew_action_pin_catches_planted_mistakes(mutant):
    with pytest.raises(AssertionError):
        check_skew_action(mutant)


# --------------------------------------------------------------------------- one step of Algorithm 1
def _fluctuating_ensemble(which, J=3, dt=0.05, mu=0.75, s=1.0):
    """Members with identical `other` field and linear fluctuations (sum zero)
    around a nonzero mean in the `which` field ("w" or "v"); nu_j = nu_m,j and
    all members alike, so the two viscous right-hand-side terms vanish."""
    mesh = unit_square(N_MESH)
    rs = np.sqrt(s)

    def fields(p):
        mean_fluct = np.stack([0.4 + 0.2 * p[:, 1], -0.3 + 0.1 * p[:, 0]], 1)
        other = np.stack([p[:, 0] ** 2, p[:, 0] * p[:, 1]], 1)
        fl = mean_fluct[None] + _linear_fluctuations(p)
        ot = np.broadcast_to(other, (J,) + other.shape)
        return (ot, fl) if which == "w" else (fl, ot)

    def u0(p):
        v, w = fields(p)
        return 0.5 * (v + w)

    def B0(p):
        v, w = fields(p)
        return 0.5 * (v - w) / rs

    zero = lambda p, t=0.0: np.zeros((J, p.shape[0], 2))
    ens = Ensemble("pin-step", mesh, np.full(J, 0.01), np.full(J, 0.01), s, dt, 1, u0=u0, B0=B0,
                   u_bc=zero, B_bc=zero, mu=mu)
    return ens


def check_step_pairing(which):
    """The eddy term of eq. weaknew1 uses l_w (from w'), that of eq. weaknew2
    uses l_v: with fluctuations in one field only, exactly one of the two
    shared matrices carries 2 mu dt (x^2 + y^2) K."""
    ens = _fluctuating_ensemble(which)
    run = OracleRun(ens)
    run.step(keep=True)
    nu_hat = 0.5 * (run.nubar + run.nubar_m)
    xy = run.S.node_xy
    Fv = _quadratic_forms(run.last["Fv"], xy)
    Fw = _quadratic_forms(run.last["Fw"], xy)
    eddy = _expected_forms(ens.dt, nu_hat, ens.mu, True)
    plain = _expected_forms(ens.dt, nu_hat, ens.mu, False)
    if which == "w":
        assert np.allclose(Fv, eddy, rtol=1e-13) and np.allclose(Fw, plain, rtol=1e-13)
    else:
        assert np.allclose(Fw, eddy, rtol=1e-13) and np.allclose(Fv, plain, rtol=1e-13)


def check_rhs_fluctuation(which):
    """Interior rows of the right-hand side of eq. weaknew1 (which = "w": the
    w members fluctuate) are M v^n / dt - b*(w'_j, v^n_j, phi_i): f = 0,
    nu_j = nu_m,j and nu'_j = 0 remove every other term.  Mirror for eq.
    weaknew2 with v'.  b* is pinned above against exact integrals."""
    ens = _fluctuating_ensemble(which)
    run = OracleRun(ens)
    run.step(keep=True)
    S, n2 = run.S, run.S.n2
    inner = ~S.is_boundary
    Z = run.last["V"] if which == "w" else run.last["W"]          # the subproblem's own field
    Y = run.last["W"] if which == "w" else run.last["V"]          # the fluctuating field
    b = run.last["bv"] if which == "w" else run.last["bw"]
    Yp = Y - Y.mean(axis=0)
    for j in range(ens.J):
        want = np.stack([run.M @ Z[j][:, d] for d in range(2)], 1) / ens.dt - skew_action(S, Yp[j], Z[j])
        got = np.stack([b[j][:n2], b[j][n2:2 * n2]], 1)
        assert np.abs(got[inner] - want[inner]).max() <= 1e-12 * np.abs(want[inner]).max()
        assert np.abs(Yp[j]).max() > 0.1                           # the term is really present
    assert np.all(b[:, 2 * n2:] == 0.0)                            # pressure rows


@pytest.mark.parametrize("which", ["w", "v"])
def test_step_eddy_term_uses_the_other_fields_fluctuation(which):
    check_step_pairing(which)


@pytest.mark.parametrize("which", ["w", "v"])
def test_step_rhs_carries_minus_fluctuation_convection(which):
    check_rhs_fluctuation(which)


def _rhs_with(action):
    """A copy of OracleRun.rhs whose fluctuation convection is `action`."""
    def rhs(self, Z, Y, Yp, f, g, j, diff_same, diff_cross):
        S = self.S
        out = np.empty((S.n2, 2))
        conv = action(self, Z, Y, Yp, j)
        for d in range(2):
            out[:, d] = (self.M @ f[j][:, d] + (self.M @ Z[j][:, d]) / self.dt - conv[:, d]
                         - 0.5 * diff_cross[j] * (self.K @ Y[j][:, d])
                         - 0.5 * diff_same[j] * (self.K @ Z[j][:, d]))
        out[S.boundary] = g[j][S.boundary]
        return np.concatenate([out[:, 0], out[:, 1], np.zeros(S.np_)])
    return rhs


RHS_MUTANTS = {
    "sign": lambda self, Z, Y, Yp, j: -skew_action(self.S, Yp[j], Z[j], self.form),
    "full field": lambda self, Z, Y, Yp, j: skew_action(self.S, Y[j], Z[j], self.form),
    "swapped arguments": lambda self, Z, Y, Yp, j: skew_action(self.S, Z[j], Yp[j], self.form),
    "dropped": lambda self, Z, Y, Yp, j: np.zeros_like(Z[j]),
}


@pytest.mark.parametrize("name", sorted(RHS_MUTANTS))
def test_rhs_pin_catches_planted_mistakes(name, monkeypatch):
    monkeypatch.setattr(OracleRun, "rhs", _rhs_with(RHS_MUTANTS[name]))
    with pytest.raises(AssertionError):
        check_rhs_fluctuation("w")


def test_step_pairing_pin_catches_swapped_mixing_lengths(monkeypatch):
    """A step that hands F_v the mixing length of v' (and F_w that of w')
    fails the pin."""
    real_step, real_F = OracleRun.step, OracleRun.shared_matrix

    def step(self, keep=False):
        mv, mw = scheme.ensemble_mean(self.V), scheme.ensemble_mean(self.W)
        swapped = iter([mixing_length_sq(self.S, self.V - mv), mixing_length_sq(self.S, self.W - mw)])
        # the step builds F_v first, then F_w
        monkeypatch.setattr(OracleRun, "shared_matrix", lambda self_, mean, l2: real_F(self_, mean, next(swapped)))
        try:
            real_step(self, keep)
        finally:
            monkeypatch.setattr(OracleRun, "shared_matrix", real_F)
    monkeypatch.setattr(OracleRun, "step", step)
    with pytest.raises(AssertionError):
        check_step_pairing("w")
