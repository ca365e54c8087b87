"""Pins of the oracle's quadrature, P2/P1 space and element integrals against
exact integration (sympy), closed forms and counting identities."""
import itertools

import numpy as np
import pytest
import sympy as sy

from oracle.quadrature import triangle_rule_deg5, monomial_integral
from oracle.fe import P2Space
from workloads.mesh import Mesh, unit_square, channel_step


def test_rule_exact_to_degree_5_and_not_6():
    xy, lam, w = triangle_rule_deg5()
    assert np.all(w > 0) and abs(w.sum() - 0.5) < 1e-15
    for d in range(6):
        for i in range(d + 1):
            j = d - i
            q = np.sum(w * xy[:, 0] ** i * xy[:, 1] ** j)
            assert abs(q - monomial_integral(i, j)) < 1e-16
    # a degree-6 monomial is not integrated exactly (the rule has degree 5)
    errs = [abs(np.sum(w * xy[:, 0] ** i * xy[:, 1] ** (6 - i)) - monomial_integral(i, 6 - i))
            for i in range(7)]
    assert max(errs) > 1e-8
    # barycentric coordinates are consistent and inside the triangle
    assert np.allclose(lam.sum(axis=1), 1.0) and np.all(lam > 0)


def test_monomial_integral_closed_form_against_sympy():
    x, y = sy.symbols("x y")
    for i, j in [(0, 0), (1, 0), (2, 3), (4, 1)]:
        exact = sy.integrate(sy.integrate(x ** i * y ** j, (y, 0, 1 - x)), (x, 0, 1))
        assert abs(float(exact) - monomial_integral(i, j)) < 1e-16


TRIANGLES = [
    [(0.0, 0.0), (1.0, 0.0), (0.0, 1.0)],
    [(0.2, -0.1), (1.3, 0.4), (0.1, 0.9)],
    [(-1.0, 0.5), (0.25, -0.75), (0.6, 1.1)],
]


def _sympy_element(verts):
    """Exact P2 mass, stiffness, convection (linear field) and divergence
    matrices on one triangle, in the canonical global numbering of a
    one-triangle mesh (vertices 0,1,2; edges (0,1),(0,2),(1,2))."""
    x, y = sy.symbols("x y")
    V = [sy.Matrix([sy.Rational(str(a)), sy.Rational(str(b))]) for a, b in verts]
    nodes = V + [(V[0] + V[1]) / 2, (V[0] + V[2]) / 2, (V[1] + V[2]) / 2]
    mons = [1, x, y, x * x, x * y, y * y]
    Vd = sy.Matrix([[m.subs({x: p[0], y: p[1]}) if m != 1 else 1 for m in mons] for p in nodes])
    C = Vd.inv()
    phi = [sum(C[k, a] * mons[k] for k in range(6)) for a in range(6)]
    # P1 basis on the vertices
    mons1 = [1, x, y]
    V1 = sy.Matrix([[1, p[0], p[1]] for p in V])
    C1 = V1.inv()
    psi = [sum(C1[k, i] * mons1[k] for k in range(3)) for i in range(3)]
    # integrate over the triangle through the affine map from the reference
    s, t = sy.symbols("s t")
    X = V[0] + (V[1] - V[0]) * s + (V[2] - V[0]) * t
    det = sy.Matrix.hstack(V[1] - V[0], V[2] - V[0]).det()

    def integ(expr):
        e = sy.expand(expr.subs({x: X[0], y: X[1]}, simultaneous=True))
        return sy.integrate(sy.integrate(e, (t, 0, 1 - s)), (s, 0, 1)) * abs(det)

    a_field = (sy.Rational(3, 10) + 2 * x - y, -1 + x / 2 + sy.Rational(7, 5) * y)
    Mm = np.zeros((6, 6)); Km = np.zeros((6, 6)); Nm = np.zeros((6, 6)); Ns = np.zeros((6, 6))
    Bx = np.zeros((3, 6)); By = np.zeros((3, 6))
    grads = [(sy.diff(p, x), sy.diff(p, y)) for p in phi]
    for a in range(6):
        for b in range(6):
            Mm[a, b] = float(integ(phi[a] * phi[b]))
            Km[a, b] = float(integ(grads[a][0] * grads[b][0] + grads[a][1] * grads[b][1]))
            adb = a_field[0] * grads[b][0] + a_field[1] * grads[b][1]
            ada = a_field[0] * grads[a][0] + a_field[1] * grads[a][1]
            Ns[a, b] = float(integ(adb * phi[a]))
            Nm[a, b] = float(integ(sy.Rational(1, 2) * (adb * phi[a] - ada * phi[b])))
    for i in range(3):
        for a in range(6):
            Bx[i, a] = float(integ(-grads[a][0] * psi[i]))
            By[i, a] = float(integ(-grads[a][1] * psi[i]))
    nodal_a = np.array([[float(a_field[0].subs({x: p[0], y: p[1]})),
                         float(a_field[1].subs({x: p[0], y: p[1]}))] for p in nodes])
    return Mm, Km, Nm, Ns, Bx, By, nodal_a


@pytest.mark.parametrize("verts", TRIANGLES)
def test_element_matrices_match_exact_integrals(verts):
    mesh = Mesh(np.array(verts, dtype=np.float64), np.array([[0, 1, 2]], dtype=np.int32))
    S = P2Space(mesh)
    Mm, Km, Nm, Ns, Bx, By, nodal_a = _sympy_element(verts)
    scale = np.abs(Km).max()
    assert np.allclose(S.mass().toarray(), Mm, rtol=0, atol=1e-14)
    assert np.allclose(S.stiffness().toarray(), Km, rtol=0, atol=1e-13 * scale)
    assert np.allclose(S.convection(nodal_a, "skew").toarray(), Nm, rtol=0, atol=1e-13)
    assert np.allclose(S.convection(nodal_a, "standard").toarray(), Ns, rtol=0, atol=1e-13)
    bx, by = S.divergence()
    assert np.allclose(bx.toarray(), Bx, atol=1e-14)
    assert np.allclose(by.toarray(), By, atol=1e-14)
    # eddy stiffness with a constant coefficient is a multiple of K
    c = np.full((1, S.nq), 2.5)
    assert np.allclose(S.eddy_stiffness(c).toarray(), 2.5 * Km, atol=1e-13 * scale)


def test_p2_numbering_and_boundary_counts():
    for N in (1, 3, 8):
        S = P2Space(unit_square(N))
        nv, nt = (N + 1) ** 2, 2 * N * N
        ne = nv + nt - 1                       # Euler: V - E + F = 1
        assert S.ne == ne and S.n2 == nv + ne
        assert S.boundary.size == 8 * N        # 4N boundary edges -> 4N vertices + 4N midpoints
        # edges are sorted lexicographically and unique
        e = S.edges
        assert np.all(e[:, 0] < e[:, 1])
        keys = e[:, 0] * S.nv + e[:, 1]
        assert np.all(np.diff(keys) > 0)
        # midpoint coordinates
        assert np.allclose(S.node_xy[S.nv:], 0.5 * (S.mesh.xy[e[:, 0]] + S.mesh.xy[e[:, 1]]))
    S = P2Space(channel_step(cells_per_unit=2))
    assert S.n2 == S.nv + S.ne and S.ne == S.nv + S.nt - 1


def test_global_identities():
    mesh = channel_step(cells_per_unit=2)
    S = P2Space(mesh)
    M, K = S.mass(), S.stiffness()
    one = np.ones(S.n2)
    area = 40 * 10 - 1
    assert abs(one @ (M @ one) - area) < 1e-10
    assert np.abs(K @ one).max() < 1e-12           # constants are in the kernel of K
    # K x = 0 for the interpolant of a linear function except on boundary rows
    lin = 0.3 + 0.7 * S.node_xy[:, 0] - 1.1 * S.node_xy[:, 1]
    r = K @ lin
    assert np.abs(r[~S.is_boundary]).max() < 1e-11
    # (x, x) over the domain through M: exact for P2 data
    xq = S.node_xy[:, 0]
    exact = sum(b ** 3 / 3 * 10 for b in [40.0]) - (6 ** 3 - 5 ** 3) / 3 * 1
    assert abs(xq @ (M @ xq) - exact) < 1e-8
    # divergence of a constant field: only boundary nodes contribute
    bx, by = S.divergence()
    assert abs((bx @ one).sum()) < 1e-11 and abs((by @ one).sum()) < 1e-11
    Mp = S.pressure_mass()
    assert abs(Mp.sum() - area) < 1e-10


def test_quadratic_fields_are_reproduced():
    S = P2Space(unit_square(5))
    x, y = S.node_xy[:, 0], S.node_xy[:, 1]
    z = np.stack([x * x - 2 * x * y + 0.5, 3 * y * y + x], axis=1)
    qx, qy = S.qpts[..., 0], S.qpts[..., 1]
    exact = np.stack([qx * qx - 2 * qx * qy + 0.5, 3 * qy * qy + qx], axis=-1)
    assert np.abs(S.at_quad(z) - exact).max() < 1e-13
    g = S.grad_at_quad(z)
    assert np.abs(g[..., 0, 0] - (2 * qx - 2 * qy)).max() < 1e-12
    assert np.abs(g[..., 0, 1] - (-2 * qx)).max() < 1e-12
    assert np.abs(g[..., 1, 1] - 6 * qy).max() < 1e-12
