"""P2 velocity spaces with a P1 pressure, element integrals and global
assembly (oracle; test infrastructure only).

Two pressure spaces (Section 2: the analysis takes the Scott-Vogelius pair,
any inf-sup stable pair is allowed):
* ``"P1"``: continuous P1 pressure (Taylor-Hood P2/P1);
* ``"P1disc"``: discontinuous P1 pressure (Scott-Vogelius P2/P1disc, stable on
  barycenter-refined meshes); the divergence of every P2 field lies in
  P1disc, so a velocity that satisfies the discrete continuity equation is
  divergence-free at every point.

Numbering convention (also the convention of the library's C ABI):
* P2 node k < nv is mesh vertex k;
* P2 node nv + e is the midpoint of edge e, where the edges are the distinct
  unordered vertex pairs of the triangulation sorted lexicographically by
  (smaller vertex, larger vertex);
* continuous P1 pressure node i is vertex i; discontinuous P1 pressure dof
  3e + i is the barycentric coordinate of local vertex i on triangle e.
Local P2 node order on a triangle (v0, v1, v2): v0, v1, v2, then the
midpoints of (v0,v1), (v1,v2), (v2,v0).

Bilinear forms (Section 2 and Algorithm 1), for scalar P2 basis functions:
  M_ab   = (phi_b, phi_a)
  K_ab   = (grad phi_b, grad phi_a)
  N(a)_ab = 1/2 [ (a . grad phi_b, phi_a) - (a . grad phi_a, phi_b) ]   (skew form)
          or (a . grad phi_b, phi_a)                                     (standard form b)
  K_T(c)_ab = (c grad phi_b, grad phi_a)
  Bx_ia = -(d phi_a / dx, psi_i),  By_ia = -(d phi_a / dy, psi_i)
All integrals use the degree-5 rule of :mod:`oracle.quadrature`.
"""
import numpy as np
import scipy.sparse as sp

from .quadrature import triangle_rule_deg5

LOCAL_EDGES = ((0, 1), (1, 2), (2, 0))


def p2_values(lam):
    """P2 basis at barycentric points lam [..., 3] -> [..., 6]."""
    l0, l1, l2 = lam[..., 0], lam[..., 1], lam[..., 2]
    return np.stack([l0 * (2 * l0 - 1), l1 * (2 * l1 - 1), l2 * (2 * l2 - 1),
                     4 * l0 * l1, 4 * l1 * l2, 4 * l2 * l0], axis=-1)


def p2_bary_derivs(lam):
    """d phi_a / d lambda_k at lam [..., 3] -> [..., 6, 3]."""
    l0, l1, l2 = lam[..., 0], lam[..., 1], lam[..., 2]
    z = np.zeros_like(l0)
    rows = [
        [4 * l0 - 1, z, z],
        [z, 4 * l1 - 1, z],
        [z, z, 4 * l2 - 1],
        [4 * l1, 4 * l0, z],
        [z, 4 * l2, 4 * l1],
        [4 * l2, z, 4 * l0],
    ]
    return np.stack([np.stack(r, axis=-1) for r in rows], axis=-2)


class P2Space:
    """P2 velocity (per component) and a continuous (``pressure="P1"``) or
    discontinuous (``pressure="P1disc"``) P1 pressure on a triangulation."""

    def __init__(self, mesh, pressure="P1"):
        if pressure not in ("P1", "P1disc"):
            raise ValueError(pressure)
        self.mesh = mesh
        self.pressure = pressure
        xy, tri = mesh.xy, mesh.tri.astype(np.int64)
        nv, nt = xy.shape[0], tri.shape[0]
        self.nv, self.nt = nv, nt
        # edges: distinct sorted pairs, lexicographic order
        pairs = np.concatenate([np.sort(tri[:, list(e)], axis=1) for e in LOCAL_EDGES], axis=0)
        uniq, inv, counts = np.unique(pairs, axis=0, return_inverse=True, return_counts=True)
        inv = inv.ravel()
        self.edges = uniq
        self.ne = uniq.shape[0]
        self.n2 = nv + self.ne
        if pressure == "P1":
            self.np_ = nv
            self.pdofs = tri                                 # [nt, 3] pressure dof per local vertex
        else:
            self.np_ = 3 * nt
            self.pdofs = np.arange(3 * nt, dtype=np.int64).reshape(nt, 3)
        edge_of = inv.reshape(3, nt).T                     # [nt, 3] edge index per local edge
        self.dofs = np.concatenate([tri, nv + edge_of], axis=1)   # [nt, 6]
        # node coordinates
        self.node_xy = np.concatenate([xy, 0.5 * (xy[uniq[:, 0]] + xy[uniq[:, 1]])], axis=0)
        # boundary: edges used by exactly one triangle
        bedges = np.nonzero(counts == 1)[0]
        bnodes = np.concatenate([uniq[bedges, 0], uniq[bedges, 1], nv + bedges])
        self.boundary = np.unique(bnodes)
        self.is_boundary = np.zeros(self.n2, dtype=bool)
        self.is_boundary[self.boundary] = True

        # geometry: affine map x = x0 + Jac (xi, eta)
        p0, p1, p2 = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
        jac = np.stack([p1 - p0, p2 - p0], axis=2)          # [nt, 2(x), 2(ref)]
        det = jac[:, 0, 0] * jac[:, 1, 1] - jac[:, 0, 1] * jac[:, 1, 0]
        assert np.all(det > 0)
        self.area = 0.5 * det
        # gradients of barycentric coordinates: grad lambda_1, lambda_2 are rows of Jac^{-T}
        inv_t = np.empty((nt, 2, 2))
        inv_t[:, 0, 0] = jac[:, 1, 1] / det
        inv_t[:, 0, 1] = -jac[:, 1, 0] / det
        inv_t[:, 1, 0] = -jac[:, 0, 1] / det
        inv_t[:, 1, 1] = jac[:, 0, 0] / det
        g1, g2 = inv_t[:, :, 0], inv_t[:, :, 1]             # grad lambda_1, grad lambda_2  [nt,2]
        glam = np.stack([-g1 - g2, g1, g2], axis=1)          # [nt, 3, 2]
        self.grad_lambda = glam

        qxy, qlam, qw = triangle_rule_deg5()
        self.qlam, self.qw_ref = qlam, qw
        self.nq = qw.shape[0]
        self.phi = p2_values(qlam)                            # [nq, 6]
        dphi_dlam = p2_bary_derivs(qlam)                      # [nq, 6, 3]
        self.gphi = np.einsum("qak,tkd->tqad", dphi_dlam, glam)   # [nt, nq, 6, 2]
        self.wq = qw[None, :] * det[:, None]                  # [nt, nq] physical weights
        self.psi = qlam                                       # P1 basis at quad points [nq, 3]
        self.qpts = np.einsum("qk,tkd->tqd", qlam, xy[tri])  # [nt, nq, 2]

    # ------------------------------------------------------------------ helpers
    def _assemble(self, local, rows_dofs, cols_dofs, nrows, ncols):
        """Sum element matrices local [nt, r, c] into a CSR matrix."""
        r = np.repeat(rows_dofs[:, :, None], cols_dofs.shape[1], axis=2)
        c = np.repeat(cols_dofs[:, None, :], rows_dofs.shape[1], axis=1)
        A = sp.coo_matrix((local.ravel(), (r.ravel(), c.ravel())), shape=(nrows, ncols))
        return A.tocsr()

    def at_quad(self, nodal):
        """Evaluate P2 fields nodal [..., n2, d] at quadrature points -> [..., nt, nq, d]."""
        loc = nodal[..., self.dofs, :]                        # [..., nt, 6, d]
        return np.einsum("qa,...tad->...tqd", self.phi, loc)

    def grad_at_quad(self, nodal):
        """Gradient of P2 fields nodal [..., n2, d] at quadrature points ->
        [..., nt, nq, d(component), 2(direction)]."""
        loc = nodal[..., self.dofs, :]
        return np.einsum("tqax,...tad->...tqdx", self.gphi, loc)

    # ------------------------------------------------------------------ matrices
    def mass(self):
        loc = np.einsum("tq,qa,qb->tab", self.wq, self.phi, self.phi)
        return self._assemble(loc, self.dofs, self.dofs, self.n2, self.n2)

    def stiffness(self):
        loc = np.einsum("tq,tqax,tqbx->tab", self.wq, self.gphi, self.gphi)
        return self._assemble(loc, self.dofs, self.dofs, self.n2, self.n2)

    def eddy_stiffness(self, c):
        """K_T(c) with c given at quadrature points [nt, nq]."""
        loc = np.einsum("tq,tq,tqax,tqbx->tab", self.wq, c, self.gphi, self.gphi)
        return self._assemble(loc, self.dofs, self.dofs, self.n2, self.n2)

    def convection(self, a_nodal, form="skew"):
        """N(a) for a P2 vector field a_nodal [n2, 2] (rows = test phi_a)."""
        aq = self.at_quad(a_nodal)                            # [nt, nq, 2]
        adg = np.einsum("tqd,tqbd->tqb", aq, self.gphi)       # a . grad phi_b  [nt, nq, 6]
        std = np.einsum("tq,tqb,qa->tab", self.wq, adg, self.phi)   # (a.grad phi_b, phi_a)
        if form == "skew":
            loc = 0.5 * (std - np.transpose(std, (0, 2, 1)))
        elif form == "standard":
            loc = std
        else:
            raise ValueError(form)
        return self._assemble(loc, self.dofs, self.dofs, self.n2, self.n2)

    def divergence(self):
        """(Bx, By), each [np, n2]."""
        out = []
        for d in range(2):
            loc = -np.einsum("tq,qi,tqa->tia", self.wq, self.psi, self.gphi[..., d])
            out.append(self._assemble(loc, self.pdofs, self.dofs, self.np_, self.n2))
        return out

    def pressure_mass(self):
        loc = np.einsum("tq,qi,qk->tik", self.wq, self.psi, self.psi)
        return self._assemble(loc, self.pdofs, self.pdofs, self.np_, self.np_)

    def divergence_sq(self, z):
        """||div z||^2 of a P2 vector field z [n2, 2], integrated exactly
        (div z is linear on each triangle, the rule is of degree 5)."""
        g = self.grad_at_quad(z)                             # [nt, nq, comp, dir]
        dv = g[..., 0, 0] + g[..., 1, 1]
        return float(np.sum(self.wq * dv * dv))

    # ------------------------------------------------------------------ norms
    def l2_sq(self, M, z):
        """Discrete L2 norm squared of a P2 vector field z [n2, 2] via the mass matrix."""
        return float(sum(z[:, d] @ (M @ z[:, d]) for d in range(2)))

    def h1semi_sq(self, K, z):
        return float(sum(z[:, d] @ (K @ z[:, d]) for d in range(2)))

    def error_sq(self, z, exact, kind):
        """Squared L2 or H1-seminorm error of P2 field z [n2, 2] against a
        closed form, integrated with the degree-5 rule.  ``exact`` is
        (values(x,y) -> [.., 2], grads(x,y) -> (d/dx [..,2], d/dy [..,2]))."""
        x, y = self.qpts[..., 0], self.qpts[..., 1]
        if kind == "l2":
            e = self.at_quad(z) - exact[0](x, y)
            return float(np.sum(self.wq[..., None] * e * e))
        gz = self.grad_at_quad(z)                           # [nt, nq, 2, 2]
        dx, dy = exact[1](x, y)
        e = gz - np.stack([dx, dy], axis=-1)
        return float(np.sum(self.wq[..., None, None] * e * e))
