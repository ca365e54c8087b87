"""Triangulations used by the experiments of Section 4 (synthetic stand-ins).

A mesh is vertex coordinates ``xy`` (float64, [nv, 2]) and counter-clockwise
triangles ``tri`` (int32, [nt, 3], 0-based).  Nothing here depends on the
finite element space built on top of the mesh.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class Mesh:
    xy: np.ndarray    # float64 [nv, 2]
    tri: np.ndarray   # int32 [nt, 3], counter-clockwise

    @property
    def nv(self):
        return self.xy.shape[0]

    @property
    def nt(self):
        return self.tri.shape[0]


def _ccw(xy, tri):
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    det = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    return det


def unit_square(N, lo=0.0, hi=1.0, diagonal="right"):
    """Uniform N x N square grid of [lo, hi]^2, each cell cut by one diagonal.

    ``diagonal="right"`` cuts every cell from its lower-left to its upper-right
    corner (the "/" diagonal); ``"alternate"`` flips the diagonal on cells of
    odd parity.  Vertex (i, k) has index i + (N+1) k.
    """
    t = np.linspace(lo, hi, N + 1)
    X, Y = np.meshgrid(t, t, indexing="xy")
    xy = np.stack([X.ravel(), Y.ravel()], axis=1).astype(np.float64)
    tris = []
    for k in range(N):
        for i in range(N):
            v00 = i + (N + 1) * k
            v10 = v00 + 1
            v01 = v00 + (N + 1)
            v11 = v01 + 1
            if diagonal == "right" or (i + k) % 2 == 0:
                tris.append((v00, v10, v11))
                tris.append((v00, v11, v01))
            else:
                tris.append((v00, v10, v01))
                tris.append((v10, v11, v01))
    tri = np.asarray(tris, dtype=np.int32)
    assert np.all(_ccw(xy, tri) > 0)
    return Mesh(xy, tri)


def _cluster(t0, a, b, toward, gamma):
    """Monotone map of [a, b] onto itself clustering points toward one end."""
    s = (t0 - a) / (b - a)
    if toward == "a":
        s = s ** gamma
    else:
        s = 1.0 - (1.0 - s) ** gamma
    return a + (b - a) * s


def channel_step(cells_per_unit=7, length=40.0, height=10.0, step=(5.0, 6.0, 1.0),
                 gamma=1.3, jitter=0.2, seed=3):
    """Channel [0, length] x [0, height] minus the step [x0, x1] x [0, sy].

    A structured grid of ``cells_per_unit`` cells per unit length, graded by
    smooth monotone maps that cluster the lines toward the step's corners
    (the lines x = x0, x = x1 and y = sy stay straight), with seeded interior
    jitter of at most ``jitter`` times the local spacing and alternating
    diagonals, so the result looks unstructured to the solver.
    """
    x0, x1, sy = step
    nx = int(round(length * cells_per_unit))
    ny = int(round(height * cells_per_unit))
    i0, i1 = int(round(x0 * cells_per_unit)), int(round(x1 * cells_per_unit))
    k1 = int(round(sy * cells_per_unit))
    xs = np.linspace(0.0, length, nx + 1)
    ys = np.linspace(0.0, height, ny + 1)
    gx = xs.copy()
    m = xs < x0
    gx[m] = _cluster(xs[m], 0.0, x0, "b", gamma)
    m = xs > x1
    gx[m] = _cluster(xs[m], x1, length, "a", gamma)
    gy = ys.copy()
    m = ys > sy
    gy[m] = _cluster(ys[m], sy, height, "a", gamma)

    def solid_cell(i, k):
        return i0 <= i < i1 and k < k1

    def solid_vertex(i, k):
        return i0 < i < i1 and k < k1

    index = -np.ones((ny + 1, nx + 1), dtype=np.int64)
    pts = []
    for k in range(ny + 1):
        for i in range(nx + 1):
            if not solid_vertex(i, k):
                index[k, i] = len(pts)
                pts.append((gx[i], gy[k]))
    xy = np.asarray(pts, dtype=np.float64)

    # seeded jitter of interior vertices (not on any boundary line)
    rng = np.random.default_rng(seed)
    for k in range(1, ny):
        for i in range(1, nx):
            v = index[k, i]
            if v < 0:
                continue
            on_step = (i in (i0, i1) and k <= k1) or (k == k1 and i0 <= i <= i1)
            if on_step:
                continue
            hx = min(gx[i] - gx[i - 1], gx[i + 1] - gx[i])
            hy = min(gy[k] - gy[k - 1], gy[k + 1] - gy[k])
            d = rng.uniform(-jitter, jitter, size=2)
            xy[v, 0] += d[0] * hx
            xy[v, 1] += d[1] * hy

    tris = []
    for k in range(ny):
        for i in range(nx):
            if solid_cell(i, k):
                continue
            v00, v10 = index[k, i], index[k, i + 1]
            v01, v11 = index[k + 1, i], index[k + 1, i + 1]
            if (i + k) % 2 == 0:
                tris.append((v00, v10, v11))
                tris.append((v00, v11, v01))
            else:
                tris.append((v00, v10, v01))
                tris.append((v10, v11, v01))
    tri = np.asarray(tris, dtype=np.int32)
    assert np.all(_ccw(xy, tri) > 0)
    return Mesh(xy, tri)


def barycentric_refine(mesh):
    """Barycenter refinement (Alfeld split) of a triangulation: every triangle
    (a, b, c) gets a new vertex at its barycenter g and is replaced by the
    three triangles (a, b, g), (b, c, g), (c, a, g), all counter-clockwise.
    New vertex nv + e is the barycenter of old triangle e; new triangle
    3e + k is the one on old local edge k.  This is the mesh on which the
    Scott-Vogelius pair (P2, P1disc) is inf-sup stable in 2D (Section 2)."""
    xy, tri = mesh.xy, mesh.tri.astype(np.int64)
    nv, nt = xy.shape[0], tri.shape[0]
    g = xy[tri].mean(axis=1)
    new_xy = np.concatenate([xy, g], axis=0)
    c = nv + np.arange(nt, dtype=np.int64)
    a, b, d = tri[:, 0], tri[:, 1], tri[:, 2]
    new_tri = np.stack([np.stack([a, b, c], axis=1), np.stack([b, d, c], axis=1),
                        np.stack([d, a, c], axis=1)], axis=1).reshape(3 * nt, 3)
    new_tri = new_tri.astype(np.int32)
    assert np.all(_ccw(new_xy, new_tri) > 0)
    return Mesh(new_xy, new_tri)
