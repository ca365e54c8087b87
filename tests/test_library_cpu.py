"""CPU tests of the library's host side: the shared object loads and
exports every function include/mhde.h declares, and the host-built discrete
structure (P2 numbering, Dirichlet nodes, patterns) matches the oracle's
independent construction.  No GPU work is done here (contexts are not bound).
"""
import ctypes

import numpy as np
import pytest
import scipy.sparse as sp

import paper_2108_05110_gb300 as P
from paper_2108_05110_gb300 import ensemble_io
from oracle.fe import P2Space
from workloads.ensembles import lid_cavity, channel
from workloads.mesh import unit_square, channel_step, barycentric_refine


def test_library_exports_every_declared_function():
    lib = P.load_library()
    names = P.declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib.lib, n), n
    assert set(names) == set(P.binding.SIGNATURES)


@pytest.mark.parametrize("mesh", [unit_square(6), channel_step(cells_per_unit=2)])
def test_host_numbering_matches_oracle(mesh):
    s = P.EnsembleSolver(mesh.xy, mesh.tri, [0.01, 0.02], [0.01, 0.03], 0.5, 0.01, bind=False)
    S = P2Space(mesh)
    assert s.sizes.n2 == S.n2 and s.sizes.np == S.np_ and s.sizes.ne == S.ne
    xy, isb = s.p2_nodes()
    assert np.array_equal(xy, S.node_xy)
    assert np.array_equal(isb, S.is_boundary)
    assert s.sizes.n_boundary == S.boundary.size
    # pattern sizes: F has the pattern of the oracle's P2 mass matrix, B of its divergence
    M = S.mass()
    Bx, _ = S.divergence()
    nnzF = sp.csr_matrix((np.ones(M.nnz), M.indices, M.indptr), shape=M.shape).nnz
    assert s.sizes.nnz_F == nnzF
    Bpat = Bx.copy()
    Bpat.data[:] = 1.0
    assert s.sizes.nnz_B == Bpat.nnz
    assert s.sizes.n_rows == 2 * S.n2 + S.np_
    assert s.sizes.amg_levels >= 1
    s.close()


def test_create_rejects_bad_input():
    m = unit_square(3)
    lib = P.load_library()
    with pytest.raises(P.MhdeError):
        P.EnsembleSolver(m.xy, m.tri, [0.01], [0.01], 1.0, -0.1, bind=False)      # dt <= 0
    with pytest.raises(P.MhdeError):
        P.EnsembleSolver(m.xy, m.tri, [0.01], [0.01], -1.0, 0.1, bind=False)      # s < 0
    bad = m.tri.copy()
    bad[0] = bad[0][::-1]                                                         # clockwise
    with pytest.raises(P.MhdeError):
        P.EnsembleSolver(m.xy, bad, [0.01], [0.01], 1.0, 0.1, bind=False)
    # alpha_j <= 0 is an error only with strict = 1 (Section 3.1)
    nu, nu_m = [0.01, 0.02], [0.2, 0.001]
    P.EnsembleSolver(m.xy, m.tri, nu, nu_m, 1.0, 0.1, bind=False).close()
    with pytest.raises(P.MhdeError) as e:
        P.EnsembleSolver(m.xy, m.tri, nu, nu_m, 1.0, 0.1, bind=False, strict=1)
    assert e.value.code == -2
    with pytest.raises(P.MhdeError):
        P.EnsembleSolver(m.xy, m.tri, [0.01], [0.01], 1.0, 0.1, bind=False, strict=1, mu=0.4)
    # option fields outside their ranges
    for bad_opt in (dict(inner_fp16=2), dict(inner_iters=17), dict(schur=3), dict(element=2),
                    dict(element=1, schur=1)):
        with pytest.raises(P.MhdeError):
            P.EnsembleSolver(m.xy, m.tri, [0.01], [0.01], 1.0, 0.1, bind=False, **bad_opt)
    P.EnsembleSolver(m.xy, m.tri, [0.01], [0.01], 1.0, 0.1, bind=False, inner_fp16=1).close()


@pytest.mark.parametrize("kw", [dict(element="SV"), dict(element="SV", schur=0), dict(schur=2)])
def test_discontinuous_pressure_and_algebraic_laplacian_host_build(kw):
    """Scott-Vogelius: three pressure dofs per triangle and the divergence
    pattern of the oracle's P1disc space; the algebraic pressure Laplacian
    B D^{-1} B^T (also taken by the least-squares commutator on Taylor-Hood)
    coarsens into a hierarchy."""
    mesh = barycentric_refine(unit_square(6))
    s = P.EnsembleSolver(mesh.xy, mesh.tri, [0.01, 0.02], [0.01, 0.03], 0.5, 0.01, bind=False, **kw)
    sv = kw.get("element") == "SV"
    S = P2Space(mesh, pressure="P1disc" if sv else "P1")
    assert s.options.element == (1 if sv else 0)
    assert s.options.schur == kw.get("schur", 0 if sv else 1)
    assert s.options.amg_sweeps == (2 if sv else 1)
    assert s.sizes.np == S.np_ == (3 * mesh.nt if sv else mesh.nv)
    Bx, _ = S.divergence()
    Bpat = Bx.copy()
    Bpat.data[:] = 1.0
    assert s.sizes.nnz_B == Bpat.nnz
    assert s.sizes.n_rows == 2 * S.n2 + S.np_
    assert s.sizes.amg_levels >= (2 if sv else 1)      # 648 / 121 pressure dofs, coarsest <= 512
    s.close()


def _pinned(L):
    L = sp.lil_matrix(L)
    L[0, :] = 0.0
    L[:, 0] = 0.0
    L[0, 0] = 1.0
    return sp.csr_matrix(L)


@pytest.mark.parametrize("kw,bary", [(dict(element="SV"), True), (dict(element="SV"), False),
                                     (dict(schur=2), True), (dict(), True)])
def test_pressure_laplacian_matches_oracle_matrices(kw, bary):
    """The library's finest pressure operator (host-built) against one formed
    here from the oracle's matrices: the P1 stiffness of the continuous
    pressure from the oracle's barycentric gradients, or B D^{-1} B^T with
    the oracle's divergence blocks B_x, B_y and D = (30/19) diag(M) on the
    interior P2 nodes (the P2 mass diagonal, area/30 at vertices and
    8 area/45 at edge midpoints, scaled to sum to the area); dof 0 pinned.
    Also the smoother's block size: 9 on barycenter-refined meshes with the
    discontinuous pressure, 3 on other meshes, 0 (point Jacobi) otherwise."""
    # more than 512 pressure dofs in the discontinuous case (648 and 600), so
    # that the finest level is not already the dense coarsest one
    mesh = barycentric_refine(unit_square(6)) if bary else unit_square(10)
    s = P.EnsembleSolver(mesh.xy, mesh.tri, [0.01, 0.02], [0.01, 0.03], 0.5, 0.01, bind=False, **kw)
    sv = kw.get("element") == "SV"
    S = P2Space(mesh, pressure="P1disc" if sv else "P1")
    rp, col, val = s.probe_laplacian()
    L = sp.csr_matrix((val, col, rp), shape=(S.np_, S.np_))
    if sv or kw.get("schur") == 2:
        Bx, By = S.divergence()
        d = S.mass().diagonal() * (30.0 / 19.0)
        dinv = sp.diags(np.where(S.is_boundary, 0.0, 1.0 / d))
        ref = _pinned(Bx @ dinv @ Bx.T + By @ dinv @ By.T)
    else:
        g = S.grad_lambda                                   # [nt, 3, 2]
        loc = S.area[:, None, None] * np.einsum("tid,tkd->tik", g, g)
        ref = _pinned(S._assemble(loc, S.pdofs, S.pdofs, S.np_, S.np_))
    diff = abs(L - ref).max()
    assert diff <= 1e-12 * abs(ref).max(), diff
    want_block = (9 if bary else 3) if sv else 0
    assert s.sizes.smoother_block == want_block
    s.close()


def test_calls_before_bind_fail_cleanly():
    ens = lid_cavity(N=4, J=2, nsteps=1)
    s = ensemble_io.solver_for(ens, bind=False)
    with pytest.raises(P.MhdeError) as e:
        s.step()
    assert e.value.code == -7
    with pytest.raises(P.MhdeError):
        s.set_initial(np.zeros((2, s.n2, 2)))
    s.close()


def test_workspace_grows_with_members_and_precision():
    m = unit_square(8)
    sizes = {}
    for J in (2, 8):
        for prec in (0, 1):
            s = P.EnsembleSolver(m.xy, m.tri, np.full(J, 0.01), np.full(J, 0.01), 1.0, 0.01, bind=False,
                                 precision=prec)
            sizes[(J, prec)] = s.workspace_size()
            s.close()
    assert sizes[(8, 1)] > sizes[(2, 1)]
    assert sizes[(8, 0)] > sizes[(8, 1)]


def test_channel_mesh_builds_hierarchy():
    ens = channel(J=2, nsteps=1, cells_per_unit=3)
    s = ensemble_io.solver_for(ens, bind=False)
    assert s.sizes.amg_levels >= 2
    s.close()


def test_block_gram_entry_points_reject_more_blocks_than_grid_rows():
    """Both Gram entry points launch one grid row per basis block, so more
    than 65535 blocks is an argument error, caught before any device work
    (the pointers below are never dereferenced)."""
    import ctypes as C
    lib = P.load_library()
    fake = C.c_void_p(256)
    nbytes = C.c_size_t()
    assert lib.mhde_block_gram_scratch_bytes(100, 1, 65536, C.byref(nbytes)) == -1
    assert lib.mhde_block_gram(fake, 400, 65536, fake, 100, 4, 1, fake, fake, 1 << 30, None) == -1
    assert lib.mhde_block_gram_noalloc(fake, 400, 65536, fake, 100, 4, 1, fake, None) == -1


def test_concurrent_host_builds_are_identical():
    """mhde_create from many threads at once (ctypes releases the GIL): the
    host-built structures (numbering, patterns, the pressure-Laplacian
    hierarchy and its smoother blocks) come out identical to a serial build,
    for both elements."""
    from concurrent.futures import ThreadPoolExecutor
    meshes = [(barycentric_refine(unit_square(6)), dict(element="SV")), (unit_square(12), dict()),
              (channel_step(cells_per_unit=2), dict(schur=2))]

    def build(i):
        mesh, kw = meshes[i % len(meshes)]
        s = P.EnsembleSolver(mesh.xy, mesh.tri, [0.01, 0.02], [0.01, 0.03], 0.5, 0.01, bind=False, **kw)
        sz = s.sizes
        out = (i % len(meshes), sz.n2, sz.np, sz.nnz_F, sz.nnz_B, sz.amg_levels, sz.nnz_L, sz.smoother_block,
               s.probe_laplacian()[2].tobytes(), s.p2_nodes()[0].tobytes())
        s.close()
        return out

    serial = {r[0]: r for r in map(build, range(len(meshes)))}
    with ThreadPoolExecutor(max_workers=12) as ex:
        results = list(ex.map(build, range(48)))
    for r in results:
        assert r == serial[r[0]]


def _vcycle(levels, cinv, l, b, nsw):
    """The library's V-cycle on the probed hierarchy: nsw smoothing sweeps
    from zero (block Jacobi where the level has blocks, else damped point
    Jacobi), restriction of the residual, the next level, prolongation, nsw
    sweeps; a dense inverse on the coarsest level."""
    L = levels[l]
    if l == len(levels) - 1:
        return cinv @ b
    A = L["A"]
    if L["bs"]:
        bs, idx, Bi, om = L["bs"], L["blk_idx"], L["blk_inv"], L["blk_omega"]

        def sm(r):
            out = np.zeros_like(r)
            out[idx] = np.einsum("bij,bj->bi", Bi, r[idx].reshape(-1, bs)).ravel()
            return om * out
    else:
        d = A.diagonal()
        dinv = np.where(d != 0, 1.0 / np.where(d != 0, d, 1.0), 0.0)
        om = L["omega"]

        def sm(r):
            return om * dinv * r
    x = sm(b)
    for _ in range(nsw - 1):
        x = x + sm(b - A @ x)
    x = x + L["P"] @ _vcycle(levels, cinv, l + 1, L["R"] @ (b - A @ x), nsw)
    for _ in range(nsw):
        x = x + sm(b - A @ x)
    return x


@pytest.mark.parametrize("mesh,kw,max_its", [
    (barycentric_refine(unit_square(24)), dict(element="SV"), 20),     # 13 measured
    (barycentric_refine(unit_square(48)), dict(element="SV"), 20),     # 13
    (unit_square(64), dict(), 20),                                     # 14 (Taylor-Hood P1 stiffness)
    (barycentric_refine(unit_square(48)), dict(), 20),                 # 12 (40 with aggregation alone)
    (barycentric_refine(channel_step(cells_per_unit=2)), dict(schur=2), 20),
])
def test_pressure_hierarchy_preconditions_its_laplacian(mesh, kw, max_its):
    """The host-built hierarchy (probed level by level), cycled as the device
    does, is an effective preconditioner for its own finest operator:
    preconditioned CG reaches 1e-8 in a mesh-independent number of steps.
    For the discontinuous pressure the first coarse space is the continuous
    P1 space on the vertices (P injects vertex values into the three dofs of
    every triangle, R = P^T), and the finest smoother works on 9-dof macro
    triangles.  For the continuous pressure on a barycenter refinement the
    first coarse space is P1 on the parent mesh (a barycenter takes the mean
    of its triangle's vertices)."""
    import scipy.sparse.linalg as sla
    s = P.EnsembleSolver(mesh.xy, mesh.tri, [0.01, 0.02], [0.01, 0.03], 0.5, 0.01, bind=False, **kw)
    levels = [s.probe_amg_level(l) for l in range(s.sizes.amg_levels)]
    assert levels[0]["levels"] == len(levels) >= 3
    if kw.get("element") == "SV":
        P0 = levels[0]["P"]
        assert levels[0]["bs"] == 9 and P0.shape == (3 * mesh.nt, mesh.nv)
        want = sp.csr_matrix((np.ones(3 * mesh.nt - 1), (np.arange(1, 3 * mesh.nt), mesh.tri.ravel()[1:])),
                             shape=P0.shape)
        assert abs(P0 - want).max() == 0.0
        assert abs(levels[0]["R"] - P0.T).max() == 0.0
    elif mesh.nt % 3 == 0 and levels[0]["A"].shape[0] == mesh.nv and mesh.nv > 4000:
        # barycenter refinement: the parent's vertices are the coarse dofs
        nparent = mesh.nv - mesh.nt // 3
        P0 = levels[0]["P"]
        assert P0.shape == (mesh.nv, nparent)
        rows = np.diff(P0.indptr)
        assert rows[0] == 0 and set(rows[1:].tolist()) <= {1, 3}
        assert np.allclose(np.asarray(P0.sum(axis=1)).ravel()[1:], 1.0)
    cinv = np.linalg.inv(levels[-1]["A"].toarray())
    A = levels[0]["A"]
    b = np.random.default_rng(1).standard_normal(A.shape[0])
    its = [0]
    M = sla.LinearOperator(A.shape, lambda r: _vcycle(levels, cinv, 0, r, s.options.amg_sweeps))
    x, info = sla.cg(A, b, M=M, rtol=1e-8, maxiter=200, callback=lambda xk: its.__setitem__(0, its[0] + 1))
    assert info == 0 and np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b) * 1.01
    assert its[0] <= max_its, its[0]
    s.close()
