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
