"""The Scott-Vogelius element (P2 velocity, discontinuous P1 pressure, on
barycenter-refined meshes; Section 2 and Section 4) on the CUDA path, and
the least-squares-commutator Schur approximation on both elements, against
the FP64 oracle:

* the saddle SpMM with three pressure dofs per triangle, element by element
  against the oracle's Scott-Vogelius saddle matrix;
* whole steps on the FP64 (rel L2 <= 1e-10) and mixed (1e-8) paths with both
  Schur approximations the discontinuous pressure admits (least-squares
  commutator, Cahouet-Chabard), J = 1, 5, 7, cavity and channel meshes, and
  the pressures (mean zero);
* the GPU's velocities are divergence-free at every point;
* the patch solution (linear pressures) is reproduced;
* Taylor-Hood with the least-squares commutator against the Taylor-Hood
  oracle;
* the benchmark's Scott-Vogelius cavity (64 x 64 refined, J = 20), first
  step, sampled members against the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2108_05110_gb300 import ensemble_io, PREC_FP64, PREC_MIXED  # noqa: E402
from oracle.scheme import OracleRun  # noqa: E402
from workloads.ensembles import lid_cavity, channel  # noqa: E402
from workloads.mesh import channel_step, barycentric_refine  # noqa: E402
from tests._gpu_common import rel_l2, gpu_run, oracle_run, oracle_first_step_sampled  # noqa: E402
from tests.test_oracle_scheme import patch_ensemble  # noqa: E402

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-8


@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (1, 2e-6)])
def test_saddle_spmm_discontinuous_pressure(precision, tol):
    import scipy.sparse as sp
    ens = lid_cavity(N=8, J=5, s=1.0, dt=0.01, Re=1000.0, barycentric=True)
    sol = ensemble_io.solver_for(ens, precision=PREC_FP64, element="SV")
    ensemble_io.feed_initial(sol, ens)
    ensemble_io.feed_step_data(sol, ens, ens.dt)
    ref = OracleRun(ens, element="SV")
    assert sol.sizes.np == ref.S.np_ == 3 * ens.mesh.nt
    for which in (0, 1):
        rp, col, val = sol.probe_matrix_F(which)
        A = ref.saddle(sp.csr_matrix((val, col, rp), shape=(sol.n2, sol.n2)))
        X = np.random.default_rng(3 + which).standard_normal((ens.J, A.shape[0]))
        Y = sol.probe_spmm(which, X, precision)
        scale = (abs(A) @ np.abs(X.T)).T
        assert np.all(np.abs(Y - (A @ X.T).T) <= tol * scale)
    sol.close()


@pytest.mark.parametrize("schur", [2, 0])
@pytest.mark.parametrize("precision,tol", [(PREC_FP64, FP64_TOL), (PREC_MIXED, MIXED_TOL)])
@pytest.mark.parametrize("J", [1, 5, 7])
def test_sv_cavity_steps_match_oracle(schur, precision, tol, J):
    ens = lid_cavity(N=12, J=J, s=1.0, dt=0.01, Re=2000.0, nsteps=4, barycentric=True, seed=20 + J)
    ref = oracle_run(ens, 4, element="SV")
    sol = gpu_run(ens, 4, precision=precision, element="SV", schur=schur)
    v, w, q, r = sol.read_state()
    assert rel_l2(v, ref.V) <= tol and rel_l2(w, ref.W) <= tol, (rel_l2(v, ref.V), rel_l2(w, ref.W))
    assert rel_l2(q, ref.zero_mean(ref.Q)) <= 1e3 * tol and rel_l2(r, ref.zero_mean(ref.R)) <= 1e3 * tol
    # pointwise divergence-free (div P2 lies in P1disc): at the level of the
    # solver's residual, far below Taylor-Hood's O(1) on this mesh
    S = ref.S
    for Z in (v, w):
        for j in range(J):
            assert S.divergence_sq(Z[j]) <= 1e-16 * S.h1semi_sq(ref.K, Z[j])
    st = sol.stats()
    assert st.steps == 4 and max(st.last_relres) <= 1e-12
    sol.close()


def test_sv_channel_mixed():
    mesh = barycentric_refine(channel_step(cells_per_unit=2))
    ens = channel(J=3, nsteps=3, dt=0.05, mesh=mesh)
    ref = oracle_run(ens, 3, element="SV")
    sol = gpu_run(ens, 3, precision=PREC_MIXED, element="SV")
    v, w, _, _ = sol.read_state()
    assert rel_l2(v, ref.V) <= MIXED_TOL and rel_l2(w, ref.W) <= MIXED_TOL
    sol.close()


@pytest.mark.parametrize("precision", [PREC_FP64, PREC_MIXED])
def test_sv_patch_solution_exact_on_gpu(precision):
    ens, vf, wf = patch_ensemble(barycentric_refine(channel_step(cells_per_unit=1)), dt=0.02)
    sol = gpu_run(ens, ens.nsteps, precision=precision, element="SV")
    xy, _ = sol.p2_nodes()
    v, w, q, _ = sol.read_state()
    t = ens.nsteps * ens.dt
    assert np.abs(v - vf(xy, t)[None]).max() <= 1e-9 * np.abs(vf(xy, t)).max()
    assert np.abs(w - wf(xy, t)[None]).max() <= 1e-9
    # q = x - y at the three vertices of every triangle, shifted to mean zero
    pxy = ens.mesh.xy[ens.mesh.tri].reshape(-1, 2)
    ref = OracleRun(ens, element="SV")
    qe = ref.zero_mean((pxy[:, 0] - pxy[:, 1])[None])[0]
    assert np.abs(q - qe[None]).max() <= 1e-7
    sol.close()


@pytest.mark.parametrize("precision,tol", [(PREC_FP64, FP64_TOL), (PREC_MIXED, MIXED_TOL)])
def test_taylor_hood_least_squares_commutator(precision, tol):
    ens = lid_cavity(N=16, J=5, s=1.0, nsteps=4, Re=2000.0)
    ref = oracle_run(ens, 4)
    sol = gpu_run(ens, 4, precision=precision, schur=2)
    v, w, _, _ = sol.read_state()
    assert rel_l2(v, ref.V) <= tol and rel_l2(w, ref.W) <= tol
    sol.close()


def test_sv_cavity_full_size_first_step():
    """64 x 64 cavity refined at the barycenters (49,409 P2 nodes, 73,728
    pressure dofs), J = 20, mixed path: members 0, 7, 19 of the first step
    against the oracle, and the divergence of every member."""
    ens = lid_cavity(N=64, J=20, s=1.0, dt=0.01, Re=15000.0, barycentric=True)
    members = [0, 7, 19]
    ref, ov, ow = oracle_first_step_sampled(ens, members, element="SV")
    sol = gpu_run(ens, 1, precision=PREC_MIXED, element="SV")
    v, w, _, _ = sol.read_state()
    assert rel_l2(v[members], ov) <= MIXED_TOL and rel_l2(w[members], ow) <= MIXED_TOL
    S = ref.S
    worst = max(S.divergence_sq(Z[j]) / S.h1semi_sq(ref.K, Z[j]) for Z in (v, w) for j in range(20))
    assert worst <= 1e-16
    sol.close()
