"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Kernel level: ensemble mean and mixing-length field, the shared matrix F,
the batched right-hand sides and the saddle SpMM are compared element by
element.  Step level: whole time steps of Algorithm 1 on the FP64 path
(rel L2 <= 1e-10) and the mixed path (rel L2 <= 1e-8), on manufactured,
cavity- and channel-shaped ensembles that span several tiles and ragged
member counts (J = 1, 3, 5, 20), plus the patch and identical-member cases.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2108_05110_gb300 import ensemble_io, PREC_FP64, PREC_MIXED  # noqa: E402
from oracle.scheme import OracleRun, ensemble_mean, mixing_length_sq  # noqa: E402
from workloads.ensembles import manufactured, lid_cavity, channel, config_manufactured_small  # noqa: E402
from workloads.mesh import unit_square, channel_step  # noqa: E402
from tests._gpu_common import rel_l2, gpu_run, oracle_run  # noqa: E402
from tests.test_oracle_scheme import patch_ensemble  # noqa: E402

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-8


def _perturbed_manufactured(N=8, J=5):
    nu = np.linspace(0.009, 0.011, J)
    nu_m = np.linspace(0.02, 0.006, J)
    c = 1.0 + np.linspace(-0.15, 0.2, J)
    return manufactured(N, J, nu, nu_m, c, dt=0.02, nsteps=3, s=0.7)


@pytest.fixture(scope="module")
def pair():
    ens = _perturbed_manufactured()
    sol = ensemble_io.solver_for(ens, precision=PREC_FP64)
    ensemble_io.feed_initial(sol, ens)
    ensemble_io.feed_step_data(sol, ens, ens.dt)
    ref = OracleRun(ens)
    return ens, sol, ref


def test_mean_and_mixing_length(pair):
    ens, sol, ref = pair
    mv, mw, lv, lw = sol.probe_mean_l2()
    omv, omw = ensemble_mean(ref.V), ensemble_mean(ref.W)
    assert np.abs(mv - omv).max() <= 1e-14 * np.abs(omv).max()
    assert np.abs(mw - omw).max() <= 1e-14 * np.abs(omw).max()
    olv = mixing_length_sq(ref.S, ref.V - omv)
    olw = mixing_length_sq(ref.S, ref.W - omw)
    assert olv.max() > 1e-3                       # fluctuations are visible
    assert np.abs(lv - olv).max() <= 1e-13 * olv.max()
    assert np.abs(lw - olw).max() <= 1e-13 * olw.max()


@pytest.mark.parametrize("which", [0, 1])
def test_shared_matrix(pair, which):
    ens, sol, ref = pair
    rp, col, val = sol.probe_matrix_F(which)
    import scipy.sparse as sp
    F = sp.csr_matrix((val, col, rp), shape=(sol.n2, sol.n2)).toarray()
    mv, mw = ensemble_mean(ref.V), ensemble_mean(ref.W)
    if which == 0:
        Fo = ref.shared_matrix(mw, mixing_length_sq(ref.S, ref.W - mw)).toarray()
    else:
        Fo = ref.shared_matrix(mv, mixing_length_sq(ref.S, ref.V - mv)).toarray()
    bnd = ref.S.is_boundary
    Fo[bnd] = 0.0
    Fo[bnd, bnd] = 1.0
    assert np.abs(F - Fo).max() <= 1e-13 * np.abs(Fo).max()


@pytest.mark.parametrize("which", [0, 1])
def test_right_hand_sides(pair, which):
    ens, sol, ref = pair
    rhs = sol.probe_rhs(which)
    t1 = ens.dt
    f1, f2, gv, gw = ref.member_data(t1)
    mv, mw = ensemble_mean(ref.V), ensemble_mean(ref.W)
    cross = ref.nu - ref.nu_m
    same = ref.nu_p + ref.nu_m_p
    n2 = ref.S.n2
    for j in range(ens.J):
        if which == 0:
            b = ref.rhs(ref.V, ref.W, ref.W - mw, f1, gv, j, same, cross)
        else:
            b = ref.rhs(ref.W, ref.V, ref.V - mv, f2, gw, j, same, cross)
        bo = np.stack([b[:n2], b[n2:2 * n2]], axis=1)
        assert np.abs(rhs[j] - bo).max() <= 1e-12 * np.abs(bo).max()


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (1, 2e-6)])
def test_saddle_spmm(pair, which, precision, tol):
    """The SpMM kernel against A X formed on the CPU from the GPU's own F
    (probed) and the oracle's constant B, B^T, Dirichlet and pin rows."""
    import scipy.sparse as sp
    ens, sol, ref = pair
    rp, col, val = sol.probe_matrix_F(which)
    Fg = sp.csr_matrix((val, col, rp), shape=(sol.n2, sol.n2))
    A = ref.saddle(Fg)
    rng = np.random.default_rng(11)
    X = rng.standard_normal((ens.J, A.shape[0]))
    Y = sol.probe_spmm(which, X, precision)
    Yo = (A @ X.T).T
    scale = (abs(A) @ np.abs(X.T)).T
    assert np.all(np.abs(Y - Yo) <= tol * scale)


@pytest.mark.parametrize("precision,tol", [(PREC_FP64, FP64_TOL), (PREC_MIXED, MIXED_TOL)])
def test_manufactured_16x16_ten_steps(precision, tol):
    ens = config_manufactured_small()
    ref = oracle_run(ens, ens.nsteps)
    sol = gpu_run(ens, ens.nsteps, precision=precision)
    v, w, q, r = sol.read_state()
    assert rel_l2(v, ref.V) <= tol and rel_l2(w, ref.W) <= tol
    st = sol.stats()
    assert st.steps == ens.nsteps and max(st.last_relres) <= 1e-12
    # pressures (mean zero) agree to the conditioning of the pressure block
    assert rel_l2(q, ref.zero_mean(ref.Q)) <= 1e3 * tol
    sol.close()


@pytest.mark.parametrize("s", [0.01, 1.0])
@pytest.mark.parametrize("precision,tol", [(PREC_FP64, FP64_TOL), (PREC_MIXED, MIXED_TOL)])
def test_lid_cavity_small(s, precision, tol):
    ens = lid_cavity(N=16, J=5, s=s, nsteps=4, Re=2000.0)
    ref = oracle_run(ens, 4)
    sol = gpu_run(ens, 4, precision=precision)
    v, w, _, _ = sol.read_state()
    assert rel_l2(v, ref.V) <= tol and rel_l2(w, ref.W) <= tol
    u, B = sol.read_mean()
    ou, oB = ref.primitive_mean()
    assert rel_l2(u, ou) <= 10 * tol and rel_l2(B, oB) <= 10 * tol / np.sqrt(s)
    assert abs(sol.energy() - ref.energy()) <= 1e-9 * ref.energy()
    sol.close()


def test_channel_small_mixed():
    ens = channel(J=3, nsteps=3, cells_per_unit=2, dt=0.05)
    ref = oracle_run(ens, 3)
    sol = gpu_run(ens, 3, precision=PREC_MIXED)
    v, w, _, _ = sol.read_state()
    assert rel_l2(v, ref.V) <= MIXED_TOL and rel_l2(w, ref.W) <= MIXED_TOL
    sol.close()


@pytest.mark.parametrize("amg_sweeps,amg_cycles", [(2, 1), (3, 2)])
def test_vcycle_sweep_counts(amg_sweeps, amg_cycles):
    """Even and odd smoothing-sweep counts and repeated V-cycles: each level's
    prolongation targets the buffer from which the post-smoothing sweeps end
    in the level's output, for either parity; the fields still reach the
    oracle's to the mixed tolerance."""
    ens = lid_cavity(N=16, J=5, s=1.0, nsteps=3, Re=2000.0)
    ref = oracle_run(ens, 3)
    sol = gpu_run(ens, 3, precision=PREC_MIXED, amg_sweeps=amg_sweeps, amg_cycles=amg_cycles)
    v, w, _, _ = sol.read_state()
    assert rel_l2(v, ref.V) <= MIXED_TOL and rel_l2(w, ref.W) <= MIXED_TOL
    assert max(sol.stats().last_relres) <= 1e-12
    sol.close()


@pytest.mark.parametrize("inner_fp16", [0, 1])
def test_inner_basis_storage(inner_fp16):
    """The mixed path with the inner GMRES basis in FP32 and in FP16: the
    basis only shapes the preconditioner, so both reach the oracle's fields to
    the mixed tolerance (the FP64 refinement sets the accuracy)."""
    ens = lid_cavity(N=16, J=5, s=1.0, nsteps=4, Re=2000.0)
    ref = oracle_run(ens, 4)
    sol = gpu_run(ens, 4, precision=PREC_MIXED, inner_fp16=inner_fp16)
    v, w, _, _ = sol.read_state()
    assert rel_l2(v, ref.V) <= MIXED_TOL and rel_l2(w, ref.W) <= MIXED_TOL
    assert max(sol.stats().last_relres) <= 1e-12
    sol.close()


def test_single_member_and_standard_form():
    ens = lid_cavity(N=8, J=1, s=0.3, nsteps=3, Re=500.0)
    ref = oracle_run(ens, 3, form="standard")
    sol = gpu_run(ens, 3, precision=PREC_FP64, conv_form=1)
    v, w, _, _ = sol.read_state()
    assert rel_l2(v, ref.V) <= FP64_TOL and rel_l2(w, ref.W) <= FP64_TOL
    sol.close()


@pytest.mark.parametrize("precision", [PREC_FP64, PREC_MIXED])
def test_patch_solution_exact_on_gpu(precision):
    # dt = 0.02 keeps the cell CFL number of the w-problem (convected by
    # <v> = (1+t)(y, x), |<v>| up to 44 on this channel) below about 1
    ens, vf, wf = patch_ensemble(channel_step(cells_per_unit=1), dt=0.02)
    sol = gpu_run(ens, ens.nsteps, precision=precision)
    xy, _ = sol.p2_nodes()
    v, w, _, _ = sol.read_state()
    t = ens.nsteps * ens.dt
    assert np.abs(v - vf(xy, t)[None]).max() <= 1e-9 * np.abs(vf(xy, t)).max()
    assert np.abs(w - wf(xy, t)[None]).max() <= 1e-9
    sol.close()


def test_identical_members_match_single_member():
    base = lid_cavity(N=8, J=1, s=0.5, nsteps=3, Re=200.0)
    one = gpu_run(base, 3, precision=PREC_FP64)
    from tests.test_oracle_scheme import _replicate
    many = gpu_run(_replicate(base, 4), 3, precision=PREC_FP64)
    v1, w1, _, _ = one.read_state()
    v4, w4, _, _ = many.read_state()
    for j in range(4):
        assert rel_l2(v4[j], v1[0]) <= 1e-11 and rel_l2(w4[j], w1[0]) <= 1e-11
    one.close()
    many.close()


def test_resume_is_bit_exact_and_runs_are_deterministic():
    ens = lid_cavity(N=12, J=3, s=0.5, nsteps=4, Re=1000.0)
    a = gpu_run(ens, 2)
    snap = a.save_state()
    ensemble_io.run(a, ens, 2, start_step=2)
    va, wa, _, _ = a.read_state()
    b = gpu_run(ens, 4)
    vb, wb, _, _ = b.read_state()
    assert np.array_equal(va, vb) and np.array_equal(wa, wb)
    b.load_state(snap)
    ensemble_io.run(b, ens, 2, start_step=2)
    vc, wc, _, _ = b.read_state()
    assert np.array_equal(va, vc) and np.array_equal(wa, wc)
    a.close()
    b.close()


def test_iteration_cap_reports_noconv_and_keeps_state():
    ens = lid_cavity(N=8, J=2, s=0.5, nsteps=1, Re=1000.0)
    sol = ensemble_io.solver_for(ens, max_iter=1, max_refine=1)
    ensemble_io.feed_initial(sol, ens)
    before = sol.read_state()[0].copy()
    ensemble_io.feed_step_data(sol, ens, ens.dt)
    import paper_2108_05110_gb300 as P
    with pytest.raises(P.MhdeError) as e:
        sol.step()
    assert e.value.code == -3
    assert np.array_equal(sol.read_state()[0], before)
    sol.close()


@pytest.mark.parametrize("n_rows,ld,r,k", [(1000, 4, 3, 1), (148739, 20, 20, 5), (5003, 64, 61, 3)])
def test_block_gram_entry_point(n_rows, ld, r, k):
    """mhde_block_gram against the FP64 definition V_i^T W (numpy)."""
    import paper_2108_05110_gb300 as P
    rng = np.random.default_rng(n_rows)
    V = rng.standard_normal((k, n_rows, ld))
    W = rng.standard_normal((n_rows, ld))
    G = P.block_gram(torch.from_numpy(V).cuda(), torch.from_numpy(W).cuda(), k, r).cpu().numpy()
    torch.cuda.synchronize()
    for i in range(k):
        ref = V[i][:, :r].T @ W[:, :r]
        scale = np.abs(V[i][:, :r]).T @ np.abs(W[:, :r])
        assert np.all(np.abs(G[i] - ref) <= 1e-13 * scale)
