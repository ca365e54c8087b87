"""The mixed path's inner solve of the velocity block (per-column GMRES(k) on
F D^{-1}, the approximate F^{-1} inside the block-triangular preconditioner)
in both of its forms: the chain of per-phase launches and the persistent
kernel (one cooperative launch whose CTAs meet at bounded grid barriers).

* Both forms against the GMRES(k) iterate computed in FP64 from the
  context's own F (probed through the C ABI) on random right-hand sides.
* Both forms, forced through MHDE_INNER_GRID at bind, reach the metric's
  1e-8 gate against the FP64 oracle after several steps on small cavity
  ensembles with member counts that exercise the column padding (J = 1, 5,
  7) and inner step counts 1, 3, 6 and 10 (both kernel instantiations), and
  at the benchmark's full size for one step; the persistent form is
  deterministic run to run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2108_05110_gb300 import PREC_MIXED  # noqa: E402
from workloads.ensembles import lid_cavity  # noqa: E402
from tests._gpu_common import rel_l2, gpu_run, oracle_run  # noqa: E402

pytestmark = pytest.mark.gpu

NSTEPS = 4


def _run_form(monkeypatch, ens, nsteps, form, **opts):
    monkeypatch.setenv("MHDE_INNER_GRID", form)
    sol = gpu_run(ens, nsteps, precision=PREC_MIXED, **opts)
    monkeypatch.delenv("MHDE_INNER_GRID")
    return sol


def _gmres_reference(F, r, k):
    """Per-column GMRES(k) on F D^{-1} from a zero start, FP64 (the
    definition both device forms compute): z = D^{-1} V_k y with y the
    minimiser of || ||r|| e_1 - H y ||."""
    import scipy.sparse as sp
    d = F.diagonal()
    A = F @ sp.diags(1.0 / d)
    beta = np.linalg.norm(r)
    if beta == 0.0:
        return np.zeros_like(r)
    V = np.zeros((r.size, k + 1))
    H = np.zeros((k + 1, k))
    V[:, 0] = r / beta
    for i in range(k):
        w = A @ V[:, i]
        for l in range(i + 1):
            H[l, i] = V[:, l] @ w
            w = w - H[l, i] * V[:, l]
        H[i + 1, i] = np.linalg.norm(w)
        if H[i + 1, i] > 0:
            V[:, i + 1] = w / H[i + 1, i]
    e1 = np.zeros(k + 1)
    e1[0] = beta
    y = np.linalg.lstsq(H, e1, rcond=None)[0]
    return (V[:, :k] @ y) / d


@pytest.mark.parametrize("J,kin", [(5, 6), (7, 3), (2, 10)])
def test_inner_solve_forms_match_gmres_definition(monkeypatch, J, kin):
    """Both FP32 forms agree with the FP64 definition, and with each other, to
    FP32 rounding of a k-step Krylov recurrence."""
    import scipy.sparse as sp
    ens = lid_cavity(N=24, J=J, s=1.0, dt=0.01, Re=5000.0, seed=90 + J)
    monkeypatch.setenv("MHDE_INNER_GRID", "1")
    sol = gpu_run(ens, 2, precision=PREC_MIXED, inner_iters=kin)
    monkeypatch.delenv("MHDE_INNER_GRID")
    n2 = sol.sizes.n2
    rng = np.random.default_rng(5 + J)
    R = rng.standard_normal((J, 2, n2))
    for which in (0, 1):
        rp, col, val = sol.probe_matrix_F(which)
        F = sp.csr_matrix((val, col, rp), shape=(n2, n2))
        Zc = sol.probe_inner(which, R, form=0)
        Zp = sol.probe_inner(which, R, form=1)
        for j in range(J):
            for d in range(2):
                ref = _gmres_reference(F, R[j, d], kin)
                ec = rel_l2(Zc[j, d], ref)
                ep = rel_l2(Zp[j, d], ref)
                assert ec <= 2e-5 and ep <= 2e-5, (which, j, d, ec, ep)
        assert rel_l2(Zp, Zc) <= 2e-5
    sol.close()


@pytest.mark.parametrize("J,kin", [(5, 6), (7, 3), (1, 6), (5, 1), (5, 10)])
def test_persistent_inner_matches_oracle_and_chain(monkeypatch, J, kin):
    ens = lid_cavity(N=16, J=J, s=1.0, dt=0.01, Re=5000.0, seed=40 + J + kin)
    ref = oracle_run(ens, NSTEPS)
    out = {}
    for form in ("1", "0"):
        sol = _run_form(monkeypatch, ens, NSTEPS, form, inner_iters=kin)
        st = sol.stats()
        assert st.inner_persistent == (1 if form == "1" else 0)
        v, w, _, _ = sol.read_state()
        assert rel_l2(v, ref.V) <= 1e-8 and rel_l2(w, ref.W) <= 1e-8, (form, rel_l2(v, ref.V), rel_l2(w, ref.W))
        out[form] = (v, w, st.total_iters)
        sol.close()
    # same method and step count: the two forms differ by FP32 rounding in the
    # preconditioner only, so the FP64-refined states agree far below the gate
    assert rel_l2(out["1"][0], out["0"][0]) <= 1e-9
    # and the outer iteration counts stay comparable (on these small meshes
    # the flexible outer iteration reacts to the rounding of its
    # preconditioner by up to ~20 %; at the benchmark's size the counts agree
    # within 1 %)
    assert abs(out["1"][2] - out["0"][2]) <= max(4, 0.3 * out["0"][2])


def test_persistent_inner_is_deterministic(monkeypatch):
    ens = lid_cavity(N=16, J=5, s=1.0, dt=0.01, Re=5000.0, seed=77)
    a = _run_form(monkeypatch, ens, 3, "1")
    b = _run_form(monkeypatch, ens, 3, "1")
    va, wa, _, _ = a.read_state()
    vb, wb, _, _ = b.read_state()
    assert np.array_equal(va, vb) and np.array_equal(wa, wb)
    a.close()
    b.close()


def test_persistent_inner_full_size(monkeypatch):
    """The benchmark's configuration (128x128 cavity, J = 20), first step,
    every member and node against the oracle."""
    ens = lid_cavity(N=128, J=20, s=1.0, dt=0.01, Re=15000.0)
    ref = oracle_run(ens, 1)
    sol = _run_form(monkeypatch, ens, 1, "1")
    assert sol.stats().inner_persistent == 1
    v, w, _, _ = sol.read_state()
    assert rel_l2(v, ref.V) <= 1e-8 and rel_l2(w, ref.W) <= 1e-8, (rel_l2(v, ref.V), rel_l2(w, ref.W))
    sol.close()
