"""Parity at the benchmark's full size: lid-driven-cavity-shaped ensemble on
the 128x128 mesh with J = 20 (n = 148,739 saddle rows), in the launch
configuration bench.py times, with the library's default tolerances.  The
oracle computes five whole steps (one SuperLU factorisation per subproblem
and step, shared by all members), so every member and every node is
compared after the first and the fifth step (errors accumulate over steps);
properties that hold at any size (discrete divergence, Dirichlet values) are
checked on the GPU result as well."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2108_05110_gb300 import ensemble_io, PREC_FP64, PREC_MIXED  # noqa: E402
from oracle.scheme import OracleRun  # noqa: E402
from workloads.ensembles import lid_cavity  # noqa: E402
from tests._gpu_common import rel_l2, gpu_run  # noqa: E402

pytestmark = pytest.mark.gpu


STEPS = (1, 5)


@pytest.fixture(scope="module")
def full():
    ens = lid_cavity(N=128, J=20, s=1.0, dt=0.01, Re=15000.0)
    ref = OracleRun(ens)
    snaps = {}
    for n in range(1, STEPS[-1] + 1):
        ref.step()
        if n in STEPS:
            snaps[n] = (ref.V.copy(), ref.W.copy())
    return ens, ref, snaps


@pytest.mark.parametrize("precision,tol", [(PREC_MIXED, 1e-8), (PREC_FP64, 1e-10)])
def test_full_size_steps(full, precision, tol):
    ens, ref, snaps = full
    sol = gpu_run(ens, 1, precision=precision)
    for n in range(1, STEPS[-1] + 1):
        if n > 1:
            ensemble_io.run(sol, ens, 1, start_step=n - 1)
        if n in snaps:
            v, w, q, r = sol.read_state()
            V, W = snaps[n]
            assert rel_l2(v, V) <= tol and rel_l2(w, W) <= tol, (n, rel_l2(v, V), rel_l2(w, W))
    # any-size properties: discrete divergence and Dirichlet values
    for Z in (v, w):
        for j in (0, 7, 19):
            div = ref.Bx @ Z[j][:, 0] + ref.By @ Z[j][:, 1]
            assert np.abs(div[1:]).max() <= 1e-9 * np.abs(Z[j]).max()
    xy = ref.S.node_xy
    bnd = ref.S.boundary
    gv = ens.u_bc(xy, ens.dt) + np.sqrt(ens.s) * ens.B_bc(xy, ens.dt)
    assert np.abs(v[:, bnd] - gv[:, bnd]).max() <= 1e-12
    sol.close()
