"""Accuracy of the mixed and FP64 paths over many steps: the cavity-shaped
ensemble at Re = 15000 on a 32x32 mesh (J = 8) for 100 steps, compared with
the FP64 oracle at every 25th step (errors accumulate over the run, so this
is the check behind the metric's rel L2 <= 1e-8 gate)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2108_05110_gb300 import ensemble_io, PREC_FP64, PREC_MIXED  # noqa: E402
from oracle.scheme import OracleRun  # noqa: E402
from workloads.ensembles import lid_cavity  # noqa: E402
from tests._gpu_common import rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu

NSTEPS = 100


@pytest.fixture(scope="module")
def reference():
    ens = lid_cavity(N=32, J=8, s=1.0, dt=0.01, Re=15000.0, nsteps=NSTEPS)
    ref = OracleRun(ens)
    snaps = {}
    for n in range(1, NSTEPS + 1):
        ref.step()
        if n % 25 == 0:
            snaps[n] = (ref.V.copy(), ref.W.copy())
    return ens, snaps


@pytest.mark.parametrize("precision,tol", [(PREC_MIXED, 1e-8), (PREC_FP64, 1e-10)])
def test_hundred_steps_with_default_tolerances(reference, precision, tol):
    # per-step solver residuals accumulate over the run; the library's
    # default rtol for each precision (1e-12 mixed, 1e-13 FP64) must keep
    # the gate over all 100 steps
    ens, snaps = reference
    sol = ensemble_io.solver_for(ens, precision=precision)
    ensemble_io.feed_initial(sol, ens)
    ensemble_io.feed_step_data(sol, ens, ens.dt)
    for n in range(1, NSTEPS + 1):
        sol.step()
        if n in snaps:
            v, w, _, _ = sol.read_state()
            V, W = snaps[n]
            assert rel_l2(v, V) <= tol and rel_l2(w, W) <= tol, (n, rel_l2(v, V), rel_l2(w, W))
    sol.close()
