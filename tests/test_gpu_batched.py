"""Batched uneven ensembles through mhde_advance_many: independent contexts of
different meshes and member counts, stepped concurrently from a pool of host
threads (each context on its own two streams), match the FP64 oracle run of
each ensemble alone, and match the same contexts stepped one after the other
bit for bit (no state is shared between contexts)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2108_05110_gb300 as P  # noqa: E402
from paper_2108_05110_gb300 import ensemble_io, PREC_FP64, PREC_MIXED  # noqa: E402
from workloads.ensembles import lid_cavity  # noqa: E402
from tests._gpu_common import rel_l2, oracle_run  # noqa: E402

pytestmark = pytest.mark.gpu

NSTEPS = 3


def _family():
    """Uneven sizes: (N, J, Re, s) with a single-member ensemble and an
    ensemble with J not a multiple of 4 (padded rows)."""
    spec = [(8, 2, 1000.0, 1.0), (12, 5, 5000.0, 0.5), (16, 1, 3000.0, 1.0), (10, 7, 15000.0, 0.1)]
    return [lid_cavity(N=N, J=J, Re=Re, s=s, dt=0.01, nsteps=NSTEPS, seed=700 + k)
            for k, (N, J, Re, s) in enumerate(spec)]


def _solvers(fam, precision):
    out = []
    for ens in fam:
        sol = ensemble_io.solver_for(ens, precision=precision)
        ensemble_io.feed_initial(sol, ens)
        ensemble_io.feed_step_data(sol, ens, ens.dt)
        out.append(sol)
    return out


@pytest.fixture(scope="module")
def references():
    fam = _family()
    return fam, [oracle_run(ens, NSTEPS) for ens in fam]


@pytest.mark.parametrize("precision,tol", [(PREC_MIXED, 1e-8), (PREC_FP64, 1e-10)])
def test_advance_many_matches_oracle_and_sequential(references, precision, tol):
    fam, refs = references
    many = _solvers(fam, precision)
    ms = P.advance_many(many, NSTEPS, nthreads=3)
    assert ms.shape == (len(fam), NSTEPS) and np.all(ms > 0)
    alone = _solvers(fam, precision)
    for sol in alone:
        sol.advance(NSTEPS)
    for sol, one, ref in zip(many, alone, refs):
        v, w, _, _ = sol.read_state()
        assert rel_l2(v, ref.V) <= tol and rel_l2(w, ref.W) <= tol, (sol.J, rel_l2(v, ref.V), rel_l2(w, ref.W))
        v1, w1, _, _ = one.read_state()
        assert np.array_equal(v, v1) and np.array_equal(w, w1)
        assert sol.stats().steps == NSTEPS
    for sol in many + alone:
        sol.close()
