"""Parity on the channel-past-a-step-shaped workload at its full size
([0,40]x[0,10] minus the step [5,6]x[0,1], 280x70 graded jittered cells,
157,838 velocity DOFs, J = 50 members with inflows scaled by 1 + eps_j,
nu = nu_m = 1/600, s = 0.01, dt = 0.05) on the mixed path, with the
library's default tolerances.  The oracle factorises each shared matrix
once and solves sampled members (first, middle, last); any-size properties
(discrete divergence, Dirichlet values) are checked on every member."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2108_05110_gb300 import ensemble_io, PREC_MIXED  # noqa: E402
from workloads.ensembles import channel  # noqa: E402
from tests._gpu_common import rel_l2, gpu_run, oracle_first_step_sampled  # noqa: E402

pytestmark = pytest.mark.gpu

MEMBERS = (0, 17, 49)


def test_channel_full_size_first_step_mixed():
    ens = channel(J=50)
    ref, V, W = oracle_first_step_sampled(ens, MEMBERS)
    sol = gpu_run(ens, 1, precision=PREC_MIXED)
    v, w, _, _ = sol.read_state()
    sol.close()
    idx = list(MEMBERS)
    assert rel_l2(v[idx], V) <= 1e-8 and rel_l2(w[idx], W) <= 1e-8, (rel_l2(v[idx], V), rel_l2(w[idx], W))
    for Z in (v, w):
        div = np.stack([ref.Bx @ Z[j][:, 0] + ref.By @ Z[j][:, 1] for j in range(ens.J)])
        assert np.abs(div[:, 1:]).max() <= 1e-9 * np.abs(Z).max()
    xy, bnd = ref.S.node_xy, ref.S.boundary
    gv = ens.u_bc(xy, ens.dt) + np.sqrt(ens.s) * ens.B_bc(xy, ens.dt)
    assert np.abs(v[:, bnd] - gv[:, bnd]).max() <= 1e-12
