"""Launch-shape invariance of the CUDA path: programmatic dependent launch
(MHDE_PDL) and the CTA shape of the staged block combination (MHDE_COMB)
change only scheduling, never arithmetic order (every reduction has a fixed
order and a combination row is summed the same way by any CTA), so the
fields after several mixed-precision steps must be bit-identical.  Both
settings are read once per process, so each run is its own process."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RUN = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
from paper_2108_05110_gb300 import ensemble_io, PREC_MIXED
from workloads.ensembles import lid_cavity
ens = lid_cavity(N=24, J=7, s=1.0, nsteps=3, Re=3000.0)
sol = ensemble_io.solver_for(ens, precision=PREC_MIXED)
ensemble_io.feed_initial(sol, ens)
ensemble_io.run(sol, ens, 3)
v, w, q, r = sol.read_state()
np.savez({out!r}, v=v, w=w, q=q, r=r, iters=np.array(sol.stats().last_iters[:]))
sol.close()
"""


def _run(tmp_path, name, env_extra):
    out = str(tmp_path / f"{name}.npz")
    env = dict(os.environ)
    env.update(env_extra)
    subprocess.run([sys.executable, "-c", _RUN.format(root=ROOT, out=out)], env=env, check=True, timeout=600)
    return np.load(out)


def test_results_do_not_depend_on_pdl_or_combine_shape(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    base = _run(tmp_path, "base", {})
    for name, extra in [("nopdl", {"MHDE_PDL": "0"}), ("comb1", {"MHDE_COMB": "1"}),
                        ("comb2", {"MHDE_COMB": "2"}), ("comb3", {"MHDE_COMB": "3"})]:
        other = _run(tmp_path, name, extra)
        for key in ("v", "w", "q", "r", "iters"):
            assert np.array_equal(base[key], other[key]), (name, key, json.dumps(extra))
