"""Helpers shared by the GPU parity tests (imported by tests only)."""
import numpy as np
import scipy.sparse as sp

from oracle.scheme import OracleRun, ensemble_mean, mixing_length_sq
from paper_2108_05110_gb300 import ensemble_io


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu_run(ens, nsteps, **opts):
    sol = ensemble_io.solver_for(ens, **opts)
    ensemble_io.feed_initial(sol, ens)
    ensemble_io.run(sol, ens, nsteps)
    return sol


def oracle_run(ens, nsteps, **kw):
    r = OracleRun(ens, **kw)
    for _ in range(nsteps):
        r.step()
    return r


def saddle_from_probe(rp, col, val, n2):
    return sp.csr_matrix((val, col, rp), shape=(n2, n2))
