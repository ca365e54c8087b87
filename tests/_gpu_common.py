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


def oracle_first_step_sampled(ens, members, form="skew", element="TH"):
    """The first step of Algorithm 1 by the oracle for a subset of members:
    the ensemble means and mixing lengths use all members, the two shared
    saddle matrices are factorised once (SuperLU) and solved for the chosen
    members only (members are independent once the shared quantities are
    known).  Returns the oracle run (its P2 space and matrices) and the new
    v, w of the chosen members [len(members), n2, 2]."""
    from scipy.sparse.linalg import splu
    run = OracleRun(ens, form=form, element=element)
    S, n2 = run.S, run.S.n2
    mv, mw = ensemble_mean(run.V), ensemble_mean(run.W)
    Vp, Wp = run.V - mv, run.W - mw
    Av = run.saddle(run.shared_matrix(mw, mixing_length_sq(S, Wp)))
    Aw = run.saddle(run.shared_matrix(mv, mixing_length_sq(S, Vp)))
    f1, f2, gv, gw = run.member_data(ens.dt)
    cross, same = run.nu - run.nu_m, run.nu_p + run.nu_m_p
    luv, luw = splu(Av), splu(Aw)
    out_v, out_w = [], []
    for j in members:
        xv = luv.solve(run.rhs(run.V, run.W, Wp, f1, gv, j, same, cross))
        xw = luw.solve(run.rhs(run.W, run.V, Vp, f2, gw, j, same, cross))
        out_v.append(np.stack([xv[:n2], xv[n2:2 * n2]], 1))
        out_w.append(np.stack([xw[:n2], xw[n2:2 * n2]], 1))
    return run, np.array(out_v), np.array(out_w)
