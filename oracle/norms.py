"""Error norms of Section 4.1 (oracle; test infrastructure only).

||<e_z>||_{2,1} = ( sum_{n=1}^{M} dt ||<z_h>^n - <z>(t^n)||_{H^1}^2 )^{1/2}, the
L^2(0,T; H^1) norm of the ensemble-average error with the full H^1 norm
(L^2 part plus seminorm); the exact ensemble average of the member fields
c_j z is <c> z.
"""
import numpy as np

from workloads.ensembles import exact_v, exact_w, _grad_rows


def _exact(which, t, scale):
    f = exact_v if which == "v" else exact_w
    sign = 1.0 if which == "v" else -1.0

    def vals(x, y):
        return scale * f(x, y, t)

    def grads(x, y):
        dx, dy = _grad_rows(x, y, t, sign)
        return scale * dx, scale * dy

    return vals, grads


def l2h1_errors(run_factory, ens, nsteps):
    """Run the oracle and accumulate sum dt ||<e>||_{H1}^2 for v and w.
    Returns (err_v, err_w, semi_v, semi_w)."""
    run = run_factory(ens)
    cbar = float(np.mean(ens.info["c"]))
    acc = {"v": 0.0, "w": 0.0, "sv": 0.0, "sw": 0.0}
    for _ in range(nsteps):
        run.step()
        t = run.n * ens.dt
        for which, Z in (("v", run.V), ("w", run.W)):
            mean = Z.sum(axis=0) / Z.shape[0]
            ex = _exact(which, t, cbar)
            l2 = run.S.error_sq(mean, ex, "l2")
            h1 = run.S.error_sq(mean, ex, "h1")
            acc[which] += ens.dt * (l2 + h1)
            acc["s" + which] += ens.dt * h1
    return tuple(np.sqrt(acc[k]) for k in ("v", "w", "sv", "sw"))
