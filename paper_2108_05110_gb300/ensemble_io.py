"""Feeding an ensemble description into the library.

An ensemble description is any object with the attributes of the problem
statement of Section 1: ``mesh`` (``xy``, ``tri``), ``nu``, ``nu_m``, ``s``,
``dt``, ``mu``, and callables ``u0(pts)``, ``B0(pts)``, ``u_bc(pts, t)``,
``B_bc(pts, t)``, ``f(pts, t)`` / ``curl_g(pts, t)`` (or None) returning
[J, P, 2] arrays at points ``pts`` [P, 2].  The callables are evaluated at
the library's P2 nodes; forcing and Dirichlet data are taken at t^{n+1}.
"""
from .binding import EnsembleSolver


def solver_for(ens, bind=True, **opts):
    opts.setdefault("mu", float(getattr(ens, "mu", 1.0)))
    return EnsembleSolver(ens.mesh.xy, ens.mesh.tri, ens.nu, ens.nu_m, ens.s, ens.dt, bind=bind, **opts)


def feed_initial(solver, ens):
    xy, _ = solver.p2_nodes()
    solver._nodes = xy
    solver.set_initial(ens.u0(xy), ens.B0(xy) if ens.s > 0 else None)


def feed_step_data(solver, ens, t):
    xy = solver._nodes
    solver.set_dirichlet(ens.u_bc(xy, t), ens.B_bc(xy, t) if ens.s > 0 else None)
    f = ens.f(xy, t) if ens.f is not None else None
    cg = ens.curl_g(xy, t) if (ens.curl_g is not None and ens.s > 0) else None
    solver.set_forcing(f, cg)


def run(solver, ens, nsteps, start_step=0, callback=None):
    """Advance ``nsteps`` steps, refreshing forcing and Dirichlet data at t^{n+1}."""
    for n in range(start_step, start_step + nsteps):
        feed_step_data(solver, ens, (n + 1) * ens.dt)
        solver.step()
        if callback is not None:
            callback(solver, n + 1)
