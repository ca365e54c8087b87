"""Pins of the oracle's Algorithm 1 against what the paper and the
mathematics fix: an exactly representable patch solution, special cases of
the ensemble (identical members, v<->w mirror, s = 0), the per-step stability
inequality of Section 3.1, and the error tables of Section 4.1."""
import json
import os

import numpy as np
import pytest
from scipy.sparse.linalg import splu

from oracle.scheme import OracleRun, ensemble_mean
from oracle.norms import l2h1_errors
from workloads.ensembles import (Ensemble, lid_cavity, convergence_study, energy_study,
                                 manufactured)
from workloads.mesh import unit_square, channel_step

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def patch_ensemble(mesh, J=3, s=1.0, dt=0.1, nsteps=3):
    """v = (1+t)(y, x), w = (a, b) constant, q = x - y, r = 2x + y for every
    member (different nu_j, nu_m,j).  All terms are exact in P2/P1 and the
    fluctuations vanish, so the discrete solution is the exact one."""
    a, b = 0.7, -0.4
    rs = np.sqrt(s)
    nu = np.array([0.01, 0.02, 0.015][:J])
    nu_m = np.array([0.03, 0.005, 0.02][:J])

    def v(pts, t):
        return (1 + t) * np.stack([pts[:, 1], pts[:, 0]], axis=1)

    def w(pts, t):
        return np.broadcast_to(np.array([a, b]), (pts.shape[0], 2))

    def rep(z):
        return np.broadcast_to(z[None], (J,) + z.shape).copy()

    def f1(pts, t):
        return (np.stack([pts[:, 1], pts[:, 0]], axis=1) + (1 + t) * np.array([b, a])
                + np.array([1.0, -1.0]))

    def f2(pts, t):
        return np.broadcast_to(np.array([2.0, 1.0]), (pts.shape[0], 2))

    u = lambda p, t: rep(0.5 * (v(p, t) + w(p, t)))
    B = lambda p, t: rep(0.5 * (v(p, t) - w(p, t)) / rs)
    f = lambda p, t: rep(0.5 * (f1(p, t) + f2(p, t)))
    cg = lambda p, t: rep(0.5 * (f1(p, t) - f2(p, t)) / rs)
    ens = Ensemble("patch", mesh, nu, nu_m, s, dt, nsteps, u0=lambda p: u(p, 0.0),
                   B0=lambda p: B(p, 0.0), u_bc=u, B_bc=B, f=f, curl_g=cg)
    return ens, v, w


@pytest.mark.parametrize("mesh", [unit_square(5), channel_step(cells_per_unit=1)])
@pytest.mark.parametrize("form", ["skew", "standard"])
def test_patch_solution_is_exact(mesh, form):
    ens, v, w = patch_ensemble(mesh)
    run = OracleRun(ens, form=form)
    xy = run.S.node_xy
    x, y = run.S.mesh.xy[:, 0], run.S.mesh.xy[:, 1]
    for _ in range(ens.nsteps):
        run.step()
        t = run.n * ens.dt
        scale = np.abs(v(xy, t)).max()
        assert np.abs(run.V - v(xy, t)[None]).max() < 1e-11 * scale
        assert np.abs(run.W - w(xy, t)[None]).max() < 1e-11
        q = run.zero_mean(run.Q)
        r = run.zero_mean(run.R)
        qe = run.zero_mean((x - y)[None])[0]
        re = run.zero_mean((2 * x + y)[None])[0]
        assert np.abs(q - qe).max() < 1e-9 and np.abs(r - re).max() < 1e-9


def _replicate(ens, J):
    rep = lambda fn: (lambda *a: np.repeat(fn(*a)[:1], J, axis=0))
    return Ensemble(ens.name + f"-x{J}", ens.mesh, np.repeat(ens.nu[:1], J),
                    np.repeat(ens.nu_m[:1], J), ens.s, ens.dt, ens.nsteps,
                    u0=rep(ens.u0), B0=rep(ens.B0), u_bc=rep(ens.u_bc), B_bc=rep(ens.B_bc))


def test_identical_members_reproduce_single_run():
    base = lid_cavity(N=8, J=1, s=0.5, nsteps=3, Re=200.0)
    base.u0 = (lambda f: (lambda p: f(p) * 50.0))(base.u0)     # visible initial field
    many = _replicate(base, 4)
    r1, r4 = OracleRun(base), OracleRun(many)
    for _ in range(3):
        r1.step(); r4.step()
    for j in range(4):
        assert np.abs(r4.V[j] - r1.V[0]).max() < 1e-13 * np.abs(r1.V).max()
        assert np.abs(r4.W[j] - r1.W[0]).max() < 1e-13 * np.abs(r1.W).max()


def test_v_w_mirror():
    ens = lid_cavity(N=8, J=3, s=0.5, nsteps=3, Re=300.0)
    mir = lid_cavity(N=8, J=3, s=0.5, nsteps=3, Re=300.0)
    mir.B0 = (lambda f: (lambda p: -f(p)))(ens.B0)
    mir.B_bc = (lambda f: (lambda p, t: -f(p, t)))(ens.B_bc)
    r, m = OracleRun(ens), OracleRun(mir)
    for _ in range(3):
        r.step(); m.step()
        assert np.abs(m.V - r.W).max() < 1e-13 * np.abs(r.W).max()
        assert np.abs(m.W - r.V).max() < 1e-13 * np.abs(r.V).max()


def test_s_zero_gives_identical_subproblems():
    ens = lid_cavity(N=8, J=3, s=0.0, nsteps=3, Re=300.0)
    r = OracleRun(ens)
    for _ in range(3):
        r.step()
        assert np.array_equal(r.V, r.W)


def test_discrete_divergence_and_dense_solve():
    ens = lid_cavity(N=2, J=2, s=1.0, nsteps=1, Re=100.0)
    r = OracleRun(ens)
    r.step(keep=True)
    A = r.last["Av"].toarray()
    for j in range(2):
        xd = np.linalg.solve(A, r.last["bv"][j])
        xs = splu(r.last["Av"]).solve(r.last["bv"][j])
        assert np.abs(xd - xs).max() < 1e-12 * np.abs(xd).max()
    ens = lid_cavity(N=8, J=3, s=1.0, nsteps=2, Re=500.0)
    r = OracleRun(ens)
    for _ in range(2):
        r.step()
    for j in range(3):
        div = r.Bx @ r.V[j][:, 0] + r.By @ r.V[j][:, 1]
        assert np.abs(div[1:]).max() < 1e-12 * np.abs(r.V[j]).max()


def test_stability_inequality_each_step():
    """Section 3.1 per-step inequality (f = 0, homogeneous data, alpha_j > 0,
    mu > 1/2), checked from the first step whose old state is in V_h."""
    ens = energy_study(N=12, J=6, dt=0.05, nsteps=8)
    r = OracleRun(ens)
    assert np.all(r.alpha() > 0)
    c = 0.5 * (r.nubar + r.nubar_m) * ens.dt
    S, M, K = r.S, r.M, r.K

    def norms(Z):
        return (np.array([S.l2_sq(M, z) for z in Z]), np.array([S.h1semi_sq(K, z) for z in Z]))

    r.step()
    energies = []
    for _ in range(ens.nsteps - 1):
        v0, gv0 = norms(r.V)
        w0, gw0 = norms(r.W)
        r.step()
        v1, gv1 = norms(r.V)
        w1, gw1 = norms(r.W)
        lhs = v1 + w1 + c * (gv1 + gw1) + 0.5 * r.alpha() * ens.dt * (gv0 + gw0)
        rhs = v0 + w0 + c * (gv0 + gw0)
        assert np.all(lhs <= rhs * (1 + 1e-12))
        energies.append(r.energy())
    assert np.all(np.diff(energies) <= 0)          # Section 4.2: energy decays


def _rates(e):
    e = np.asarray(e)
    return np.log2(e[:-1] / e[1:])


def test_spatial_errors_match_table1_for_pressure_free_velocity():
    """Table 1 (eps = 0): the paper's Scott-Vogelius velocity error does not
    depend on the pressure, so Taylor-Hood with the same velocity and zero
    pressure must give the same errors and rate 2."""
    g = json.load(open(os.path.join(GOLDEN, "table1_spatial_eps0.json")))
    ev, ew = [], []
    for N in (4, 8, 16, 32):
        ens = convergence_study(N, 2, dt=0.001 / 8, nsteps=8, eps=0.0, with_pressure=False)
        a, b, _, _ = l2h1_errors(OracleRun, ens, 8)
        ev.append(a); ew.append(b)
    assert np.allclose(ev, g["e_v"][:4], rtol=0.05)
    assert np.allclose(ew, g["e_w"][:4], rtol=0.05)
    assert np.all(np.abs(_rates(ev) - 2.0) < 0.1) and np.all(np.abs(_rates(ew) - 2.0) < 0.1)


def test_spatial_rates_with_pressure_are_second_order_preasymptotic():
    """With the printed pressure, Taylor-Hood is not pressure-robust: the rate
    on coarse meshes sits between 1.6 and 2 and the errors exceed the
    pressure-free ones."""
    ev = []
    for N in (4, 8, 16):
        ens = convergence_study(N, 2, dt=0.001 / 8, nsteps=8, eps=0.01)
        a, _, _, _ = l2h1_errors(OracleRun, ens, 8)
        ev.append(a)
    r = _rates(ev)
    assert np.all((r > 1.6) & (r < 2.1))


def test_temporal_errors_match_table4():
    """Table 4 (eps = 0): temporal errors dominate at h = 1/16, so the values
    of both samples are reproduced and the rate tends to 1."""
    g = json.load(open(os.path.join(GOLDEN, "table4_temporal_eps0.json")))
    for sample, tol in ((1, 0.05), (2, 0.10)):
        ev, ew = [], []
        for k in (2, 4, 8, 16):
            ens = convergence_study(16, 4, dt=1.0 / k, nsteps=k, eps=0.0, sample=sample)
            a, b, _, _ = l2h1_errors(OracleRun, ens, k)
            ev.append(a); ew.append(b)
        ref = g[f"sample{sample}"]
        assert np.allclose(ev, ref["e_v"][:4], rtol=tol)
        assert np.allclose(ew, ref["e_w"][:4], rtol=tol)
        assert np.all(np.diff(ev) < 0) and np.all((_rates(ev) > 0.7) & (_rates(ev) < 1.1))
