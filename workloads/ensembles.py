"""Seeded ensemble descriptions for the experiments of Section 4 and the
benchmark workloads shaped like them.

An :class:`Ensemble` carries the problem statement of Section 1 (eq. gov1-gov5
and the Elsaesser change of variables): a mesh, J members with their
viscosities nu_j and magnetic diffusivities nu_{m,j}, the coupling number s,
the time step dt, and closed-form initial, Dirichlet and forcing fields in
primitive variables (u, B, f, curl g).  Field callables take points
``pts`` [P, 2] (and a time) and return arrays [J, P, 2].

Random draws use ``numpy.random.default_rng(seed)``; the recipes are stated
next to each generator.
"""
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

from .mesh import unit_square, channel_step, barycentric_refine, Mesh


@dataclass
class Ensemble:
    name: str
    mesh: Mesh
    nu: np.ndarray           # [J]
    nu_m: np.ndarray         # [J]
    s: float
    dt: float
    nsteps: int
    u0: Callable             # pts -> [J, P, 2]
    B0: Callable
    u_bc: Callable           # (pts, t) -> [J, P, 2], used on boundary nodes only
    B_bc: Callable
    f: Optional[Callable] = None        # (pts, t) -> [J, P, 2]; None = 0
    curl_g: Optional[Callable] = None   # (pts, t) -> [J, P, 2]; None = 0
    mu: float = 1.0
    info: dict = field(default_factory=dict)

    @property
    def J(self):
        return int(self.nu.shape[0])


def perturbation_factor(J, eps):
    """c_j = 1 + (-1)^(j+1) ceil(j/2) eps / 5 for j = 1..J (Section 4.1)."""
    j = np.arange(1, J + 1)
    return 1.0 + ((-1.0) ** (j + 1)) * np.ceil(j / 2.0) * eps / 5.0


# ---------------------------------------------------------------------------
# Manufactured solution of Section 4.1 (eq. exact-solution) in Elsaesser form
#   v = (cos y + (1+e^t) sin y, sin x + (1+e^t) cos x)
#   w = (cos y - (1+e^t) sin y, sin x - (1+e^t) cos x)
#   q = r = p = sin(x+y)(1+e^t)        (lambda = 0)
# member j scales v and w by c_j; p is not scaled.
# ---------------------------------------------------------------------------

def exact_v(x, y, t):
    a = 1.0 + np.exp(t)
    return np.stack([np.cos(y) + a * np.sin(y), np.sin(x) + a * np.cos(x)], axis=-1)


def exact_w(x, y, t):
    a = 1.0 + np.exp(t)
    return np.stack([np.cos(y) - a * np.sin(y), np.sin(x) - a * np.cos(x)], axis=-1)


def exact_p(x, y, t):
    return np.sin(x + y) * (1.0 + np.exp(t))


def _grad_rows(x, y, t, sign):
    """Rows of grad z for z = v (sign=+1) or w (sign=-1): returns (dz/dx, dz/dy),
    each [.., 2]."""
    a = 1.0 + np.exp(t)
    dzdx = np.stack([np.zeros_like(x), np.cos(x) - sign * a * np.sin(x)], axis=-1)
    dzdy = np.stack([-np.sin(y) + sign * a * np.cos(y), np.zeros_like(y)], axis=-1)
    return dzdx, dzdy


def manufactured_forcing(x, y, t, c, nu, nu_m, with_pressure=True):
    """f1, f2 of eq. els1-els2 for the member fields c v, c w (Delta v = -v,
    Delta w = -w), with the member's (nu, nu_m).  Returns (f1, f2), [.., 2].
    ``with_pressure=False`` drops grad p (the same velocity with q = r = 0)."""
    e = np.exp(t)
    v, w = exact_v(x, y, t), exact_w(x, y, t)
    vt = np.stack([e * np.sin(y), e * np.cos(x)], axis=-1)
    wt = -vt
    gp = (1.0 + e) * np.cos(x + y)
    gradp = np.stack([gp, gp], axis=-1) if with_pressure else 0.0
    vx, vy = _grad_rows(x, y, t, +1.0)
    wx, wy = _grad_rows(x, y, t, -1.0)
    w_grad_v = w[..., :1] * vx + w[..., 1:] * vy
    v_grad_w = v[..., :1] * wx + v[..., 1:] * wy
    sp, sm = 0.5 * (nu + nu_m), 0.5 * (nu - nu_m)
    f1 = c * vt + c * c * w_grad_v + c * sp * v + c * sm * w + gradp
    f2 = c * wt + c * c * v_grad_w + c * sp * w + c * sm * v + gradp
    return f1, f2


def manufactured(N, J, nu, nu_m, c, dt, nsteps, s=1.0, mu=1.0, name="manufactured",
                 homogeneous=False, zero_forcing=False, with_pressure=True, mesh=None):
    """Ensemble whose member j has the exact Elsaesser fields c_j v, c_j w.

    Primitive data follow from u = (v+w)/2 and sqrt(s) B = (v-w)/2, and
    f = (f1+f2)/2, sqrt(s) curl g = (f1-f2)/2 (Section 1).
    ``homogeneous`` / ``zero_forcing`` give the energy test of Section 4.2.
    ``mesh`` replaces the N x N unit square (e.g. by its barycenter refinement).
    """
    mesh = unit_square(N) if mesh is None else mesh
    nu = np.asarray(nu, dtype=np.float64)
    nu_m = np.asarray(nu_m, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    rs = np.sqrt(s)

    def vw(pts, t):
        x, y = pts[:, 0], pts[:, 1]
        v = c[:, None, None] * exact_v(x, y, t)[None]
        w = c[:, None, None] * exact_w(x, y, t)[None]
        return v, w

    def u_at(pts, t):
        v, w = vw(pts, t)
        return 0.5 * (v + w)

    def B_at(pts, t):
        v, w = vw(pts, t)
        return 0.5 * (v - w) / rs

    def zero(pts, t=0.0):
        return np.zeros((len(c), pts.shape[0], 2))

    def forcing(pts, t):
        x, y = pts[:, 0], pts[:, 1]
        f1 = np.empty((len(c), pts.shape[0], 2))
        f2 = np.empty_like(f1)
        for j in range(len(c)):
            f1[j], f2[j] = manufactured_forcing(x, y, t, c[j], nu[j], nu_m[j], with_pressure)
        return f1, f2

    def f_at(pts, t):
        f1, f2 = forcing(pts, t)
        return 0.5 * (f1 + f2)

    def cg_at(pts, t):
        f1, f2 = forcing(pts, t)
        return 0.5 * (f1 - f2) / rs

    return Ensemble(
        name=name, mesh=mesh, nu=nu, nu_m=nu_m, s=float(s), dt=float(dt), nsteps=int(nsteps),
        u0=lambda pts: u_at(pts, 0.0), B0=lambda pts: B_at(pts, 0.0),
        u_bc=zero if homogeneous else u_at, B_bc=zero if homogeneous else B_at,
        f=None if zero_forcing else f_at, curl_g=None if zero_forcing else cg_at,
        mu=mu, info={"N": N, "c": c, "with_pressure": with_pressure},
    )


def config_manufactured_small():
    """16x16 right-diagonal unit square, J=3, nu_j = nu_m,j = 0.01 (1+delta_j),
    delta in {-0.1, 0, 0.1}, s = 1, dt = 0.01, 10 steps, member fields
    scaled by c_j = 1 + eps_j with eps in {-1e-3, 0, 1e-3}."""
    delta = np.array([-0.1, 0.0, 0.1])
    nu = 0.01 * (1.0 + delta)
    c = 1.0 + np.array([-1e-3, 0.0, 1e-3])
    return manufactured(16, 3, nu, nu.copy(), c, dt=0.01, nsteps=10, s=1.0,
                        name="manufactured-16x16-J3")


def convergence_study(N, J, dt, nsteps, eps=0.0, sample=1, seed=0, with_pressure=True,
                      mesh=None):
    """Section 4.1: (nu_j, nu_m,j) uniform in [0.009,0.011] x [0.09,0.11]
    (sample 1) or [0.009,0.011] x [0.0009,0.0011] (sample 2); c_j from
    :func:`perturbation_factor`."""
    rng = np.random.default_rng(seed)
    nu = rng.uniform(0.009, 0.011, J)
    nu_m = rng.uniform(0.09, 0.11, J) if sample == 1 else rng.uniform(0.0009, 0.0011, J)
    c = perturbation_factor(J, eps)
    return manufactured(N, J, nu, nu_m, c, dt=dt, nsteps=nsteps, s=1.0,
                        name=f"convergence-N{N}-J{J}", with_pressure=with_pressure, mesh=mesh)


def energy_study(N=32, J=20, dt=0.05, nsteps=20, seed=0):
    """Section 4.2: manufactured initial data with eps = 0.01, homogeneous
    Dirichlet data, zero forcing, (nu, nu_m) from sample 1."""
    rng = np.random.default_rng(seed)
    nu = rng.uniform(0.009, 0.011, J)
    nu_m = rng.uniform(0.09, 0.11, J)
    c = perturbation_factor(J, 0.01)
    return manufactured(N, J, nu, nu_m, c, dt=dt, nsteps=nsteps, s=1.0, homogeneous=True,
                        zero_forcing=True, name=f"energy-N{N}-J{J}")


def _stream_perturbation(pts):
    """Divergence-free field curl(psi) = (d psi/dy, -d psi/dx) with
    psi = sin^2(pi x) sin^2(pi y); vanishes on the boundary of the unit square."""
    x, y = pts[:, 0], pts[:, 1]
    px = 2 * np.pi * np.sin(np.pi * x) * np.cos(np.pi * x) * np.sin(np.pi * y) ** 2
    py = 2 * np.pi * np.sin(np.pi * y) * np.cos(np.pi * y) * np.sin(np.pi * x) ** 2
    return np.stack([py, -px], axis=-1)


def lid_cavity(N=128, J=20, s=1.0, dt=0.01, nsteps=200, Re=15000.0, seed=2, spread=0.1,
               barycentric=False):
    """Lid-driven-cavity-shaped workload (shape of Section 4.3).

    Unit square N x N right-diagonal; nu_j = nu_m,j = (1/Re)(1+delta_j),
    delta_j ~ U[-spread, spread]; lid u = (1, 0) on y = 1 for 0 < x < 1 (the
    two top corners take the wall value 0), u = 0 on the other sides;
    B = (0, 1) on the whole boundary; initial u_j = eps_j curl(psi),
    B_j = eps'_j curl(psi), eps, eps' ~ N(0, sigma = 1e-3); no forcing.
    ``barycentric=True`` takes the barycenter refinement of the N x N mesh
    (the meshes of Section 4, for the Scott-Vogelius element).
    """
    rng = np.random.default_rng(seed)
    delta = rng.uniform(-spread, spread, J)
    nu = (1.0 / Re) * (1.0 + delta)
    nu_m = nu.copy()
    eps_u = rng.normal(0.0, 1e-3, J)
    eps_B = rng.normal(0.0, 1e-3, J)
    mesh = unit_square(N)
    if barycentric:
        mesh = barycentric_refine(mesh)

    def u0(pts):
        return eps_u[:, None, None] * _stream_perturbation(pts)[None]

    def B0(pts):
        return eps_B[:, None, None] * _stream_perturbation(pts)[None]

    def u_bc(pts, t):
        x, y = pts[:, 0], pts[:, 1]
        lid = (y == 1.0) & (x > 0.0) & (x < 1.0)
        out = np.zeros((J, pts.shape[0], 2))
        out[:, lid, 0] = 1.0
        return out

    def B_bc(pts, t):
        out = np.zeros((J, pts.shape[0], 2))
        out[:, :, 1] = 1.0
        return out

    # the amplitudes are read when u0 / B0 are called, so a caller may change
    # info["eps_u"] / info["eps_B"] in place (finite-difference perturbations)
    return Ensemble(name=f"lid-cavity-N{N}{'-bary' if barycentric else ''}-J{J}-s{s:g}", mesh=mesh, nu=nu, nu_m=nu_m, s=float(s),
                    dt=float(dt), nsteps=int(nsteps), u0=u0, B0=B0, u_bc=u_bc, B_bc=B_bc,
                    info={"N": N, "Re": Re, "seed": seed, "eps_u": eps_u, "eps_B": eps_B,
                          "perturbation_shape": _stream_perturbation})


def channel(J=50, dt=0.05, nsteps=400, s=0.01, nu=1.0 / 600, nu_m=1.0 / 600, seed=3,
            cells_per_unit=7, eps_range=0.05, mesh=None):
    """Channel-past-a-step workload (shape of Section 4.4).

    [0,40] x [0,10] minus [5,6] x [0,1], graded jittered mesh; c_j = 1+eps_j,
    eps_j ~ U[-eps_range, eps_range]; initial u_j = c_j (y(10-y)/25, 0),
    B_j = 0; Dirichlet: walls u = 0, inlet x = 0 and outlet x = 40
    u = c_j (y(10-y)/25, 0); B = c_j (0, 1) on the whole boundary; no forcing.
    """
    rng = np.random.default_rng(seed)
    eps = rng.uniform(-eps_range, eps_range, J)
    c = 1.0 + eps
    mesh = mesh if mesh is not None else channel_step(cells_per_unit=cells_per_unit, seed=seed)
    nuv = np.full(J, nu)
    numv = np.full(J, nu_m)
    xmax = float(mesh.xy[:, 0].max())

    def profile(pts):
        y = pts[:, 1]
        return y * (10.0 - y) / 25.0

    def u0(pts):
        out = np.zeros((J, pts.shape[0], 2))
        out[:, :, 0] = c[:, None] * profile(pts)[None]
        return out

    def B0(pts):
        return np.zeros((J, pts.shape[0], 2))

    def u_bc(pts, t):
        x = pts[:, 0]
        io = (x == 0.0) | (x == xmax)
        out = np.zeros((J, pts.shape[0], 2))
        out[:, io, 0] = c[:, None] * profile(pts)[io][None]
        return out

    def B_bc(pts, t):
        out = np.zeros((J, pts.shape[0], 2))
        out[:, :, 1] = c[:, None]
        return out

    return Ensemble(name=f"channel-J{J}", mesh=mesh, nu=nuv, nu_m=numv, s=float(s), dt=float(dt),
                    nsteps=int(nsteps), u0=u0, B0=B0, u_bc=u_bc, B_bc=B_bc,
                    info={"c": c, "seed": seed})


def sensitivity(N=64, J=8, s=0.5, dt=0.01, nsteps=40, seed=4):
    """Sensitivity workload: lid-cavity data with nu_j, nu_m,j = 0.005 (1+delta),
    delta ~ U[-0.2, 0.2] drawn independently for nu and nu_m."""
    rng = np.random.default_rng(seed)
    nu = 0.005 * (1.0 + rng.uniform(-0.2, 0.2, J))
    nu_m = 0.005 * (1.0 + rng.uniform(-0.2, 0.2, J))
    base = lid_cavity(N=N, J=J, s=s, dt=dt, nsteps=nsteps, seed=seed)
    base.nu, base.nu_m = nu, nu_m
    base.name = f"sensitivity-N{N}-J{J}"
    return base


def batched_family(count=64, seed=5000, Ns=(32, 64, 128, 256), Jmax=64, nsteps=50):
    """Batched uneven ensembles: ensemble k uses seed ``seed + k`` to draw
    J_k ~ U{1..Jmax}, N_k from ``Ns`` and Re_k ~ U[1000, 15000], with the
    lid-cavity data of :func:`lid_cavity`."""
    out = []
    for k in range(count):
        rng = np.random.default_rng(seed + k)
        Jk = int(rng.integers(1, Jmax + 1))
        Nk = int(rng.choice(Ns))
        Re = float(rng.uniform(1000.0, 15000.0))
        out.append(lid_cavity(N=Nk, J=Jk, Re=Re, nsteps=nsteps, seed=seed + k))
    return out
