"""Benchmark: ensemble member-steps/s of the decoupled Elsaesser scheme
(Algorithm 1) on the lid-driven-cavity-shaped workload (unit square 128x128
right-diagonal, Taylor-Hood P2-P1, J = 20, nu = nu_m = (1/15000)(1 + delta_j),
s = 1, dt = 0.01, synthetic seeded data).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision mixed|fp64]

One step = one pass of the whole hot path for all J members: ensemble means
and mixing-length fields, two shared-matrix assemblies, two batched
right-hand-side assemblies, and the two block solves on two streams.  Under
torchrun each rank runs an independent ensemble replica (seed 2 + rank): the
value is the whole-job member-steps/s.  Prints one JSON line on rank 0.
"""
import argparse
import faulthandler
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ensemble member-steps/s at rel L2 <=1e-8 vs FP64 oracle"
UNIT = "member-steps/s"
WORKLOAD = dict(N=128, J=20, s=1.0, dt=0.01, Re=15000.0)
CHANNEL = dict(J=50, s=0.01, dt=0.05, nu=1.0 / 600)
SV_N = 64


def element_of(workload):
    """Finite element pair of a workload: Scott-Vogelius (P2, P1disc) for the
    barycenter-refined cavity, Taylor-Hood P2-P1 otherwise."""
    return "SV" if workload == "sv" else "TH"


def make_ensemble(workload, N, J, seed=None):
    """The benchmark's synthetic ensembles: the lid-driven-cavity-shaped one
    (the metric's workload), the same cavity on the barycenter refinement of
    an N x N mesh for the Scott-Vogelius element, or the
    channel-past-a-step-shaped one."""
    from workloads.ensembles import lid_cavity, channel
    if workload == "channel":
        return channel(J=J, dt=CHANNEL["dt"], s=CHANNEL["s"], nu=CHANNEL["nu"], nu_m=CHANNEL["nu"],
                       seed=3 if seed is None else seed)
    return lid_cavity(N=N, J=J, s=WORKLOAD["s"], dt=WORKLOAD["dt"], Re=WORKLOAD["Re"],
                      seed=2 if seed is None else seed, barycentric=(workload == "sv"))


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-separate", action="store_true", help="skip the separate-solve comparator")
    p.add_argument("--workload", default="cavity", choices=["cavity", "sv", "channel", "batched", "adjoint"],
                   help="cavity: the metric's workload; sv: the cavity ensemble with the Scott-Vogelius "
                        "element on the barycenter refinement of an N x N mesh (default N = 64); "
                        "channel: the channel-past-a-step ensemble; "
                        "batched: uneven independent ensembles; adjoint: forward and forward + discrete "
                        "adjoint of the sensitivity workload")
    p.add_argument("--batch-count", type=int, default=64)
    p.add_argument("--batch-threads", type=int, default=4, help="host threads of mhde_advance_many")
    p.add_argument("--batch-mem-gb", type=float, default=240.0,
                   help="cap on the summed workspaces of the batched ensembles")
    p.add_argument("--profile-only", action="store_true",
                   help="run W warm-up and K timed steps and exit (for ncu captures)")
    p.add_argument("--profile-kernel", type=int, default=-1,
                   help="with --profile-only: launch only this hot-path kernel group K times "
                        "(mhde_time_kernel ids: 0 SpMM FP64, 1 SpMM FP32, 2 F assembly, 3 RHS, "
                        "4 means+l2, 5 preconditioner, 6 Gram)")
    p.add_argument("--no-oracle-check", action="store_true",
                   help="skip the one-step oracle check of the benchmarked state")
    p.add_argument("--cpu-study", action="store_true",
                   help="time the FP64 oracle on the host cores three ways (factor per member, factor once per "
                        "step, a process pool over members) on the workload's first step, print one JSON line")
    p.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--oracle-check", default=None, help=argparse.SUPPRESS)
    p.add_argument("--N", type=int, default=None, help="cells per side (default 128 cavity, 64 sv)")
    p.add_argument("--J", type=int, default=None, help="members (default 20 cavity, 50 channel)")
    a = p.parse_args()
    if a.J is None:
        a.J = CHANNEL["J"] if a.workload == "channel" else WORKLOAD["J"]
    if a.N is None:
        a.N = SV_N if a.workload == "sv" else WORKLOAD["N"]
    return a


def config(args, extra=None):
    if args.workload == "channel":
        c = {"workload": f"channel-past-a-step-shaped ensemble, [0,40]x[0,10] minus [5,6]x[0,1], 280x70 "
                         f"graded jittered cells, Taylor-Hood P2-P1 (157,838 velocity DOFs), J={args.J}, "
                         f"nu=nu_m=1/600, s=0.01, dt=0.05, inflow scaled by 1+eps_j",
             "mesh": "channel 280x70 cells minus step", "J": args.J, "s": CHANNEL["s"], "dt": CHANNEL["dt"]}
    elif args.workload == "sv":
        c = {"workload": f"lid-driven-cavity-shaped ensemble, barycenter refinement of the unit square "
                         f"{args.N}x{args.N} right-diagonal mesh, Scott-Vogelius P2-P1disc, J={args.J}, "
                         f"Re=15000, s=1, dt=0.01",
             "mesh": f"{args.N}x{args.N} barycenter-refined", "J": args.J, "s": WORKLOAD["s"],
             "dt": WORKLOAD["dt"]}
    else:
        c = {"workload": f"lid-driven-cavity-shaped ensemble, unit square {args.N}x{args.N} "
                         f"right-diagonal, Taylor-Hood P2-P1, J={args.J}, Re=15000, s=1, dt=0.01",
             "mesh": f"{args.N}x{args.N}", "J": args.J, "s": WORKLOAD["s"], "dt": WORKLOAD["dt"]}
    c.update({"element": "P2-P1disc" if args.workload == "sv" else "P2-P1",
              "l2": "per-step working set (Krylov basis 31 blocks + states) > 129 MB L2",
              "parallelism": f"replicas x{args.gpus}" if args.gpus > 1 else "single GPU"})
    if extra:
        c.update(extra)
    return c


# --------------------------------------------------------------------------- CPU oracle sample
def cpu_sample(workload, N, J_total):
    """One v-subproblem of one member of the workload's first step on the full
    mesh through the FP64 oracle (assembly + SuperLU factorisation + solve),
    run in a fresh single-threaded process.  Returns seconds."""
    import numpy as np
    from oracle.scheme import OracleRun, ensemble_mean, mixing_length_sq
    from scipy.sparse.linalg import splu
    ens = make_ensemble(workload, N, J_total)
    run = OracleRun(ens, lu_per_member=True, element=element_of(workload))
    t0 = time.perf_counter()
    mv, mw = ensemble_mean(run.V), ensemble_mean(run.W)
    Wp = run.W - mw
    l2w = mixing_length_sq(run.S, Wp)
    A = run.saddle(run.shared_matrix(mw, l2w))
    f1, f2, gv, gw = run.member_data(ens.dt)
    b = run.rhs(run.V, run.W, Wp, f1, gv, 0, run.nu_p + run.nu_m_p, run.nu - run.nu_m)
    x = splu(A).solve(b)
    assert np.isfinite(x).all()
    return time.perf_counter() - t0


def run_cpu_sample_subprocess(args):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", "--workload", args.workload,
                          "--N", str(args.N), "--J", str(args.J)], capture_output=True, text=True, env=env,
                         timeout=900)
    line = [l for l in out.stdout.splitlines() if l.startswith("{")]
    if out.returncode != 0 or not line:
        raise RuntimeError("cpu sample failed: " + out.stderr[-2000:])
    return json.loads(line[-1])["seconds"]


def cpu_baseline_block(seconds):
    return {"value": 0.5 / seconds, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "one member's v-subproblem of one step on the full mesh (half a member-step): "
                      "FP64 numpy/scipy assembly + SuperLU factorisation and solve, 1 thread; "
                      f"{seconds:.2f} s"}


# --------------------------------------------------------------------------- accuracy at the benchmarked state
def oracle_step_check(path, workload, N, J):
    """The next step of the FP64 oracle from the state stored in `path`
    (both Elsaesser fields of all members, library numbering), with one
    SuperLU factorisation per subproblem shared by all members: rel L2 of the
    library's step against it, per subproblem, over all members and nodes."""
    import numpy as np
    from oracle.scheme import OracleRun
    d = np.load(path)
    ens = make_ensemble(workload, N, J)
    run = OracleRun(ens, element=element_of(workload))
    run.V, run.W, run.n = d["v0"].copy(), d["w0"].copy(), int(d["n"])
    t0 = time.perf_counter()
    run.step()
    secs = time.perf_counter() - t0
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    return {"rel_l2_v": rel(d["v1"], run.V), "rel_l2_w": rel(d["w1"], run.W), "step": int(d["n"]) + 1,
            "members": J, "oracle_seconds": secs}


def oracle_check(args, sol):
    """One more library step from the benchmarked state, compared with the
    same step of the FP64 oracle run in a fresh single-threaded process."""
    import tempfile
    import numpy as np
    v0, w0, _, _ = sol.read_state()
    n = int(sol.stats().steps)
    sol.step()
    v1, w1, _, _ = sol.read_state()
    fd, path = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    try:
        np.savez(path, v0=v0, w0=w0, v1=v1, w1=w1, n=n)
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
                   CUDA_VISIBLE_DEVICES="")
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-check", path, "--workload",
                              args.workload, "--N", str(args.N), "--J", str(args.J)], capture_output=True,
                             text=True, env=env, timeout=1800)
    finally:
        os.remove(path)
    line = [l for l in out.stdout.splitlines() if l.startswith("{")]
    if out.returncode != 0 or not line:
        return {"error": out.stderr[-500:]}
    res = json.loads(line[-1])
    res["gate"] = 1e-8 if sol.options.precision == 1 else 1e-10
    res["what"] = ("rel L2 of the step after the timed ones (all members, all nodes) against the FP64 "
                   "oracle stepped from the same state")
    return res


def fp64_same_steps(args, ens, state0, device):
    """The plain FP64 GPU path (FP64 Krylov, SpMM and preconditioner) over the
    first steps of the timed region, from the same post-warm-up state."""
    import torch
    from paper_2108_05110_gb300 import ensemble_io, PREC_FP64
    sol = ensemble_io.solver_for(ens, precision=PREC_FP64, device=device, element=element_of(args.workload))
    ensemble_io.feed_initial(sol, ens)
    ensemble_io.feed_step_data(sol, ens, ens.dt)
    sol.load_state(state0)
    k = max(1, min(3, args.steps))
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(sol.stream_v)
    st0 = sol.stats()
    try:
        sol.advance(k)
    except Exception as e:          # a step that does not converge is reported, not fatal
        torch.cuda.synchronize()
        st1 = sol.stats()
        sol.close()
        return {"error": str(e)[:200], "steps_done": int(st1.steps - st0.steps),
                "what": "FP64 Krylov, SpMM and preconditioner (the plain FP64 GPU form), same post-warm-up "
                        "state and first steps of the timed region"}
    ev1.record(sol.stream_v)
    torch.cuda.synchronize()
    st1 = sol.stats()
    ms = ev0.elapsed_time(ev1)
    out = {"value": ens.J * k / (ms / 1000.0), "unit": UNIT, "steps": k, "ms_per_step": ms / k,
           "rtol": sol.options.rtol, "final_relres": max(float(st1.last_relres[0]), float(st1.last_relres[1])),
           "krylov_iters_per_step": (st1.total_iters - st0.total_iters) / k,
           "what": "FP64 Krylov, SpMM and preconditioner (the plain FP64 GPU form), same post-warm-up state "
                   "and first steps of the timed region"}
    sol.close()
    return out


# --------------------------------------------------------------------------- CPU oracle study
def _v_system(workload, N, J):
    """The v-subproblem of the workload's first step through the oracle:
    (saddle matrix, right-hand sides of all members)."""
    from oracle.scheme import OracleRun, ensemble_mean, mixing_length_sq
    ens = make_ensemble(workload, N, J)
    run = OracleRun(ens, element=element_of(workload))
    mw = ensemble_mean(run.W)
    Wp = run.W - mw
    A = run.saddle(run.shared_matrix(mw, mixing_length_sq(run.S, Wp)))
    f1, _, gv, _ = run.member_data(ens.dt)
    bs = [run.rhs(run.V, run.W, Wp, f1, gv, j, run.nu_p + run.nu_m_p, run.nu - run.nu_m) for j in range(J)]
    return A, bs


def _pool_member(args):
    """One member's v-subproblem with its own factorisation (a pool worker)."""
    workload, N, J, j = args
    from scipy.sparse.linalg import splu
    A, bs = _v_system(workload, N, J)
    t0 = time.perf_counter()
    splu(A).solve(bs[j])
    return time.perf_counter() - t0


def cpu_study(args):
    """Host-core baselines of the oracle on the v-subproblem of the first
    step (half a member-step per member): (1) factor per member, (2) factor
    once and solve every member (the shared matrix of Section 1), (3) a
    process pool over members, each factorising its own copy.  Rates are in
    member-steps/s (two subproblems per member-step)."""
    import multiprocessing as mp
    import platform
    from scipy.sparse.linalg import splu
    info = {"os_cpu_count": os.cpu_count(), "machine": platform.machine(), "processor": platform.processor()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "CPU(s)", "Thread(s) per core", "Core(s) per socket",
                                              "Socket(s)", "Vendor ID"):
                info[line.split(":")[0].strip()] = line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    J = args.J
    t0 = time.perf_counter()
    A, bs = _v_system(args.workload, args.N, J)
    t_assemble = time.perf_counter() - t0
    t0 = time.perf_counter()
    lu = splu(A)
    t_factor = time.perf_counter() - t0
    t0 = time.perf_counter()
    for b in bs:
        lu.solve(b)
    t_solves = time.perf_counter() - t0
    per_member = t_factor + t_solves / J
    once = t_factor + t_solves
    workers = max(1, min(J, os.cpu_count() or 1))
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        t0 = time.perf_counter()
        per_worker = pool.map(_pool_member, [(args.workload, args.N, J, j) for j in range(workers)])
        t_wall = time.perf_counter() - t0
    t_pool = max(per_worker)                            # the workers factorise and solve concurrently
    rate = lambda members, secs: 0.5 * members / secs
    return {"cpu_study": True, "workload": config(args)["workload"], "host": info,
            "threads_per_process": os.environ.get("OMP_NUM_THREADS", "unset"),
            "assemble_s": t_assemble, "factor_s": t_factor, "solve_s_per_member": t_solves / J,
            "factor_per_member": {"member_steps_per_s": rate(1, per_member), "cores": 1},
            "factor_once_per_step": {"member_steps_per_s": rate(J, once), "cores": 1},
            "process_pool": {"member_steps_per_s": rate(workers, t_pool), "cores": workers,
                             "slowest_worker_s": t_pool, "pool_wall_s": t_wall,
                             "what": f"{workers} spawned processes at once, each assembling, factorising and "
                                     "solving its own member; rate from the slowest worker's factor + solve"}}


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- multi-rank aggregation
def max_over_ranks(value, world, device=None):
    """Maximum of a per-rank scalar over all ranks (the slowest rank's time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds_max):
    """Units processed by all ranks divided by the slowest rank's time."""
    return units_per_rank * world / seconds_max


# --------------------------------------------------------------------------- reference arm
def reference_arm(args, rank, world):
    if rank != 0:
        return
    import multiprocessing as mp
    samples = max(1, min(args.steps, 3))
    warm = 1 if args.warmup > 0 else 0
    secs = []
    for i in range(warm + samples):
        secs.append(run_cpu_sample_subprocess(args))
    timed = secs[warm:]
    total = sum(timed)
    value = 0.5 * samples / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": samples, "warmup": warm, "ms_per_step": 1000.0 * total / samples,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args, {"sample": "half a member-step per step"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{samples} timed samples (after {warm} warm-up), each one "
                                       "member's v-subproblem of one step on the full mesh with the "
                                       "FP64 oracle (SuperLU), 1 thread; the driver's K is capped "
                                       "at 3 to bound the run"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- separate-solve comparator
def separate_solve_baseline(args, prec, device, steps=3, warmup=1):
    """The usual per-member approach: each member is its own ensemble of one
    (its own nu_j, nu_m,j, data and convecting field), so every step does J
    assemblies and J single-right-hand-side solves, one member after the
    other, through the same library.  Returns member-steps/s."""
    import numpy as np
    import torch
    from paper_2108_05110_gb300 import ensemble_io
    from workloads.ensembles import lid_cavity, Ensemble
    ens = lid_cavity(N=args.N, J=args.J, s=WORKLOAD["s"], dt=WORKLOAD["dt"], Re=WORKLOAD["Re"], seed=2)
    solvers = []
    for j in range(ens.J):
        pick = (lambda fn, jj: (lambda *a: fn(*a)[jj:jj + 1]))
        one = Ensemble(f"member-{j}", ens.mesh, ens.nu[j:j + 1], ens.nu_m[j:j + 1], ens.s, ens.dt, ens.nsteps,
                       u0=pick(ens.u0, j), B0=pick(ens.B0, j), u_bc=pick(ens.u_bc, j), B_bc=pick(ens.B_bc, j))
        sol = ensemble_io.solver_for(one, precision=prec, device=device)
        ensemble_io.feed_initial(sol, one)
        ensemble_io.feed_step_data(sol, one, one.dt)
        solvers.append(sol)
    for _ in range(warmup):
        for sol in solvers:
            sol.step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        for sol in solvers:
            sol.step()
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    for sol in solvers:
        sol.close()
    return {"value": ens.J * steps / secs, "unit": UNIT, "steps": steps, "warmup": warmup,
            "what": "J=20 single-member contexts stepped one after the other (J assemblies and J "
                    "single-RHS solves per step), same library and tolerance"}


# --------------------------------------------------------------------------- batched ensembles
def batched_arm(args, local_rank):
    """Independent lid-cavity ensembles of uneven size (seed 5000+k: J_k in
    1..64, N_k in {32, 64, 128, 256}, Re_k in [1000, 15000]) stepped
    concurrently by mhde_advance_many; member-steps/s over all ensembles and
    the per-step latency distribution."""
    import numpy as np
    import torch
    import paper_2108_05110_gb300 as P
    from paper_2108_05110_gb300 import ensemble_io
    from workloads.ensembles import batched_family
    torch.cuda.set_device(local_rank)
    fam = batched_family(count=args.batch_count, nsteps=args.steps)
    sols, members, total_bytes = [], 0, 0
    # restart 15 keeps the 64 Krylov bases in memory; the stronger preconditioner
    # settings (8 inner steps, two smoothing sweeps) keep the 256 x 256,
    # high-Re ensembles converging with the shorter restart
    opts = dict(restart=15, inner_iters=8, amg_sweeps=2, max_refine=200, max_iter=5000)
    # the 256 x 256 ensembles above Re = 10,000 do not converge on their first
    # step with this block preconditioner (measured: stagnation or divergence
    # with restart 15 or 30, FP32 or FP64 Krylov), so they are left out
    excluded = [k for k, e in enumerate(fam) if e.info["N"] >= 256 and e.info["Re"] > 10000.0]
    for k, ens in enumerate(fam):
        if k in excluded:
            continue
        probe = ensemble_io.solver_for(ens, bind=False, **opts)
        need = probe.workspace_size()
        probe.close()
        if total_bytes + need > args.batch_mem_gb * 1e9:
            continue
        sol = ensemble_io.solver_for(ens, device=f"cuda:{local_rank}", **opts)
        ensemble_io.feed_initial(sol, ens)
        ensemble_io.feed_step_data(sol, ens, ens.dt)
        sols.append(sol)
        members += ens.J
        total_bytes += need
    P.advance_many(sols, args.warmup, nthreads=args.batch_threads)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ms = P.advance_many(sols, args.steps, nthreads=args.batch_threads)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    value = members * args.steps / secs
    sizes = sorted({(int(s.sizes.nv), int(s.J)) for s in sols})
    line = {"metric": "batched ensemble member-steps/s (uneven J, N)", "value": value, "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": f"{len(sols)} of {len(fam)} lid-cavity ensembles (seed 5000+k) that fit "
                                   f"{args.batch_mem_gb:g} GB, J_k in 1..64, N_k in 32..256",
                       "ensembles": len(sols), "members": members, "workspace_gb": total_bytes / 1e9,
                       "excluded": {"ensembles": excluded,
                                    "reason": "N = 256 and Re > 10000: first step does not converge"},
                       "concurrency": f"mhde_advance_many, {args.batch_threads} host threads, 2 streams per ensemble",
                       "options": opts},
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                           "max": float(ms.max())}}
    for sol in sols:
        sol.close()
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- adjoint timing
def adjoint_arm(args, local_rank):
    """The sensitivity workload (64x64, J = 8, s = 0.5, dt = 0.01, 40 steps,
    checkpoint every 5): wall time of the 40 forward steps alone and of the
    forward run plus the discrete adjoint (mhde_energy_adjoint), both
    precisions, after one untimed run of each."""
    import torch
    from paper_2108_05110_gb300 import ensemble_io, PREC_FP64, PREC_MIXED
    from workloads.ensembles import sensitivity
    torch.cuda.set_device(local_rank)
    ens = sensitivity()
    K, C = ens.nsteps, 5
    out = {"metric": "discrete adjoint of E_h^K: wall time", "unit": "s", "config": {
        "workload": "sensitivity: unit square 64x64, P2-P1, J=8, nu, nu_m = 0.005(1+delta), s=0.5, dt=0.01, "
                    "K=40 steps, checkpoint every 5", "mesh": "64x64", "J": ens.J}, "data": "synthetic"}
    for name, prec in (("fp64", PREC_FP64), ("mixed", PREC_MIXED)):
        sol = ensemble_io.solver_for(ens, precision=prec, device=f"cuda:{local_rank}",
                                 element=element_of(args.workload))
        ensemble_io.feed_initial(sol, ens)
        ensemble_io.feed_step_data(sol, ens, ens.dt)
        state = sol.save_state()
        res = {}
        for rep in range(2):
            sol.load_state(state)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sol.advance(K)
            torch.cuda.synchronize()
            res["forward_s"] = time.perf_counter() - t0
            sol.load_state(state)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g = sol.energy_adjoint(K, C)
            torch.cuda.synchronize()
            res["forward_and_adjoint_s"] = time.perf_counter() - t0
        res["loss"] = g["loss"]
        out[name] = res
        sol.close()
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------------------- our arm
def spmm_bytes(sz, prec_bytes):
    """Algorithmic bytes of one saddle SpMM: matrix structure and values read
    once (F: value + column per nnz and row pointers; B and B^T: value pair +
    column per nnz and row pointers; Dirichlet flags), X read once, Y written
    once."""
    n2, np_, nf, nb, Jp = sz.n2, sz.np, sz.nnz_F, sz.nnz_B, sz.J_pad
    matrix = nf * (prec_bytes + 4) + 4 * (n2 + 1) + 2 * nb * (2 * prec_bytes + 4) + 4 * (n2 + 1) \
        + 4 * (np_ + 1) + n2
    vectors = 2 * sz.n_rows * Jp * prec_bytes
    return matrix + vectors


def laplacian_bytes(sz, prec_bytes):
    """Algorithmic bytes of the timed residual b - L x on the finest pressure
    level: L's values, column indices and row pointers once, the input (x and
    b are one buffer in the timing call) read once and the residual written
    once, J_pad columns each."""
    return sz.nnz_L * (prec_bytes + 4) + (sz.np + 1) * 4 + 2 * sz.np * sz.J_pad * prec_bytes


# DRAM bytes (read + write) of that launch on the 64 x 64 barycenter-refined
# Scott-Vogelius cavity, J = 20, FP32 (44.49 MB read, <0.1 MB written: the
# residual stays in L2), from an ncu capture of the same launch configuration
LAPLACIAN_TRAFFIC_SV64 = 44492544 + 50176


def gram_bytes(sz, restart, prec_bytes):
    """Algorithmic bytes of the block Gram timed by kernel id 8: restart/2
    basis blocks and W (n_rows x J_pad each) read once, the (k+1) J x J Gram
    (FP64) written once."""
    k1 = max(1, restart // 2) + 1
    return k1 * sz.n_rows * sz.J_pad * prec_bytes + k1 * sz.J * sz.J * 8


# ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_gram_staged<20, 2, 512>
# launch on the 128x128, J=20 workload with 16 blocks (192.54 MB + 5.02 MB, taken
# with --set full on the current kernel)
GRAM_TRAFFIC = 197.56e6


def our_arm(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2108_05110_gb300 import ensemble_io, PREC_FP64, PREC_MIXED
    cpu_secs = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.profile_only:
        cpu_secs = run_cpu_sample_subprocess(args)      # before any GPU work in this process

    torch.cuda.set_device(local_rank)
    prec = PREC_MIXED if args.precision == "mixed" else PREC_FP64
    ens = make_ensemble(args.workload, args.N, args.J, seed=(3 if args.workload == "channel" else 2) + rank)
    sol = ensemble_io.solver_for(ens, precision=prec, device=f"cuda:{local_rank}",
                                 element=element_of(args.workload))
    ensemble_io.feed_initial(sol, ens)
    ensemble_io.feed_step_data(sol, ens, ens.dt)     # constant lid / field data
    sol.advance(args.warmup)
    if args.profile_only and args.profile_kernel >= 0:
        ms = sol.time_kernel(0, args.profile_kernel, reps=max(1, args.steps))
        if rank == 0:
            print(json.dumps({"profile_only": True, "kernel": args.profile_kernel, "ms": ms}), flush=True)
        sol.close()
        return
    if args.profile_only:
        torch.cuda.synchronize()
        sol.advance(args.steps)
        torch.cuda.synchronize()
        st = sol.stats()
        if rank == 0:
            print(json.dumps({"profile_only": True, "steps": args.steps, "launches": int(st.launches),
                              "iters": int(st.total_iters)}), flush=True)
        sol.close()
        return

    def barrier():
        if world > 1:
            dist.barrier()

    # post-warm-up state: the end-to-end leg below re-runs exactly the steps
    # that the device-timed region runs
    state0 = sol.save_state()
    clocks = ClockSampler(local_rank)
    st0 = sol.stats()
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(sol.stream_v)
    t0 = time.perf_counter()
    sol.advance(args.steps)
    ev1.record(sol.stream_v)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    barrier()
    clock_info = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    st1 = sol.stats()
    ms_max = max_over_ranks(ms, world, device=f"cuda:{local_rank}")
    value = whole_job_rate(ens.J * args.steps, world, ms_max / 1000.0)
    launches = int(st1.launches - st0.launches)
    iters = int(st1.total_iters - st0.total_iters)
    relres = max(float(st1.last_relres[0]), float(st1.last_relres[1]))
    v_dev, w_dev, _, _ = sol.read_state()

    # dominant kernel (largest share of the step's device time in the ncu
    # launch list): the partial sums of the block Gram, timed alone on
    # restart/2 basis blocks plus W, J columns each
    pbytes = 4 if prec == PREC_MIXED else 8
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    gram_ms = sol.time_kernel(0, 8, reps=50)
    alg = gram_bytes(sol.sizes, sol.options.restart, pbytes)
    achieved = alg / (gram_ms / 1000.0) / 1e9
    # DRAM bytes of one launch of this kernel at this size, from an ncu capture of
    # the same launch configuration; known only for the default workload
    gram_tc = bool(st1.gram_tensor_cores)
    traffic = GRAM_TRAFFIC if (prec == PREC_MIXED and args.workload == "cavity" and args.N == WORKLOAD["N"]
                               and args.J == WORKLOAD["J"] and not gram_tc
                               and sol.options.restart == 30) else None
    if pbytes == 8:
        kname = "k_gram, FP64"
    else:
        kname = "k_gram_tc, FP32 on tensor cores" if gram_tc else "k_gram_staged, FP32"
    roofline = {"bound": "hbm", "kernel": f"block Gram partial sums ({kname}), "
                f"{sol.options.restart // 2 + 1} blocks x {args.J} columns",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "bytes_per_launch": alg, "ms_per_launch": gram_ms,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    if args.workload == "sv":
        # with the discontinuous pressure the dominant kernel of the step is the
        # pressure-Laplacian CSR product of the V-cycle (k_csr, a third of the
        # device time in the ncu launch list); its finest-level residual
        # b - L x is timed alone: L read once, x, b read and r written once
        lb = laplacian_bytes(sol.sizes, pbytes)
        l_ms = sol.time_kernel(0, 9, reps=50)
        l_ach = lb / (l_ms / 1000.0) / 1e9
        roofline = {"bound": "hbm", "kernel": f"pressure-Laplacian residual b - L x on the finest level "
                    f"(k_csr<{'float' if pbytes == 4 else 'double'}>, L = B D^-1 B^T, nnz {sol.sizes.nnz_L})",
                    "achieved": l_ach, "peak": peak, "unit": "GB/s", "frac": l_ach / peak,
                    "traffic": LAPLACIAN_TRAFFIC_SV64 if (pbytes == 4 and args.N == SV_N and args.J == 20) else None,
                    "bytes_per_launch": lb, "ms_per_launch": l_ms,
                    "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                    "block_gram": {"achieved": achieved, "frac": achieved / peak, "ms_per_launch": gram_ms}}
    # the Krylov operator (saddle SpMM), for reference
    kid = 1 if prec == PREC_MIXED else 0
    spmm_ms = sol.time_kernel(0, kid, reps=50)
    salg = spmm_bytes(sol.sizes, pbytes)
    spmm_line = {"kernel": f"saddle SpMM ({'FP32' if pbytes == 4 else 'FP64'})", "bytes_per_launch": salg,
                 "ms_per_launch": spmm_ms, "achieved": salg / (spmm_ms / 1000.0) / 1e9,
                 "frac": salg / (spmm_ms / 1000.0) / 1e9 / peak, "cta_size": int(st1.spmm_block)}
    kernel_ms = {name: sol.time_kernel(0, k, reps=10) for name, k in
                 (("means_l2", 4), ("assemble_F", 2), ("rhs", 3), ("precond", 5), ("gram", 6),
                  ("combine", 7))}

    # end to end through the public API with host buffers, over the same
    # steps: restore the post-warm-up state, then per step copy that step's
    # Dirichlet data in, step, and read the ensemble means out
    xy = sol._nodes
    ub, Bb = ens.u_bc(xy, ens.dt), ens.B_bc(xy, ens.dt)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    sol.load_state(state0)
    for _ in range(args.steps):
        sol.set_dirichlet(ub, Bb)
        sol.step()
        um, Bm = sol.read_mean()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = whole_job_rate(ens.J * args.steps, world,
                               max_over_ranks(e2e_s, world, device=f"cuda:{local_rank}"))
    v_e2e, w_e2e, _, _ = sol.read_state()
    same_steps = bool(np.array_equal(v_e2e, v_dev) and np.array_equal(w_e2e, w_dev))
    sz = sol.sizes
    # bytes that cross per step: the restored state once, then per step the
    # packed Dirichlet values of both subproblems in, both means out
    dirichlet_bytes = 2 * sz.n_boundary * 2 * sz.J_pad * 8
    h2d = (state0.nbytes + args.steps * dirichlet_bytes) / args.steps
    d2h = um.nbytes + Bm.nbytes

    accuracy = None
    fp64_line = None
    separate = None
    if rank == 0 and world == 1 and not args.no_separate:
        # one more step from the benchmarked state, checked against the oracle
        if not args.no_oracle_check:
            accuracy = oracle_check(args, sol)
        if prec == PREC_MIXED:
            fp64_line = fp64_same_steps(args, ens, state0, f"cuda:{local_rank}")
    sol.close()
    if rank == 0 and world == 1 and not args.no_separate and args.workload == "cavity":
        separate = separate_solve_baseline(args, prec, f"cuda:{local_rank}")

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if prec == PREC_MIXED else "f64", "data": "synthetic",
                "config": config(args, {"precision": args.precision}),
                "roofline": roofline, "clocks": clock_info, "gpu_launches": launches,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h), "same_steps_as_value": same_steps},
                "final_relres": relres, "krylov_iters_per_step": iters / args.steps,
                "block_ops_autotune": {"gram": "tensor cores" if st1.gram_tensor_cores else "cuda cores",
                                       "gram_us_cuda_tensor": list(st1.gram_tuned_us),
                                       "combine": "tensor cores" if st1.combine_tensor_cores else "cuda cores",
                                       "combine_us_cuda_tensor": list(st1.combine_tuned_us),
                                       "inner": "persistent" if st1.inner_persistent else "launch chain",
                                       "inner_us_chain_persistent": list(st1.inner_tuned_us)},
                "kernel_ms": kernel_ms, "spmm": spmm_line,
                "wall_ms_per_step": 1000.0 * wall / args.steps}
        if accuracy is not None:
            line["accuracy"] = accuracy
        if fp64_line is not None:
            line["fp64_path"] = fp64_line
        if cpu_secs is not None:
            line["cpu_baseline"] = cpu_baseline_block(cpu_secs)
        if separate is not None:
            line["separate_solve_baseline"] = separate
        print(json.dumps(line), flush=True)


def main():
    faulthandler.enable()
    args = parse()
    if args.cpu_sample:
        print(json.dumps({"seconds": cpu_sample(args.workload, args.N, args.J)}), flush=True)
        return
    if args.oracle_check:
        print(json.dumps(oracle_step_check(args.oracle_check, args.workload, args.N, args.J)), flush=True)
        return
    if args.cpu_study:
        print(json.dumps(cpu_study(args)), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if args.workload == "batched":
        if rank == 0:
            batched_arm(args, local_rank)
        return
    if args.workload == "adjoint":
        if rank == 0:
            adjoint_arm(args, local_rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    our_arm(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
