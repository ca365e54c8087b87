"""ctypes binding of libmhde (include/mhde.h) with the same function names.

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch provides the device workspace (one uint8 tensor) and
the two CUDA streams of the v and w subproblems.  There is no CPU fallback:
a missing library or a missing GPU raises.
"""
import atexit
import ctypes as C
import os
import re
import weakref

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "..", "include", "mhde.h")
PREC_FP64, PREC_MIXED = 0, 1

ERRORS = {0: "MHDE_OK", -1: "MHDE_EINVAL", -2: "MHDE_ESTAB", -3: "MHDE_ENOCONV", -4: "MHDE_ENAN",
          -5: "MHDE_ECUDA", -6: "MHDE_EWORKSPACE", -7: "MHDE_ESTATE"}


class MhdeError(RuntimeError):
    def __init__(self, code, where, msg=""):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} {msg}".strip())


class Mesh(C.Structure):
    _fields_ = [("nv", C.c_int), ("nt", C.c_int), ("xy", C.POINTER(C.c_double)),
                ("tri", C.POINTER(C.c_int))]


class Options(C.Structure):
    _fields_ = [("mu", C.c_double), ("conv_form", C.c_int), ("precision", C.c_int),
                ("rtol", C.c_double), ("inner_rtol", C.c_double), ("restart", C.c_int),
                ("max_iter", C.c_int), ("max_refine", C.c_int), ("jacobi_sweeps", C.c_int),
                ("jacobi_omega", C.c_double), ("amg_sweeps", C.c_int), ("amg_cycles", C.c_int),
                ("inner_iters", C.c_int),
                ("schur", C.c_int), ("strict", C.c_int), ("inner_fp16", C.c_int),
                ("element", C.c_int)]

ELEMENTS = {"TH": 0, "SV": 1}     # Taylor-Hood P2/P1, Scott-Vogelius P2/P1disc


class Sizes(C.Structure):
    _fields_ = [("nv", C.c_int), ("nt", C.c_int), ("ne", C.c_int), ("n2", C.c_int), ("np", C.c_int),
                ("n_rows", C.c_int), ("J", C.c_int), ("J_pad", C.c_int), ("nnz_F", C.c_longlong),
                ("nnz_B", C.c_longlong), ("nnz_saddle", C.c_longlong), ("n_boundary", C.c_int),
                ("amg_levels", C.c_int), ("nnz_L", C.c_longlong), ("smoother_block", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("steps", C.c_longlong), ("last_iters", C.c_int * 2), ("last_refine", C.c_int * 2),
                ("last_relres", C.c_double * 2), ("total_iters", C.c_longlong),
                ("last_step_ms", C.c_double), ("launches", C.c_longlong),
                ("spmm_block", C.c_int), ("spmm_tuned_us", C.c_double * 3),
                ("gram_tensor_cores", C.c_int), ("combine_tensor_cores", C.c_int),
                ("gram_tuned_us", C.c_double * 2), ("combine_tuned_us", C.c_double * 2),
                ("inner_persistent", C.c_int), ("inner_tuned_us", C.c_double * 2)]


def library_path():
    return os.path.join(HERE, "libmhde.so")


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_U8 = C.POINTER(C.c_ubyte)
SIGNATURES = {
    "mhde_default_options": (None, [C.POINTER(Options)]),
    "mhde_create": (C.c_int, [C.POINTER(Mesh), C.c_int, _D, _D, C.c_double, C.c_double,
                              C.POINTER(Options), C.POINTER(_P)]),
    "mhde_get_sizes": (C.c_int, [_P, C.POINTER(Sizes)]),
    "mhde_workspace_size": (C.c_int, [_P, C.POINTER(C.c_size_t)]),
    "mhde_bind": (C.c_int, [_P, _P, C.c_size_t, _P, _P]),
    "mhde_p2_nodes": (C.c_int, [_P, _D, _U8]),
    "mhde_set_initial": (C.c_int, [_P, _D, _D]),
    "mhde_set_forcing": (C.c_int, [_P, _D, _D]),
    "mhde_set_viscosity": (C.c_int, [_P, _D, _D]),
    "mhde_adjoint_workspace_size": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
    "mhde_energy_adjoint": (C.c_int, [_P, C.c_int, C.c_int, _P, C.c_size_t, _D, _D, _D, _D, _D]),
    "mhde_set_dirichlet": (C.c_int, [_P, _D, _D]),
    "mhde_step": (C.c_int, [_P]),
    "mhde_advance": (C.c_int, [_P, C.c_int]),
    "mhde_advance_many": (C.c_int, [C.POINTER(_P), C.c_int, C.c_int, C.c_int, _D]),
    "mhde_read_mean": (C.c_int, [_P, _D, _D]),
    "mhde_read_state": (C.c_int, [_P, _D, _D, _D, _D]),
    "mhde_read_member": (C.c_int, [_P, C.c_int, _D, _D, _D, _D]),
    "mhde_energy": (C.c_int, [_P, _D]),
    "mhde_get_stats": (C.c_int, [_P, C.POINTER(Stats)]),
    "mhde_state_bytes": (C.c_int, [_P, C.POINTER(C.c_size_t)]),
    "mhde_save_state": (C.c_int, [_P, _P]),
    "mhde_load_state": (C.c_int, [_P, _P]),
    "mhde_last_error": (C.c_char_p, [_P]),
    "mhde_destroy": (None, [_P]),
    "mhde_probe_mean_l2": (C.c_int, [_P, _D, _D, _D, _D]),
    "mhde_probe_matrix_F": (C.c_int, [_P, C.c_int, _I, _I, _D]),
    "mhde_probe_laplacian": (C.c_int, [_P, _I, _I, _D]),
    "mhde_probe_amg_level": (C.c_int, [_P, C.c_int, C.POINTER(C.c_longlong), _D, _I, _I, _D, _I, _I, _D, _I, _I,
                                       _D, _I, _D]),
    "mhde_probe_rhs": (C.c_int, [_P, C.c_int, _D]),
    "mhde_probe_spmm": (C.c_int, [_P, C.c_int, C.c_int, _D, _D]),
    "mhde_probe_inner": (C.c_int, [_P, C.c_int, C.c_int, _D, _D]),
    "mhde_time_kernel": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _D]),
    "mhde_block_gram_scratch_bytes": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
    "mhde_block_gram": (C.c_int, [_P, C.c_size_t, C.c_int, _P, C.c_int, C.c_int, C.c_int, _P, _P,
                                  C.c_size_t, _P]),
    "mhde_block_gram_noalloc": (C.c_int, [_P, C.c_size_t, C.c_int, _P, C.c_int, C.c_int, C.c_int, _P, _P]),
    "mhde_block_gram_f32_scratch_bytes": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
    "mhde_block_gram_f32": (C.c_int, [_P, C.c_size_t, C.c_int, _P, C.c_int, C.c_int, C.c_int, _P, _P, C.c_size_t,
                                      C.c_int, _P]),
    "mhde_fp64_fma_rate": (C.c_int, [_P, C.POINTER(C.c_double)]),
    "mhde_block_combine_f32": (C.c_int, [_P, _P, C.c_float, _P, C.c_size_t, C.c_int, C.c_int, _P, C.c_int, C.c_int,
                                         C.c_int, C.c_int, _P, C.c_size_t, C.c_int, _P]),
}


def declared_functions(header=HEADER):
    """Names of the functions declared in include/mhde.h."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mhde_[A-Za-z0-9_]+)\s*\(", text)))


class Library:
    def __init__(self, path=None):
        path = path or library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libmhde is not built ({path}); run __graft_entry__.build()")
        self.path = path
        self.lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(self.lib, name)
            fn.restype = res
            fn.argtypes = args

    def __getattr__(self, name):
        if name.startswith("mhde_"):
            return getattr(self.lib, name)
        raise AttributeError(name)


_LIB = None


def load_library():
    global _LIB
    if _LIB is None:
        _LIB = Library()
    return _LIB


def _dptr(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def default_options(**kw):
    """mhde_default_options with fields replaced by keyword.  ``element`` may
    be given as "TH" / "SV"; unless given otherwise, the Scott-Vogelius
    element takes the Cahouet-Chabard Schur approximation (schur = 0) with
    two smoothing sweeps per level (amg_sweeps = 2): on the 64 x 64
    barycenter-refined cavity ensemble (J = 20) 240 ms per step against 275
    ms with one sweep and 400 ms for the least-squares commutator (schur = 2,
    two sweeps and two cycles), which takes fewer iterations (313 against
    416) at twice the cost per application."""
    lib = load_library()
    o = Options()
    lib.mhde_default_options(C.byref(o))
    kw = dict(kw)
    if isinstance(kw.get("element"), str):
        kw["element"] = ELEMENTS[kw["element"]]
    if kw.get("element", 0) == 1:
        kw.setdefault("schur", 0)
        kw.setdefault("amg_sweeps", 2)
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def advance_many(solvers, nsteps, nthreads=8):
    """Step independent ensembles concurrently through mhde_advance_many;
    returns per-step wall times [len(solvers), nsteps] in ms."""
    lib = load_library()
    arr = (_P * len(solvers))(*[s.ctx for s in solvers])
    ms = np.zeros((len(solvers), nsteps))
    rc = lib.mhde_advance_many(arr, len(solvers), int(nsteps), int(nthreads), _dptr(ms))
    if rc != 0:
        raise MhdeError(rc, "mhde_advance_many")
    return ms


def block_gram(V, W, kblocks, r, stream=None):
    """G_i = V_i^T W through mhde_block_gram.  V: torch float64 CUDA tensor
    [kblocks, n_rows, ld], W: [n_rows, ld]; returns a torch tensor
    [kblocks, r, r].  Scratch comes from torch."""
    import torch
    lib = load_library()
    k, n_rows, ld = V.shape
    nbytes = C.c_size_t()
    rc = lib.mhde_block_gram_scratch_bytes(n_rows, r, kblocks, C.byref(nbytes))
    if rc != 0:
        raise MhdeError(rc, "mhde_block_gram_scratch_bytes")
    scratch = torch.empty(max(int(nbytes.value), 1), dtype=torch.uint8, device=V.device)
    G = torch.empty((kblocks, r, r), dtype=torch.float64, device=V.device)
    st = stream if stream is not None else torch.cuda.current_stream(V.device)
    rc = lib.mhde_block_gram(C.c_void_p(V.data_ptr()), n_rows * ld, kblocks, C.c_void_p(W.data_ptr()), n_rows,
                             ld, r, C.c_void_p(G.data_ptr()), C.c_void_p(scratch.data_ptr()), nbytes.value,
                             C.c_void_p(st.cuda_stream))
    if rc != 0:
        raise MhdeError(rc, "mhde_block_gram")
    return G


def block_gram_f32(V, W, kblocks, r, tensor_cores=True, stream=None):
    """G_i = V_i^T W (FP64 result) from FP32 blocks through mhde_block_gram_f32:
    V torch float32 CUDA tensor [kblocks, n_rows, ld], W [n_rows, ld]; the
    tensor-core kernel or the CUDA-core kernels.  Scratch comes from torch."""
    import torch
    lib = load_library()
    k, n_rows, ld = V.shape
    nbytes = C.c_size_t()
    rc = lib.mhde_block_gram_f32_scratch_bytes(n_rows, r, kblocks, C.byref(nbytes))
    if rc != 0:
        raise MhdeError(rc, "mhde_block_gram_f32_scratch_bytes")
    scratch = torch.empty(int(nbytes.value), dtype=torch.uint8, device=V.device)
    G = torch.empty((kblocks, r, r), dtype=torch.float64, device=V.device)
    st = stream if stream is not None else torch.cuda.current_stream(V.device)
    rc = lib.mhde_block_gram_f32(C.c_void_p(V.data_ptr()), n_rows * ld, kblocks, C.c_void_p(W.data_ptr()), n_rows,
                                 ld, r, C.c_void_p(G.data_ptr()), C.c_void_p(scratch.data_ptr()), nbytes.value,
                                 1 if tensor_cores else 0, C.c_void_p(st.cuda_stream))
    if rc != 0:
        raise MhdeError(rc, "mhde_block_gram_f32")
    return G


def block_combine_f32(out, V, coef, r_in, r_out, in_=None, alpha=0.0, v_stride=None, tensor_cores=True,
                      stream=None):
    """out = alpha in + sum_i V_i coef_i through mhde_block_combine_f32.  V:
    torch float32 CUDA tensor whose leading dimension holds the blocks ([k,
    n_rows, ldv]; or give v_stride in elements); coef: float32 [k, r_in,
    r_out]; out / in_: float32 [n_rows, ldo] (may alias each other or a
    block of V)."""
    import torch
    lib = load_library()
    k = coef.shape[0]
    n_rows, ldo = out.shape
    ldv = V.shape[-1]
    if v_stride is None:
        v_stride = V.shape[1] * ldv
    scratch = torch.empty(256, dtype=torch.uint8, device=out.device)
    st = stream if stream is not None else torch.cuda.current_stream(out.device)
    ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
    rc = lib.mhde_block_combine_f32(ptr(out), ptr(in_), float(alpha), ptr(V), int(v_stride), int(k), int(r_in),
                                    ptr(coef), int(r_out), int(n_rows), int(ldv), int(ldo), ptr(scratch), 256,
                                    1 if tensor_cores else 0, C.c_void_p(st.cuda_stream))
    if rc != 0:
        raise MhdeError(rc, "mhde_block_combine_f32")
    return out


def fp64_fma_rate(stream=None):
    """Measured FP64 FMA rate of the current device (TFLOP/s), mhde_fp64_fma_rate."""
    import torch
    lib = load_library()
    st = stream if stream is not None else torch.cuda.current_stream()
    out = C.c_double()
    rc = lib.mhde_fp64_fma_rate(C.c_void_p(st.cuda_stream), C.byref(out))
    if rc != 0:
        raise MhdeError(rc, "mhde_fp64_fma_rate")
    return out.value


def block_gram_noalloc(V, W, kblocks, r, G=None, stream=None):
    """G_i = V_i^T W through mhde_block_gram_noalloc, which uses the library's
    fixed device scratch instead of allocating.  V: torch float64 CUDA
    tensor [kblocks, n_rows, ld], W: [n_rows, ld]; G: optional output
    [kblocks, r, r] (the caller's memory)."""
    import torch
    lib = load_library()
    k, n_rows, ld = V.shape
    if G is None:
        G = torch.empty((kblocks, r, r), dtype=torch.float64, device=V.device)
    st = stream if stream is not None else torch.cuda.current_stream(V.device)
    rc = lib.mhde_block_gram_noalloc(C.c_void_p(V.data_ptr()), n_rows * ld, kblocks, C.c_void_p(W.data_ptr()),
                                     n_rows, ld, r, C.c_void_p(G.data_ptr()), C.c_void_p(st.cuda_stream))
    if rc != 0:
        raise MhdeError(rc, "mhde_block_gram_noalloc")
    return G


_LIVE = weakref.WeakSet()


def _close_live_solvers():
    """Destroy the contexts still open at interpreter exit, before the CUDA
    runtime and torch's streams are torn down."""
    for s in list(_LIVE):
        try:
            s.close()
        except Exception:
            pass


atexit.register(_close_live_solvers)


class EnsembleSolver:
    """One ensemble (mesh, J members) on one GPU, through the C ABI.

    ``bind=False`` builds the host-side structure only (no GPU needed), which
    is what the CPU tests use to check numbering and sizes.
    """

    def __init__(self, xy, tri, nu, nu_m, s, dt, options=None, bind=True, device=None, **opt_kw):
        self.lib = load_library()
        xy = _f64(xy)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        self._keep = (xy, tri)
        mesh = Mesh(xy.shape[0], tri.shape[0], xy.ctypes.data_as(_D), tri.ctypes.data_as(_I))
        nu = _f64(nu).ravel()
        nu_m = _f64(nu_m).ravel()
        self.J = nu.shape[0]
        self.s = float(s)
        opts = options if options is not None else default_options(**opt_kw)
        self.options = opts
        ctx = _P()
        rc = self.lib.mhde_create(C.byref(mesh), self.J, _dptr(nu), _dptr(nu_m), float(s), float(dt),
                                  C.byref(opts), C.byref(ctx))
        if rc != 0:
            raise MhdeError(rc, "mhde_create")
        self.ctx = ctx
        _LIVE.add(self)
        self.sizes = Sizes()
        self._check(self.lib.mhde_get_sizes(self.ctx, C.byref(self.sizes)), "mhde_get_sizes")
        self.bound = False
        if bind:
            self.bind(device)

    # ------------------------------------------------------------------ plumbing
    def _check(self, rc, where):
        if rc != 0:
            msg = self.lib.mhde_last_error(self.ctx) if getattr(self, "ctx", None) else b""
            raise MhdeError(rc, where, (msg or b"").decode())

    def bind(self, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libmhde needs a CUDA device; none is available")
        dev = torch.device(device or "cuda:0")
        torch.cuda.set_device(dev)
        nbytes = C.c_size_t()
        self._check(self.lib.mhde_workspace_size(self.ctx, C.byref(nbytes)), "mhde_workspace_size")
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=dev)
        self.stream_v = torch.cuda.Stream(device=dev)
        self.stream_w = torch.cuda.Stream(device=dev)
        self._check(self.lib.mhde_bind(self.ctx, C.c_void_p(self.workspace.data_ptr()), nbytes.value,
                                       C.c_void_p(self.stream_v.cuda_stream),
                                       C.c_void_p(self.stream_w.cuda_stream)), "mhde_bind")
        self.bound = True
        self.workspace_bytes = int(nbytes.value)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.mhde_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ mesh
    @property
    def n2(self):
        return self.sizes.n2

    @property
    def np_(self):
        return self.sizes.np

    def p2_nodes(self):
        xy = np.empty((self.n2, 2))
        isb = np.empty(self.n2, dtype=np.uint8)
        self._check(self.lib.mhde_p2_nodes(self.ctx, _dptr(xy), isb.ctypes.data_as(_U8)), "mhde_p2_nodes")
        return xy, isb.astype(bool)

    def workspace_size(self):
        nbytes = C.c_size_t()
        self._check(self.lib.mhde_workspace_size(self.ctx, C.byref(nbytes)), "mhde_workspace_size")
        return int(nbytes.value)

    # ------------------------------------------------------------------ data
    def set_initial(self, u0, B0=None):
        shp = (self.J, self.n2, 2)
        u0, B0 = _f64(u0, shp), _f64(B0, shp)
        self._check(self.lib.mhde_set_initial(self.ctx, _dptr(u0), _dptr(B0)), "mhde_set_initial")

    def set_forcing(self, f=None, curl_g=None):
        shp = (self.J, self.n2, 2)
        f, cg = _f64(f, shp), _f64(curl_g, shp)
        self._check(self.lib.mhde_set_forcing(self.ctx, _dptr(f), _dptr(cg)), "mhde_set_forcing")

    def set_dirichlet(self, u_bc=None, B_bc=None):
        shp = (self.J, self.n2, 2)
        u, B = _f64(u_bc, shp), _f64(B_bc, shp)
        self._check(self.lib.mhde_set_dirichlet(self.ctx, _dptr(u), _dptr(B)), "mhde_set_dirichlet")

    def set_viscosity(self, nu, nu_m):
        nu = np.ascontiguousarray(nu, dtype=np.float64).reshape(self.J)
        nu_m = np.ascontiguousarray(nu_m, dtype=np.float64).reshape(self.J)
        self._check(self.lib.mhde_set_viscosity(self.ctx, _dptr(nu), _dptr(nu_m)), "mhde_set_viscosity")

    # ------------------------------------------------------------------ adjoint
    def energy_adjoint(self, nsteps, checkpoint_every=5):
        """L = E_h after ``nsteps`` steps from the current state and its
        gradient (mhde_energy_adjoint): dict with loss, grad_nu, grad_nu_m
        [J] and grad_u0, grad_B0 [J, n2, 2].  The device workspace is a torch
        tensor held for the call."""
        import torch
        nbytes = C.c_size_t()
        self._check(self.lib.mhde_adjoint_workspace_size(self.ctx, int(nsteps), int(checkpoint_every),
                                                         C.byref(nbytes)), "mhde_adjoint_workspace_size")
        ws = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.workspace.device)
        loss = C.c_double()
        gnu, gnum = np.empty(self.J), np.empty(self.J)
        gu, gB = np.empty((self.J, self.n2, 2)), np.empty((self.J, self.n2, 2))
        torch.cuda.synchronize(self.workspace.device)
        self._check(self.lib.mhde_energy_adjoint(self.ctx, int(nsteps), int(checkpoint_every),
                                                 C.c_void_p(ws.data_ptr()), nbytes.value, C.byref(loss),
                                                 _dptr(gnu), _dptr(gnum), _dptr(gu), _dptr(gB)),
                    "mhde_energy_adjoint")
        del ws
        return {"loss": loss.value, "grad_nu": gnu, "grad_nu_m": gnum, "grad_u0": gu, "grad_B0": gB}

    # ------------------------------------------------------------------ stepping
    def step(self):
        self._check(self.lib.mhde_step(self.ctx), "mhde_step")

    def advance(self, nsteps):
        self._check(self.lib.mhde_advance(self.ctx, int(nsteps)), "mhde_advance")

    # ------------------------------------------------------------------ read-out
    def read_mean(self, with_B=True):
        u = np.empty((self.n2, 2))
        B = np.empty((self.n2, 2)) if with_B else None
        self._check(self.lib.mhde_read_mean(self.ctx, _dptr(u), _dptr(B)), "mhde_read_mean")
        return u, B

    def read_state(self):
        v = np.empty((self.J, self.n2, 2))
        w = np.empty((self.J, self.n2, 2))
        q = np.empty((self.J, self.np_))
        r = np.empty((self.J, self.np_))
        self._check(self.lib.mhde_read_state(self.ctx, _dptr(v), _dptr(w), _dptr(q), _dptr(r)),
                    "mhde_read_state")
        return v, w, q, r

    def read_member(self, j):
        u = np.empty((self.n2, 2))
        p = np.empty(self.np_)
        B = np.empty((self.n2, 2)) if self.s > 0 else None
        lam = np.empty(self.np_) if self.s > 0 else None
        self._check(self.lib.mhde_read_member(self.ctx, int(j), _dptr(u), _dptr(B), _dptr(p), _dptr(lam)),
                    "mhde_read_member")
        return u, B, p, lam

    def energy(self):
        e = C.c_double()
        self._check(self.lib.mhde_energy(self.ctx, C.byref(e)), "mhde_energy")
        return e.value

    def stats(self):
        st = Stats()
        self._check(self.lib.mhde_get_stats(self.ctx, C.byref(st)), "mhde_get_stats")
        return st

    def save_state(self):
        nb = C.c_size_t()
        self._check(self.lib.mhde_state_bytes(self.ctx, C.byref(nb)), "mhde_state_bytes")
        buf = np.empty(nb.value, dtype=np.uint8)
        self._check(self.lib.mhde_save_state(self.ctx, C.c_void_p(buf.ctypes.data)), "mhde_save_state")
        return buf

    def load_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(self.lib.mhde_load_state(self.ctx, C.c_void_p(buf.ctypes.data)), "mhde_load_state")

    # ------------------------------------------------------------------ probes
    def probe_mean_l2(self):
        nt = self.sizes.nt
        mv, mw = np.empty((self.n2, 2)), np.empty((self.n2, 2))
        lv, lw = np.empty((nt, 7)), np.empty((nt, 7))
        self._check(self.lib.mhde_probe_mean_l2(self.ctx, _dptr(mv), _dptr(mw), _dptr(lv), _dptr(lw)),
                    "mhde_probe_mean_l2")
        return mv, mw, lv, lw

    def probe_matrix_F(self, which):
        rp = np.empty(self.n2 + 1, dtype=np.int32)
        col = np.empty(self.sizes.nnz_F, dtype=np.int32)
        val = np.empty(self.sizes.nnz_F)
        self._check(self.lib.mhde_probe_matrix_F(self.ctx, int(which), rp.ctypes.data_as(_I),
                                                 col.ctypes.data_as(_I), _dptr(val)), "mhde_probe_matrix_F")
        return rp, col, val

    def probe_laplacian(self):
        """Finest pressure-Laplacian operator (host data; works before bind)."""
        np_ = self.sizes.np
        rp = np.empty(np_ + 1, dtype=np.int32)
        col = np.empty(self.sizes.nnz_L, dtype=np.int32)
        val = np.empty(self.sizes.nnz_L)
        self._check(self.lib.mhde_probe_laplacian(self.ctx, rp.ctypes.data_as(_I), col.ctypes.data_as(_I),
                                                  _dptr(val)), "mhde_probe_laplacian")
        return rp, col, val

    def probe_amg_level(self, level):
        """One level of the pressure-Laplacian hierarchy (host data; works
        before bind): dict with A, P, R (scipy CSR; P, R None on the coarsest
        level), omega, block size bs, block damping, blk_idx, blk_inv, levels."""
        import scipy.sparse as sp
        counts = (C.c_longlong * 6)()
        scal = (C.c_double * 2)()
        self._check(self.lib.mhde_probe_amg_level(self.ctx, int(level), counts, scal, *([None] * 11)),
                    "mhde_probe_amg_level")
        n, nnzA, nnzP, nnzR, bs, nlev = (int(v) for v in counts)
        nxt = None
        if nnzP:
            c2 = (C.c_longlong * 6)()
            self._check(self.lib.mhde_probe_amg_level(self.ctx, int(level) + 1, c2, None, *([None] * 11)),
                        "mhde_probe_amg_level")
            nxt = int(c2[0])
        arr = {}
        for name, rows, nnz in (("A", n, nnzA), ("P", n, nnzP), ("R", nxt or 0, nnzR)):
            arr[name] = (np.zeros(rows + 1, dtype=np.int32), np.zeros(nnz, dtype=np.int32), np.zeros(nnz))
        bidx = np.zeros(n if bs else 0, dtype=np.int32)
        binv = np.zeros((n // bs) * bs * bs if bs else 0)
        ptrs = []
        for name in ("A", "P", "R"):
            rp, col, val = arr[name]
            ptrs += [rp.ctypes.data_as(_I), col.ctypes.data_as(_I), _dptr(val)]
        self._check(self.lib.mhde_probe_amg_level(self.ctx, int(level), counts, scal, *ptrs,
                                                  bidx.ctypes.data_as(_I), _dptr(binv)), "mhde_probe_amg_level")
        A = sp.csr_matrix((arr["A"][2], arr["A"][1], arr["A"][0]), shape=(n, n))
        P = sp.csr_matrix((arr["P"][2], arr["P"][1], arr["P"][0]), shape=(n, nxt)) if nnzP else None
        R = sp.csr_matrix((arr["R"][2], arr["R"][1], arr["R"][0]), shape=(nxt, n)) if nnzP else None
        return {"A": A, "P": P, "R": R, "omega": scal[0], "bs": bs, "blk_omega": scal[1],
                "blk_idx": bidx, "blk_inv": binv.reshape(-1, bs, bs) if bs else None, "levels": nlev}

    def probe_rhs(self, which):
        out = np.empty((self.J, self.n2, 2))
        self._check(self.lib.mhde_probe_rhs(self.ctx, int(which), _dptr(out)), "mhde_probe_rhs")
        return out

    def time_kernel(self, which, kernel, reps=20):
        ms = C.c_double()
        self._check(self.lib.mhde_time_kernel(self.ctx, int(which), int(kernel), int(reps), C.byref(ms)),
                    "mhde_time_kernel")
        return ms.value

    def probe_inner(self, which, R, form=0):
        """Inner solve of the velocity block (mixed path): R, Z [J][2][n2];
        form 0 the launch chain, 1 the persistent kernel."""
        R = _f64(R, (self.J, 2, self.sizes.n2))
        Z = np.empty_like(R)
        self._check(self.lib.mhde_probe_inner(self.ctx, int(which), int(form), _dptr(R), _dptr(Z)),
                    "mhde_probe_inner")
        return Z

    def probe_spmm(self, which, X, precision=0):
        X = _f64(X, (self.J, self.sizes.n_rows))
        Y = np.empty_like(X)
        self._check(self.lib.mhde_probe_spmm(self.ctx, int(which), int(precision), _dptr(X), _dptr(Y)),
                    "mhde_probe_spmm")
        return Y
