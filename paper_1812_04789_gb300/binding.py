"""ctypes binding of libdgpmg.so (the C ABI of include/dg.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device buffers are passed as integer device pointers, or as torch
CUDA tensors (contiguous float64), whose data_ptr() is taken.  The library is
loaded on first use and a missing library raises: there is no CPU path.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdgpmg.so")

DG_OK, DG_ERR_INVALID, DG_ERR_OOM, DG_ERR_CUDA, DG_ERR_NONPHYSICAL = 0, 1, 2, 3, 4
DG_ERR_NOT_CONVERGED, DG_ERR_BREAKDOWN, DG_ERR_TIMEOUT, DG_ERR_UNSUPPORTED = 5, 6, 7, 8
STATUS_NAMES = {0: "DG_OK", 1: "DG_ERR_INVALID", 2: "DG_ERR_OOM", 3: "DG_ERR_CUDA",
                4: "DG_ERR_NONPHYSICAL", 5: "DG_ERR_NOT_CONVERGED", 6: "DG_ERR_BREAKDOWN",
                7: "DG_ERR_TIMEOUT", 8: "DG_ERR_UNSUPPORTED"}
JVP_EXACT, JVP_FD, JVP_FD_SCALED, JVP_EXACT_FP32 = 0, 1, 2, 3
CYCLE_FMG, CYCLE_V, CYCLE_BJ = 0, 1, 2
PREC_FP64, PREC_MIXED = 0, 1
SPACE_P, SPACE_Q = 0, 1
BLOCKS_DIAG_INV, BLOCKS_NEIGHBOUR, BLOCKS_DIAG = 0, 1, 2
COARSE_BJ, COARSE_BILU = 0, 1
ORDER_MDF, ORDER_NATURAL, ORDER_COLOUR = 0, 1, 2
STORE_NATIVE, STORE_BF16 = 0, 1
KT_FACE_JVP, KT_VOLUME_JVP, KT_BLOCK_JACOBI, KT_OPERATOR, KT_SMOOTH = 0, 1, 2, 3, 4

EXPORTED = ["dg_mesh_create", "dg_mesh_destroy", "dg_mesh_info", "dg_residual", "dg_jvp",
            "dg_pmg_setup", "dg_pmg_apply", "dg_pmg_destroy", "dg_fgmres_step", "dg_status_sync",
            "dg_pmg_bytes", "dg_pmg_export_blocks", "dg_bdf2_rhs", "dg_axpy", "dg_launch_count", "dg_pmg_refresh", "dg_residual_noalloc",
            "dg_esdirk3_rhs", "dg_esdirk3_step", "dg_bilu_order", "dg_pmg_bilu_order", "dg_mesh_create_tri",
            "dg_pmg_operator", "dg_pmg_kernel_time"]


class DGError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__("%s returned %s" % (fn, STATUS_NAMES.get(code, code)))
        self.code = code


class MeshDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("p", ctypes.c_int), ("nq1d", ctypes.c_int),
                ("space", ctypes.c_int)]


class TriDesc(ctypes.Structure):
    _fields_ = [("n_vert", ctypes.c_int), ("X", ctypes.POINTER(ctypes.c_double)), ("n_tri", ctypes.c_int),
                ("tri", ctypes.POINTER(ctypes.c_int)), ("shift", ctypes.POINTER(ctypes.c_int)),
                ("lo", ctypes.c_double * 2), ("hi", ctypes.c_double * 2), ("p", ctypes.c_int),
                ("nq1d", ctypes.c_int)]


class PhysicsDesc(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("Pr", ctypes.c_double), ("mu", ctypes.c_double),
                ("Rgas", ctypes.c_double), ("eta_br2", ctypes.c_double), ("roe_delta", ctypes.c_double)]


class PmgOpts(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int), ("p_level", ctypes.c_int * 8), ("nu_pre", ctypes.c_int * 8),
                ("nu_post", ctypes.c_int * 8), ("nu_coarse", ctypes.c_int), ("cycle", ctypes.c_int),
                ("precision", ctypes.c_int), ("fgmres_restart", ctypes.c_int), ("coarse_precond", ctypes.c_int),
                ("coarse_order", ctypes.c_int), ("block_storage", ctypes.c_int)]


class KrylovOpts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("max_restarts", ctypes.c_int), ("rtol", ctypes.c_double),
                ("atol", ctypes.c_double), ("jvp_mode", ctypes.c_int)]


class KrylovStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("res0", ctypes.c_double), ("res_final", ctypes.c_double),
                ("rho", ctypes.c_double), ("status", ctypes.c_int), ("ms_total", ctypes.c_float),
                ("ms_setup", ctypes.c_float)]


_lib = None
P = ctypes.c_void_p


def load(path=None):
    """Load the shared library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libdgpmg.so not found at %s: build it with "
                           "paper_1812_04789_gb300.build.build() (there is no CPU fallback)" % path)
    lib = ctypes.CDLL(path)
    sig = {
        "dg_mesh_create": [ctypes.POINTER(MeshDesc), ctypes.POINTER(PhysicsDesc), P, ctypes.POINTER(P)],
        "dg_mesh_destroy": [P],
        "dg_mesh_info": [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_size_t)],
        "dg_residual": [P, P, P, P, P],
        "dg_jvp": [P, P, P, ctypes.c_double, P, P, ctypes.c_int, P],
        "dg_pmg_setup": [P, P, ctypes.c_double, ctypes.POINTER(PmgOpts), P, ctypes.POINTER(P)],
        "dg_pmg_apply": [P, P, P, P],
        "dg_pmg_destroy": [P],
        "dg_fgmres_step": [P, P, P, P, ctypes.c_double, ctypes.POINTER(KrylovOpts), P,
                           ctypes.POINTER(KrylovStats), P],
        "dg_status_sync": [P, P],
        "dg_pmg_bytes": [P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)],
        "dg_pmg_export_blocks": [P, ctypes.c_int, ctypes.c_int, P, ctypes.c_size_t, P],
        "dg_bdf2_rhs": [P, P, P, P, ctypes.c_double, P, P],
        "dg_axpy": [P, ctypes.c_double, P, P, P],
        "dg_launch_count": [ctypes.POINTER(ctypes.c_ulonglong)],
        "dg_pmg_refresh": [P, P, ctypes.c_double, P],
        "dg_residual_noalloc": [P, P, P, P, P],
        "dg_esdirk3_rhs": [P, P, P, ctypes.c_double, P, P, P],
        "dg_esdirk3_step": [P, P, P, ctypes.c_double, ctypes.c_int, ctypes.POINTER(KrylovOpts), P, ctypes.c_size_t,
                            P, ctypes.POINTER(KrylovStats), P],
        "dg_bilu_order": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                          ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(ctypes.c_int)],
        "dg_pmg_bilu_order": [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), P],
        "dg_mesh_create_tri": [ctypes.POINTER(TriDesc), ctypes.POINTER(PhysicsDesc), P, ctypes.POINTER(P)],
        "dg_pmg_operator": [P, ctypes.c_int, P, P, P],
        "dg_pmg_kernel_time": [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_float), P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(x):
    """Device pointer of a torch CUDA tensor (checked contiguous) or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("device buffers must be contiguous")
        return x.data_ptr()
    raise TypeError("expected a device pointer or a tensor, got %r" % type(x))


def _stream(stream):
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(fn, code):
    if code != DG_OK:
        raise DGError(fn, code)


class Mesh:
    """Owns a dg_mesh handle (periodic structured mesh + basis tables)."""

    def __init__(self, dim, n, lo, hi, p, nq1d=0, gamma=1.4, Pr=0.72, mu=0.0, Rgas=1.0, eta=0.0,
                 roe_delta=0.1, stream=None, space="P"):
        lib = load()
        d = MeshDesc()
        d.dim = dim
        n = list(n) + [1] * (3 - len(n))
        lo = list(lo) + [0.0] * (3 - len(lo))
        hi = list(hi) + [1.0] * (3 - len(hi))
        for k in range(3):
            d.n[k], d.lo[k], d.hi[k] = int(n[k]), float(lo[k]), float(hi[k])
        d.p, d.nq1d = int(p), int(nq1d)
        d.space = SPACE_Q if space == "Q" else SPACE_P
        ph = PhysicsDesc(gamma, Pr, mu, Rgas, eta, roe_delta)
        h = P()
        _check("dg_mesh_create", lib.dg_mesh_create(ctypes.byref(d), ctypes.byref(ph), _stream(stream),
                                                    ctypes.byref(h)))
        self.h = h
        self.dim, self.p = dim, p
        E, nm, m, N = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        _check("dg_mesh_info", lib.dg_mesh_info(h, ctypes.byref(E), ctypes.byref(nm), ctypes.byref(m),
                                                ctypes.byref(N)))
        self.E, self.nm, self.m, self.ndofs = E.value, nm.value, m.value, N.value

    @classmethod
    def triangles(cls, X, tri, shift, lo, hi, p, nq1d=0, gamma=1.4, Pr=0.72, mu=0.0, Rgas=1.0, eta=0.0,
                  roe_delta=0.1, stream=None):
        """A periodic triangulation (dg_mesh_create_tri): X (nv, 2) vertex
        coordinates, tri (E, 3) counter-clockwise vertex ids, shift (E, 3, 2)
        integer lattice shifts, box [lo, hi]^2, full-order degree p."""
        import numpy as np
        lib = load()
        Xc = np.ascontiguousarray(X, dtype=np.float64)
        Tc = np.ascontiguousarray(tri, dtype=np.int32)
        Sc = np.ascontiguousarray(shift, dtype=np.int32)
        d = TriDesc()
        d.n_vert, d.n_tri = len(Xc), len(Tc)
        d.X = Xc.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.tri = Tc.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        d.shift = Sc.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        for k in range(2):
            d.lo[k], d.hi[k] = float(lo[k]), float(hi[k])
        d.p, d.nq1d = int(p), int(nq1d)
        ph = PhysicsDesc(gamma, Pr, mu, Rgas, eta, roe_delta)
        h = P()
        _check("dg_mesh_create_tri", lib.dg_mesh_create_tri(ctypes.byref(d), ctypes.byref(ph), _stream(stream),
                                                            ctypes.byref(h)))
        self = cls.__new__(cls)
        self.h = h
        self.dim, self.p = 2, p
        E, nm, m, N = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        _check("dg_mesh_info", lib.dg_mesh_info(h, ctypes.byref(E), ctypes.byref(nm), ctypes.byref(m),
                                                ctypes.byref(N)))
        self.E, self.nm, self.m, self.ndofs = E.value, nm.value, m.value, N.value
        return self

    @classmethod
    def from_tri_workload(cls, mesh, phys, p, stream=None):
        """From workloads.tri_mesh(...) / workloads.tri_physics(...) dicts."""
        return cls.triangles(mesh["X"], mesh["tri"], mesh["shift"], mesh["lo"], mesh["hi"], p,
                             gamma=phys["gamma"], Pr=phys["Pr"], mu=phys["mu"], Rgas=phys["Rgas"],
                             eta=phys.get("eta", 0.0) or 0.0, roe_delta=phys["roe_delta"], stream=stream)

    @classmethod
    def from_workload(cls, desc, phys, stream=None):
        """From workloads.mesh_desc(...) / workloads.physics(...) dicts."""
        return cls(desc["dim"], desc["n"], desc["lo"], desc["hi"], desc["p"], desc.get("nq1d", 0),
                   gamma=phys["gamma"], Pr=phys["Pr"], mu=phys["mu"], Rgas=phys["Rgas"],
                   eta=phys.get("eta", 0.0) or 0.0, roe_delta=phys["roe_delta"], stream=stream,
                   space=desc.get("space", "P"))

    @property
    def shape(self):
        return (self.E, self.m, self.nm)

    def close(self):
        if getattr(self, "h", None):
            load().dg_mesh_destroy(self.h)
            self.h = None

    __del__ = close

    def residual(self, W, R, S=None, stream=None):
        _check("dg_residual", load().dg_residual(self.h, _ptr(W), _ptr(S), _ptr(R), _stream(stream)))

    def residual_noalloc(self, W, R, S=None, stream=None):
        """The residual with the face scratch in the library's fixed device array
        (no allocation at any call; meshes up to E*d*2*m*n_m = 2^20 doubles)."""
        _check("dg_residual_noalloc", load().dg_residual_noalloc(self.h, _ptr(W), _ptr(S), _ptr(R),
                                                                 _stream(stream)))

    def jvp(self, W, v, Kv, sigma, mode=JVP_EXACT, R_W=None, stream=None):
        _check("dg_jvp", load().dg_jvp(self.h, _ptr(W), _ptr(R_W), float(sigma), _ptr(v), _ptr(Kv),
                                       int(mode), _stream(stream)))

    def bdf2_rhs(self, Wk, Wn, Wnm1, dt, b, stream=None):
        """b = -[M (3 Wk - 4 Wn + Wnm1)/(2 dt) + R(Wk)] (BDF2 Newton right-hand side)."""
        _check("dg_bdf2_rhs", load().dg_bdf2_rhs(self.h, _ptr(Wk), _ptr(Wn), _ptr(Wnm1), float(dt), _ptr(b),
                                                 _stream(stream)))

    def esdirk3_rhs(self, Wk, Wn, sigma, racc, b, stream=None):
        """b = -[sigma M (Wk - Wn) + racc + R(Wk)] (ESDIRK stage Newton right-hand side)."""
        _check("dg_esdirk3_rhs", load().dg_esdirk3_rhs(self.h, _ptr(Wk), _ptr(Wn), float(sigma), _ptr(racc),
                                                       _ptr(b), _stream(stream)))

    def axpy(self, alpha, x, y, stream=None):
        _check("dg_axpy", load().dg_axpy(self.h, float(alpha), _ptr(x), _ptr(y), _stream(stream)))

    def status_sync(self, stream=None):
        return load().dg_status_sync(self.h, _stream(stream))


def launch_count():
    """Kernels launched by the library so far in this process."""
    c = ctypes.c_ulonglong()
    _check("dg_launch_count", load().dg_launch_count(ctypes.byref(c)))
    return c.value


def pmg_opts(p_levels, nu_pre=10, nu_post=10, nu_coarse=30, cycle=CYCLE_FMG, precision=PREC_FP64,
             fgmres_restart=30, coarse=COARSE_BJ, order=ORDER_MDF, storage=0):
    o = PmgOpts()
    o.n_levels = len(p_levels)
    for l, p in enumerate(p_levels):
        o.p_level[l] = int(p)
        o.nu_pre[l] = int(nu_pre[l] if hasattr(nu_pre, "__len__") else nu_pre)
        o.nu_post[l] = int(nu_post[l] if hasattr(nu_post, "__len__") else nu_post)
    o.nu_coarse = int(nu_coarse)
    o.cycle = int(cycle)
    o.precision = int(precision)
    o.fgmres_restart = int(fgmres_restart)
    o.coarse_precond = int(coarse)
    o.coarse_order = int(order)
    o.block_storage = int(storage)
    return o


def bilu_order(nbr, kind, c=None):
    """Host ordering of a block ILU(0) (dg_bilu_order): nbr int array
    [n_elem, n_faces], c float array of the same shape (MDF only).  Returns
    (order, level, n_levels) as numpy arrays / int."""
    import numpy as np
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    E, nf = nbr.shape
    order = np.zeros(E, dtype=np.int32)
    level = np.zeros(E, dtype=np.int32)
    nl = ctypes.c_int()
    cp = None
    if c is not None:
        c = np.ascontiguousarray(c, dtype=np.float64)
        cp = c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    ip = ctypes.POINTER(ctypes.c_int)
    _check("dg_bilu_order", load().dg_bilu_order(E, nf, nbr.ctypes.data_as(ip), cp, int(kind),
                                                 order.ctypes.data_as(ip), level.ctypes.data_as(ip),
                                                 ctypes.byref(nl)))
    return order, level, nl.value


class PMG:
    """Owns a dg_pmg handle: blocks, inverses and workspace set up at (W, sigma)."""

    def __init__(self, mesh, W, sigma, opts, stream=None):
        h = P()
        _check("dg_pmg_setup", load().dg_pmg_setup(mesh.h, _ptr(W), float(sigma), ctypes.byref(opts),
                                                   _stream(stream), ctypes.byref(h)))
        self.h = h
        self.mesh = mesh
        self.sigma = sigma
        self.opts = opts

    def close(self):
        if getattr(self, "h", None):
            load().dg_pmg_destroy(self.h)
            self.h = None

    __del__ = close

    def refresh(self, W, sigma, stream=None):
        """Recompute the preconditioner at (W, sigma) in the handle's buffers (async)."""
        _check("dg_pmg_refresh", load().dg_pmg_refresh(self.h, _ptr(W), float(sigma), _stream(stream)))
        self.sigma = sigma

    def apply(self, r, z, stream=None):
        _check("dg_pmg_apply", load().dg_pmg_apply(self.h, _ptr(r), _ptr(z), _stream(stream)))

    def bilu_order(self, stream=None):
        """(order, n_levels) of the coarsest block ILU(0) now in use."""
        import numpy as np
        order = np.zeros(self.mesh.E, dtype=np.int32)
        nl = ctypes.c_int()
        _check("dg_pmg_bilu_order", load().dg_pmg_bilu_order(self.h, order.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                                             ctypes.byref(nl), _stream(stream)))
        return order, nl.value

    def bytes(self):
        a, b = ctypes.c_size_t(), ctypes.c_size_t()
        _check("dg_pmg_bytes", load().dg_pmg_bytes(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def operator(self, level, x, y, stream=None):
        """y = A_level x (dg_pmg_operator): the operator the level's smoother uses."""
        _check("dg_pmg_operator", load().dg_pmg_operator(self.h, int(level), _ptr(x), _ptr(y), _stream(stream)))

    def kernel_time(self, kernel, level=0, reps=10, stream=None):
        """Mean device ms of one kernel of the solve path (dg_pmg_kernel_time)."""
        ms = ctypes.c_float()
        _check("dg_pmg_kernel_time", load().dg_pmg_kernel_time(self.h, int(kernel), int(level), int(reps),
                                                               ctypes.byref(ms), _stream(stream)))
        return ms.value

    def export_blocks(self, level, which, out, stream=None):
        nbytes = out.numel() * out.element_size()
        _check("dg_pmg_export_blocks", load().dg_pmg_export_blocks(self.h, int(level), int(which), _ptr(out),
                                                                   nbytes, _stream(stream)))

    def fgmres(self, W, b, dW, sigma=None, restart=30, max_restarts=0, rtol=1e-5, atol=0.0,
               jvp_mode=JVP_EXACT, stream=None, raise_on_error=True):
        """Solve K dW = b; returns the KrylovStats as a dict."""
        ko = KrylovOpts(int(restart), int(max_restarts), float(rtol), float(atol), int(jvp_mode))
        st = KrylovStats()
        code = load().dg_fgmres_step(self.mesh.h, self.h, _ptr(W), _ptr(b),
                                     float(self.sigma if sigma is None else sigma), ctypes.byref(ko),
                                     _ptr(dW), ctypes.byref(st), _stream(stream))
        out = dict(iters=st.iters, res0=st.res0, res_final=st.res_final, rho=st.rho, status=code,
                   ms_total=st.ms_total, ms_setup=st.ms_setup)
        if raise_on_error and code != DG_OK:
            raise DGError("dg_fgmres_step", code)
        return out

    def esdirk3_step(self, Wn, dt, Wout, newton=2, restart=30, max_restarts=4, rtol=1e-5, atol=0.0,
                     work=None, stream=None, raise_on_error=True):
        """One ESDIRK3 step from Wn into Wout (preconditioner refreshed at Wn and
        lagged over the step); `work` (device FP64, >= 6 n_dofs) is allocated here
        when not given.  Returns the summed KrylovStats as a dict."""
        if work is None:
            work = Wn.new_empty((6 * Wn.numel(),))
        ko = KrylovOpts(int(restart), int(max_restarts), float(rtol), float(atol), JVP_EXACT)
        st = KrylovStats()
        code = load().dg_esdirk3_step(self.mesh.h, self.h, _ptr(Wn), float(dt), int(newton), ctypes.byref(ko),
                                      _ptr(work), work.numel() * work.element_size(), _ptr(Wout), ctypes.byref(st),
                                      _stream(stream))
        out = dict(iters=st.iters, res_final=st.res_final, status=code, ms_total=st.ms_total)
        if raise_on_error and code != DG_OK:
            raise DGError("dg_esdirk3_step", code)
        return out



class ServerResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("status", ctypes.c_int), ("latency_ms", ctypes.c_double),
                ("queue_ms", ctypes.c_double), ("fgmres_iters", ctypes.c_int), ("ndofs", ctypes.c_longlong)]


_SERVER_SIGS = {
    "dg_server_create": [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(P)],
    "dg_server_submit": [P, ctypes.c_longlong, ctypes.POINTER(MeshDesc), ctypes.POINTER(PhysicsDesc),
                         ctypes.POINTER(PmgOpts), P, P, ctypes.c_double, ctypes.c_int, ctypes.c_double, P],
    "dg_server_poll": [P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ServerResult), ctypes.c_int,
                       ctypes.POINTER(ctypes.c_int)],
    "dg_server_stats": [P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int),
                        ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)],
    "dg_server_destroy": [P],
}
EXPORTED += list(_SERVER_SIGS)


def _server_lib():
    lib = load()
    for name, args in _SERVER_SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    return lib


def mesh_desc_struct(desc):
    d = MeshDesc()
    d.dim = desc["dim"]
    n = list(desc["n"]) + [1] * (3 - len(desc["n"]))
    lo = list(desc["lo"]) + [0.0] * (3 - len(desc["lo"]))
    hi = list(desc["hi"]) + [1.0] * (3 - len(desc["hi"]))
    for k in range(3):
        d.n[k], d.lo[k], d.hi[k] = int(n[k]), float(lo[k]), float(hi[k])
    d.p, d.nq1d = int(desc["p"]), int(desc.get("nq1d", 0))
    d.space = SPACE_Q if desc.get("space", "P") == "Q" else SPACE_P
    return d


def physics_struct(phys):
    return PhysicsDesc(phys["gamma"], phys["Pr"], phys["mu"], phys["Rgas"], phys.get("eta", 0.0) or 0.0,
                       phys["roe_delta"])


class Server:
    """Continuous-batching request loop over implicit steps (dg_server_*).
    Host arrays passed to submit() are kept referenced until their completion
    has been polled."""

    def __init__(self, budget_bytes, workers=4):
        self.lib = _server_lib()
        h = P()
        _check("dg_server_create", self.lib.dg_server_create(int(budget_bytes), int(workers), ctypes.byref(h)))
        self.h = h
        self._keep = {}

    def submit(self, rid, desc, phys, opts, Wn, Wnm1, dt, Wout, newton=2, rtol=1e-5):
        import numpy as np
        for a in (Wn, Wnm1, Wout):
            assert isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
        d, p = mesh_desc_struct(desc), physics_struct(phys)
        self._keep[rid] = (Wn, Wnm1, Wout, d, p, opts)
        _check("dg_server_submit", self.lib.dg_server_submit(
            self.h, int(rid), ctypes.byref(d), ctypes.byref(p), ctypes.byref(opts), Wn.ctypes.data,
            Wnm1.ctypes.data, float(dt), int(newton), float(rtol), Wout.ctypes.data))

    def poll(self, min_done=1, timeout_ms=-1, cap=256):
        buf = (ServerResult * cap)()
        n = ctypes.c_int()
        self.lib.dg_server_poll(self.h, int(min_done), int(timeout_ms), buf, cap, ctypes.byref(n))
        out = []
        for i in range(n.value):
            r = buf[i]
            out.append(dict(id=r.id, status=r.status, latency_ms=r.latency_ms, queue_ms=r.queue_ms,
                            fgmres_iters=r.fgmres_iters, ndofs=r.ndofs))
            self._keep.pop(r.id, None)
        return out

    def stats(self):
        u, s, a, b = ctypes.c_size_t(), ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong()
        _check("dg_server_stats", self.lib.dg_server_stats(self.h, ctypes.byref(u), ctypes.byref(s),
                                                           ctypes.byref(a), ctypes.byref(b)))
        return dict(used_bytes=u.value, resident_slots=s.value, submitted=a.value, completed=b.value)

    def close(self):
        if getattr(self, "h", None):
            self.lib.dg_server_destroy(self.h)
            self.h = None

    __del__ = close
