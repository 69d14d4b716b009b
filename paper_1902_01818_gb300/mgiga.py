"""ctypes binding of libmgiga (include/mgiga.h): argument marshalling only.

Every step of the solver runs in the compiled library; this module converts
Python problem descriptions and arrays into the C structs and pointers of the
C ABI.  Importing it loads libmgiga.so and raises if the library is missing:
there is no Python fallback.

Host-pointer calls take numpy float64 arrays; the *_d calls take CUDA tensors
(torch) and pass their device pointers.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "_lib", "libmgiga.so")

if not os.path.exists(LIBPATH):
    raise ImportError(f"libmgiga.so not found at {LIBPATH}; build it with paper_1902_01818_gb300.build.build()")
_lib = C.CDLL(LIBPATH)

# status codes
OK, EINVAL, ENOMEM, ECUDA, ENOTSPD, ENOCONV, EBREAKDOWN, ETIMEOUT, ESTATE = range(9)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENOTSPD", "ENOCONV", "EBREAKDOWN", "ETIMEOUT", "ESTATE"]
CONFORMING, SIPG = 0, 1
SMOOTHER = {"scms": 0, "gs": 1, "hybrid": 2}
OUTER = {"pcg": 0, "direct": 1}
PRECISION = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}
STAGE = {"band": 0, "fd": 1, "pieces": 2, "gs": 3, "restrict": 4, "prolong": 5, "coarse": 6, "vcycle": 7,
         "residual": 8}
OP = {"residual": 0, "matvec": 1, "smooth": 2, "gs_fwd": 3, "gs_bwd": 4, "restrict": 5, "prolong": 6,
      "coarse": 7, "cycle_residual": 8}


class MgigaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class _Interface(C.Structure):
    _fields_ = [("patch_a", C.c_int), ("side_a", C.c_int), ("patch_b", C.c_int), ("side_b", C.c_int),
                ("orient", C.c_uint)]


class _Problem(C.Structure):
    _fields_ = [("dim", C.c_int), ("num_patches", C.c_int), ("degree", C.c_int),
                ("num_knots", C.POINTER(C.c_int)), ("knots", C.POINTER(C.c_double)),
                ("geo_degree", C.c_int), ("geo_num_knots", C.POINTER(C.c_int)),
                ("geo_knots", C.POINTER(C.c_double)), ("geo_ctrl", C.POINTER(C.c_double)),
                ("num_interfaces", C.c_int), ("interfaces", C.POINTER(_Interface)),
                ("coupling", C.c_int), ("sipg_penalty", C.c_double), ("degrees", C.POINTER(C.c_int))]


class _Options(C.Structure):
    _fields_ = [("levels", C.c_int), ("smoother", C.c_int), ("nu", C.c_int), ("mu", C.c_int),
                ("outer", C.c_int), ("precision", C.c_int), ("max_iter", C.c_int),
                ("tau", C.c_double), ("delta", C.c_double), ("hbm_budget", C.c_size_t),
                ("stream", C.c_void_p), ("gs_cluster", C.c_int), ("autotune", C.c_int),
                ("matrix_free", C.c_int)]


_H = C.c_void_p
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_SIGS = {
    "mgiga_default_options": (None, [C.POINTER(_Options)]),
    "mgiga_create": (C.c_int, [C.POINTER(_Problem), C.POINTER(_Options), C.POINTER(_H)]),
    "mgiga_assemble": (C.c_int, [_H]),
    "mgiga_load": (C.c_int, [_H, C.c_void_p, C.c_void_p, _D]),
    "mgiga_source_sinprod": (C.c_double, [_D, C.c_void_p]),
    "mgiga_vcycle": (C.c_int, [_H, _D, _D]),
    "mgiga_vcycle_d": (C.c_int, [_H, C.c_void_p, C.c_void_p]),
    "mgiga_solve": (C.c_int, [_H, _D, _D, C.c_double, _I, _D]),
    "mgiga_solve_d": (C.c_int, [_H, C.c_void_p, C.c_void_p, C.c_double, _I, _D]),
    "mgiga_solve_batch_d": (C.c_int, [C.POINTER(_H), C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                      C.c_double, C.c_int, _I, _D, _I]),
    "mgiga_apply": (C.c_int, [_H, C.c_int, C.c_int, _D, _D, _D]),
    "mgiga_apply_d": (C.c_int, [_H, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mgiga_residual_noalloc_d": (C.c_int, [_H, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mgiga_kernel_launches": (C.c_int, [_H, C.POINTER(C.c_longlong)]),
    "mgiga_check_wait_expiry": (C.c_int, [_H, C.c_longlong, _D]),
    "mgiga_residual_history": (C.c_int, [_H, _D, C.c_int, _I]),
    "mgiga_time_stage": (C.c_int, [_H, C.c_int, C.c_int, C.c_int, _D]),
    "mgiga_stage_work": (C.c_int, [_H, C.c_int, C.c_int, _D, _D]),
    "mgiga_num_levels": (C.c_int, [_H, _I]),
    "mgiga_ndof": (C.c_int, [_H, C.c_int, C.POINTER(C.c_long)]),
    "mgiga_dof_map": (C.c_int, [_H, C.c_int, _I, _I]),
    "mgiga_colours": (C.c_int, [_H, C.c_int, _I]),
    "mgiga_pieces": (C.c_int, [_H, C.c_int, _I, _I]),
    "mgiga_device_bytes": (C.c_int, [_H, C.POINTER(C.c_size_t)]),
    "mgiga_last_error": (C.c_char_p, [_H]),
    "mgiga_destroy": (None, [_H]),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args

EXPORTED = sorted(_SIGS)


def _dptr(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _tensor_ptr(t):
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise TypeError("device entry points take CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    import torch
    if t.dtype != torch.float64:
        raise TypeError("tensor must be float64")
    return C.c_void_p(t.data_ptr())


def marshal_problem(prob):
    """C problem struct (and the arrays it points to) from a problem dict."""
    d, K, p = prob["dim"], len(prob["knots"]), prob["degree"]
    nk = np.array([len(prob["knots"][k][a]) for k in range(K) for a in range(d)], dtype=np.int32)
    kn = _f64(np.concatenate([np.asarray(prob["knots"][k][a], float) for k in range(K) for a in range(d)]))
    gnk = np.array([len(prob["geo_knots"][k][a]) for k in range(K) for a in range(d)], dtype=np.int32)
    gkn = _f64(np.concatenate([np.asarray(prob["geo_knots"][k][a], float) for k in range(K) for a in range(d)]))
    gctrl = _f64(np.concatenate([np.asarray(prob["geo_ctrl"][k], float).ravel() for k in range(K)]))
    ifs = (_Interface * max(1, len(prob["interfaces"])))()
    for i, (pa, sa, pb, sb, o) in enumerate(prob["interfaces"]):
        ifs[i] = _Interface(pa, sa, pb, sb, o)
    degs = None
    if prob.get("degrees") is not None:  # one degree per patch; `degree` is their largest
        degs = np.ascontiguousarray(prob["degrees"], dtype=np.int32)
    keep = (nk, kn, gnk, gkn, gctrl, ifs, degs)
    cp = _Problem(d, K, p, nk.ctypes.data_as(_I), _dptr(kn), prob["geo_degree"], gnk.ctypes.data_as(_I),
                  _dptr(gkn), _dptr(gctrl), len(prob["interfaces"]), ifs,
                  CONFORMING if prob["coupling"] == "conforming" else SIPG, float(prob.get("sipg_penalty", 0.0)),
                  degs.ctypes.data_as(_I) if degs is not None else None)
    return cp, keep


class Solver:
    """One problem on the GPU: mgiga_create + mgiga_assemble, then solves.

    levels=0 chooses the number of levels automatically; smoother 'scms' |
    'gs' | 'hybrid'; outer 'pcg' | 'direct'; stream: an int cudaStream_t.
    """

    def __init__(self, prob, levels=0, smoother="scms", tau=1.0, delta=0.12, nu=1, mu=1, outer="pcg",
                 precision="fp64", max_iter=1000, hbm_budget=0, stream=None, assemble=True, gs_cluster=0,
                 autotune=False, matrix_free=False):
        self.prob = prob
        self.precision = precision
        cp, self._keep = marshal_problem(prob)
        opts = _Options()
        _lib.mgiga_default_options(C.byref(opts))
        opts.levels, opts.smoother, opts.nu, opts.mu = levels, SMOOTHER[smoother], nu, mu
        opts.outer, opts.precision, opts.max_iter = OUTER[outer], PRECISION[precision], max_iter
        opts.tau, opts.delta, opts.hbm_budget = tau, delta, hbm_budget
        opts.stream = C.c_void_p(stream) if stream else None
        opts.gs_cluster = gs_cluster
        opts.autotune = 1 if autotune else 0
        opts.matrix_free = 1 if matrix_free else 0
        self._h = _H()
        st = _lib.mgiga_create(C.byref(cp), C.byref(opts), C.byref(self._h))
        if st != OK:
            msg = self.last_error()
            self.close()
            raise MgigaError(st, msg)
        self.levels = self._num_levels()
        if assemble:
            self.assemble()

    # -- lifecycle ----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.mgiga_destroy(self._h)
            self._h = _H()

    def __del__(self):
        self.close()

    def last_error(self):
        return _lib.mgiga_last_error(self._h).decode()

    def _check(self, st, allow=()):
        if st != OK and st not in allow:
            raise MgigaError(st, self.last_error())
        return st

    def assemble(self):
        self._check(_lib.mgiga_assemble(self._h))

    # -- sizes and integer maps --------------------------------------------
    def _num_levels(self):
        n = C.c_int()
        self._check(_lib.mgiga_num_levels(self._h, C.byref(n)))
        return n.value

    def ndof(self, level=-1):
        level = level % self.levels
        n = C.c_long()
        self._check(_lib.mgiga_ndof(self._h, level, C.byref(n)))
        return n.value

    def dof_map(self, level=-1):
        level = level % self.levels
        n = self.ndof(level)
        patch = np.zeros(n, dtype=np.int32)
        local = np.zeros(n, dtype=np.int32)
        self._check(_lib.mgiga_dof_map(self._h, level, patch.ctypes.data_as(_I), local.ctypes.data_as(_I)))
        return patch, local

    def colours(self, level=-1):
        level = level % self.levels
        out = np.zeros(self.ndof(level), dtype=np.int32)
        self._check(_lib.mgiga_colours(self._h, level, out.ctypes.data_as(_I)))
        return out

    def pieces(self, level=-1):
        level = level % self.levels
        out = np.zeros(self.ndof(level), dtype=np.int32)
        n = C.c_int()
        self._check(_lib.mgiga_pieces(self._h, level, out.ctypes.data_as(_I), C.byref(n)))
        return out, n.value

    def check_wait_expiry(self, iterations):
        """One bounded device wait on a barrier nothing completes: (status, ms)."""
        ms = C.c_double()
        st = _lib.mgiga_check_wait_expiry(self._h, iterations, C.byref(ms))
        return st, ms.value

    def residual_history(self):
        """Relative residuals of the last solve: initial, then per outer iteration."""
        n = C.c_int()
        self._check(_lib.mgiga_residual_history(self._h, None, 0, C.byref(n)))
        out = np.zeros(n.value)
        if n.value:
            self._check(_lib.mgiga_residual_history(self._h, _dptr(out), n.value, C.byref(n)))
        return out

    def kernel_launches(self):
        n = C.c_longlong()
        self._check(_lib.mgiga_kernel_launches(self._h, C.byref(n)))
        return n.value

    def time_stage(self, stage, level=-1, reps=20):
        """Average device milliseconds of one application of a stage."""
        ms = C.c_double()
        self._check(_lib.mgiga_time_stage(self._h, STAGE[stage], level % self.levels, reps, C.byref(ms)))
        return ms.value

    def stage_work(self, stage, level=-1):
        """(algorithmic flops, algorithmic bytes) of one application of a stage."""
        fl, by = C.c_double(), C.c_double()
        self._check(_lib.mgiga_stage_work(self._h, STAGE[stage], level % self.levels, C.byref(fl), C.byref(by)))
        return fl.value, by.value

    def device_bytes(self):
        b = C.c_size_t()
        self._check(_lib.mgiga_device_bytes(self._h, C.byref(b)))
        return b.value

    # -- compute (host arrays) ---------------------------------------------
    def load_sinprod(self):
        """Load vector of f = d pi^2 prod sin(pi x_a) (built-in source)."""
        out = np.zeros(self.ndof())
        dim = C.c_int(self.prob["dim"])
        fn = C.cast(_lib.mgiga_source_sinprod, C.c_void_p)
        self._check(_lib.mgiga_load(self._h, fn, C.cast(C.byref(dim), C.c_void_p), _dptr(out)))
        return out

    def vcycle(self, r):
        r = _f64(r)
        z = np.zeros_like(r)
        self._check(_lib.mgiga_vcycle(self._h, _dptr(r), _dptr(z)))
        return z

    def solve(self, rhs, u0=None, tol=1e-8, allow_noconv=False):
        """Returns (u, iterations, final relative residual, status)."""
        rhs = _f64(rhs)
        u = np.zeros_like(rhs) if u0 is None else _f64(u0).copy()
        it = C.c_int()
        rel = C.c_double()
        st = _lib.mgiga_solve(self._h, _dptr(rhs), _dptr(u), tol, C.byref(it), C.byref(rel))
        self._check(st, allow=(ENOCONV,) if allow_noconv else ())
        return u, it.value, rel.value, st

    def apply(self, op, level, a, b=None):
        level = level % self.levels
        a = _f64(a)
        bb = _f64(b) if b is not None else None
        if op == "restrict":
            nout = self.ndof(level - 1)
        else:
            nout = self.ndof(level)
        out = np.zeros(nout)
        self._check(_lib.mgiga_apply(self._h, OP[op], level, _dptr(a), _dptr(bb) if bb is not None else None,
                                     _dptr(out)))
        return out

    # -- compute (device tensors) -------------------------------------------
    def solve_d(self, rhs, u, tol=1e-8, allow_noconv=False):
        it = C.c_int()
        rel = C.c_double()
        st = _lib.mgiga_solve_d(self._h, _tensor_ptr(rhs), _tensor_ptr(u), tol, C.byref(it), C.byref(rel))
        self._check(st, allow=(ENOCONV,) if allow_noconv else ())
        return it.value, rel.value, st

    def vcycle_d(self, r, z):
        self._check(_lib.mgiga_vcycle_d(self._h, _tensor_ptr(r), _tensor_ptr(z)))

    def residual_noalloc_d(self, level, f, u, out):
        """out = f - A_level u with the allocation-free entry point (fixed scratch)."""
        self._check(_lib.mgiga_residual_noalloc_d(self._h, level % self.levels, _tensor_ptr(f), _tensor_ptr(u),
                                                  _tensor_ptr(out)))

    def apply_d(self, op, level, a, b, out):
        level = level % self.levels
        self._check(_lib.mgiga_apply_d(self._h, OP[op], level, _tensor_ptr(a),
                                       _tensor_ptr(b) if b is not None else None, _tensor_ptr(out)))


BATCH_ONE_GRAPH = 1


def solve_batch_d(solvers, rhs, u, tol=1e-8, one_graph=False):
    """mgiga_solve_batch_d: solve every (solver, rhs, u) of the lists (CUDA float64 tensors, u the
    initial guess and the solution); returns (iterations, final relative residuals, statuses) as
    lists.  one_graph: all solves as the branches of one graph launch."""
    n = len(solvers)
    hs = (_H * max(n, 1))(*[s._h for s in solvers])
    rp = (C.c_void_p * max(n, 1))(*[_tensor_ptr(x).value for x in rhs])
    up = (C.c_void_p * max(n, 1))(*[_tensor_ptr(x).value for x in u])
    it = np.zeros(max(n, 1), dtype=np.int32)
    rel = np.zeros(max(n, 1))
    st = np.zeros(max(n, 1), dtype=np.int32)
    _lib.mgiga_solve_batch_d(hs, n, rp, up, tol, BATCH_ONE_GRAPH if one_graph else 0, it.ctypes.data_as(_I),
                             _dptr(rel), st.ctypes.data_as(_I))
    return it[:n].tolist(), rel[:n].tolist(), st[:n].tolist()
