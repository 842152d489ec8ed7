"""Python binding of libdgmg (ctypes): argument marshalling only.

Every computation runs in the CUDA library; this module converts torch tensors
to device pointers and raises ``DGMGError`` on any non-zero return code. There
is no fallback: if ``libdgmg.so`` is missing the import fails loudly.
"""
import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libdgmg.so")

DGMG_OK = 0
DGMG_EINVAL = -1
DGMG_ENOMEM = -2
DGMG_EBUDGET = -3
DGMG_ENOTCONVERGED = -4
DGMG_ENONFINITE = -5
DGMG_ECUDA = -6
DGMG_ETIMEOUT = -7
DGMG_FP64 = 0
DGMG_MIXED_FP32 = 1
DGMG_OUTER_AUTO = 0
DGMG_OUTER_PCG = 1
DGMG_OUTER_RELIABLE = 2
DGMG_OUTER_MGMULT = 3
DGMG_OUTER_MGMULT_PREC = 4
DGMG_BASIS_GLL = 0
DGMG_BASIS_GL = 1
DGMG_PENDING = 0
DGMG_RUNNING = 1
DGMG_DONE = 2
DGMG_FAILED = 3
DGMG_BLOCK_EXACT = 0
DGMG_BLOCK_INTERIOR_ONLY = 1


class DGMGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dgmg error {code}: {msg}")
        self.code = code


class Mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3)]


class Opts(ctypes.Structure):
    _fields_ = [("omega_dg", ctypes.c_double), ("omega_cg", ctypes.c_double),
                ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int), ("precision", ctypes.c_int),
                ("block_inverse", ctypes.c_int), ("coarsening", ctypes.c_int),
                ("rtol", ctypes.c_double), ("maxit", ctypes.c_int), ("outer", ctypes.c_int),
                ("delta", ctypes.c_double), ("autotune", ctypes.c_int), ("p_coarsening", ctypes.c_int),
                ("basis", ctypes.c_int), ("recompute_block", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("p", ctypes.c_int), ("q", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("ncell", ctypes.c_int64), ("ndof", ctypes.c_int64), ("nlevels_cg", ctypes.c_int),
                ("nvert0", ctypes.c_int64), ("ncoarse", ctypes.c_int64),
                ("omega_dg", ctypes.c_double), ("omega_cg", ctypes.c_double),
                ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int), ("precision", ctypes.c_int),
                ("block_inverse", ctypes.c_int), ("coarsening", ctypes.c_int),
                ("device_bytes", ctypes.c_size_t), ("outer", ctypes.c_int), ("dg_levels", ctypes.c_int),
                ("tiles", ctypes.c_int * 6)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("rel_residual_recursive", ctypes.c_double), ("prec_residual", ctypes.c_double),
                ("seconds", ctypes.c_double), ("fp64_applies", ctypes.c_int), ("queue_seconds", ctypes.c_double)]


class ServerInfo(ctypes.Structure):
    _fields_ = [("pending", ctypes.c_int), ("active", ctypes.c_int), ("done", ctypes.c_longlong),
                ("failed", ctypes.c_longlong), ("admitted", ctypes.c_longlong), ("cache_entries", ctypes.c_int),
                ("cache_hits", ctypes.c_longlong), ("cache_misses", ctypes.c_longlong),
                ("evictions", ctypes.c_longlong), ("bytes_in_use", ctypes.c_size_t), ("budget", ctypes.c_size_t)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("groups", ctypes.c_int), ("ndof", ctypes.c_int64),
                ("device_bytes", ctypes.c_size_t), ("max_levels", ctypes.c_int),
                ("kernels_per_iteration", ctypes.c_longlong), ("group_q", ctypes.c_int * 4),
                ("group_tiles", (ctypes.c_int * 3) * 4)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SIGS = {
    "dgmg_version": (ctypes.c_char_p, []),
    "dgmg_last_error": (ctypes.c_char_p, []),
    "dgmg_default_opts": (None, [ctypes.POINTER(Opts)]),
    "dgmg_create": (_I, [ctypes.POINTER(Mesh), _I, _P, ctypes.POINTER(Opts), ctypes.POINTER(_P)]),
    "dgmg_destroy": (_I, [_P]),
    "dgmg_info": (_I, [_P, ctypes.POINTER(Info)]),
    "dgmg_gll_nodes": (_I, [_P, _P]),
    "dgmg_update_kappa": (_I, [_P, _P]),
    "dgmg_apply": (_I, [_P, _P, _P, _P]),
    "dgmg_residual": (_I, [_P, _P, _P, _P, _P]),
    "dgmg_smooth": (_I, [_P, _P, _P, _I, _P]),
    "dgmg_vcycle": (_I, [_P, _P, _P, _P]),
    "dgmg_solve": (_I, [_P, _P, _P, ctypes.POINTER(Stats), _P]),
    "dgmg_solve_host": (_I, [_P, _P, _P, ctypes.POINTER(Stats), _P]),
    "dgmg_quad_points": (_I, [_P, _P, _P]),
    "dgmg_load_vector": (_I, [_P, _P, _P, _P]),
    "dgmg_project": (_I, [_P, _P, _P, _P, _P]),
    "dgmg_residual_restrict": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "dgmg_residual_restrict_noalloc": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "dgmg_cg_smooth": (_I, [_P, _I, _P, _P, _I, _P]),
    "dgmg_cg_residual": (_I, [_P, _I, _P, _P, _P, _P]),
    "dgmg_h_restrict": (_I, [_P, _I, _P, _P, _P]),
    "dgmg_h_prolong": (_I, [_P, _I, _P, _P, _P]),
    "dgmg_coarse_solve": (_I, [_P, _P, _P, _P]),
    "dgmg_cg_size": (ctypes.c_int64, [_P, _I]),
    "dgmg_volume_residual_f32": (_I, [_P, _P, _P, _P, _I, _P]),
    "dgmg_apply_f32": (_I, [_P, _P, _P, _I, _P]),
    "dgmg_estimate_bytes": (_I, [ctypes.POINTER(Mesh), _I, ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_size_t)]),
    "dgmg_server_create": (_I, [ctypes.c_size_t, _I, ctypes.POINTER(Opts), ctypes.POINTER(_P)]),
    "dgmg_submit": (_I, [_P, ctypes.POINTER(Mesh), _I, _P, _P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "dgmg_poll": (_I, [_P, ctypes.c_uint64, ctypes.POINTER(_I), ctypes.POINTER(Stats)]),
    "dgmg_server_info": (_I, [_P, ctypes.POINTER(ServerInfo)]),
    "dgmg_server_destroy": (_I, [_P]),
    "dgmg_batch_create": (_I, [_I, _P, _P, _P, ctypes.POINTER(Opts), ctypes.POINTER(_P)]),
    "dgmg_batch_info": (_I, [_P, ctypes.POINTER(BatchInfo)]),
    "dgmg_batch_solve": (_I, [_P, _P, _P, _P, _P]),
    "dgmg_batch_destroy": (_I, [_P]),
    "dgmg_profile": (_I, [_P, _I]),
    "dgmg_profile_read": (_I, [_P, _P, _P, _I]),
    "dgmg_kernel_launches": (ctypes.c_longlong, []),
    "dgmg_wait_timeouts": (_I, [ctypes.POINTER(ctypes.c_ulonglong)]),
    "dgmg_fma_peak": (_I, [_I, ctypes.POINTER(ctypes.c_double), _P]),
}

STAGES = ("project", "smooth", "residual", "cg_levels", "vector")


def kernel_launches():
    """Kernels launched by libdgmg in this process."""
    return int(load().dgmg_kernel_launches())


def fma_peak(kind, stream=None):
    """Measured FMA-loop peak of the current device in TFLOP/s: kind 0 FP64,
    1 FP32, 2 FP32 on packed pairs."""
    v = ctypes.c_double(0.0)
    _check(load().dgmg_fma_peak(int(kind), ctypes.byref(v), _stream(stream)))
    return float(v.value)


def wait_timeouts():
    """Device-side bounded waits that ran out on the current device (0 when healthy)."""
    v = ctypes.c_ulonglong(0)
    _check(load().dgmg_wait_timeouts(ctypes.byref(v)))
    return int(v.value)

_lib = None


def load(path=LIB_PATH):
    """Load libdgmg.so (raises OSError if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libdgmg.so not found at {path}; build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc, allow=()):
    if rc != DGMG_OK and rc not in allow:
        raise DGMGError(rc, load().dgmg_last_error().decode())
    return rc


def _ptr(t, n=None, dtype=None):
    """Device pointer of a contiguous CUDA tensor of `dtype` (float64 unless
    given) holding at least `n` elements (the length the library reads or
    writes; unchecked when n is None or negative)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("tensor must be a contiguous CUDA tensor")
    if t.dtype != (torch.float64 if dtype is None else dtype):
        raise ValueError(f"tensor must be {torch.float64 if dtype is None else dtype}")
    if n is not None and n >= 0 and t.numel() < n:
        raise ValueError(f"tensor holds {t.numel()} elements, {n} needed")
    return ctypes.c_void_p(t.data_ptr())


def _f32(t, n):
    import torch
    return _ptr(t, n, torch.float32)


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _mesh(n):
    m = Mesh()
    m.dim = len(n)
    for a in range(3):
        m.n[a] = int(n[a]) if a < len(n) else 1
    return m


def _ncell(n):
    c = 1
    for v in n:
        c *= int(v)
    return c


def _ndof(n, p):
    return _ncell(n) * (int(p) + 1) ** len(n)


def _kappa(kappa, n):
    """Contiguous float64 copy of one coefficient per cell of mesh n."""
    import numpy as np
    k = np.ascontiguousarray(np.asarray(kappa, dtype=np.float64).reshape(-1))
    if k.size != _ncell(n):
        raise ValueError("kappa needs one value per cell")
    return k


def _opts(**opts):
    o = Opts()
    load().dgmg_default_opts(ctypes.byref(o))
    for k, v in opts.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def estimate_bytes(n, p, **opts):
    b = ctypes.c_size_t()
    _check(load().dgmg_estimate_bytes(ctypes.byref(_mesh(n)), int(p), ctypes.byref(_opts(**opts)), ctypes.byref(b)))
    return int(b.value)


class Server:
    """A dgmg_server: continuous batching of independent solves."""

    def __init__(self, budget_bytes, max_active, **opts):
        self.lib = load()
        self.opts = _opts(**opts)
        h = ctypes.c_void_p()
        _check(self.lib.dgmg_server_create(ctypes.c_size_t(int(budget_bytes)), int(max_active),
                                           ctypes.byref(self.opts), ctypes.byref(h)))
        self.h = h
        self._keep = {}

    def submit(self, n, p, b, x, kappa=None):
        """Queue a solve; b, x: contiguous CUDA float64 tensors kept alive until done."""
        kp = None
        if kappa is not None:
            k = _kappa(kappa, n)
            kp = k.ctypes.data_as(ctypes.c_void_p)
        t = ctypes.c_uint64()
        nd = _ndof(n, p)
        _check(self.lib.dgmg_submit(self.h, ctypes.byref(_mesh(n)), int(p), kp, _ptr(b, nd), _ptr(x, nd),
                                    ctypes.byref(t)))
        self._keep[t.value] = (b, x)
        return int(t.value)

    def poll(self, ticket):
        """(status, Stats or None); raises DGMGError if the request failed."""
        st = ctypes.c_int()
        stats = Stats()
        rc = self.lib.dgmg_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(st), ctypes.byref(stats))
        if st.value in (DGMG_DONE, DGMG_FAILED):
            self._keep.pop(ticket, None)
        _check(rc)
        return st.value, (stats if st.value == DGMG_DONE else None)

    def info(self):
        inf = ServerInfo()
        _check(self.lib.dgmg_server_info(self.h, ctypes.byref(inf)))
        return inf

    def close(self):
        if getattr(self, "h", None):
            self.lib.dgmg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A dgmg_batch: independent problems solved together, one launch per stage."""

    def __init__(self, problems, **opts):
        """problems: list of (n, p, kappa or None); all meshes of one dimension."""
        self.lib = load()
        self.opts = _opts(**opts)
        k = len(problems)
        meshes = (Mesh * k)()
        ps = (ctypes.c_int * k)()
        kps = (ctypes.c_void_p * k)()
        self._kappa_keep = []
        self._ndof = []
        for i, (n, p, kappa) in enumerate(problems):
            meshes[i] = _mesh(n)
            ps[i] = int(p)
            self._ndof.append(_ndof(n, p))
            if kappa is not None:
                a = _kappa(kappa, n)
                self._kappa_keep.append(a)
                kps[i] = a.ctypes.data
        h = ctypes.c_void_p()
        _check(self.lib.dgmg_batch_create(k, ctypes.cast(meshes, _P), ctypes.cast(ps, _P), ctypes.cast(kps, _P),
                                          ctypes.byref(self.opts), ctypes.byref(h)))
        self.h = h
        self.count = k

    def info(self):
        inf = BatchInfo()
        _check(self.lib.dgmg_batch_info(self.h, ctypes.byref(inf)))
        return inf

    def solve(self, bs, xs, stream=None, allow_notconverged=False):
        """bs, xs: lists of contiguous CUDA float64 tensors, one per problem.
        Returns (list of Stats, return code)."""
        k = self.count
        if len(bs) != k or len(xs) != k:
            raise ValueError("one b and one x per problem")
        bp = (ctypes.c_void_p * k)(*[_ptr(t, nd).value for t, nd in zip(bs, self._ndof)])
        xp = (ctypes.c_void_p * k)(*[_ptr(t, nd).value for t, nd in zip(xs, self._ndof)])
        st = (Stats * k)()
        allow = (DGMG_ENOTCONVERGED,) if allow_notconverged else ()
        rc = _check(self.lib.dgmg_batch_solve(self.h, ctypes.cast(bp, _P), ctypes.cast(xp, _P), ctypes.cast(st, _P),
                                              _stream(stream)), allow)
        return list(st), rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.dgmg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def default_opts():
    o = Opts()
    load().dgmg_default_opts(ctypes.byref(o))
    return o


class Context:
    """A dgmg_ctx: the hierarchy for one mesh, degree and kappa field."""

    def __init__(self, n, p, kappa=None, **opts):
        lib = load()
        self.lib = lib
        m = Mesh()
        m.dim = len(n)
        for a in range(3):
            m.n[a] = int(n[a]) if a < len(n) else 1
        o = default_opts()
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        self.opts = o
        kap_ptr = None
        self._kappa_keep = None
        if kappa is not None:
            k = _kappa(kappa, n)
            self._kappa_keep = k
            kap_ptr = k.ctypes.data_as(ctypes.c_void_p)
        h = ctypes.c_void_p()
        _check(lib.dgmg_create(ctypes.byref(m), int(p), kap_ptr, ctypes.byref(o), ctypes.byref(h)))
        self.h = h
        self.info = self.get_info()
        self.n = tuple(int(v) for v in n)
        self.p = int(p)
        self.ndof = int(self.info.ndof)

    def get_info(self):
        inf = Info()
        _check(self.lib.dgmg_info(self.h, ctypes.byref(inf)))
        return inf

    def close(self):
        if getattr(self, "h", None):
            self.lib.dgmg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update_kappa(self, kappa):
        """New per-cell coefficients for the same mesh and degree (dgmg_update_kappa)."""
        k = _kappa(kappa, self.n)
        _check(self.lib.dgmg_update_kappa(self.h, k.ctypes.data_as(ctypes.c_void_p)))
        self._kappa_keep = k

    def gll_nodes(self):
        import numpy as np
        x = np.zeros(self.info.q)
        _check(self.lib.dgmg_gll_nodes(self.h, x.ctypes.data_as(ctypes.c_void_p)))
        return x

    def cg_size(self, level):
        return int(self.lib.dgmg_cg_size(self.h, int(level)))

    def apply(self, u, y, stream=None):
        n = self.ndof
        _check(self.lib.dgmg_apply(self.h, _ptr(u, n), _ptr(y, n), _stream(stream)))

    def residual(self, u, b, r, stream=None):
        n = self.ndof
        _check(self.lib.dgmg_residual(self.h, _ptr(u, n), _ptr(b, n), _ptr(r, n), _stream(stream)))

    def smooth(self, u, b, nsteps, stream=None):
        n = self.ndof
        _check(self.lib.dgmg_smooth(self.h, _ptr(u, n), _ptr(b, n), int(nsteps), _stream(stream)))

    def vcycle(self, r, e, stream=None):
        n = self.ndof
        _check(self.lib.dgmg_vcycle(self.h, _ptr(r, n), _ptr(e, n), _stream(stream)))

    def solve(self, b, x, stream=None, allow_notconverged=False):
        st = Stats()
        allow = (DGMG_ENOTCONVERGED,) if allow_notconverged else ()
        n = self.ndof
        rc = _check(self.lib.dgmg_solve(self.h, _ptr(b, n), _ptr(x, n), ctypes.byref(st), _stream(stream)), allow)
        return st, rc

    def solve_host(self, b_host, x_host, stream=None):
        """b_host, x_host: CPU float64 torch tensors (pinned for best speed)."""
        import torch
        for t in (b_host, x_host):
            if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
                raise ValueError("host tensors must be contiguous CPU float64")
            if t.numel() < self.ndof:
                raise ValueError(f"host tensor holds {t.numel()} elements, {self.ndof} needed")
        st = Stats()
        _check(self.lib.dgmg_solve_host(self.h, ctypes.c_void_p(b_host.data_ptr()),
                                        ctypes.c_void_p(x_host.data_ptr()), ctypes.byref(st), _stream(stream)))
        return st

    def _quad_per_cell(self):
        return (self.info.p + 2) ** self.info.dim

    def quad_points(self, xq, stream=None):
        n = int(self.info.ncell) * self._quad_per_cell() * self.info.dim
        _check(self.lib.dgmg_quad_points(self.h, _ptr(xq, n), _stream(stream)))

    def load_vector(self, fq, b, stream=None):
        n = int(self.info.ncell) * self._quad_per_cell()
        _check(self.lib.dgmg_load_vector(self.h, _ptr(fq, n), _ptr(b, self.ndof), _stream(stream)))

    def project(self, u, e, traces, stream=None):
        _check(self.lib.dgmg_project(self.h, _ptr(u, self.ndof), _ptr(e, int(self.info.nvert0)),
                                     _ptr(traces, self.trace_size()), _stream(stream)))

    def _rr_args(self, u, b, traces, r, rc):
        n = self.ndof
        return (_ptr(u, n), _ptr(b, n), _ptr(traces, self.trace_size()), _ptr(r, n), _ptr(rc, int(self.info.nvert0)))

    def residual_restrict(self, u, b, traces, r, rc, stream=None):
        _check(self.lib.dgmg_residual_restrict(self.h, *self._rr_args(u, b, traces, r, rc), _stream(stream)))

    def residual_restrict_noalloc(self, u, b, traces, r, rc, stream=None):
        """As residual_restrict, with the scratch in the library's fixed device
        array instead of the context's (allocates nothing; see dgmg.h)."""
        _check(self.lib.dgmg_residual_restrict_noalloc(self.h, *self._rr_args(u, b, traces, r, rc), _stream(stream)))

    def volume_residual_f32(self, u, b, r, method, stream=None):
        """r = b - kappa_K E u_K per cell (FP32 tensors; method 0 sum-factorised,
        1 tensor cores, TF32): the volume term of the operator alone."""
        n = self.ndof
        _check(self.lib.dgmg_volume_residual_f32(self.h, _f32(u, n), _f32(b, n), _f32(r, n), int(method),
                                                 _stream(stream)))

    def apply_f32(self, u, y, form=0, stream=None):
        """y = A u in FP32 (mixed-precision ctx): the operator of the FP32 CG
        recurrences; form 0 the solver's choice, 1 per pencil, 2 one thread per
        cell through the fast-diagonalisation factors."""
        n = self.ndof
        _check(self.lib.dgmg_apply_f32(self.h, _f32(u, n), _f32(y, n), int(form), _stream(stream)))

    def cg_smooth(self, level, u, b, nsteps, stream=None):
        n = self.cg_size(level)
        _check(self.lib.dgmg_cg_smooth(self.h, int(level), _ptr(u, n), _ptr(b, n), int(nsteps), _stream(stream)))

    def cg_residual(self, level, u, b, r, stream=None):
        n = self.cg_size(level)
        _check(self.lib.dgmg_cg_residual(self.h, int(level), _ptr(u, n), _ptr(b, n), _ptr(r, n), _stream(stream)))

    def h_restrict(self, level, rf, rc, stream=None):
        _check(self.lib.dgmg_h_restrict(self.h, int(level), _ptr(rf, self.cg_size(level)),
                                        _ptr(rc, self.cg_size(level + 1)), _stream(stream)))

    def h_prolong(self, level, ec, uf, stream=None):
        _check(self.lib.dgmg_h_prolong(self.h, int(level), _ptr(ec, self.cg_size(level + 1)),
                                       _ptr(uf, self.cg_size(level)), _stream(stream)))

    def coarse_solve(self, r, e, stream=None):
        n = int(self.info.ncoarse)
        _check(self.lib.dgmg_coarse_solve(self.h, _ptr(r, n), _ptr(e, n), _stream(stream)))

    def profile(self, enable=True):
        _check(self.lib.dgmg_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        """{stage: (milliseconds, launches)} since the last read."""
        import numpy as np
        ms = np.zeros(len(STAGES))
        cnt = np.zeros(len(STAGES), dtype=np.int64)
        _check(self.lib.dgmg_profile_read(self.h, ms.ctypes.data_as(ctypes.c_void_p),
                                          cnt.ctypes.data_as(ctypes.c_void_p), len(STAGES)))
        return {s: (float(ms[i]), int(cnt[i])) for i, s in enumerate(STAGES)}

    def trace_size(self):
        d, q = self.info.dim, self.info.q
        return int(self.info.ncell) * 2 * d * 2 * q ** (d - 1)
