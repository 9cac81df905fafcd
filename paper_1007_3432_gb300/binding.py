"""ctypes binding of ``libhubhmc.so``: argument marshalling only.

Every function here forwards to the C ABI declared in ``include/hubhmc.h``
with the same name; tensors are passed as raw device (or host) pointers and
the CUDA stream as the raw ``cudaStream_t`` handle.  There is no CPU fallback:
if the library cannot be loaded, the import raises.
"""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libhubhmc.so")
# The debug build with index checks (HH_BOUNDS_CHECK=1 selects it).
LIB_CHECK_PATH = os.path.join(HERE, "lib", "libhubhmc_check.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "hubhmc.h")

HH_OK, HH_EINVAL, HH_ENOMEM, HH_ECUDA = 0, -1, -2, -3
HH_ENOCONV, HH_ENUMERIC, HH_ETIMEOUT, HH_EBUSY, HH_ESIZE, HH_EBOUNDS = -4, -5, -6, -7, -8, -9
HH_BOUNDS_READ, HH_BOUNDS_SELFTEST = 0, 1
HH_NOALLOC_MAX_SITES = 262144
HH_FP64, HH_MIXED, HH_MIXED_BF16LINK, HH_MIXED_FIX16LINK = 0, 1, 2, 3
PRECISIONS = {"fp64": HH_FP64, "mixed": HH_MIXED, "mixed-bf16link": HH_MIXED_BF16LINK,
              "mixed-fix16link": HH_MIXED_FIX16LINK}
HH_OP_M, HH_OP_MT, HH_OP_MTM = 0, 1, 2
HH_DTYPE_F64, HH_DTYPE_F32 = 0, 1


class HHError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, _strerror(code), code))


class hh_lattice(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("nx", ctypes.c_int), ("ntau", ctypes.c_int)]


class hh_params(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dtau", ctypes.c_double), ("A", ctypes.c_double),
                ("precision", ctypes.c_int), ("cg_tol", ctypes.c_double), ("cg_maxit", ctypes.c_int),
                ("reliable_delta", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("n_pf", ctypes.c_int), ("chain_id", ctypes.c_uint64),
                ("cheb_degree", ctypes.c_int), ("cheb_eps", ctypes.c_double), ("integrator", ctypes.c_int),
                ("chrono", ctypes.c_int), ("link_order", ctypes.c_int)]


class hh_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("true_relres", ctypes.c_double), ("converged", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hh_traj_info(ctypes.Structure):
    _fields_ = [("H0", ctypes.c_double), ("H1", ctypes.c_double), ("dH", ctypes.c_double),
                ("u", ctypes.c_double), ("accepted", ctypes.c_int), ("cg_iterations", ctypes.c_int),
                ("n_solves", ctypes.c_int), ("max_true_relres", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hh_obs_info(ctypes.Structure):
    _fields_ = [("trace_Minv", ctypes.c_double), ("trace_err", ctypes.c_double),
                ("one_minus_g_sq", ctypes.c_double), ("mean_sin", ctypes.c_double),
                ("mean_sin2", ctypes.c_double), ("n_noise", ctypes.c_int), ("cg_iterations", ctypes.c_int),
                ("max_true_relres", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hh_counters(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_longlong), ("engine_launches", ctypes.c_longlong),
                ("engine_ms", ctypes.c_double), ("cg_steps", ctypes.c_longlong),
                ("ru_steps", ctypes.c_longlong), ("solves", ctypes.c_longlong),
                ("fp64_steps", ctypes.c_longlong), ("sites", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hh_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("lat", hh_lattice), ("prm", hh_params),
                ("sigma", ctypes.c_void_p), ("b", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("n_md", ctypes.c_int), ("dt", ctypes.c_double), ("traj_index", ctypes.c_uint64)]


class hh_result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("kind", ctypes.c_int), ("status", ctypes.c_int),
                ("cg_iterations", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("n_solves", ctypes.c_int), ("max_true_relres", ctypes.c_double),
                ("H0", ctypes.c_double), ("H1", ctypes.c_double), ("dH", ctypes.c_double),
                ("u", ctypes.c_double), ("accepted", ctypes.c_int), ("queue_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hh_batch_config(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_size_t),
                ("chunk_iters", ctypes.c_int), ("tile_sites", ctypes.c_int),
                ("max_active_sites", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_size_t)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int)


EXCHANGE_DEV_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_size_t, ctypes.c_void_p)
ALLREDUCE_DEV_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p)


class hh_comm(ctypes.Structure):
    _fields_ = [("exchange", EXCHANGE_FN), ("allreduce_sum", ALLREDUCE_FN), ("user", ctypes.c_void_p),
                ("exchange_device", EXCHANGE_DEV_FN), ("allreduce_sum_device", ALLREDUCE_DEV_FN)]


class _CudaBuffer:
    """A device buffer given by its address, viewed by torch.as_tensor without
    a copy (CUDA array interface)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def _device_doubles(ptr, n):
    import torch
    return torch.as_tensor(_CudaBuffer(ptr, n), device="cuda")


def _stream_of(handle):
    import torch
    return torch.cuda.ExternalStream(int(handle)) if handle else torch.cuda.default_stream()


HH_REQ_SOLVE, HH_REQ_TRAJECTORY = 0, 1
HH_LEAPFROG, HH_OMELYAN = 0, 1
INTEGRATORS = {"leapfrog": HH_LEAPFROG, "omelyan": HH_OMELYAN}

_lib = None


def load(path: str = None):
    """Load the CUDA library (the index-checking debug build when
    HH_BOUNDS_CHECK=1); raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = LIB_CHECK_PATH if os.environ.get("HH_BOUNDS_CHECK") == "1" else LIB_PATH
    if not os.path.exists(path):
        raise ImportError("%s not built (run __graft_entry__.build()): %s" % (os.path.basename(path), path))
    L = ctypes.CDLL(path)
    vp, i, d, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
    sig = {
        "hh_default_params": (None, [ctypes.POINTER(hh_params)]),
        "hh_strerror": (ctypes.c_char_p, [i]),
        "hh_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(hh_lattice), ctypes.POINTER(hh_params), vp]),
        "hh_destroy": (i, [vp]),
        "hh_nsites": (ctypes.c_longlong, [vp]),
        "hh_set_field": (i, [vp, vp, i]),
        "hh_get_field": (i, [vp, vp, i]),
        "hh_init_field_random": (i, [vp, u64]),
        "hh_apply": (i, [vp, i, vp, vp, i]),
        "hh_apply_multi": (i, [vp, i, vp, vp, i, i]),
        "hh_solve": (i, [vp, vp, vp, i, ctypes.POINTER(hh_solve_info)]),
        "hh_solve_guess": (i, [vp, vp, vp, i, ctypes.POINTER(hh_solve_info)]),
        "hh_force": (i, [vp, vp, i, vp, ctypes.POINTER(hh_solve_info)]),
        "hh_action": (i, [vp, vp, i, ctypes.POINTER(d), ctypes.POINTER(hh_solve_info)]),
        "hh_trajectory": (i, [vp, i, d, u64, ctypes.POINTER(hh_traj_info)]),
        "hh_observables": (i, [vp, i, u64, ctypes.POINTER(hh_obs_info)]),
        "hh_leapfrog": (i, [vp, vp, vp, i, i, d, ctypes.POINTER(hh_solve_info)]),
        "hh_set_timeout": (i, [vp, d]),
        "hh_batch_set_timeout": (i, [vp, d]),
        "hh_counters_reset": (i, [vp, i]),
        "hh_counters_get": (i, [vp, ctypes.POINTER(hh_counters)]),
        "hh_bounds_check": (i, [i, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_longlong)]),
        "hh_solve_noalloc": (i, [ctypes.POINTER(hh_lattice), ctypes.POINTER(hh_params), vp, vp, vp, vp,
                                 ctypes.POINTER(hh_solve_info)]),
        "hh_slab_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(hh_lattice), ctypes.POINTER(hh_params), i, i,
                               ctypes.POINTER(hh_comm), vp]),
        "hh_slab_destroy": (i, [vp]),
        "hh_slab_set_field": (i, [vp, vp, i]),
        "hh_slab_apply": (i, [vp, i, vp, vp]),
        "hh_slab_solve": (i, [vp, vp, vp, ctypes.POINTER(hh_solve_info)]),
        "hh_batch_default_config": (None, [ctypes.POINTER(hh_batch_config)]),
        "hh_batch_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(hh_batch_config), vp]),
        "hh_batch_destroy": (i, [vp]),
        "hh_batch_submit": (i, [vp, ctypes.POINTER(hh_request), ctypes.POINTER(u64)]),
        "hh_batch_step": (i, [vp, ctypes.POINTER(i)]),
        "hh_batch_start": (i, [vp]),
        "hh_batch_stop": (i, [vp]),
        "hh_batch_poll": (i, [vp, ctypes.POINTER(hh_result), i, ctypes.POINTER(i)]),
        "hh_batch_pending": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(i)]),
        "hh_batch_autotune": (i, [ctypes.POINTER(hh_request), i, ctypes.c_size_t, i, ctypes.c_char_p, vp,
                                  ctypes.POINTER(hh_batch_config)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _strerror(code):
    if _lib is None:
        return "error"
    return _lib.hh_strerror(code).decode()


def header_symbols(path: str = HEADER):
    """Names of the functions declared in a public header."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hh_[a-z0-9_]+)\s*\(", text)))


def check(code, what, allow=()):
    if code != HH_OK and code not in allow:
        raise HHError(code, what)
    return code


def _ptr(t):
    """Raw pointer of a torch tensor or an integer address."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class MetricsLog:
    """Per-call records as JSON lines (one object per line): solves
    (iterations, reliable updates, true relative residual), trajectories
    (H0, dH, u, accept, CG iterations, solves), served results (status,
    latency, queueing, service) with the queue depth when they were polled.
    target: a path (appended to) or an open text file."""

    def __init__(self, target):
        self._own = isinstance(target, (str, os.PathLike))
        self._f = open(target, "a") if self._own else target

    def write(self, record, **fields):
        """One line: {"record": record, "time": unix seconds, **fields}."""
        import json
        import time
        rec = {"record": record, "time": time.time()}
        rec.update(fields)
        self._f.write(json.dumps(rec) + "\n")
        self._f.flush()

    def close(self):
        if self._own and not self._f.closed:
            self._f.close()


def _as_log(log):
    return log if log is None or isinstance(log, MetricsLog) else MetricsLog(log)


class Context:
    """One lattice and one Markov chain on the current CUDA device.  log: a
    MetricsLog (or a path for one) that receives a record per solve, force,
    action and trajectory."""

    def __init__(self, d, nx, ntau, t=1.0, dtau=0.05, A=0.5, precision=HH_FP64, cg_tol=1e-10,
                 cg_maxit=1000000, reliable_delta=0.1, seed=0, n_pf=2, chain_id=0, stream=None,
                 cheb_degree=0, cheb_eps=1e-3, integrator="leapfrog", chrono=0, link_order=0, log=None):
        L = load()
        self._lib = L
        self.log = _as_log(log)
        self.lat = hh_lattice(d, nx, ntau)
        p = hh_params()
        L.hh_default_params(ctypes.byref(p))
        p.t, p.dtau, p.A = t, dtau, A
        p.precision = PRECISIONS.get(precision, precision)
        p.cg_tol, p.cg_maxit, p.reliable_delta = cg_tol, cg_maxit, reliable_delta
        p.seed, p.n_pf, p.chain_id = seed, n_pf, chain_id
        p.cheb_degree, p.cheb_eps = cheb_degree, cheb_eps
        p.integrator = INTEGRATORS.get(integrator, integrator)
        p.chrono = chrono
        p.link_order = link_order
        self.params = p
        self.stream = stream
        h = ctypes.c_void_p()
        check(L.hh_create(ctypes.byref(h), ctypes.byref(self.lat), ctypes.byref(p),
                          _stream_handle(stream)), "hh_create")
        self._h = h
        self.N = int(L.hh_nsites(h))

    def _record(self, record, info, **extra):
        if self.log is not None and info is not None:
            self.log.write(record, d=self.lat.d, nx=self.lat.nx, ntau=self.lat.ntau,
                           precision=int(self.params.precision), **extra, **info)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- field ----
    def set_field(self, sigma, on_device=None):
        if on_device is None:
            on_device = getattr(sigma, "is_cuda", False)
        ptr = _ptr(sigma) if not hasattr(sigma, "ctypes") else sigma.ctypes.data
        check(self._lib.hh_set_field(self._h, ptr, int(bool(on_device))), "hh_set_field")

    def get_field(self, out, on_device=None):
        if on_device is None:
            on_device = getattr(out, "is_cuda", False)
        ptr = _ptr(out) if not hasattr(out, "ctypes") else out.ctypes.data
        check(self._lib.hh_get_field(self._h, ptr, int(bool(on_device))), "hh_get_field")
        return out

    def init_field_random(self, seed):
        check(self._lib.hh_init_field_random(self._h, seed), "hh_init_field_random")

    # ---- operators and solves ----
    def apply(self, op, x, y, dtype=None):
        if dtype is None:
            import torch
            dtype = HH_DTYPE_F32 if x.dtype == torch.float32 else HH_DTYPE_F64
        check(self._lib.hh_apply(self._h, op, _ptr(x), _ptr(y), dtype), "hh_apply")

    def apply_multi(self, op, x, y, n_vec, dtype=None):
        """y_v = op(x_v) for n_vec vectors stored back to back (hh_apply_multi)."""
        if dtype is None:
            import torch
            dtype = HH_DTYPE_F32 if x.dtype == torch.float32 else HH_DTYPE_F64
        check(self._lib.hh_apply_multi(self._h, op, _ptr(x), _ptr(y), n_vec, dtype), "hh_apply_multi")

    def solve(self, b, x, n_rhs=1, info=True, allow=(), guess=False):
        """guess: start from the x passed in (hh_solve_guess) instead of zero."""
        inf = hh_solve_info() if info else None
        fn = self._lib.hh_solve_guess if guess else self._lib.hh_solve
        rc = fn(self._h, _ptr(b), _ptr(x), n_rhs, ctypes.byref(inf) if info else None)
        check(rc, "hh_solve_guess" if guess else "hh_solve", allow)
        if not info:
            return rc
        out = inf.as_dict()
        self._record("solve", out, status=rc, n_rhs=n_rhs)
        return rc, out

    def force(self, chi, n_rhs, F, info=True):
        inf = hh_solve_info() if info else None
        rc = self._lib.hh_force(self._h, _ptr(chi), n_rhs, _ptr(F), ctypes.byref(inf) if info else None)
        check(rc, "hh_force")
        out = inf.as_dict() if info else None
        self._record("force", out, n_rhs=n_rhs)
        return out

    def action(self, chi, n_rhs):
        S = ctypes.c_double()
        inf = hh_solve_info()
        check(self._lib.hh_action(self._h, _ptr(chi), n_rhs, ctypes.byref(S), ctypes.byref(inf)), "hh_action")
        out = inf.as_dict()
        self._record("action", out, S=S.value, n_rhs=n_rhs)
        return S.value, out

    def leapfrog(self, pi, chi, n_rhs, n_md, dt, info=True):
        inf = hh_solve_info() if info else None
        rc = self._lib.hh_leapfrog(self._h, _ptr(pi), _ptr(chi), n_rhs, n_md, dt,
                                   ctypes.byref(inf) if info else None)
        check(rc, "hh_leapfrog")
        return inf.as_dict() if info else None

    def trajectory(self, n_md, dt, traj_index, info=True, allow=()):
        inf = hh_traj_info() if info else None
        rc = self._lib.hh_trajectory(self._h, n_md, dt, traj_index, ctypes.byref(inf) if info else None)
        check(rc, "hh_trajectory", allow)
        out = inf.as_dict() if info else None
        self._record("trajectory", out, status=rc, n_md=n_md, dt=dt, traj_index=traj_index)
        return out

    def observables(self, n_noise, traj=0):
        """Noise estimators of diag M^{-1} at the current field (hh_observables)."""
        inf = hh_obs_info()
        check(self._lib.hh_observables(self._h, n_noise, traj, ctypes.byref(inf)), "hh_observables")
        return inf.as_dict()

    def set_timeout(self, seconds):
        """Bound of every device-side wait (hh_set_timeout)."""
        check(self._lib.hh_set_timeout(self._h, float(seconds)), "hh_set_timeout")

    def counters_reset(self, profile_engine=False):
        check(self._lib.hh_counters_reset(self._h, int(bool(profile_engine))), "hh_counters_reset")

    def counters(self):
        c = hh_counters()
        check(self._lib.hh_counters_get(self._h, ctypes.byref(c)), "hh_counters_get")
        return c.as_dict()


def bounds_check(selftest=False):
    """Index-check records of the debug build: (status, enabled, record);
    status HH_EBOUNDS if a check failed since the last call."""
    L = load()
    en = ctypes.c_int(0)
    rec = ctypes.c_longlong(0)
    rc = L.hh_bounds_check(HH_BOUNDS_SELFTEST if selftest else HH_BOUNDS_READ, ctypes.byref(en),
                           ctypes.byref(rec))
    if rc not in (HH_OK, HH_EBOUNDS):
        check(rc, "hh_bounds_check")
    return rc, en.value, rec.value


def solve_noalloc(d, nx, ntau, sigma, b, x, t=1.0, dtau=0.05, A=0.5, cg_tol=1e-10, cg_maxit=1000000,
                  stream=None, info=True):
    """hh_solve_noalloc: FP64 CG for Q x = b with no allocation by the library.
    sigma, b, x: device tensors of N doubles.  Returns (rc, info dict)."""
    L = load()
    lat = hh_lattice(d, nx, ntau)
    p = hh_params()
    L.hh_default_params(ctypes.byref(p))
    p.t, p.dtau, p.A, p.cg_tol, p.cg_maxit = t, dtau, A, cg_tol, cg_maxit
    inf = hh_solve_info()
    rc = L.hh_solve_noalloc(ctypes.byref(lat), ctypes.byref(p), _ptr(sigma), _ptr(b), _ptr(x),
                            _stream_handle(stream), ctypes.byref(inf) if info else None)
    return rc, (inf.as_dict() if info else None)


def make_params(t=1.0, dtau=0.05, A=0.5, precision=HH_FP64, cg_tol=1e-10, cg_maxit=1000000,
                reliable_delta=0.1, seed=0, n_pf=2, chain_id=0, cheb_degree=0, cheb_eps=1e-3,
                integrator="leapfrog", chrono=0, link_order=0):
    L = load()
    p = hh_params()
    L.hh_default_params(ctypes.byref(p))
    p.t, p.dtau, p.A = t, dtau, A
    p.precision = PRECISIONS.get(precision, precision)
    p.cg_tol, p.cg_maxit, p.reliable_delta = cg_tol, cg_maxit, reliable_delta
    p.seed, p.n_pf, p.chain_id = seed, n_pf, chain_id
    p.cheb_degree, p.cheb_eps = cheb_degree, cheb_eps
    p.integrator = INTEGRATORS.get(integrator, integrator)
    p.chrono = chrono
    p.link_order = link_order
    return p


def make_request(kind, d, nx, ntau, sigma=None, b=None, out=None, n_md=0, dt=0.0, traj_index=0, **prm):
    """An hh_request.  sigma, b: host float64 NumPy arrays (copied at submit);
    out: host float64 NumPy array written on completion (kept alive by the caller)."""
    r = hh_request()
    r.kind = kind
    r.lat = hh_lattice(d, nx, ntau)
    r.prm = make_params(**prm)
    r.sigma = sigma.ctypes.data if sigma is not None else None
    r.b = b.ctypes.data if b is not None else None
    r.out = out.ctypes.data if out is not None else None
    r.n_md, r.dt, r.traj_index = n_md, dt, traj_index
    return r


class Batch:
    """Batched multi-chain engine / serving loop (hh_batch_*).  log: a
    MetricsLog (or a path for one) that receives a record per polled result,
    with the queue depth (queued and active requests) at that poll."""

    def __init__(self, max_slots=64, hbm_budget_bytes=4 << 30, chunk_iters=32, tile_sites=4096,
                 max_active_sites=0, stream=None, log=None):
        L = load()
        self._lib = L
        self.log = _as_log(log)
        cfg = hh_batch_config()
        L.hh_batch_default_config(ctypes.byref(cfg))
        cfg.max_slots, cfg.hbm_budget_bytes = max_slots, hbm_budget_bytes
        cfg.chunk_iters, cfg.tile_sites, cfg.max_active_sites = chunk_iters, tile_sites, max_active_sites
        self.config = cfg
        h = ctypes.c_void_p()
        check(L.hh_batch_create(ctypes.byref(h), ctypes.byref(cfg), _stream_handle(stream)), "hh_batch_create")
        self._h = h
        self._keep = {}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hh_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, req, keep=None, allow=()):
        t = ctypes.c_uint64()
        rc = self._lib.hh_batch_submit(self._h, ctypes.byref(req), ctypes.byref(t))
        check(rc, "hh_batch_submit", allow)
        if rc == HH_OK and keep is not None:
            self._keep[t.value] = keep
        return rc, t.value

    def step(self, allow=()):
        n = ctypes.c_int()
        rc = self._lib.hh_batch_step(self._h, ctypes.byref(n))
        check(rc, "hh_batch_step", allow)
        return n.value

    def set_timeout(self, seconds):
        """Bound of every device-side wait of the engine launches (hh_batch_set_timeout)."""
        check(self._lib.hh_batch_set_timeout(self._h, float(seconds)), "hh_batch_set_timeout")

    def start(self):
        check(self._lib.hh_batch_start(self._h), "hh_batch_start")

    def stop(self):
        check(self._lib.hh_batch_stop(self._h), "hh_batch_stop")

    def poll(self, max_results=256):
        arr = (hh_result * max_results)()
        n = ctypes.c_int()
        check(self._lib.hh_batch_poll(self._h, arr, max_results, ctypes.byref(n)), "hh_batch_poll")
        out = [arr[j].as_dict() for j in range(n.value)]
        for r in out:
            self._keep.pop(r["ticket"], None)
        if self.log is not None and out:
            queued, active = self.pending()
            for r in out:
                self.log.write("result", queued=queued, active=active, **r)
        return out

    def pending(self):
        q, a = ctypes.c_int(), ctypes.c_int()
        check(self._lib.hh_batch_pending(self._h, ctypes.byref(q), ctypes.byref(a)), "hh_batch_pending")
        return q.value, a.value

    def run_until_idle(self, max_steps=10 ** 7, allow=()):
        results = []
        for _ in range(max_steps):
            busy = self.step(allow)
            results += self.poll()
            if busy == 0:
                break
        return results + self.poll()


def autotune(requests, hbm_budget_bytes=4 << 30, rounds=8, cache_path=None, stream=None):
    """hh_batch_autotune on copies of the given solve requests; returns the
    chosen configuration as a dict."""
    L = load()
    arr = (hh_request * len(requests))(*requests)
    best = hh_batch_config()
    check(L.hh_batch_autotune(arr, len(requests), hbm_budget_bytes, rounds,
                              cache_path.encode() if cache_path else None, _stream_handle(stream),
                              ctypes.byref(best)), "hh_batch_autotune")
    return best.as_dict()


class TorchDistComm:
    """The two host-side callbacks of a time slab (hh_comm) over
    torch.distributed with CPU tensors (gloo): exchange of one time slice with
    the neighbouring ranks of the ring, and the sum of a few doubles over all
    ranks.  With one rank the exchange copies send into recv."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.error = None

    def exchange_host(self, direction, send, recv):
        """send, recv: 1-D CPU tensors of the same size."""
        if self.world == 1:
            recv.copy_(send)
            return
        nxt, prv = (self.rank + 1) % self.world, (self.rank - 1) % self.world
        to, frm = (nxt, prv) if direction > 0 else (prv, nxt)
        req = self.dist.isend(send, to, group=self.group)
        self.dist.recv(recv, frm, group=self.group)
        req.wait()

    def allreduce_host(self, vals):
        if self.world > 1:
            self.dist.all_reduce(vals, op=self.dist.ReduceOp.SUM, group=self.group)

    def device_capable(self):
        """The device form needs one rank or an NCCL group."""
        return self.world == 1 or self.dist.get_backend(self.group) == "nccl"

    def exchange_device(self, direction, send, recv):
        """send, recv: CUDA tensors; enqueued on the current stream."""
        if self.world == 1:
            recv.copy_(send, non_blocking=True)
            return
        nxt, prv = (self.rank + 1) % self.world, (self.rank - 1) % self.world
        to, frm = (nxt, prv) if direction > 0 else (prv, nxt)
        ops = [self.dist.P2POp(self.dist.isend, send, to, self.group),
               self.dist.P2POp(self.dist.irecv, recv, frm, self.group)]
        for w in self.dist.batch_isend_irecv(ops):
            w.wait()   # NCCL: the current stream waits, not the host

    def allreduce_device(self, vals):
        if self.world > 1:
            self.dist.all_reduce(vals, op=self.dist.ReduceOp.SUM, group=self.group)

    def c_callbacks(self, device=False):
        """An hh_comm whose callbacks call the methods above (keep the returned
        object alive while the slab exists); device=True adds the device form
        (the slab then uses it)."""
        import torch

        def _exchange(user, direction, send, recv, nbytes):
            try:
                n = int(nbytes) // 8
                s = torch.frombuffer((ctypes.c_double * n).from_address(send), dtype=torch.float64)
                r = torch.frombuffer((ctypes.c_double * n).from_address(recv), dtype=torch.float64)
                self.exchange_host(int(direction), s.clone(), r)
                return 0
            except Exception as e:   # no exception may cross the C ABI
                self.error = e
                return 1

        def _allreduce(user, vals, n):
            try:
                v = torch.frombuffer((ctypes.c_double * int(n)).from_address(ctypes.addressof(vals.contents)),
                                     dtype=torch.float64)
                t = v.clone()
                self.allreduce_host(t)
                v.copy_(t)
                return 0
            except Exception as e:
                self.error = e
                return 1

        self._ex = EXCHANGE_FN(_exchange)
        self._ar = ALLREDUCE_FN(_allreduce)
        if not device:
            return hh_comm(self._ex, self._ar, None, EXCHANGE_DEV_FN(), ALLREDUCE_DEV_FN())

        # With several ranks the transfers are not captured into the slab's
        # CUDA graph: a callback refuses before enqueuing anything, on every
        # rank alike, and the slab then launches its iterations directly.
        def _refuse_capture():
            return self.world > 1 and torch.cuda.is_current_stream_capturing()

        def _exchange_dev(user, direction, send, recv, nbytes, stream):
            try:
                n = int(nbytes) // 8
                with torch.cuda.stream(_stream_of(stream)):
                    if _refuse_capture():
                        return 1
                    self.exchange_device(int(direction), _device_doubles(send, n), _device_doubles(recv, n))
                return 0
            except Exception as e:
                self.error = e
                return 1

        def _allreduce_dev(user, vals, n, stream):
            try:
                with torch.cuda.stream(_stream_of(stream)):
                    if _refuse_capture():
                        return 1
                    self.allreduce_device(_device_doubles(vals, n))
                return 0
            except Exception as e:
                self.error = e
                return 1

        self._exd = EXCHANGE_DEV_FN(_exchange_dev)
        self._ard = ALLREDUCE_DEV_FN(_allreduce_dev)
        return hh_comm(self._ex, self._ar, None, self._exd, self._ard)


class Slab:
    """The slices [tau0, tau1) of one lattice on this rank (hh_slab_*)."""

    def __init__(self, d, nx, ntau, tau0, tau1, comm=None, stream=None, device_comm=False, **prm):
        L = load()
        self._lib = L
        self.comm = comm if comm is not None else TorchDistComm()
        if device_comm and not self.comm.device_capable():
            raise ValueError("the device form of the callbacks needs one rank or an NCCL group")
        self._c = self.comm.c_callbacks(device=device_comm)
        self.lat = hh_lattice(d, nx, ntau)
        p = make_params(**prm)
        h = ctypes.c_void_p()
        check(L.hh_slab_create(ctypes.byref(h), ctypes.byref(self.lat), ctypes.byref(p), tau0, tau1,
                               ctypes.byref(self._c), _stream_handle(stream)), "hh_slab_create")
        self._h = h
        self.V = nx ** d
        self.n = self.V * (tau1 - tau0)

    def _check(self, rc, what):
        if rc != HH_OK and self.comm.error is not None:
            err, self.comm.error = self.comm.error, None
            raise HHError(rc, what + " (callback: %r)" % (err,))
        check(rc, what)
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hh_slab_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_field(self, sigma_slab):
        on_device = getattr(sigma_slab, "is_cuda", False)
        ptr = _ptr(sigma_slab) if not hasattr(sigma_slab, "ctypes") else sigma_slab.ctypes.data
        self._check(self._lib.hh_slab_set_field(self._h, ptr, int(bool(on_device))), "hh_slab_set_field")

    def apply(self, op, x, y):
        self._check(self._lib.hh_slab_apply(self._h, op, _ptr(x), _ptr(y)), "hh_slab_apply")

    def solve(self, b, x, allow=()):
        inf = hh_solve_info()
        rc = self._lib.hh_slab_solve(self._h, _ptr(b), _ptr(x), ctypes.byref(inf))
        if rc not in allow:
            self._check(rc, "hh_slab_solve")
        return rc, inf.as_dict()

