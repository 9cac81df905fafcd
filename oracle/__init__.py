"""Python access to the FP64 CPU oracle (``hubbard_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may import this package.  The
CUDA library and its binding never import it, and it imports nothing from them.

The arrays are NumPy float64, laid out with the site index
``i = x + Nx*(y + Nx*(z + Nx*tau))`` (``i = x + Nx*tau`` for d = 1).
"""
import ctypes
import os

import numpy as np

from . import build_oracle

_lib = None


class Lattice(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("nx", ctypes.c_int), ("ntau", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dtau", ctypes.c_double), ("A", ctypes.c_double),
                ("cg_tol", ctypes.c_double), ("cg_maxit", ctypes.c_int), ("n_pf", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("chain", ctypes.c_uint64), ("integrator", ctypes.c_int),
                ("chrono", ctypes.c_int), ("link_order", ctypes.c_int)]


class TrajInfo(ctypes.Structure):
    _fields_ = [("H0", ctypes.c_double), ("H1", ctypes.c_double), ("dH", ctypes.c_double),
                ("u", ctypes.c_double), ("accepted", ctypes.c_int),
                ("cg_iterations", ctypes.c_int), ("n_solves", ctypes.c_int),
                ("max_relres", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_dp = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        L.oracle_nsites.restype = ctypes.c_long
        L.oracle_uniform.restype = ctypes.c_double
        L.oracle_action.restype = ctypes.c_double
        L.oracle_cheb_poly.restype = ctypes.c_double
        L.oracle_cheb_poly.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        _lib = L
    return _lib


def _ptr(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def lattice(d, nx, ntau):
    return Lattice(d, nx, ntau)


def params(t=1.0, dtau=0.05, A=0.5, cg_tol=1e-10, cg_maxit=100000, n_pf=2, seed=1007, chain=0, integrator=0,
           chrono=0, link_order=0):
    """integrator: 0 leapfrog (Sec. 4.1), 1 Omelyan's second-order minimum-norm scheme.
    chrono: initial guess of the MD solves (0 zero, 1 last solution, 2 linear extrapolation).
    link_order: form of M (0 reading R1; 1, 2 the exact-block form expanded to that order)."""
    return Params(t, dtau, A, cg_tol, cg_maxit, n_pf, seed, chain, integrator, chrono, link_order)


def nsites(lat):
    return lat.nx ** lat.d * lat.ntau


def links(lat, A, sigma):
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    L = np.empty(nsites(lat))
    lib().oracle_links(ctypes.byref(lat), ctypes.c_double(A), _ptr(sigma), _ptr(L))
    return L


def _apply(fn, lat, h, L, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    y = np.empty(nsites(lat))
    fn(ctypes.byref(lat), ctypes.c_double(h), _ptr(L), _ptr(x), _ptr(y))
    return y


def apply_M(lat, h, L, x):
    return _apply(lib().oracle_apply_M, lat, h, L, x)


def apply_MT(lat, h, L, x):
    return _apply(lib().oracle_apply_MT, lat, h, L, x)


def apply_MTM(lat, h, L, x):
    return _apply(lib().oracle_apply_MTM, lat, h, L, x)


def _apply_ex(fn, lat, h, L, order, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    y = np.empty(nsites(lat))
    fn(ctypes.byref(lat), ctypes.c_double(h), _ptr(L), ctypes.c_int(order), _ptr(x), _ptr(y))
    return y


def apply_M_ex(lat, h, L, order, x):
    return _apply_ex(lib().oracle_apply_M_ex, lat, h, L, order, x)


def apply_MT_ex(lat, h, L, order, x):
    return _apply_ex(lib().oracle_apply_MT_ex, lat, h, L, order, x)


def apply_MTM_ex(lat, h, L, order, x):
    return _apply_ex(lib().oracle_apply_MTM_ex, lat, h, L, order, x)


def cg_ex(lat, h, L, order, b, x0=None, tol=1e-10, maxit=100000):
    """CG for the M of the given order, from zero or from x0."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    x = np.zeros(nsites(lat)) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = lib().oracle_cg_ex(ctypes.byref(lat), ctypes.c_double(h), _ptr(L), ctypes.c_int(order), _ptr(b), _ptr(x),
                            ctypes.c_int(0 if x0 is None else 1), ctypes.c_double(tol), ctypes.c_int(maxit),
                            ctypes.byref(it), ctypes.byref(rr))
    return x, st, it.value, rr.value


def cg(lat, h, L, b, tol=1e-10, maxit=100000):
    """Returns (x, status, iterations, true_relres)."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    x = np.empty(nsites(lat))
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = lib().oracle_cg(ctypes.byref(lat), ctypes.c_double(h), _ptr(L), _ptr(b), _ptr(x),
                         ctypes.c_double(tol), ctypes.c_int(maxit), ctypes.byref(it),
                         ctypes.byref(rr))
    return x, st, it.value, rr.value


def cg_guess(lat, h, L, b, x0, tol=1e-10, maxit=100000):
    """CG from the initial guess x0; returns (x, status, iterations, true_relres)."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    x = np.array(x0, dtype=np.float64, copy=True)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = lib().oracle_cg_guess(ctypes.byref(lat), ctypes.c_double(h), _ptr(L), _ptr(b), _ptr(x),
                               ctypes.c_double(tol), ctypes.c_int(maxit), ctypes.byref(it), ctypes.byref(rr))
    return x, st, it.value, rr.value


def gershgorin_lambda_max(d, h, A):
    """Upper bound of the spectrum of Q = M^T M: ||Q|| <= ||M||_1 ||M||_inf,
    each at most 1 + 2 d h + (1 + A) (unit diagonal, 2d hops, one link)."""
    return (2.0 + 2.0 * d * h + A) ** 2


def cheb_poly(n, eps, z):
    return lib().oracle_cheb_poly(n, eps, z)


def cheb_apply(lat, h, L, n, eps, lam, x):
    assert 0 <= n <= 64
    x = np.ascontiguousarray(x, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    y = np.empty(nsites(lat))
    lib().oracle_cheb_apply(ctypes.byref(lat), ctypes.c_double(h), _ptr(L), ctypes.c_int(n),
                            ctypes.c_double(eps), ctypes.c_double(lam), _ptr(x), _ptr(y))
    return y


def pcg(lat, h, L, b, n, eps, lam, tol=1e-10, maxit=100000):
    """Chebyshev-preconditioned CG; returns (x, status, iterations, true_relres)."""
    assert 0 <= n <= 64
    b = np.ascontiguousarray(b, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    x = np.empty(nsites(lat))
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = lib().oracle_pcg(ctypes.byref(lat), ctypes.c_double(h), _ptr(L), ctypes.c_int(n),
                          ctypes.c_double(eps), ctypes.c_double(lam), _ptr(b), _ptr(x),
                          ctypes.c_double(tol), ctypes.c_int(maxit), ctypes.byref(it), ctypes.byref(rr))
    return x, st, it.value, rr.value


def philox4x64(ctr, key):
    c = (ctypes.c_uint64 * 4)(*[int(v) for v in ctr])
    k = (ctypes.c_uint64 * 2)(*[int(v) for v in key])
    o = (ctypes.c_uint64 * 4)()
    lib().oracle_philox4x64(c, k, o)
    return [int(v) for v in o]


def gaussian(seed, tag, a, traj, chain, n):
    out = np.empty(n)
    lib().oracle_gaussian(ctypes.c_uint64(seed), ctypes.c_int(tag), ctypes.c_int(a),
                          ctypes.c_uint64(traj), ctypes.c_uint64(chain), ctypes.c_long(n), _ptr(out))
    return out


def uniform(seed, tag, traj, chain, i):
    return lib().oracle_uniform(ctypes.c_uint64(seed), ctypes.c_int(tag), ctypes.c_uint64(traj),
                                ctypes.c_uint64(chain), ctypes.c_long(i))


def init_field(seed, chain, n):
    out = np.empty(n)
    lib().oracle_init_field(ctypes.c_uint64(seed), ctypes.c_uint64(chain), ctypes.c_long(n), _ptr(out))
    return out


def heatbath(lat, prm, sigma, traj):
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    chi = np.empty(prm.n_pf * nsites(lat))
    lib().oracle_heatbath(ctypes.byref(lat), ctypes.byref(prm), _ptr(sigma), ctypes.c_uint64(traj), _ptr(chi))
    return chi.reshape(prm.n_pf, -1)


def action(lat, prm, sigma, chi):
    """Returns (S_pf, cg_iterations, max_true_relres, status)."""
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    chi = np.ascontiguousarray(chi, dtype=np.float64).reshape(-1)
    it, rr, st = ctypes.c_int(0), ctypes.c_double(0.0), ctypes.c_int(0)
    S = lib().oracle_action(ctypes.byref(lat), ctypes.byref(prm), _ptr(sigma), _ptr(chi),
                            ctypes.byref(it), ctypes.byref(rr), ctypes.byref(st))
    return S, it.value, rr.value, st.value


def force(lat, prm, sigma, chi):
    """Returns (F, cg_iterations, max_true_relres, status)."""
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    chi = np.ascontiguousarray(chi, dtype=np.float64).reshape(-1)
    F = np.empty(nsites(lat))
    it, rr, st = ctypes.c_int(0), ctypes.c_double(0.0), ctypes.c_int(0)
    lib().oracle_force(ctypes.byref(lat), ctypes.byref(prm), _ptr(sigma), _ptr(chi), _ptr(F),
                       ctypes.byref(it), ctypes.byref(rr), ctypes.byref(st))
    return F, it.value, rr.value, st.value


def leapfrog(lat, prm, sigma, pi, chi, n_md, dt):
    """Evolves copies of (sigma, pi); returns (sigma, pi, cg_iterations, relres, status)."""
    sigma = np.array(sigma, dtype=np.float64, copy=True)
    pi = np.array(pi, dtype=np.float64, copy=True)
    chi = np.ascontiguousarray(chi, dtype=np.float64).reshape(-1)
    it, rr, st = ctypes.c_int(0), ctypes.c_double(0.0), ctypes.c_int(0)
    lib().oracle_leapfrog(ctypes.byref(lat), ctypes.byref(prm), _ptr(sigma), _ptr(pi), _ptr(chi),
                          ctypes.c_int(n_md), ctypes.c_double(dt), ctypes.byref(it),
                          ctypes.byref(rr), ctypes.byref(st))
    return sigma, pi, it.value, rr.value, st.value


def trajectory(lat, prm, sigma, n_md, dt, traj):
    """Runs one trajectory on a copy of sigma; returns (sigma_out, info_dict)."""
    sigma = np.array(sigma, dtype=np.float64, copy=True)
    info = TrajInfo()
    lib().oracle_trajectory(ctypes.byref(lat), ctypes.byref(prm), _ptr(sigma), ctypes.c_int(n_md),
                            ctypes.c_double(dt), ctypes.c_uint64(traj), ctypes.byref(info))
    return sigma, info.as_dict()


def z2_noise(seed, k, traj, chain, n):
    """Z2 noise vector k of the observables (Philox tag 6)."""
    out = np.empty(n)
    lib().oracle_z2_noise(ctypes.c_uint64(seed), ctypes.c_int(k), ctypes.c_uint64(traj), ctypes.c_uint64(chain),
                          ctypes.c_long(n), _ptr(out))
    return out


def observables(lat, prm, sigma, n_noise, traj):
    """Noise estimators (reading R13); returns a dict with trace_Minv (mean of
    (1/N) eta_k . M^{-1} eta_k), trace_err, one_minus_g_sq, mean_sin,
    mean_sin2, cg_iterations, max_relres, status."""
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    out = np.zeros(5)
    it, rr = ctypes.c_int(0), ctypes.c_double(0.0)
    st = lib().oracle_observables(ctypes.byref(lat), ctypes.byref(prm), _ptr(sigma), ctypes.c_int(n_noise),
                                  ctypes.c_uint64(traj), _ptr(out), ctypes.byref(it), ctypes.byref(rr))
    return {"trace_Minv": out[0], "trace_err": out[1], "one_minus_g_sq": out[2], "mean_sin": out[3],
            "mean_sin2": out[4], "cg_iterations": it.value, "max_relres": rr.value, "status": st}


def dense(lat, h, L, which="M", order=0):
    """Dense matrix of M, M^T or M^T M built column by column (small lattices only)."""
    n = nsites(lat)
    fn = {"M": apply_M, "MT": apply_MT, "MTM": apply_MTM}[which]
    if order:
        ex = {"M": apply_M_ex, "MT": apply_MT_ex, "MTM": apply_MTM_ex}[which]
        fn = lambda lat_, h_, L_, x_: ex(lat_, h_, L_, order, x_)
    D = np.empty((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        D[:, j] = fn(lat, h, L, e)
        e[j] = 0.0
    return D
