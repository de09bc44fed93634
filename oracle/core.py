"""ctypes wrapper of the C oracle (``residual.c``): residual f(y), FD-JVP, volumes.

TEST INFRASTRUCTURE ONLY.  Lorenz-96 (appendix) is written in NumPy here.
"""
import ctypes
import ctypes.util

import numpy as np

from . import build as _build

_lib = None


class _Problem(ctypes.Structure):
    _fields_ = [
        ('nx', ctypes.c_int), ('ny', ctypes.c_int),
        ('curvilinear', ctypes.c_int), ('viscous', ctypes.c_int),
        ('bc', ctypes.c_int * 4),
        ('dx', ctypes.c_double), ('dy', ctypes.c_double),
        ('xv', ctypes.POINTER(ctypes.c_double)), ('yv', ctypes.POINTER(ctypes.c_double)),
        ('gamma', ctypes.c_double), ('prandtl', ctypes.c_double),
        ('mu_ref', ctypes.c_double), ('t_ref', ctypes.c_double), ('suth_s', ctypes.c_double),
        ('q_inf', ctypes.c_double * 4),
        ('kappa', ctypes.c_double), ('efix', ctypes.c_double),
    ]


_parallel = False


def use_parallel_build(threads):
    """Switch the residual to the OpenMP build of the same source (identical
    bits) with `threads` threads, or back to the plain build (threads=None).
    Only the CPU-baseline timing uses this."""
    global _lib, _parallel
    want = threads is not None
    if want != _parallel:
        _lib = None
        _parallel = want
    lib()
    if want:
        ctypes.CDLL(ctypes.util.find_library('gomp') or 'libgomp.so.1').omp_set_num_threads(int(threads))


def lib():
    global _lib
    if _lib is None:
        path = _build.build_parallel() if _parallel else _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        L.oracle_residual.argtypes = [ctypes.POINTER(_Problem), dp, dp]
        L.oracle_residual.restype = ctypes.c_int
        L.oracle_jvp_fd.argtypes = [ctypes.POINTER(_Problem), dp, dp, dp, ctypes.c_double, dp]
        L.oracle_jvp_fd.restype = ctypes.c_int
        L.oracle_cell_volumes.argtypes = [ctypes.POINTER(_Problem), dp]
        L.oracle_cell_volumes.restype = ctypes.c_int
        L.oracle_roe_flux.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, dp]
        L.oracle_roe_flux.restype = None
        L.oracle_jvp_cs.argtypes = [ctypes.POINTER(_Problem), dp, dp, ctypes.c_double, dp]
        L.oracle_jvp_cs.restype = ctypes.c_int
        L.oracle_residual_cx.argtypes = [ctypes.POINTER(_Problem), dp, dp, dp, dp]
        L.oracle_residual_cx.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class _Desc:
    """Holds the ctypes struct and keeps the vertex arrays alive."""

    def __init__(self, prob):
        s = _Problem()
        s.nx, s.ny = prob.nx, prob.ny
        s.curvilinear = 1 if prob.xv is not None else 0
        s.viscous = 1 if prob.kind == 1 else 0
        for k in range(4):
            s.bc[k] = int(prob.bc[k])
            s.q_inf[k] = float(prob.q_inf[k])
        s.dx = prob.lx / prob.nx
        s.dy = prob.ly / prob.ny
        self._xv = self._yv = None
        if prob.xv is not None:
            self._xv = np.ascontiguousarray(prob.xv, dtype=np.float64)
            self._yv = np.ascontiguousarray(prob.yv, dtype=np.float64)
            s.xv, s.yv = _dp(self._xv), _dp(self._yv)
        s.gamma, s.prandtl = prob.gamma, prob.prandtl
        s.mu_ref, s.t_ref, s.suth_s = prob.mu, prob.t_ref, prob.sutherland_s
        s.kappa, s.efix = prob.muscl_kappa, prob.entropy_fix
        self.s = s


_cache = {}


def _desc(prob):
    key = id(prob)
    d = _cache.get(key)
    if d is None or d[0] is not prob:
        d = (prob, _Desc(prob))
        _cache[key] = d
    return d[1]


def lorenz96_rhs(prob, u):
    """Lorenz-96 (appendix): du_i/dt = (u_{i+1} - u_{i-2}) u_{i-1} - u_i + F, periodic."""
    return (np.roll(u, -1) - np.roll(u, 2)) * np.roll(u, 1) - u + prob.lorenz_f


def residual(prob, y):
    """f(y) for the problem; y has ``prob.shape``; returns a new float64 array
    (complex128 for a complex y: the same residual continued analytically, for
    complex-step derivatives of the integrators)."""
    if np.iscomplexobj(y):
        return _residual_complex(prob, y)
    y = np.ascontiguousarray(y, dtype=np.float64)
    if prob.kind == 2:
        return lorenz96_rhs(prob, y)
    f = np.empty_like(y)
    rc = lib().oracle_residual(ctypes.byref(_desc(prob).s), _dp(y), _dp(f))
    if rc != 0:
        raise MemoryError('oracle_residual failed')
    return f


def _residual_complex(prob, y):
    y = np.ascontiguousarray(y, dtype=np.complex128)
    if prob.kind == 2:
        return lorenz96_rhs(prob, y)
    q_re, q_im = np.ascontiguousarray(y.real), np.ascontiguousarray(y.imag)
    f_re, f_im = np.empty_like(q_re), np.empty_like(q_re)
    rc = lib().oracle_residual_cx(ctypes.byref(_desc(prob).s), _dp(q_re), _dp(q_im), _dp(f_re), _dp(f_im))
    if rc != 0:
        raise MemoryError('oracle_residual_cx failed')
    return f_re + 1j * f_im


def jvp_fd(prob, y, v, f0, eps):
    """Eq. matvecFD: (f(y + eps v) - f0) / eps."""
    if np.iscomplexobj(y) or np.iscomplexobj(v) or np.iscomplexobj(f0):
        return (_residual_complex(prob, np.asarray(y) + eps * np.asarray(v)) - f0) / eps
    y = np.ascontiguousarray(y, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    f0 = np.ascontiguousarray(f0, dtype=np.float64)
    if prob.kind == 2:
        return (lorenz96_rhs(prob, y + eps * v) - f0) / eps
    w = np.empty_like(y)
    rc = lib().oracle_jvp_fd(ctypes.byref(_desc(prob).s), _dp(y), _dp(v), _dp(f0), float(eps), _dp(w))
    if rc != 0:
        raise MemoryError('oracle_jvp_fd failed')
    return w


def jvp_exact(prob, y, v, h=1e-100):
    """Exact Jacobian-vector product J(y) v: the complex-step derivative
    Im f(y + i h v) / h of the same residual (no cancellation, exact to
    rounding); analytic for Lorenz-96."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    if prob.kind == 2:
        return (np.roll(v, -1) - np.roll(v, 2)) * np.roll(y, 1) + (np.roll(y, -1) - np.roll(y, 2)) * np.roll(v, 1) - v
    w = np.empty_like(y)
    rc = lib().oracle_jvp_cs(ctypes.byref(_desc(prob).s), _dp(y), _dp(v), float(h), _dp(w))
    if rc != 0:
        raise MemoryError('oracle_jvp_cs failed')
    return w


def cell_volumes(prob):
    vol = np.empty((prob.ny, prob.nx))
    lib().oracle_cell_volumes(ctypes.byref(_desc(prob).s), _dp(vol))
    return vol


def roe_flux(WL, WR, nx, ny, gamma=1.4, efix=0.1):
    """Roe face flux for primitive states (rho, u, v, p) and unit normal (nx, ny)."""
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    F = np.empty(4)
    lib().oracle_roe_flux(_dp(WL), _dp(WR), float(nx), float(ny), float(gamma), float(efix), _dp(F))
    return F


class System:
    """f and the FD Jacobian-vector product of one problem, as callables on
    arrays of ``prob.shape`` (the integrators only see this interface)."""

    def __init__(self, prob):
        self.prob = prob
        self.shape = prob.shape

    def f(self, y):
        return residual(self.prob, y)

    def jvp(self, y, v, f0, eps):
        return jvp_fd(self.prob, y, v, f0, eps)


class ExactSystem(System):
    """The same f with the exact (complex-step) Jacobian-vector product."""

    def jvp(self, y, v, f0, eps):
        return jvp_exact(self.prob, y, v)
