"""Thin ctypes binding of ``librok.so`` (C ABI in ``include/rok.h``).

Argument marshalling only: every function forwards to the C entry point of
the same name with raw device pointers and sizes; all arithmetic runs in the
library's CUDA kernels.  State tensors are float64 CUDA tensors of shape
``problem.shape`` (contiguous).  CPU tensors are accepted by the step calls
for end-to-end use: they are copied to a device buffer, stepped and copied
back (host<->device copies, nothing else, on the host side).

Importing this module loads the library and raises if it has not been built
(``python -c "import __graft_entry__ as g; g.build()"``); there is no CPU
fallback.
"""
import ctypes
import os

import numpy as np
import torch

from . import workloads as _W

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), '_lib', 'librok.so')
if not os.path.exists(_LIB_PATH):
    raise ImportError('librok.so is not built (%s); run __graft_entry__.build()' % _LIB_PATH)
_lib = ctypes.CDLL(_LIB_PATH)

ROK_OK, ROK_ERR_INVALID_ARG, ROK_ERR_CUDA, ROK_ERR_NONFINITE = 0, 1, 2, 3
ROK_ERR_NOT_CONVERGED, ROK_ERR_TIMEOUT, ROK_ERR_UNSUPPORTED, ROK_ERR_NOMEM = 4, 5, 6, 7
ROK_JVP_FD, ROK_JVP_EXACT = 0, 1
ROK_ROUND_FAST, ROK_ROUND_STRICT = 0, 1
ROK_BASIS_FP64, ROK_BASIS_FP32 = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)


class ProblemDesc(ctypes.Structure):
    _fields_ = [
        ('kind', ctypes.c_int), ('nx', ctypes.c_int), ('ny', ctypes.c_int),
        ('xv', _dp), ('yv', _dp), ('lx', ctypes.c_double), ('ly', ctypes.c_double),
        ('bc', ctypes.c_int * 4),
        ('gamma', ctypes.c_double), ('prandtl', ctypes.c_double), ('mu', ctypes.c_double),
        ('t_ref', ctypes.c_double), ('sutherland_s', ctypes.c_double),
        ('q_inf', ctypes.c_double * 4),
        ('muscl_kappa', ctypes.c_double), ('entropy_fix', ctypes.c_double), ('lorenz_f', ctypes.c_double),
        ('krylov_max', ctypes.c_int), ('rounding', ctypes.c_int), ('basis', ctypes.c_int),
        ('jvp', ctypes.c_int),
    ]


class StepInfo(ctypes.Structure):
    _fields_ = [('status', ctypes.c_int), ('m_eff', ctypes.c_int), ('residual_evals', ctypes.c_int),
                ('jvps', ctypes.c_int), ('newton_iters', ctypes.c_int), ('gmres_iters', ctypes.c_int),
                ('eps', ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class EsdirkOpts(ctypes.Structure):
    _fields_ = [('gmres_m', ctypes.c_int), ('gmres_tol', ctypes.c_double), ('gmres_restarts', ctypes.c_int),
                ('newton_tol', ctypes.c_double), ('newton_max', ctypes.c_int)]


class Counters(ctypes.Structure):
    _fields_ = [('launches', ctypes.c_longlong), ('stencil_launches', ctypes.c_longlong),
                ('stencil_ms', ctypes.c_double), ('stencil_timed', ctypes.c_longlong)]


class AdaptOpts(ctypes.Structure):
    _fields_ = [('atol', ctypes.c_double), ('rtol', ctypes.c_double), ('h0', ctypes.c_double),
                ('safety', ctypes.c_double), ('facmin', ctypes.c_double), ('facmax', ctypes.c_double),
                ('max_steps', ctypes.c_int)]


class AdaptInfo(ctypes.Structure):
    _fields_ = [('accepted', ctypes.c_int), ('rejected', ctypes.c_int), ('t', ctypes.c_double),
                ('h_next', ctypes.c_double), ('residual_evals', ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


ROK_TILE_32x8, ROK_TILE_16x16, ROK_TILE_64x4 = 0, 1, 2
CHUNKS_PER_CTA = (1, 2, 4, 8)


class BatchTuning(ctypes.Structure):
    _fields_ = [('tile', ctypes.c_int * 3), ('chunks_per_cta', ctypes.c_int), ('vec_chunks_per_cta', ctypes.c_int),
                ('stencil_ms', (ctypes.c_float * 3) * 3), ('mgs_ms', ctypes.c_float * 4),
                ('vec_ms', ctypes.c_float * 4)]

    def as_dict(self):
        return {'tile': list(self.tile), 'chunks_per_cta': self.chunks_per_cta,
                'vec_chunks_per_cta': self.vec_chunks_per_cta,
                'stencil_ms': [list(r) for r in self.stencil_ms], 'mgs_ms': list(self.mgs_ms),
                'vec_ms': list(self.vec_ms)}


_vp = ctypes.c_void_p
_sig = {
    'rok_init': (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(ProblemDesc), _vp]),
    'rok_destroy': (ctypes.c_int, [_vp]),
    'rok_set_stream': (ctypes.c_int, [_vp, _vp]),
    'rok_residual': (ctypes.c_int, [_vp, _vp, _vp]),
    'rok_jvp': (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_int]),
    'rok_arnoldi': (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.POINTER(ctypes.c_int)]),
    'rok_step': (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.c_int, ctypes.POINTER(StepInfo)]),
    'rk_step': (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.POINTER(StepInfo)]),
    'esdirk_step': (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.POINTER(EsdirkOpts), ctypes.POINTER(StepInfo)]),
    'ros_step': (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.c_int, ctypes.POINTER(EsdirkOpts),
                                ctypes.POINTER(StepInfo)]),
    'rok_dt_from_cfl': (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    'rok_sync': (ctypes.c_int, [_vp, ctypes.POINTER(StepInfo)]),
    'rok_set_graph': (ctypes.c_int, [_vp, ctypes.c_int]),
    'rok_set_persistent': (ctypes.c_int, [_vp, ctypes.c_int]),
    'rok_get_counters': (ctypes.c_int, [_vp, ctypes.POINTER(Counters), ctypes.c_int]),
    'rok_set_stencil_timing': (ctypes.c_int, [_vp, ctypes.c_int]),
    'rok_status_string': (ctypes.c_char_p, [ctypes.c_int]),
    'rok_fp64_fma_peak': (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    'rok_integrate': (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.c_int, ctypes.POINTER(AdaptOpts),
                                     ctypes.POINTER(AdaptInfo)]),
    'dopri5_integrate': (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.POINTER(AdaptOpts),
                                        ctypes.POINTER(AdaptInfo)]),
    'rok_vjp': (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_double)]),
    'rok_step_vjp': (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.c_int, _vp, _vp, ctypes.POINTER(ctypes.c_double)]),
    'rok_tape_bytes': (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    'rok_step_record': (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.c_int, _vp]),
    'rok_step_vjp_tape': (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_double)]),
    'rok_batch_init': (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(ProblemDesc), ctypes.c_int, _vp]),
    'rok_batch_destroy': (ctypes.c_int, [_vp]),
    'rok_batch_layout': (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    'rok_batch_residual': (ctypes.c_int, [_vp, _vp, _vp]),
    'rok_batch_step': (ctypes.c_int, [_vp, _vp, _dp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(StepInfo)]),
    'rok_batch_tune': (ctypes.c_int, [_vp, _vp, ctypes.POINTER(BatchTuning)]),
    'rok_batch_set_tuning': (ctypes.c_int, [_vp, ctypes.POINTER(BatchTuning)]),
    'rok_batch_get_tuning': (ctypes.c_int, [_vp, ctypes.POINTER(BatchTuning)]),
    'rok_batch_set_graph': (ctypes.c_int, [_vp, ctypes.c_int]),
    'rok_batch_get_launches': (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]),
    'rok_jvp_noalloc': (ctypes.c_int, [ctypes.POINTER(ProblemDesc), _vp, _vp, _vp, _vp, ctypes.c_double, _vp, _vp]),
    'rok_selftest_wait': (ctypes.c_int, [_vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    'rok_selftest_rcp': (ctypes.c_int, [_vp, _vp, ctypes.c_longlong, _vp]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sig)


class RokError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__('%s: %s (status %d)' % (where, rok_status_string(status), status))


def rok_status_string(status):
    return _lib.rok_status_string(int(status)).decode()


def _check(status, where):
    if status != ROK_OK:
        raise RokError(status, where)


def _ptr(t, numel=None, dtype=torch.float64):
    """Raw device pointer of a tensor after checking what the C ABI cannot:
    a contiguous tensor of `dtype` on the current CUDA device, with `numel`
    entries when given.  A CPU tensor or one of the wrong size would otherwise
    reach the kernels as an out-of-bounds or host address."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError('expected a torch tensor, got %s' % type(t).__name__)
    if not t.is_contiguous() or t.dtype != dtype:
        raise ValueError('expected a contiguous %s tensor' % dtype)
    if not t.is_cuda:
        raise ValueError('expected a CUDA tensor (device memory), got one on %s' % t.device)
    if t.device.index != torch.cuda.current_device():
        raise ValueError('tensor on %s but the current device is cuda:%d' % (t.device, torch.cuda.current_device()))
    if numel is not None and t.numel() != numel:
        raise ValueError('expected %d entries, got %d' % (numel, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """Owns one ``rok_ctx``; created by :func:`rok_init`."""

    def __init__(self, handle, problem, stream):
        self.handle = handle
        self.problem = problem
        self.stream = stream
        self._stage = None

    def __del__(self):
        try:
            if self.handle:
                _lib.rok_destroy(self.handle)
                self.handle = None
        except Exception:
            pass

    def _dev_state(self, y):
        """Device view of a state; CPU tensors are staged through a device buffer."""
        if y.is_cuda:
            return y, None
        if self._stage is None or self._stage.shape != y.shape:
            self._stage = torch.empty(y.shape, dtype=torch.float64, device='cuda')
        self._stage.copy_(y, non_blocking=True)
        return self._stage, y


def _desc(problem, krylov_max, rounding, basis=0, jvp=0):
    d = ProblemDesc()
    d.kind = int(problem.kind)
    d.nx, d.ny = int(problem.nx), int(problem.ny)
    keep = []
    if problem.xv is not None:
        xv = np.ascontiguousarray(problem.xv, dtype=np.float64)
        yv = np.ascontiguousarray(problem.yv, dtype=np.float64)
        keep = [xv, yv]
        d.xv = xv.ctypes.data_as(_dp)
        d.yv = yv.ctypes.data_as(_dp)
    d.lx, d.ly = float(problem.lx), float(problem.ly)
    for k in range(4):
        d.bc[k] = int(problem.bc[k])
        d.q_inf[k] = float(problem.q_inf[k])
    d.gamma, d.prandtl, d.mu = float(problem.gamma), float(problem.prandtl), float(problem.mu)
    d.t_ref, d.sutherland_s = float(problem.t_ref), float(problem.sutherland_s)
    d.muscl_kappa, d.entropy_fix, d.lorenz_f = float(problem.muscl_kappa), float(problem.entropy_fix), float(problem.lorenz_f)
    d.krylov_max = int(krylov_max)
    d.rounding = int(rounding)
    d.basis = int(basis)
    d.jvp = int(jvp)
    return d, keep


def rok_init(problem, krylov_max=20, rounding=ROK_ROUND_FAST, stream=None, basis=ROK_BASIS_FP64, jvp=ROK_JVP_FD):
    """Create a context (``rok_init``) for a :class:`workloads.FlowProblem`."""
    if stream is None:
        stream = torch.cuda.current_stream()
    d, keep = _desc(problem, krylov_max, rounding, basis, jvp)
    h = ctypes.c_void_p()
    _check(_lib.rok_init(ctypes.byref(h), ctypes.byref(d), ctypes.c_void_p(stream.cuda_stream)), 'rok_init')
    del keep
    return Context(h, problem, stream)


def rok_destroy(ctx):
    _check(_lib.rok_destroy(ctx.handle), 'rok_destroy')
    ctx.handle = None


def rok_set_stream(ctx, stream):
    ctx.stream = stream
    _check(_lib.rok_set_stream(ctx.handle, ctypes.c_void_p(stream.cuda_stream)), 'rok_set_stream')


def rok_residual(ctx, y, f=None):
    if f is None:
        f = torch.empty_like(y)
    n = ctx.problem.ndof
    _check(_lib.rok_residual(ctx.handle, _ptr(y, n), _ptr(f, n)), 'rok_residual')
    return f


def rok_jvp(ctx, y, v, fy=None, eps=0.0, mode=ROK_JVP_FD, out=None):
    if out is None:
        out = torch.empty_like(y)
    n = ctx.problem.ndof
    _check(_lib.rok_jvp(ctx.handle, _ptr(y, n), _ptr(fy, n), _ptr(v, n), _ptr(out, n), float(eps), int(mode)),
           'rok_jvp')
    return out


def rok_arnoldi(ctx, y, M):
    """Returns (V[M_eff, N], H[M, M], M_eff)."""
    N = y.numel()
    V = torch.zeros((M, N), dtype=torch.float64, device=y.device)
    H = torch.zeros((M, M), dtype=torch.float64, device=y.device)
    me = ctypes.c_int(0)
    _check(_lib.rok_arnoldi(ctx.handle, _ptr(y, ctx.problem.ndof), int(M), _ptr(V), _ptr(H), ctypes.byref(me)),
           'rok_arnoldi')
    return V[:me.value], H, me.value


def _step_call(ctx, y, where, call, info):
    yd, host = ctx._dev_state(y)
    _ptr(yd, ctx.problem.ndof)
    si = StepInfo()
    st = call(yd, ctypes.byref(si) if (info or host is not None) else None)
    if host is not None:
        host.copy_(yd, non_blocking=False)
    _check(st, where)
    return si.as_dict() if info else None


def rok_step(ctx, y, h, M, info=False):
    """One ROK4 step in place (``rok_step``); returns the step info dict when info=True."""
    return _step_call(ctx, y, 'rok_step', lambda yd, ip: _lib.rok_step(ctx.handle, _ptr(yd), float(h), int(M), ip), info)


def rk_step(ctx, y, h, info=False):
    return _step_call(ctx, y, 'rk_step', lambda yd, ip: _lib.rk_step(ctx.handle, _ptr(yd), float(h), ip), info)


def esdirk_step(ctx, y, h, gmres_m=30, gmres_tol=1e-6, gmres_restarts=5, newton_tol=1e-10, newton_max=10, info=False):
    o = EsdirkOpts(int(gmres_m), float(gmres_tol), int(gmres_restarts), float(newton_tol), int(newton_max))
    return _step_call(ctx, y, 'esdirk_step',
                      lambda yd, ip: _lib.esdirk_step(ctx.handle, _ptr(yd), float(h), ctypes.byref(o), ip), info)


ROK_ROS_ROS4 = 0
ROK_ROS_ROW = 1


def ros_step(ctx, y, h, method=ROK_ROS_ROS4, gmres_m=30, gmres_tol=1e-6, gmres_restarts=5, info=False):
    """``ros_step``: one Rosenbrock (ROS4) or Rosenbrock-W (ROW) step, Eq. ROS."""
    o = EsdirkOpts(int(gmres_m), float(gmres_tol), int(gmres_restarts), 1e-10, 10)
    return _step_call(ctx, y, 'ros_step',
                      lambda yd, ip: _lib.ros_step(ctx.handle, _ptr(yd), float(h), int(method), ctypes.byref(o), ip),
                      info)


def rok_dt_from_cfl(ctx, y, cfl):
    dt = ctypes.c_double(0.0)
    _check(_lib.rok_dt_from_cfl(ctx.handle, _ptr(y, ctx.problem.ndof), float(cfl), ctypes.byref(dt)), 'rok_dt_from_cfl')
    return dt.value


def rok_sync(ctx):
    si = StepInfo()
    _check(_lib.rok_sync(ctx.handle, ctypes.byref(si)), 'rok_sync')
    return si.as_dict()


def rok_set_graph(ctx, enable):
    _check(_lib.rok_set_graph(ctx.handle, int(bool(enable))), 'rok_set_graph')


def rok_set_persistent(ctx, enable):
    """``rok_set_persistent``: one cooperative launch per Arnoldi column (and
    per reverse column) where it fits (True, default) or one launch per
    Gram-Schmidt pass (False)."""
    _check(_lib.rok_set_persistent(ctx.handle, int(bool(enable))), 'rok_set_persistent')


def rok_get_counters(ctx, reset=False):
    c = Counters()
    _check(_lib.rok_get_counters(ctx.handle, ctypes.byref(c), int(bool(reset))), 'rok_get_counters')
    return {k: getattr(c, k) for k, _ in c._fields_}


def rok_set_stencil_timing(ctx, enable):
    _check(_lib.rok_set_stencil_timing(ctx.handle, int(bool(enable))), 'rok_set_stencil_timing')


def _adapt(atol, rtol, h0, safety, facmin, facmax, max_steps):
    return AdaptOpts(float(atol), float(rtol), float(h0), float(safety), float(facmin), float(facmax), int(max_steps))


def rok_integrate(ctx, y, T, M, atol, rtol, h0, safety=0.9, facmin=0.2, facmax=5.0, max_steps=100000):
    """``rok_integrate``: adaptive ROK4 from 0 to T in place; returns the info dict."""
    o = _adapt(atol, rtol, h0, safety, facmin, facmax, max_steps)
    info = AdaptInfo()
    _check(_lib.rok_integrate(ctx.handle, _ptr(y, ctx.problem.ndof), float(T), int(M), ctypes.byref(o), ctypes.byref(info)),
           'rok_integrate')
    return info.as_dict()


def dopri5_integrate(ctx, y, T, atol, rtol, h0, safety=0.9, facmin=0.2, facmax=5.0, max_steps=100000):
    """``dopri5_integrate``: adaptive Dormand-Prince 5(4) from 0 to T in place."""
    o = _adapt(atol, rtol, h0, safety, facmin, facmax, max_steps)
    info = AdaptInfo()
    _check(_lib.dopri5_integrate(ctx.handle, _ptr(y, ctx.problem.ndof), float(T), ctypes.byref(o), ctypes.byref(info)),
           'dopri5_integrate')
    return info.as_dict()


def rok_vjp(ctx, y, ubar, out=None, mubar=False):
    """``rok_vjp``: J(y)^T ubar (and, with mubar=True, also ubar . df/dmu;
    returns (ybar, mubar) then)."""
    if out is None:
        out = torch.empty_like(y)
    mb = ctypes.c_double(0.0)
    n = ctx.problem.ndof
    _check(_lib.rok_vjp(ctx.handle, _ptr(y, n), _ptr(ubar, n), _ptr(out, n), ctypes.byref(mb) if mubar else None),
           'rok_vjp')
    return (out, mb.value) if mubar else out


def rok_step_vjp(ctx, y, h, M, ybar, out=None):
    """``rok_step_vjp``: reverse of one ROK4 step from y_n = y; returns
    (ybar_n, mubar of the step)."""
    if out is None:
        out = torch.empty_like(y)
    mb = ctypes.c_double(0.0)
    n = ctx.problem.ndof
    _check(_lib.rok_step_vjp(ctx.handle, _ptr(y, n), float(h), int(M), _ptr(ybar, n), _ptr(out, n), ctypes.byref(mb)),
           'rok_step_vjp')
    return out, mb.value


def rok_tape_bytes(ctx, M):
    """``rok_tape_bytes``: bytes of a tape for Krylov dimension M."""
    n = ctypes.c_size_t(0)
    _check(_lib.rok_tape_bytes(ctx.handle, int(M), ctypes.byref(n)), 'rok_tape_bytes')
    return n.value


def _tape_ptr(tape):
    return _ptr(tape, None, torch.uint8)


def rok_step_record(ctx, y, h, M, tape=None):
    """``rok_step_record``: one ROK4 step of y in place that also writes the
    step's tape (a uint8 device tensor of ``rok_tape_bytes(ctx, M)`` bytes,
    allocated when None); returns the tape."""
    if tape is None:
        tape = torch.empty(rok_tape_bytes(ctx, M), dtype=torch.uint8, device=y.device)
    _check(_lib.rok_step_record(ctx.handle, _ptr(y, ctx.problem.ndof), float(h), int(M), _tape_ptr(tape)),
           'rok_step_record')
    return tape


def rok_step_vjp_tape(ctx, tape, ybar, out=None):
    """``rok_step_vjp_tape``: reverse of the step a tape recorded; returns
    (ybar_n, mubar of the step)."""
    if out is None:
        out = torch.empty_like(ybar)
    mb = ctypes.c_double(0.0)
    n = ctx.problem.ndof
    _check(_lib.rok_step_vjp_tape(ctx.handle, _tape_ptr(tape), _ptr(ybar, n), _ptr(out, n), ctypes.byref(mb)),
           'rok_step_vjp_tape')
    return out, mb.value


class Batch:
    """Owns one ``rok_batch`` (many independent problems stepped together);
    created by :func:`rok_batch_init`.  ``offsets[k]`` is the first entry of
    instance k in the flat state vector of ``total`` entries."""

    def __init__(self, handle, problems, stream, total, offsets):
        self.handle = handle
        self.problems = list(problems)
        self.stream = stream
        self.total = total
        self.offsets = offsets

    def __del__(self):
        try:
            if self.handle:
                _lib.rok_batch_destroy(self.handle)
                self.handle = None
        except Exception:
            pass

    def view(self, y, k):
        """Instance k's state inside the flat vector y, shape problems[k].shape."""
        p = self.problems[k]
        n = 4 * p.nx * p.ny
        return y[self.offsets[k]:self.offsets[k] + n].view(p.shape)

    def pack(self, states, device='cuda'):
        """Flat state vector from per-instance states (NumPy arrays or tensors)."""
        y = torch.zeros(self.total, dtype=torch.float64, device=device)
        for k, s in enumerate(states):
            t = s if isinstance(s, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(s, dtype=np.float64))
            self.view(y, k).copy_(t.reshape(self.problems[k].shape))
        return y

    def unpack(self, y):
        """Per-instance NumPy states of a flat vector."""
        yh = y.detach().cpu()
        return [self.view(yh, k).numpy().copy() for k in range(len(self.problems))]


def rok_batch_init(problems, krylov_max=16, rounding=ROK_ROUND_FAST, stream=None):
    """Create a batch (``rok_batch_init``) of uniform periodic problems."""
    if stream is None:
        stream = torch.cuda.current_stream()
    n = len(problems)
    arr = (ProblemDesc * n)()
    for k, p in enumerate(problems):
        d, _ = _desc(p, krylov_max, rounding)
        arr[k] = d
    h = ctypes.c_void_p()
    _check(_lib.rok_batch_init(ctypes.byref(h), arr, n, ctypes.c_void_p(stream.cuda_stream)), 'rok_batch_init')
    total = ctypes.c_size_t(0)
    offs = (ctypes.c_size_t * n)()
    _check(_lib.rok_batch_layout(h, ctypes.byref(total), offs), 'rok_batch_layout')
    return Batch(h, problems, stream, total.value, [int(o) for o in offs])


def rok_batch_layout(b):
    """(total, offsets) of the flat state vector."""
    total = ctypes.c_size_t(0)
    offs = (ctypes.c_size_t * len(b.problems))()
    _check(_lib.rok_batch_layout(b.handle, ctypes.byref(total), offs), 'rok_batch_layout')
    return total.value, [int(o) for o in offs]


def rok_batch_destroy(b):
    _check(_lib.rok_batch_destroy(b.handle), 'rok_batch_destroy')
    b.handle = None


def rok_batch_residual(b, y, f=None):
    if f is None:
        f = torch.zeros_like(y)
    _check(_lib.rok_batch_residual(b.handle, _ptr(y, b.total), _ptr(f, b.total)), 'rok_batch_residual')
    return f


def rok_batch_step(b, y, h, M, nsteps=1, info=False):
    """``nsteps`` ROK4 steps of every instance in place; h: one step size per
    instance (or one for all).  info=True synchronises and returns the
    per-instance info dicts (a failed instance shows in its ``status``);
    info=False raises only on argument or CUDA errors."""
    hv = np.ascontiguousarray(np.broadcast_to(np.asarray(h, dtype=np.float64), (len(b.problems),)))
    si = (StepInfo * len(b.problems))() if info else None
    st = _lib.rok_batch_step(b.handle, _ptr(y, b.total), hv.ctypes.data_as(_dp), int(M), int(nsteps), si)
    if not info:
        _check(st, 'rok_batch_step')
        return None
    out = [s.as_dict() for s in si]
    if st not in (ROK_OK, ROK_ERR_NONFINITE, ROK_ERR_TIMEOUT):
        _check(st, 'rok_batch_step')
    return out


def rok_batch_tune(b, y):
    t = BatchTuning()
    _check(_lib.rok_batch_tune(b.handle, _ptr(y, b.total), ctypes.byref(t)), 'rok_batch_tune')
    return t.as_dict()


def rok_batch_set_tuning(b, tile=(0, 0, 0), chunks_per_cta=1, vec_chunks_per_cta=1):
    t = BatchTuning()
    for g in range(3):
        t.tile[g] = int(tile[g])
    t.chunks_per_cta, t.vec_chunks_per_cta = int(chunks_per_cta), int(vec_chunks_per_cta)
    _check(_lib.rok_batch_set_tuning(b.handle, ctypes.byref(t)), 'rok_batch_set_tuning')


def rok_batch_get_tuning(b):
    t = BatchTuning()
    _check(_lib.rok_batch_get_tuning(b.handle, ctypes.byref(t)), 'rok_batch_get_tuning')
    return t.as_dict()


def rok_batch_set_graph(b, enable):
    _check(_lib.rok_batch_set_graph(b.handle, int(bool(enable))), 'rok_batch_set_graph')


def rok_batch_get_launches(b, reset=False):
    n = ctypes.c_longlong(0)
    _check(_lib.rok_batch_get_launches(b.handle, ctypes.byref(n), int(bool(reset))), 'rok_batch_get_launches')
    return n.value


ROK_NOALLOC_MAX_N = 4096 * 2048


def rok_jvp_noalloc(problem, y, v, fy, out, eps=0.0, status=None, rounding=ROK_ROUND_FAST, stream=None):
    """``rok_jvp_noalloc``: FD Jacobian-vector product without any device
    allocation by the library (no context; scratch in a static device array).
    ``y``, ``v``, ``fy`` and ``out`` are float64 CUDA tensors of
    ``problem.ndof`` entries on the current device; ``out`` (and the optional
    one-entry int32 CUDA tensor ``status``) are the caller's.  Every tensor is
    checked here before the call: the C entry point has no context that could
    catch a size or device mismatch."""
    if stream is None:
        stream = torch.cuda.current_stream()
    d, keep = _desc(problem, 0, rounding)
    n = problem.ndof
    st = _ptr(status, 1, torch.int32) if status is not None else None
    _check(_lib.rok_jvp_noalloc(ctypes.byref(d), _ptr(y, n), _ptr(fy, n), _ptr(v, n), _ptr(out, n), float(eps), st,
                                ctypes.c_void_p(stream.cuda_stream)), 'rok_jvp_noalloc')
    del keep
    return out


def rok_fp64_fma_peak(repeats=20):
    """Measured FP64 FMA throughput of the current device, TFLOP/s."""
    t = ctypes.c_double(0.0)
    _check(_lib.rok_fp64_fma_peak(ctypes.byref(t), int(repeats)), 'rok_fp64_fma_peak')
    return t.value


def rok_selftest_wait(ctx, polls=20000):
    """``rok_selftest_wait``: run the bounded wait of the persistent kernels on
    a counter nothing advances; returns (expired, GPU ms)."""
    ex = ctypes.c_int(0)
    ms = ctypes.c_double(0.0)
    _check(_lib.rok_selftest_wait(ctx.handle, int(polls), ctypes.byref(ex), ctypes.byref(ms)), 'rok_selftest_wait')
    return ex.value, ms.value


def state_tensor(y, device='cuda'):
    """float64 tensor of a NumPy state on the device (helper for callers)."""
    return torch.from_numpy(np.ascontiguousarray(y, dtype=np.float64)).to(device)


def rok_selftest_rcp(x, out=None, stream=None):
    """``rok_selftest_rcp``: the FMA-build stencil's reciprocal of every entry of
    the float64 CUDA tensor x."""
    if stream is None:
        stream = torch.cuda.current_stream()
    if out is None:
        out = torch.empty_like(x)
    n = x.numel()
    _check(_lib.rok_selftest_rcp(_ptr(x, n), _ptr(out, n), int(n), ctypes.c_void_p(stream.cuda_stream)),
           'rok_selftest_rcp')
    return out
