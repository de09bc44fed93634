"""Gradients of a functional of the state after K ROK4 steps, through
``torch.autograd``: forward K steps with ``rok_step``, backward with
``rok_step_vjp`` (the discrete adjoint of each step, Sec. 2.2.2 / Eq. ROK with
the finite-difference JVP of Eq. matvecFD, eps held constant).

Memory: the forward keeps the state every ``checkpoint_every`` steps; the
backward re-runs one segment at a time from its checkpoint and reverses it
step by step.  With tapes (the default) the re-run records each step's
internals (stages, basis, Hessenberg matrix, stage solves: about 10 + M state
vectors a step, ``rok_step_record``) and the reverse reads them back
(``rok_step_vjp_tape``); the forward records the last segment itself, so it
is not re-run.  Without tapes the re-run keeps only the states and each
reverse step recomputes its own internals (``rok_step_vjp``).  Both give the
same bits.
Argument marshalling and bookkeeping only: every step and every reverse step
runs in the library's kernels.
"""
import torch

from . import rok


class _Integrate(torch.autograd.Function):
    @staticmethod
    def forward(fctx, y0, mu, rctx, h, M, nsteps, every, tapes):
        if abs(float(mu) - float(rctx.problem.mu)) > 0.0:
            raise ValueError('mu must be the viscosity of the context problem')
        y = y0.detach().clone().contiguous()
        checkpoints, last = [], []
        last0 = ((nsteps - 1) // every) * every if nsteps > 0 else 0
        for n in range(nsteps):
            if n % every == 0:
                checkpoints.append(y.clone())
            if tapes and n >= last0:
                last.append(rok.rok_step_record(rctx, y, h, M))
            else:
                rok.rok_step(rctx, y, h, M)
        fctx.rctx, fctx.h, fctx.M, fctx.nsteps, fctx.every = rctx, h, M, nsteps, every
        fctx.checkpoints, fctx.tapes, fctx.last = checkpoints, tapes, last
        return y

    @staticmethod
    def backward(fctx, ybar):
        rctx, h, M, nsteps, every = fctx.rctx, fctx.h, fctx.M, fctx.nsteps, fctx.every
        yb = ybar.detach().contiguous().clone()
        mub = 0.0
        nseg = len(fctx.checkpoints)
        pool = fctx.last   # the last segment's tapes, reused for the earlier segments
        for s in range(nseg - 1, -1, -1):
            n0 = s * every
            n1 = min(n0 + every, nsteps)
            if fctx.tapes:
                if s < nseg - 1:
                    y = fctx.checkpoints[s].clone()
                    for n in range(n0, n1):
                        k = n - n0
                        if k < len(pool):
                            rok.rok_step_record(rctx, y, h, M, pool[k])
                        else:
                            pool.append(rok.rok_step_record(rctx, y, h, M))
                for n in range(n1 - 1, n0 - 1, -1):
                    yb, mb = rok.rok_step_vjp_tape(rctx, pool[n - n0], yb, out=yb)
                    mub += mb
                continue
            states = []
            y = fctx.checkpoints[s].clone()
            for n in range(n0, n1):
                states.append(y.clone())
                if n + 1 < n1:
                    rok.rok_step(rctx, y, h, M)
            for n in range(n1 - 1, n0 - 1, -1):
                yb, mb = rok.rok_step_vjp(rctx, states[n - n0], h, M, yb, out=yb)
                mub += mb
        fctx.checkpoints = fctx.last = None
        return yb, torch.tensor(mub, dtype=torch.float64), None, None, None, None, None, None


def integrate(rctx, y0, mu, h, M, nsteps, checkpoint_every=10, tapes=True):
    """y_K after ``nsteps`` ROK4 steps of size h (Krylov dimension M) from y0,
    differentiable with respect to y0 and mu (a 0-d float64 tensor equal to
    the context problem's viscosity: the constant one, or under Sutherland's
    law the viscosity at t_ref).  ``tapes``: keep each re-run
    step's internals for its reverse (faster, about (10 + M) state vectors per
    step of a segment) instead of recomputing them."""
    return _Integrate.apply(y0, mu, rctx, float(h), int(M), int(nsteps), int(checkpoint_every), bool(tapes))


def kinetic_energy(y):
    """Total kinetic energy sum (rho u^2 + rho v^2) / (2 rho) of a state (differentiable)."""
    return 0.5 * ((y[1] * y[1] + y[2] * y[2]) / y[0]).sum()
