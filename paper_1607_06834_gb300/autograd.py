"""Gradients of a functional of the state after K ROK4 steps, through
``torch.autograd``: forward K steps with ``rok_step``, backward with
``rok_step_vjp`` (the discrete adjoint of each step, Sec. 2.3.3 / Eq. ROK with
the finite-difference JVP of Eq. matvecFD, eps held constant).

Memory: the forward keeps the state every ``checkpoint_every`` steps; the
backward re-runs one segment at a time from its checkpoint, keeping that
segment's states, and reverses it step by step (each reverse step recomputes
its own stages, basis and stage solves from the step's start state).
Argument marshalling and bookkeeping only: every step and every reverse step
runs in the library's kernels.
"""
import torch

from . import rok


class _Integrate(torch.autograd.Function):
    @staticmethod
    def forward(fctx, y0, mu, rctx, h, M, nsteps, every):
        if abs(float(mu) - float(rctx.problem.mu)) > 0.0:
            raise ValueError('mu must be the viscosity of the context problem')
        y = y0.detach().clone().contiguous()
        checkpoints = []
        for n in range(nsteps):
            if n % every == 0:
                checkpoints.append(y.clone())
            rok.rok_step(rctx, y, h, M)
        fctx.rctx, fctx.h, fctx.M, fctx.nsteps, fctx.every = rctx, h, M, nsteps, every
        fctx.checkpoints = checkpoints
        return y

    @staticmethod
    def backward(fctx, ybar):
        rctx, h, M, nsteps, every = fctx.rctx, fctx.h, fctx.M, fctx.nsteps, fctx.every
        yb = ybar.detach().contiguous().clone()
        mub = 0.0
        nseg = len(fctx.checkpoints)
        for s in range(nseg - 1, -1, -1):
            n0 = s * every
            n1 = min(n0 + every, nsteps)
            states = []
            y = fctx.checkpoints[s].clone()
            for n in range(n0, n1):
                states.append(y.clone())
                if n + 1 < n1:
                    rok.rok_step(rctx, y, h, M)
            for n in range(n1 - 1, n0 - 1, -1):
                yb, mb = rok.rok_step_vjp(rctx, states[n - n0], h, M, yb, out=yb)
                mub += mb
        fctx.checkpoints = None
        return yb, torch.tensor(mub, dtype=torch.float64), None, None, None, None, None


def integrate(rctx, y0, mu, h, M, nsteps, checkpoint_every=10):
    """y_K after ``nsteps`` ROK4 steps of size h (Krylov dimension M) from y0,
    differentiable with respect to y0 and mu (a 0-d float64 tensor equal to
    the context problem's constant viscosity)."""
    return _Integrate.apply(y0, mu, rctx, float(h), int(M), int(nsteps), int(checkpoint_every))


def kinetic_energy(y):
    """Total kinetic energy sum (rho u^2 + rho v^2) / (2 rho) of a state (differentiable)."""
    return 0.5 * ((y[1] * y[1] + y[2] * y[2]) / y[0]).sum()
