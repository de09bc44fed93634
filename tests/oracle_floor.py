"""Oracle trajectories for the multi-step parity tests (and one ESDIRK3 step of
the comparator test), and the oracle's own
rounding floor.

The FD Jacobian-vector product (Eq. matvecFD) divides a difference of two
residuals by eps ~ sqrt(u ||y||), so a last-bit change of f becomes a change
of ~u/eps in the Krylov vectors; over several ROK4 steps (Eq. ROK) the
trajectory is fixed by the binary64 arithmetic only to that level.  The
rounding floor of a configuration is measured on the oracle itself: the
relative L2 distance after `steps` steps between its trajectory from y0 and
from y0 with every entry moved by one ulp (seeded random direction).  Any
arithmetic that does not repeat the oracle's operations one by one (fused
multiply-adds, another summation order) lands at about that distance.

Trajectories run in spawned worker processes (safe after CUDA is initialised
in the test process), several at once.
"""
import multiprocessing as mp
from concurrent.futures import ProcessPoolExecutor

import numpy as np


def one_ulp_everywhere(y0, seed=0):
    """y0 with every entry moved by one ulp up or down (seeded)."""
    up = np.random.default_rng(seed).random(y0.shape) < 0.5
    return np.where(up, np.nextafter(y0, np.inf), np.nextafter(y0, -np.inf))


def trajectory(args):
    """`steps` oracle ROK4 steps from y0 (optionally perturbed); returns the state."""
    from oracle import core
    from oracle import integrators as I
    prob, y0, h, M, steps, basis32, perturb_seed = args
    y = y0 if perturb_seed is None else one_ulp_everywhere(y0, perturb_seed)
    sys_ = core.System(prob)
    for _ in range(steps):
        y = I.rok_step(sys_, y, h, M, basis=np.float32 if basis32 else np.float64)
    return y


def run_all(tasks, workers=8):
    """Run `trajectory` for every task tuple, in parallel; results in order."""
    ctx = mp.get_context('spawn')
    with ProcessPoolExecutor(max_workers=min(workers, len(tasks)), mp_context=ctx) as ex:
        return list(ex.map(trajectory, tasks))


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def esdirk_task(args):
    """One oracle ESDIRK3 Newton-GMRES(30) step; returns (state, info)."""
    from oracle import core
    from oracle import integrators as I
    prob, y0, h = args
    info = {}
    y = I.esdirk_step(core.System(prob), y0, h, info=info)
    return y, info


def ke_complex_step_task(args):
    """d/dt KE(y_K) at t = 0 by the complex step through the oracle's K ROK4
    steps: along the state direction d (y0 + i t d), or along the viscosity
    (mu + i t, f affine in mu) when d is None."""
    from oracle import adjoint as A
    from oracle import core
    from oracle import integrators as I
    prob, y0, h, M, K, d = args
    hc = 1e-30
    if d is not None:
        sys_ = core.System(prob)
        y = y0 + 1j * hc * d
    else:
        class MuStep(core.System):
            def f(self, yy):
                return core.residual(prob, yy) + 1j * hc * A.residual_dmu(prob, yy)

            def jvp(self, yy, v, f0, eps):
                return (self.f(np.asarray(yy) + eps * np.asarray(v)) - f0) / eps
        sys_ = MuStep(prob)
        y = y0.astype(complex)
    for _ in range(K):
        y = I.rok_step(sys_, y, h, M)
    ke = 0.5 * np.sum((y[1] ** 2 + y[2] ** 2) / y[0])
    return float(np.imag(ke) / hc)
