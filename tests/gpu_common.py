"""Helpers of the GPU parity tests (inputs only; no arithmetic of the method)."""
import numpy as np
import torch

from paper_1607_06834_gb300 import workloads as W

U = 2.0 ** -53


def dev(y):
    return torch.from_numpy(np.ascontiguousarray(y, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def flux_scale(prob, y):
    """Largest physical face-flux magnitude divided by the smallest cell width:
    the size of the terms whose cancellation forms f (rounding reference)."""
    if prob.kind == W.LORENZ96:
        return float(np.max(np.abs(y)) ** 2 + prob.lorenz_f)
    g = prob.gamma
    rho = y[0]
    u, v = y[1] / rho, y[2] / rho
    p = (g - 1) * (y[3] - 0.5 * rho * (u * u + v * v))
    c = np.sqrt(g * p / rho)
    F = np.max(np.abs(y[1:3]) * (np.abs(u) + np.abs(v)) + p) + np.max((y[3] + p) * (np.abs(u) + np.abs(v)))
    F += np.max(np.abs(y[0]) * (np.abs(u) + np.abs(v) + c))
    if prob.xv is None:
        h = min(prob.lx / prob.nx, prob.ly / prob.ny)
    else:
        ex = np.hypot(np.diff(prob.xv, axis=0), np.diff(prob.yv, axis=0))
        ey = np.hypot(np.diff(prob.xv, axis=1), np.diff(prob.yv, axis=1))
        h = min(ex.min(), ey.min())
    return float(F / h)


def parity_problems():
    """(name, problem, state) cases spanning several tiles and a ragged tail."""
    out = []
    p, y = W.isentropic_vortex(64)
    out.append(('vortex64', p, y))
    p, y = W.taylor_green(48, reynolds=400.0)
    p = W.FlowProblem(**{**p.__dict__, 'ny': 40, 'ly': p.ly * 40 / 48})
    y = y[:, :40, :]
    y = np.ascontiguousarray(y + 0.01 * W.random_smooth_state(p, seed=1))
    out.append(('tgv48x40', p, y))
    p2 = W.FlowProblem(**{**p.__dict__, 'sutherland_s': 0.4, 't_ref': 1.0 / 1.4, 'mu': 0.01})
    out.append(('tgv48x40-sutherland', p2, y))
    xv, yv = W.perturbed_box_grid(40, 36, 2.0, 1.8, amp=0.3, seed=4)
    p3 = W.FlowProblem(kind=W.NAVIER_STOKES, nx=40, ny=36, xv=xv, yv=yv, mu=0.02)
    out.append(('curv40x36', p3, W.random_smooth_state(p3, seed=7, amp=0.08)))
    p4, y4, _ = W.cylinder_ogrid(24, 72)
    y4 = np.ascontiguousarray(y4 + 0.02 * W.random_smooth_state(p4, seed=3))
    out.append(('ogrid24x72', p4, y4))
    p5, y5 = W.lorenz96(40)
    out.append(('lorenz40', p5, y5))
    return out
