"""GPU reverse mode against the oracle's discrete adjoint and against the
complex-step derivative of the oracle's step map, through the C ABI.

Bars: the residual VJP equals the oracle's (exact transposed Jacobian) to 1e-12
of its size and satisfies <u, J v> = <J^T u, v> against the exact (dual-number)
JVP at 256^2; one reverse ROK4 step and multi-step gradients with
checkpointing agree with the oracle to 1e-5 relative (both are exact
derivatives of the same discrete map; the finite-difference quotients inside
make them differ at the u / eps level).  Multi-step checks use states where
the derivative of the map is well conditioned (it is not on the low-Mach
Taylor-Green state at CFL 4 and above)."""
import numpy as np
import pytest

from oracle import adjoint as A
from oracle import core
from oracle import integrators as I
from paper_1607_06834_gb300 import workloads as W
from tests.gpu_common import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def rok():
    from paper_1607_06834_gb300 import rok as r
    return r


def _cases():
    p, y = W.taylor_green(40, reynolds=300.0)
    p = W.FlowProblem(**{**p.__dict__, 'ny': 36, 'ly': p.ly * 36 / 40})
    y = np.ascontiguousarray(y[:, :36, :] + 0.01 * W.random_smooth_state(p, seed=3))
    out = [('ns-40x36', p, y)]
    # Sutherland's law, temperatures away from t_ref (g(T) = mu(T) / mu_ref != 1)
    ps = W.FlowProblem(**{**p.__dict__, 'sutherland_s': 0.4, 't_ref': 0.5})
    out.append(('ns-sutherland-40x36', ps, y))
    p, y = W.isentropic_vortex(33)
    out.append(('euler-33', p, y))
    # curvilinear grids (reverse sweep) and Lorenz-96 (compressed Jacobian)
    out.extend(_off_uniform_cases())
    return out


def _off_uniform_cases():
    xv, yv = W.perturbed_box_grid(40, 36, 2.0, 1.8, amp=0.3, seed=4)
    p3 = W.FlowProblem(kind=W.NAVIER_STOKES, nx=40, ny=36, xv=xv, yv=yv, mu=0.02)
    out = [('curv-40x36', p3, W.random_smooth_state(p3, seed=7, amp=0.08))]
    # O-grid 32 x 16 (periodic in theta, wall and far field), Sutherland's law
    p4, y4, _ = W.cylinder_ogrid(16, 32)
    out.append(('ogrid-32x16', p4, np.ascontiguousarray(y4 + 0.02 * W.random_smooth_state(p4, seed=2))))
    # walls on three sides and a far field (i-walls: corner ghosts mirrored twice)
    q_inf = (1.0, 0.3, 0.1, 2.5)
    xw, yw = W.perturbed_box_grid(20, 18, 2.0, 1.8, amp=0.3, seed=5)
    p6 = W.FlowProblem(kind=W.NAVIER_STOKES, nx=20, ny=18, xv=xw, yv=yw, mu=0.02, q_inf=q_inf,
                       bc=(W.WALL, W.FARFIELD, W.WALL, W.WALL), sutherland_s=0.4, t_ref=0.5)
    out.append(('box-walls-20x18', p6, W.random_smooth_state(p6, seed=8, amp=0.08)))
    p7 = W.FlowProblem(**{**p3.__dict__, 'kind': W.EULER, 'mu': 0.0})
    out.append(('curv-euler-40x36', p7, W.random_smooth_state(p7, seed=9, amp=0.08)))
    p5, y5 = W.lorenz96(40)
    out.append(('lorenz-40', p5, y5))
    return out


@pytest.mark.parametrize('name,prob,y', _cases(), ids=[c[0] for c in _cases()])
def test_residual_vjp_matches_oracle(rok, name, prob, y):
    u = np.random.default_rng(5).standard_normal(y.shape)
    ctx = rok.rok_init(prob, krylov_max=4, rounding=rok.ROK_ROUND_STRICT)
    got, mub = rok.rok_vjp(ctx, dev(y), dev(u), mubar=True)
    ref = A.residual_vjp(prob, y, u)
    assert np.abs(host(got) - ref).max() <= 1e-12 * np.abs(ref).max()
    mref = float(np.sum(u * A.residual_dmu(prob, y)))
    assert abs(mub - mref) <= 1e-12 * np.sum(np.abs(u * A.residual_dmu(prob, y))), (mub, mref)


def test_residual_vjp_adjoint_identity_full_size(rok):
    # 256^2 Taylor-Green at Re = 1000 (the gradient workload): <u, J v> with J v
    # by the dual-number kernel equals <J^T u, v> by the reverse kernels
    prob, y = W.taylor_green(256, reynolds=1000.0)
    ctx = rok.rok_init(prob, krylov_max=4)
    rng = np.random.default_rng(8)
    u, v = dev(rng.standard_normal(y.shape)), dev(rng.standard_normal(y.shape))
    yd = dev(y)
    jv = rok.rok_jvp(ctx, yd, v, mode=rok.ROK_JVP_EXACT)
    jtu = rok.rok_vjp(ctx, yd, u)
    lhs, rhs = float((u * jv).sum()), float((jtu * v).sum())
    scale = float((u.abs() * rok.rok_jvp(ctx, yd, v.abs(), mode=rok.ROK_JVP_EXACT).abs()).sum())
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs, scale)


@pytest.mark.parametrize('M,sutherland', [(0, False), (4, False), (10, False), (4, True)])
def test_step_vjp_matches_oracle_adjoint(rok, M, sutherland):
    prob, y = W.taylor_green(24, reynolds=400.0)
    if sutherland:
        prob = W.FlowProblem(**{**prob.__dict__, 'sutherland_s': 0.4, 't_ref': 0.5})
    y = np.ascontiguousarray(y + 0.01 * W.random_smooth_state(prob, seed=5))
    h = I.dt_from_cfl(prob, y, 5.0)
    c = np.random.default_rng(M + 1).standard_normal(y.shape)
    ctx = rok.rok_init(prob, krylov_max=max(M, 1), rounding=rok.ROK_ROUND_STRICT)
    yb, mub = rok.rok_step_vjp(ctx, dev(y), h, M, dev(c))
    ref, mref = A.rok_step_vjp(prob, y, h, M, c)
    yb = host(yb)
    assert np.linalg.norm(yb - ref) <= 1e-5 * np.linalg.norm(ref), np.linalg.norm(yb - ref) / np.linalg.norm(ref)
    assert abs(mub - mref) <= 1e-5 * abs(mref), (mub, mref)


def _adjoint_self_sensitivity(prob, y, h, M, c):
    """How far the oracle's own reverse step moves when every state entry moves
    by one ulp: the FD quotients of the recomputed forward step re-round, as they
    do when the FMA build evaluates the residual with other rounding."""
    rng = np.random.default_rng(21)
    yp = y + rng.choice([-1.0, 1.0], size=y.shape) * np.spacing(y)
    ra, _ = A.rok_step_vjp(prob, y, h, M, c)
    rb, _ = A.rok_step_vjp(prob, yp, h, M, c)
    return np.linalg.norm(ra - rb) / np.linalg.norm(ra)


@pytest.mark.parametrize('mode', ['strict', 'fast'])
def test_step_vjp_euler_vortex(rok, mode):
    # strict: the forward recompute is the oracle's step bit for bit, the bar is
    # the 1e-5 of the reverse arithmetic; FMA build: the recomputed step carries
    # the FD noise of its own residual rounding (Eq. matvecFD divides it by
    # eps), bounded by 4 x the oracle's own change under one-ulp changes of the
    # state (3.3e-5 here: the old 1e-5 bar held for the FMA build by chance)
    prob, y = W.isentropic_vortex(32)
    h = I.dt_from_cfl(prob, y, 5.0)
    c = np.random.default_rng(3).standard_normal(y.shape)
    ctx = rok.rok_init(prob, krylov_max=8, rounding=getattr(rok, 'ROK_ROUND_' + mode.upper()))
    yb, mub = rok.rok_step_vjp(ctx, dev(y), h, 8, dev(c))
    ref, _ = A.rok_step_vjp(prob, y, h, 8, c)
    err = np.linalg.norm(host(yb) - ref) / np.linalg.norm(ref)
    bar = 1e-5 if mode == 'strict' else max(1e-5, 4 * _adjoint_self_sensitivity(prob, y, h, 8, c))
    assert err <= bar, (err, bar)
    assert mub == 0.0


def _ke(yy):
    return 0.5 * np.sum((yy[1] ** 2 + yy[2] ** 2) / yy[0])


def _gpu_gradient(rok, prob, y0, h, M, K, every):
    import torch

    from paper_1607_06834_gb300 import autograd as G
    ctx = rok.rok_init(prob, krylov_max=M, rounding=rok.ROK_ROUND_STRICT)
    y = dev(y0).requires_grad_(True)
    mu = torch.tensor(prob.mu, dtype=torch.float64, requires_grad=True)
    J = G.kinetic_energy(G.integrate(ctx, y, mu, h, M, K, checkpoint_every=every))
    J.backward()
    return host(y.grad), float(mu.grad)


def test_gradient_on_the_cylinder_ogrid_matches_oracle_complex_step(rok):
    # curvilinear reverse sweep inside the differentiable integration: J =
    # kinetic energy after 4 ROK4 steps (M = 4, CFL 2) on a 32 x 16 O-grid
    # (wall, far field, Sutherland's law), checkpoints every 2 steps; dJ/dy0 . d
    # and dJ/dmu_ref against the complex step through the oracle's 4 steps (in
    # the state, and in mu_ref through the affine continuation f + i d df/dmu)
    prob, y0, _ = W.cylinder_ogrid(16, 32)
    y0 = np.ascontiguousarray(y0 + 0.02 * W.random_smooth_state(prob, seed=2))
    h = I.dt_from_cfl(prob, y0, 2.0)
    M, K = 4, 4
    g, gmu = _gpu_gradient(rok, prob, y0, h, M, K, 2)
    d = np.random.default_rng(11).standard_normal(y0.shape)
    yc = y0 + 1e-30j * d
    for _ in range(K):
        yc = I.rok_step(core.System(prob), yc, h, M)
    cs = float(np.imag(_ke(yc)) / 1e-30)
    assert abs(np.sum(g * d) - cs) <= 1e-5 * abs(cs), (np.sum(g * d), cs)

    class MuStep(core.System):
        def f(self, yy):
            return core.residual(prob, yy) + 1e-30j * A.residual_dmu(prob, yy)

        def jvp(self, yy, v, f0, eps):
            return (self.f(np.asarray(yy) + eps * np.asarray(v)) - f0) / eps
    yc = y0.astype(complex)
    for _ in range(K):
        yc = I.rok_step(MuStep(prob), yc, h, M)
    csm = float(np.imag(_ke(yc)) / 1e-30)
    assert abs(gmu - csm) <= 1e-5 * abs(csm), (gmu, csm)


def test_gradient_wrt_state_with_checkpoints_matches_oracle_complex_step(rok):
    # J = kinetic energy after 6 ROK4 steps (M = 8, CFL 1) of the Euler vortex,
    # checkpoint every 2 steps: dJ/dy0 . d against the complex-step derivative of
    # the oracle's own 6-step integration.  (On the low-Mach Taylor-Green state
    # this derivative is not a well-posed check: it moves by O(1) under 1e-12
    # changes of y0, see test_oracle_adjoint.)
    prob, y0 = W.isentropic_vortex(20)
    h = I.dt_from_cfl(prob, y0, 1.0)
    M, K = 8, 6
    g, gmu = _gpu_gradient(rok, prob, y0, h, M, K, 2)
    assert gmu == 0.0
    d = np.random.default_rng(11).standard_normal(y0.shape)
    sys_ = core.System(prob)
    yc = y0 + 1e-30j * d
    for _ in range(K):
        yc = I.rok_step(sys_, yc, h, M)
    cs = float(np.imag(_ke(yc)) / 1e-30)
    assert abs(np.sum(g * d) - cs) <= 1e-5 * abs(cs), (np.sum(g * d), cs)


def test_gradient_wrt_viscosity_with_checkpoints_matches_oracle_complex_step(rok):
    # Navier-Stokes Taylor-Green, 4 steps (M = 4, CFL 1), checkpoint every 2:
    # dJ/dmu against the complex step in mu through the oracle's integration
    # (f is affine in mu: f(y; mu + i d) = f(y; mu) + i d df/dmu(y))
    prob, y0 = W.taylor_green(20, reynolds=200.0)
    y0 = np.ascontiguousarray(y0 + 0.01 * W.random_smooth_state(prob, seed=9))
    h = I.dt_from_cfl(prob, y0, 1.0)
    M, K = 4, 4
    _, gmu = _gpu_gradient(rok, prob, y0, h, M, K, 2)

    class MuStep(core.System):
        def f(self, yy):
            return core.residual(prob, yy) + 1e-30j * A.residual_dmu(prob, yy)

        def jvp(self, yy, v, f0, eps):
            return (self.f(np.asarray(yy) + eps * np.asarray(v)) - f0) / eps
    yc = y0.astype(complex)
    for _ in range(K):
        yc = I.rok_step(MuStep(prob), yc, h, M)
    csm = float(np.imag(_ke(yc)) / 1e-30)
    assert abs(gmu - csm) <= 1e-5 * abs(csm), (gmu, csm)


@pytest.mark.parametrize('name', ['ogrid-32x16', 'lorenz-40'])
@pytest.mark.parametrize('mode', ['strict', 'fast'])
def test_step_vjp_off_uniform_grids_matches_oracle_adjoint(rok, name, mode):
    prob, y = {c[0]: (c[1], c[2]) for c in _off_uniform_cases()}[name]
    M = 4
    h = I.dt_from_cfl(prob, y, 2.0) if prob.kind != 2 else 0.01
    c = np.random.default_rng(11).standard_normal(y.shape)
    ctx = rok.rok_init(prob, krylov_max=M, rounding=getattr(rok, 'ROK_ROUND_' + mode.upper()))
    yb, mub = rok.rok_step_vjp(ctx, dev(y), h, M, dev(c))
    ref, mref = A.rok_step_vjp(prob, y, h, M, c)
    yb = host(yb)
    err = np.linalg.norm(yb - ref) / np.linalg.norm(ref)
    print(name, mode, 'relative L2 of ybar', err, 'mubar', mub, mref)
    assert err <= 1e-5, err
    if prob.kind == 2:
        assert mub == 0.0 and mref == 0.0
    else:
        assert abs(mub - mref) <= 1e-5 * abs(mref), (mub, mref)


@pytest.mark.parametrize('name', ['tgv-24', 'ogrid-32x16'])
@pytest.mark.parametrize('mode', ['strict', 'fast'])
def test_step_vjp_binary32_basis_matches_oracle_adjoint(rok, name, mode):
    # the reverse on the widened binary32 basis: the derivative of the exact
    # Arnoldi process at the rounded basis, against the oracle's binary64
    # adjoint (the basis rounding, relative 2^-24, enters the JVP directions,
    # not the FD increment, so no 1/eps amplification).  FMA build: the bar of
    # test_step_vjp_euler_vortex, the recomputed step's FD noise (the oracle's
    # own reverse moves by 1.3e-5 under one-ulp state changes on Taylor-Green)
    if name == 'tgv-24':
        prob, y = W.taylor_green(24, reynolds=400.0)
        y = np.ascontiguousarray(y + 0.01 * W.random_smooth_state(prob, seed=5))
    else:
        prob, y = {c[0]: (c[1], c[2]) for c in _off_uniform_cases()}[name]
    M = 4
    h = I.dt_from_cfl(prob, y, 2.0)
    c = np.random.default_rng(12).standard_normal(y.shape)
    ctx = rok.rok_init(prob, krylov_max=M, rounding=getattr(rok, 'ROK_ROUND_' + mode.upper()),
                       basis=rok.ROK_BASIS_FP32)
    yb, mub = rok.rok_step_vjp(ctx, dev(y), h, M, dev(c))
    ref, mref = A.rok_step_vjp(prob, y, h, M, c)
    err = np.linalg.norm(host(yb) - ref) / np.linalg.norm(ref)
    print(name, mode, 'binary32 basis: relative L2 of ybar', err, 'mubar', mub, mref)
    bar = 1e-5 if mode == 'strict' else max(1e-5, 4 * _adjoint_self_sensitivity(prob, y, h, M, c))
    assert err <= bar, (err, bar)
    assert abs(mub - mref) <= bar * abs(mref), (mub, mref)


def test_vjp_unsupported_cases(rok):
    # the reverse step of the exact-JVP step (second derivatives of f)
    prob, y = W.taylor_green(24, reynolds=400.0)
    h = I.dt_from_cfl(prob, y, 2.0)
    ctx = rok.rok_init(prob, krylov_max=4, jvp=rok.ROK_JVP_EXACT)
    with pytest.raises(rok.RokError) as e:
        rok.rok_step_vjp(ctx, dev(y), h, 4, dev(y))
    assert e.value.status == rok.ROK_ERR_UNSUPPORTED


def _ns_case():
    prob, y = W.taylor_green(40, reynolds=300.0)
    prob = W.FlowProblem(**{**prob.__dict__, 'ny': 36, 'ly': prob.ly * 36 / 40})
    y = np.ascontiguousarray(y[:, :36, :] + 0.01 * W.random_smooth_state(prob, seed=9))
    return prob, y


@pytest.mark.parametrize('mode', ['strict', 'fast'])
def test_recorded_step_and_its_reverse_are_bit_identical_to_the_recomputed_ones(rok, mode):
    # two steps recorded on tapes, reversed in the opposite order: each y_{n+1}
    # equals rok_step's and each reverse equals rok_step_vjp's, bit for bit (the
    # same kernels on the same data; the tape only moves the internals)
    import torch
    prob, y = _ns_case()
    h = I.dt_from_cfl(prob, y, 4.0)
    M = 6
    ctx = rok.rok_init(prob, krylov_max=M, rounding=getattr(rok, 'ROK_ROUND_' + mode.upper()))
    nbytes = rok.rok_tape_bytes(ctx, M)
    assert nbytes >= (10 + M) * y.size * 8
    ys = [dev(y)]
    for _ in range(2):
        ys.append(ys[-1].clone())
        rok.rok_step(ctx, ys[-1], h, M)
    yr = dev(y)
    tapes = [rok.rok_step_record(ctx, yr, h, M)]
    assert torch.equal(yr, ys[1])
    tapes.append(rok.rok_step_record(ctx, yr, h, M))
    assert torch.equal(yr, ys[2])
    c = dev(np.random.default_rng(4).standard_normal(y.shape))
    ref1, m1 = rok.rok_step_vjp(ctx, ys[1], h, M, c)
    ref0, m0 = rok.rok_step_vjp(ctx, ys[0], h, M, ref1)
    got1, g1 = rok.rok_step_vjp_tape(ctx, tapes[1], c)
    got0, g0 = rok.rok_step_vjp_tape(ctx, tapes[0], got1, out=got1)
    assert torch.equal(got0, ref0)
    assert (g1, g0) == (m1, m0)
    assert m0 != 0.0


def test_tape_rejects_bad_arguments(rok):
    import torch
    prob, y = _ns_case()
    h = I.dt_from_cfl(prob, y, 4.0)
    ctx = rok.rok_init(prob, krylov_max=4)
    tape = torch.empty(rok.rok_tape_bytes(ctx, 4) + 512, dtype=torch.uint8, device='cuda')
    yd = dev(y)
    c = dev(np.ones(y.shape))

    def status(call):
        with pytest.raises(rok.RokError) as e:
            call()
        return e.value.status

    assert status(lambda: rok.rok_tape_bytes(ctx, 5)) == rok.ROK_ERR_INVALID_ARG      # M > krylov_max
    assert status(lambda: rok.rok_step_record(ctx, yd, h, 4, tape[8:])) == rok.ROK_ERR_INVALID_ARG  # unaligned
    assert status(lambda: rok.rok_step_record(ctx, yd, -h, 4, tape)) == rok.ROK_ERR_INVALID_ARG
    assert torch.equal(yd, dev(y))
    tape.zero_()
    assert status(lambda: rok.rok_step_vjp_tape(ctx, tape, c)) == rok.ROK_ERR_INVALID_ARG  # no header
    rok.rok_step_record(ctx, yd, h, 4, tape)
    alias = tape[1024:1024 + y.size * 8].view(torch.float64)
    assert status(lambda: rok.rok_step_vjp_tape(ctx, tape, c, out=alias)) == rok.ROK_ERR_INVALID_ARG
    # a tape of another problem (other N)
    p2, y2 = W.taylor_green(32, reynolds=300.0)
    ctx2 = rok.rok_init(p2, krylov_max=4)
    assert status(lambda: rok.rok_step_vjp_tape(ctx2, tape, dev(np.ones(y2.shape)))) == rok.ROK_ERR_INVALID_ARG
    # the exact-JVP step has no reverse
    ctx3 = rok.rok_init(prob, krylov_max=4, jvp=rok.ROK_JVP_EXACT)
    assert status(lambda: rok.rok_step_record(ctx3, dev(y), h, 4, tape)) == rok.ROK_ERR_UNSUPPORTED


def test_gradient_with_tapes_is_bit_identical_to_recomputation(rok):
    # 7 steps, checkpoint every 3 (segments 3, 3, 1): the tape path records the
    # ragged last segment in the forward and reuses its tapes for the others
    import torch

    from paper_1607_06834_gb300 import autograd as G
    prob, y0 = _ns_case()
    h = I.dt_from_cfl(prob, y0, 2.0)
    ctx = rok.rok_init(prob, krylov_max=6)
    grads = []
    for tapes in (True, False):
        y = dev(y0).requires_grad_(True)
        mu = torch.tensor(prob.mu, dtype=torch.float64, requires_grad=True)
        G.kinetic_energy(G.integrate(ctx, y, mu, h, 6, 7, checkpoint_every=3, tapes=tapes)).backward()
        grads.append((y.grad.clone(), float(mu.grad)))
    assert torch.equal(grads[0][0], grads[1][0])
    assert grads[0][1] == grads[1][1]


def _full_length_case(viscous):
    prob, y0 = W.isentropic_vortex(64)
    if viscous:
        prob = W.FlowProblem(**{**prob.__dict__, 'kind': W.NAVIER_STOKES, 'mu': 0.01})
    return prob, y0, I.dt_from_cfl(prob, y0, 0.5)


def _cell_ke(t):
    a = host(t)
    return 0.5 * (a[1] * a[1] + a[2] * a[2]) / a[0]


@pytest.mark.parametrize('viscous', [False, True], ids=['euler', 'navier-stokes'])
def test_gradient_full_length_well_conditioned(rok, viscous):
    # The gradient workload's shape (100 ROK4 steps, checkpoint every 10) on a
    # map whose derivative is well conditioned: the isentropic vortex 64^2,
    # M = 12, CFL 0.5 (Euler; Navier-Stokes with mu = 0.01 for dJ/dmu), J the
    # final kinetic energy.  Checks, strict and FMA builds:
    #  - 100 steps: dJ/dy0 . d and dJ/dmu against the complex-step derivative of
    #    the oracle's own 100-step map, 1e-5;
    #  - 10 steps: dJ/dy0 . d against central differences (h = 1e-6) of the
    #    GPU's forward map, 1e-5 (their spread under one-ulp changes of y0 is
    #    ~1e-6 there; after 100 steps it grows to ~2e-5 and the differences
    #    are only reported);
    #  - 100 steps: dJ/dmu against central differences in mu (relative step
    #    1e-4; the map is smooth in mu), 1e-5.
    # (At CFL >= 2, or on the low-Mach Taylor-Green state, complex step and
    # central differences of the same map disagree by O(1): the FD-JVP
    # Krylov map is not smooth at that scale.)
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    import torch

    from paper_1607_06834_gb300 import autograd as G
    from tests.oracle_floor import ke_complex_step_task
    prob, y0, h = _full_length_case(viscous)
    M, every = 12, 10
    d = np.random.default_rng(0).standard_normal(y0.shape)
    d /= np.linalg.norm(d)

    def grad(ctx, K):
        y = dev(y0).requires_grad_(True)
        mu = torch.tensor(prob.mu, dtype=torch.float64, requires_grad=True)
        G.kinetic_energy(G.integrate(ctx, y, mu, h, M, K, checkpoint_every=every)).backward()
        return float(np.sum(host(y.grad) * d)), float(mu.grad)

    def forward(ctx, start, K):
        yy = dev(start)
        for _ in range(K):
            rok.rok_step(ctx, yy, h, M)
        return _cell_ke(yy)

    with ProcessPoolExecutor(max_workers=2, mp_context=mp.get_context('spawn')) as ex:
        f_cs = ex.submit(ke_complex_step_task, (prob, y0, h, M, 100, d))
        f_csm = ex.submit(ke_complex_step_task, (prob, y0, h, M, 100, None)) if viscous else None
        res = {}
        for mode in ('strict', 'fast'):
            rounding = getattr(rok, 'ROK_ROUND_' + mode.upper())
            ctx = rok.rok_init(prob, krylov_max=M, rounding=rounding)
            gd100, gmu100 = grad(ctx, 100)
            gd10, _ = grad(ctx, 10)
            fd10 = float(np.sum(forward(ctx, y0 + 1e-6 * d, 10) - forward(ctx, y0 - 1e-6 * d, 10))) / 2e-6
            fd100 = float(np.sum(forward(ctx, y0 + 1e-6 * d, 100) - forward(ctx, y0 - 1e-6 * d, 100))) / 2e-6
            fdm = None
            if viscous:
                vm = []
                for sgn in (1.0, -1.0):
                    pm = W.FlowProblem(**{**prob.__dict__, 'mu': prob.mu * (1.0 + sgn * 1e-4)})
                    vm.append(forward(rok.rok_init(pm, krylov_max=M, rounding=rounding), y0, 100))
                fdm = float(np.sum(vm[0] - vm[1])) / (2e-4 * prob.mu)
            res[mode] = (gd100, gmu100, gd10, fd10, fd100, fdm)
        cs = f_cs.result()
        csm = f_csm.result() if viscous else None
    for mode, (gd100, gmu100, gd10, fd10, fd100, fdm) in res.items():
        tag = 'NS' if viscous else 'Euler'
        print('\n[grad] vortex 64^2 %s, %s build: 100 steps dJ/dy0.d %.10g vs complex step %.10g (rel %.2e), '
              'central FD %.10g (rel %.2e, reported); 10 steps %.10g vs central FD %.10g (rel %.2e)'
              % (tag, mode, gd100, cs, abs(gd100 - cs) / abs(cs), fd100, abs(gd100 - fd100) / abs(gd100),
                 gd10, fd10, abs(gd10 - fd10) / abs(gd10)))
        assert abs(gd100 - cs) <= 1e-5 * abs(cs)
        assert abs(gd10 - fd10) <= 1e-5 * abs(gd10)
        if viscous:
            print('[grad]   100 steps dJ/dmu %.10g vs complex step %.10g (rel %.2e), central FD %.10g (rel %.2e)'
                  % (gmu100, csm, abs(gmu100 - csm) / abs(csm), fdm, abs(gmu100 - fdm) / abs(gmu100)))
            assert abs(gmu100 - csm) <= 1e-5 * abs(csm)
            assert abs(gmu100 - fdm) <= 1e-5 * abs(gmu100)
        else:
            assert gmu100 == 0.0
