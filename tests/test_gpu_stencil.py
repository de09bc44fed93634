"""GPU parity of the residual f(y) (Sec. 3.2) and the FD Jacobian-vector product
(Eq. matvecFD) through the C ABI against the CPU oracle.

Strict rounding (no FMA contraction) must be bit-exact.  The default build may
contract multiply-adds: its residual differs from the oracle only by rounding
of the face-flux terms, bounded here by 64 u max|F|/h (u = 2^-53, F the
physical flux, h the smallest cell width) per entry and by 1e-12 relative in
L2 (the denominator floored at 1e-3 of the face-flux scale); the FD quotient
amplifies that by 1/eps."""
import numpy as np
import pytest

from oracle import core
from oracle import integrators as I
from tests.gpu_common import U, dev, flux_scale, host, parity_problems

pytestmark = pytest.mark.gpu

CASES = parity_problems()
IDS = [c[0] for c in CASES]


@pytest.fixture(scope='module')
def rok():
    from paper_1607_06834_gb300 import rok as r
    return r


@pytest.mark.parametrize('case', CASES, ids=IDS)
def test_residual_strict_bitexact(rok, case):
    name, prob, y = case
    ctx = rok.rok_init(prob, krylov_max=4, rounding=rok.ROK_ROUND_STRICT)
    f = host(rok.rok_residual(ctx, dev(y)))
    fo = core.residual(prob, y)
    assert np.array_equal(f, fo), (name, np.abs(f - fo).max())


@pytest.mark.parametrize('case', CASES, ids=IDS)
def test_residual_fast_within_rounding(rok, case):
    name, prob, y = case
    ctx = rok.rok_init(prob, krylov_max=4, rounding=rok.ROK_ROUND_FAST)
    f = host(rok.rok_residual(ctx, dev(y)))
    fo = core.residual(prob, y)
    tol = 64 * U * flux_scale(prob, y)
    assert np.abs(f - fo).max() <= tol, (name, np.abs(f - fo).max(), tol)
    # 1e-12 relative, the denominator floored at 1e-3 of the face-flux scale:
    # where the fluxes nearly cancel (a slowly varying flow) f is small next to
    # the terms whose rounding it inherits
    den = max(np.linalg.norm(fo), 1e-3 * np.sqrt(fo.size) * flux_scale(prob, y))
    rel = np.linalg.norm(f - fo) / den
    print('\n[residual] %s FMA build: rel L2 %.3e (plain %.3e)' % (name, rel, np.linalg.norm(f - fo) / np.linalg.norm(fo)))
    assert rel <= 1e-12, (name, rel)


@pytest.mark.parametrize('case', CASES, ids=IDS)
def test_jvp_strict_bitexact(rok, case):
    name, prob, y = case
    ctx = rok.rok_init(prob, krylov_max=4, rounding=rok.ROK_ROUND_STRICT)
    rng = np.random.default_rng(11)
    v = rng.normal(size=y.shape)
    v /= np.linalg.norm(v)
    f0 = core.residual(prob, y)
    eps = I.fd_eps(I.norm(y))
    w = host(rok.rok_jvp(ctx, dev(y), dev(v), fy=dev(f0), eps=eps))
    wo = core.jvp_fd(prob, y, v, f0, eps)
    assert np.array_equal(w, wo), (name, np.abs(w - wo).max())
    # automatic increment (fy computed by the library): same power of two
    w2 = host(rok.rok_jvp(ctx, dev(y), dev(v)))
    e2 = I.fd_eps(I.norm(y), I.norm(v))
    assert np.array_equal(w2, core.jvp_fd(prob, y, v, f0, e2))


@pytest.mark.parametrize('case', CASES, ids=IDS)
def test_jvp_fast_within_amplified_rounding(rok, case):
    name, prob, y = case
    ctx = rok.rok_init(prob, krylov_max=4, rounding=rok.ROK_ROUND_FAST)
    rng = np.random.default_rng(12)
    v = rng.normal(size=y.shape)
    v /= np.linalg.norm(v)
    f0 = core.residual(prob, y)
    eps = I.fd_eps(I.norm(y))
    w = host(rok.rok_jvp(ctx, dev(y), dev(v), fy=dev(f0), eps=eps))
    wo = core.jvp_fd(prob, y, v, f0, eps)
    tol = 64 * U * flux_scale(prob, y) / eps
    assert np.abs(w - wo).max() <= tol, (name, np.abs(w - wo).max(), tol)


def test_residual_full_size_taylor_green(rok):
    # the 512 x 512 Navier-Stokes Taylor-Green case of the benchmark, both builds
    from paper_1607_06834_gb300 import workloads as W
    prob, y = W.taylor_green(512, reynolds=1600.0)
    fo = core.residual(prob, y)
    for mode in (rok.ROK_ROUND_STRICT, rok.ROK_ROUND_FAST):
        ctx = rok.rok_init(prob, krylov_max=2, rounding=mode)
        f = host(rok.rok_residual(ctx, dev(y)))
        if mode == rok.ROK_ROUND_STRICT:
            assert np.array_equal(f, fo)
        else:
            assert np.abs(f - fo).max() <= 64 * U * flux_scale(prob, y)


def test_nonfinite_detected(rok):
    from paper_1607_06834_gb300 import workloads as W
    prob, y = W.isentropic_vortex(32)
    y = y.copy()
    y[0, 5, 7] = np.nan
    ctx = rok.rok_init(prob, krylov_max=4)
    rok.rok_residual(ctx, dev(y))
    with pytest.raises(rok.RokError) as e:
        rok.rok_sync(ctx)
    assert e.value.status == rok.ROK_ERR_NONFINITE
    rok.rok_sync(ctx)   # latched status was cleared


# ---- exact JVP (forward-mode dual numbers) vs the complex-step oracle ----------

@pytest.mark.parametrize('mode', ['fast', 'strict'])
@pytest.mark.parametrize('case', CASES, ids=IDS)
def test_exact_jvp_matches_complex_step(rok, case, mode):
    # both are the derivative of the same discrete residual to rounding: 1e-12
    name, prob, y = case
    ctx = rok.rok_init(prob, krylov_max=4, rounding=getattr(rok, 'ROK_ROUND_' + mode.upper()))
    rng = np.random.default_rng(21)
    v = rng.normal(size=y.shape)
    w = host(rok.rok_jvp(ctx, dev(y), dev(v), mode=rok.ROK_JVP_EXACT))
    wo = core.jvp_exact(prob, y, v)
    assert np.linalg.norm(w - wo) <= 1e-12 * np.linalg.norm(wo), (name, np.linalg.norm(w - wo) / np.linalg.norm(wo))
