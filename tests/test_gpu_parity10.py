"""Ten-step parity of the ROK4 step (Sec. 2.2.2, Eq. ROK) on the three
single-grid configurations at their full sizes, through the C ABI, against
the CPU oracle:

- Euler isentropic vortex, periodic 64 x 64, ROK4 M = 12, CFL 5;
- Navier-Stokes Taylor-Green vortex, periodic 512 x 512, Re 1600, M 0.1,
  ROK4 M = 20, CFL 8 (the benchmark workload);
- Navier-Stokes cylinder, O-grid 256 x 512, Sutherland, wall and far field,
  ROK4 M = 30, CFL 10.

Bars:
- strict rounding (no contraction, IEEE division and square root, the
  oracle's operation order): bit-exact after 10 steps, binary64 basis and
  binary32 basis;
- FMA build (the benchmarked build): 1e-9 relative L2 after 10 steps where
  the oracle's own rounding floor allows it, else within 10x that floor
  (tests/oracle_floor.py: the oracle's distance from itself after 10 steps
  when every entry of y0 moves by one ulp).  The floor is measured here, per
  configuration, and printed beside the error;
- binary32 basis (mixed precision) against the binary64 oracle: 1e-6
  relative L2 after 10 steps.
"""
import numpy as np
import pytest

from oracle import integrators as I
from paper_1607_06834_gb300 import workloads as W
from tests.gpu_common import dev, host
from tests.oracle_floor import rel_l2, run_all

pytestmark = pytest.mark.gpu

STEPS = 10


def _configs():
    out = {}
    p, y = W.isentropic_vortex(64)
    out['vortex64-M12-cfl5'] = (p, y, I.dt_from_cfl(p, y, 5.0), 12)
    p, y = W.taylor_green(512, reynolds=1600.0)
    out['tgv512-M20-cfl8'] = (p, y, I.dt_from_cfl(p, y, 8.0), 20)
    p, y, _ = W.cylinder_ogrid(256, 512)
    out['cylinder256x512-M30-cfl10'] = (p, y, I.dt_from_cfl(p, y, 10.0), 30)
    return out


CONFIGS = _configs()
NAMES = list(CONFIGS)
MIXED = NAMES[1:]


@pytest.fixture(scope='module')
def rok():
    from paper_1607_06834_gb300 import rok as r
    return r


@pytest.fixture(scope='module')
def oracle_runs():
    keys, tasks = [], []
    for name, (p, y0, h, M) in CONFIGS.items():
        keys += [(name, 'fp64'), (name, 'floor')]
        tasks += [(p, y0, h, M, STEPS, False, None), (p, y0, h, M, STEPS, False, 1)]
        if name in MIXED:
            keys.append((name, 'fp32'))
            tasks.append((p, y0, h, M, STEPS, True, None))
    return dict(zip(keys, run_all(tasks)))


def _gpu_steps(rok, name, rounding, basis):
    p, y0, h, M = CONFIGS[name]
    ctx = rok.rok_init(p, krylov_max=M, rounding=rounding, basis=basis)
    rok.rok_set_graph(ctx, True)
    y = dev(y0)
    for _ in range(STEPS):
        info = rok.rok_step(ctx, y, h, M, info=True)
        assert info['m_eff'] == M
    return host(y)


@pytest.mark.parametrize('name', NAMES)
def test_strict_ten_steps_bitexact(rok, oracle_runs, name):
    y = _gpu_steps(rok, name, rok.ROK_ROUND_STRICT, rok.ROK_BASIS_FP64)
    yo = oracle_runs[(name, 'fp64')]
    assert np.array_equal(y, yo), (name, rel_l2(y, yo))


@pytest.mark.parametrize('name', MIXED)
def test_strict_mixed_ten_steps_bitexact(rok, oracle_runs, name):
    y = _gpu_steps(rok, name, rok.ROK_ROUND_STRICT, rok.ROK_BASIS_FP32)
    yo = oracle_runs[(name, 'fp32')]
    assert np.array_equal(y, yo), (name, rel_l2(y, yo))


@pytest.mark.parametrize('name', NAMES)
def test_fma_ten_steps_within_the_rounding_floor(rok, oracle_runs, name):
    y = _gpu_steps(rok, name, rok.ROK_ROUND_FAST, rok.ROK_BASIS_FP64)
    yo = oracle_runs[(name, 'fp64')]
    err = rel_l2(y, yo)
    floor = rel_l2(oracle_runs[(name, 'floor')], yo)
    tol = 1e-9 if floor < 1e-10 else max(1e-9, 10.0 * floor)
    print('\n[parity10] %s FMA build, %d steps: rel L2 vs oracle %.3e; oracle rounding floor %.3e; bar %.1e'
          % (name, STEPS, err, floor, tol))
    assert err <= tol, (name, err, floor)


@pytest.mark.parametrize('name', MIXED)
def test_mixed_precision_ten_steps_vs_binary64_oracle(rok, oracle_runs, name):
    y = _gpu_steps(rok, name, rok.ROK_ROUND_FAST, rok.ROK_BASIS_FP32)
    err = rel_l2(y, oracle_runs[(name, 'fp64')])
    print('\n[parity10] %s binary32 basis (FMA build), %d steps: rel L2 vs binary64 oracle %.3e'
          % (name, STEPS, err))
    assert err <= 1e-6, (name, err)
