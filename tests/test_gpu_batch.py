"""GPU parity of the batched ROK4 step (many independent problems, every
launch covering all of them) against the CPU oracle, instance by instance,
and against the single-problem entry point, through the C ABI.

Bars: under strict rounding every instance equals the oracle's ROK4 step bit
for bit (the batch keeps each instance's reduction trees); every launch-shape
candidate of the tuner gives the same bits; graph replay and eager launches
give the same bits; under the FMA build (and on the full 64-instance
workload) every sampled instance is within 1e-9 relative L2 of the oracle,
or within 10x the oracle's own rounding floor where that floor is above
1e-10."""
import numpy as np
import pytest

from oracle import core
from oracle import integrators as I
from paper_1607_06834_gb300 import workloads as W
from tests.gpu_common import dev, host, rel_l2
from tests.oracle_floor import one_ulp_everywhere

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def rok():
    from paper_1607_06834_gb300 import rok as r
    return r


def _mixed_instances():
    """Euler vortices and Navier-Stokes Taylor-Green grids (constant viscosity
    and Sutherland), square and rectangular, sizes that leave ragged tiles and
    ragged 2048-entry chunks."""
    out = []
    p, y = W.isentropic_vortex(32, centre=(3.0, 7.0))
    out.append((p, y, 3.0))
    p, y = W.taylor_green(40, reynolds=300.0)
    out.append((p, y, 4.0))
    p, y = W.taylor_green(48, reynolds=700.0)
    p = W.FlowProblem(**{**p.__dict__, 'ny': 40, 'ly': p.ly * 40 / 48})
    y = np.ascontiguousarray(y[:, :40, :] + 0.01 * W.random_smooth_state(p, seed=2))
    out.append((p, y, 2.0))
    p, y = W.isentropic_vortex(37, centre=(6.5, 2.0))
    out.append((p, y, 5.0))
    p, y = W.taylor_green(36, reynolds=200.0)
    p = W.FlowProblem(**{**p.__dict__, 'sutherland_s': 0.4, 't_ref': 1.0 / 1.4})
    out.append((p, y, 3.5))
    p, y = W.isentropic_vortex(50)
    out.append((p, y, 1.5))
    return out


def _dts(cases):
    return [I.dt_from_cfl(p, y, c) for p, y, c in cases]


def test_batch_strict_bitexact_vs_oracle(rok):
    cases = _mixed_instances()
    M, steps = 8, 3
    b = rok.rok_batch_init([p for p, _, _ in cases], krylov_max=M, rounding=rok.ROK_ROUND_STRICT)
    y = b.pack([yy for _, yy, _ in cases])
    hs = _dts(cases)
    for _ in range(steps):
        info = rok.rok_batch_step(b, y, hs, M, info=True)
        assert all(i['status'] == 0 and i['m_eff'] == M for i in info), info
    got = b.unpack(y)
    for k, (p, y0, _) in enumerate(cases):
        sys_ = core.System(p)
        yo = y0
        for _ in range(steps):
            yo = I.rok_step(sys_, yo, hs[k], M)
        assert np.array_equal(got[k], yo), (k, rel_l2(got[k], yo))


def _oracle_steps(prob, y0, h, M, steps):
    sys_ = core.System(prob)
    y = y0
    for _ in range(steps):
        y = I.rok_step(sys_, y, h, M)
    return y


def _single_fast(rok, prob, y0, h, M, steps):
    ctx = rok.rok_init(prob, krylov_max=M, rounding=rok.ROK_ROUND_FAST)
    ys = dev(y0)
    for _ in range(steps):
        rok.rok_step(ctx, ys, h, M)
    return host(ys)


def _check_fast(rok, prob, y0, h, M, steps, got, label):
    """The FMA build may contract a formula differently in the batched and the
    single-problem kernels; the FD quotients amplify those last-bit differences.
    Bar: 1e-9 relative L2, or, where the oracle's own rounding floor (its
    distance from itself when every entry of y0 moves by one ulp) is above
    1e-10, within 10x that floor."""
    yo = _oracle_steps(prob, y0, h, M, steps)
    e_b = rel_l2(got, yo)
    e_s = rel_l2(_single_fast(rok, prob, y0, h, M, steps), yo)
    floor = rel_l2(_oracle_steps(prob, one_ulp_everywhere(y0, 1), h, M, steps), yo)
    tol = 1e-9 if floor < 1e-10 else max(1e-9, 10.0 * floor)
    print('\n[batch] instance %s: batched %.3e, single %.3e, oracle floor %.3e, bar %.1e'
          % (label, e_b, e_s, floor, tol))
    assert e_b <= tol, (label, e_b, e_s, floor, tol)


def test_batch_fast_as_close_to_oracle_as_single_path(rok):
    cases = _mixed_instances()
    M, steps = 8, 2
    b = rok.rok_batch_init([p for p, _, _ in cases], krylov_max=M, rounding=rok.ROK_ROUND_FAST)
    y = b.pack([yy for _, yy, _ in cases])
    hs = _dts(cases)
    rok.rok_batch_step(b, y, hs, M, nsteps=steps)
    got = b.unpack(y)
    for k, (p, y0, _) in enumerate(cases):
        _check_fast(rok, p, y0, hs[k], M, steps, got[k], k)


@pytest.mark.parametrize('mode', ['strict', 'fast'])
def test_batch_every_tuning_candidate_same_bits(rok, mode):
    cases = _mixed_instances()
    M = 6
    b = rok.rok_batch_init([p for p, _, _ in cases], krylov_max=M,
                           rounding=getattr(rok, 'ROK_ROUND_' + mode.upper()))
    y0 = b.pack([yy for _, yy, _ in cases])
    hs = _dts(cases)
    ref = None
    for tile in (rok.ROK_TILE_32x8, rok.ROK_TILE_16x16, rok.ROK_TILE_64x4):
        for cpc in rok.CHUNKS_PER_CTA:
            rok.rok_batch_set_tuning(b, tile=(tile, tile, tile), chunks_per_cta=cpc,
                                     vec_chunks_per_cta=rok.CHUNKS_PER_CTA[-1 - rok.CHUNKS_PER_CTA.index(cpc)])
            y = y0.clone()
            rok.rok_batch_step(b, y, hs, M, nsteps=2)
            r = host(y)
            if ref is None:
                ref = r
            assert np.array_equal(r, ref), (tile, cpc)
    t = rok.rok_batch_tune(b, y0)
    assert all(s in (0, 1, 2) for s in t['tile']) and t['chunks_per_cta'] in rok.CHUNKS_PER_CTA
    assert all(ms > 0 for ms in t['mgs_ms']) and all(ms > 0 for ms in t['vec_ms'])
    assert t['stencil_ms'][0][0] > 0 and t['stencil_ms'][1][0] > 0 and t['stencil_ms'][2][0] > 0
    assert rok.rok_batch_get_tuning(b)['tile'] == t['tile']
    y = y0.clone()
    rok.rok_batch_step(b, y, hs, M, nsteps=2)
    assert np.array_equal(host(y), ref)


def test_batch_graph_replay_and_step_runs(rok):
    cases = _mixed_instances()
    M = 6
    b = rok.rok_batch_init([p for p, _, _ in cases], krylov_max=M)
    y0 = b.pack([yy for _, yy, _ in cases])
    hs = _dts(cases)
    ya = y0.clone()
    rok.rok_batch_get_launches(b, reset=True)
    for _ in range(3):
        rok.rok_batch_step(b, ya, hs, M)
    eager = rok.rok_batch_get_launches(b, reset=True)
    rok.rok_batch_set_graph(b, True)
    yb = y0.clone()
    rok.rok_batch_step(b, yb, hs, M, nsteps=3)        # captured once, replayed
    replay = rok.rok_batch_get_launches(b, reset=True)
    yc = y0.clone()
    info = rok.rok_batch_step(b, yc, hs, M, nsteps=3, info=True)
    assert np.array_equal(host(ya), host(yb)) and np.array_equal(host(ya), host(yc))
    assert all(i['status'] == 0 and i['jvps'] == 3 * M for i in info)
    # a replay counts its kernel nodes: the same kernels as the eager steps, per
    # step one stencil launch per physics group and pass, not one per instance
    assert eager == replay
    per_step = eager // 3
    assert 3 * (1 + M + 3) <= per_step < 3 * (1 + M + 3) + 2 * M + (M * (M + 1)) // 2 + 40


def test_batch_failed_instance_is_isolated(rok):
    cases = _mixed_instances()
    M = 6
    b = rok.rok_batch_init([p for p, _, _ in cases], krylov_max=M, rounding=rok.ROK_ROUND_STRICT)
    states = [yy.copy() for _, yy, _ in cases]
    states[2][1, 5, 7] = np.nan
    y = b.pack(states)
    hs = _dts([(p, yy if k != 2 else cases[2][1], c) for k, (p, yy, c) in enumerate(cases)])
    info = rok.rok_batch_step(b, y, hs, M, nsteps=2, info=True)
    got = b.unpack(y)
    assert info[2]['status'] == rok.ROK_ERR_NONFINITE
    assert np.array_equal(got[2], states[2], equal_nan=True)
    for k, (p, y0, _) in enumerate(cases):
        if k == 2:
            continue
        assert info[k]['status'] == 0
        sys_ = core.System(p)
        yo = I.rok_step(sys_, I.rok_step(sys_, y0, hs[k], M), hs[k], M)
        assert np.array_equal(got[k], yo), k
    # statuses were cleared by the info call: the next clean run reports OK
    y = b.pack([yy for _, yy, _ in cases])
    info = rok.rok_batch_step(b, y, hs, M, info=True)
    assert all(i['status'] == 0 for i in info)


def test_batch_invalid_arguments(rok):
    cases = _mixed_instances()[:2]
    b = rok.rok_batch_init([p for p, _, _ in cases], krylov_max=4)
    y = b.pack([yy for _, yy, _ in cases])
    with pytest.raises(rok.RokError):
        rok.rok_batch_step(b, y, [1e-3, -1.0], 4)
    with pytest.raises(rok.RokError):
        rok.rok_batch_step(b, y, [1e-3, 1e-3], 5)
    with pytest.raises(rok.RokError):
        rok.rok_batch_set_tuning(b, tile=(0, 0, 0), chunks_per_cta=3)
    p, _, _ = W.cylinder_ogrid(16, 32)
    with pytest.raises(rok.RokError) as e:
        rok.rok_batch_init([p], krylov_max=4)
    assert e.value.status == rok.ROK_ERR_UNSUPPORTED


def test_batch_full_workload(rok):
    # 64 Euler-vortex / Navier-Stokes Taylor-Green instances, sides 32..384, ROK4
    # M = 16, tuned launch shapes, graph replay: the launch configuration the
    # benchmark times.  Sampled instances (the three smallest, the two largest)
    # against the oracle; mass conservation for all.
    inst = W.batched_instances()
    M, steps = 16, 2
    probs = [i.problem for i in inst]
    b = rok.rok_batch_init(probs, krylov_max=M)
    y = b.pack([i.y0 for i in inst])
    hs = [I.dt_from_cfl(i.problem, i.y0, i.cfl) for i in inst]
    rok.rok_batch_tune(b, y)
    rok.rok_batch_set_graph(b, True)
    info = rok.rok_batch_step(b, y, hs, M, nsteps=steps, info=True)
    assert all(i['status'] == 0 and i['m_eff'] == M for i in info)
    got = b.unpack(y)
    order = np.argsort([p.nx for p in probs])
    for k in list(order[:3]) + list(order[-2:]):
        _check_fast(rok, probs[k], inst[k].y0, hs[k], M, steps, got[k], (k, probs[k].nx))
    for k in range(len(inst)):
        m0, m1 = inst[k].y0[0].sum(), got[k][0].sum()
        assert abs(m1 - m0) <= 1e-9 * abs(m0), k
