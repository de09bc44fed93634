"""Benchmark of the ROK4 hot path on GB300.

Workload (one step = one ROK4 step, rows a1-a7 of the hot path): decaying 2-D
Navier-Stokes Taylor-Green vortex, periodic 512 x 512 uniform grid, M = 0.1,
Re = 1600, FP64 state, Krylov dimension M = 20, time step at CFL 8.  Synthetic
data from the closed-form initial condition.  Metric: cells x JVPs per second
of whole ROK4 steps (Mcell-JVP/s), with the roofline of the dominant kernel
(the FP64 residual/JVP stencil) and the RK4 / ESDIRK3 comparators on the same
state.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain FP64 evaluation of the same
step) on this host's cores.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID, RE, MACH, KRYLOV, CFL = 512, 1600.0, 0.1, 20, 8.0
METRIC = 'time-to-fixed-L2-error ROK4 vs RK4/ESDIRK; Mcell-JVP/s; % HBM peak'
UNIT = 'Mcell-JVP/s'
WORKLOAD = 'ns2d-taylor-green-512x512-Re1600-M0.1-rok4-M20-cfl8'

# Algorithmic FP64 operations per cell of one stencil launch, Navier-Stokes on a
# uniform grid (divisions and square roots counted as one operation each; each
# face counted once).  Per face: MUSCL 44, Roe averages 42, Roe dissipation and
# flux 75, viscous flux 34 -> 195; two faces per cell 390; primitives 10; face
# balance 20; JVP state formation y + eps v 8 and quotient 8.
FLOPS_RESIDUAL_NS = 390 + 10 + 20
FLOPS_JVP_NS = FLOPS_RESIDUAL_NS + 8 + 8
BYTES_RESIDUAL, BYTES_JVP = 64, 128

# DRAM bytes (read + write) of one FD-JVP launch of the Navier-Stokes stencil at
# 512 x 512, from an ncu capture of this workload (dram__bytes_read.sum +
# dram__bytes_write.sum, cold L2): the three inputs y, v, f(y) are read once
# (25.17 MB algorithmic); the 8.4 MB output stays in L2 within the launch.
STENCIL_JVP_DRAM_BYTES_512 = 25243136 + 0


def _peaks():
    path = os.path.join(ROOT, 'MEASURED_PEAKS.json')
    if os.path.exists(path):
        try:
            with open(path) as fh:
                d = json.load(fh)
            return d, 'measured'
        except Exception:
            pass
    return {'hbm_gbs': 6800.0, 'bf16_tflops': 1900.0}, 'fallback'


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms from before the
    warm-up; only the samples taken inside the timed window are summarised."""
    Q = ('timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
         'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
         'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.window = None

    def start(self):
        try:
            self.proc = subprocess.Popen(['nvidia-smi', '-i', str(self.index), '--query-gpu=' + self.Q,
                                          '--format=csv,noheader,nounits', '-lms', '50'],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(',')]))

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def stop(self):
        if self.proc is None:
            return {'sm_mhz': None, 'sm_max_mhz': None, 'reasons': ['nvidia-smi unavailable']}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [(t, r) for t, r in self.rows if len(r) >= 10]
        inside = [(t, r) for t, r in rows if self.window and self.window[0] <= t <= self.window[1] + 0.06]
        use = inside if inside else rows[-3:]
        num = lambda x: float(x) if x.replace('.', '').isdigit() else None
        sm = [num(r[2]) for _, r in use if num(r[2]) is not None]
        mx = [num(r[3]) for _, r in use if num(r[3]) is not None]
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        reasons = set()
        for _, r in use:
            for k, nm in enumerate(names):
                if r[6 + k].lower() == 'active':
                    reasons.add(nm)
        return {'sm_mhz': statistics.median(sm) if sm else None, 'sm_max_mhz': max(mx) if mx else None,
                'reasons': sorted(reasons), 'samples': len(use), 'samples_in_window': len(inside)}


def _dist():
    ws = int(os.environ.get('WORLD_SIZE', '1'))
    rank = int(os.environ.get('RANK', '0'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    return ws, rank, local


def reduce_timing(ms_local, units_local, dist_ok):
    """Whole-job timing of N replicas: the step time is the maximum over ranks,
    the value the units all ranks processed divided by that time (weak scaling,
    no data-path collective: only this scalar reduction and the barriers)."""
    import torch
    import torch.distributed as dist
    dev = 'cuda' if dist_ok and dist.get_backend() == 'nccl' else 'cpu'
    t = torch.tensor([ms_local, units_local], dtype=torch.float64, device=dev)
    if dist_ok:
        mx = t[:1].clone()
        tot = t[1:].clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        return float(mx.item()), float(tot.item())
    return float(ms_local), float(units_local)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1607_06834_gb300 import rok
    from paper_1607_06834_gb300 import workloads as W

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group('nccl' if dist.is_nccl_available() else 'gloo')

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    prob, y0 = W.taylor_green(N_GRID, mach=MACH, reynolds=RE)
    cells = prob.ncells
    stream = torch.cuda.current_stream()
    rounding = rok.ROK_ROUND_STRICT if args.rounding == 'strict' else rok.ROK_ROUND_FAST
    ctx = rok.rok_init(prob, krylov_max=max(KRYLOV, 30), rounding=rounding, stream=stream)
    y = rok.state_tensor(y0)
    h = rok.rok_dt_from_cfl(ctx, y, CFL)
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device='cuda')

    fp64_peak = rok.rok_fp64_fma_peak(20) if rank == 0 else None

    sampler = ClockSampler(local)
    sampler.start()
    if args.graph:
        rok.rok_set_graph(ctx, True)
    for _ in range(args.warmup):
        rok.rok_step(ctx, y, h, KRYLOV)
    info = rok.rok_step(ctx, y, h, KRYLOV, info=True)
    assert info['m_eff'] == KRYLOV

    rok.rok_get_counters(ctx, reset=True)
    rok.rok_set_stencil_timing(ctx, not args.graph)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    t_wall0 = time.perf_counter()
    t_epoch0 = time.time()
    for k in range(args.steps):
        flush.fill_(float(k))           # evict L2 between timed steps (outside the events)
        ev[k][0].record(stream)
        rok.rok_step(ctx, y, h, KRYLOV)
        ev[k][1].record(stream)
    barrier()
    wall = time.perf_counter() - t_wall0
    sampler.mark(t_epoch0, time.time())
    clocks = sampler.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    cnt = rok.rok_get_counters(ctx, reset=True)
    rok.rok_set_stencil_timing(ctx, False)
    rok.rok_sync(ctx)
    if args.graph:
        # graph replays carry no per-kernel events: time the stencil launches of
        # the same steps in a second, eager pass
        rok.rok_set_graph(ctx, False)
        rok.rok_set_stencil_timing(ctx, True)
        for k in range(args.steps):
            rok.rok_step(ctx, y, h, KRYLOV)
        c2 = rok.rok_get_counters(ctx, reset=True)
        rok.rok_set_stencil_timing(ctx, False)
        cnt['stencil_ms'], cnt['stencil_timed'] = c2['stencil_ms'], c2['stencil_timed']
        rok.rok_set_graph(ctx, True)
    # whole job: the slowest rank's time, the cell-JVPs of all ranks
    ms, units = reduce_timing(ms, float(cells * KRYLOV * args.steps), ws > 1)
    ms_per_step = ms / args.steps
    value = units / (ms * 1e-3) / 1e6

    # dominant kernel: the residual / JVP stencil (1 + M + 3 launches per step)
    n_res, n_jvp = 4, KRYLOV
    flops_step = cells * (n_res * FLOPS_RESIDUAL_NS + n_jvp * FLOPS_JVP_NS)
    stencil_ms_per_launch = cnt['stencil_ms'] / max(cnt['stencil_timed'], 1)
    achieved = flops_step / (n_res + n_jvp) / (stencil_ms_per_launch * 1e-3) / 1e12
    # algorithmic bytes of the average launch: a residual reads q and writes f
    # (64 B per cell), an FD JVP reads y, v, f(y) and writes Jv (128 B per cell)
    bytes_launch = cells * (n_res * BYTES_RESIDUAL + n_jvp * BYTES_JVP) / (n_res + n_jvp)

    # end to end through the public API with host buffers (pinned), copies inside
    yh = torch.from_numpy(y0.copy()).pin_memory()
    e2e_steps = max(2, min(args.steps, 5))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        rok.rok_step(ctx, yh, h, KRYLOV)   # host tensor: H2D, step, D2H
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_value = ws * cells * KRYLOV * e2e_steps / e2e_s / 1e6

    # comparators on the same state: classical RK4 and ESDIRK3 Newton-GMRES(30)
    yc = rok.state_tensor(y0)
    h_rk = rok.rok_dt_from_cfl(ctx, yc, 1.0)
    rok.rk_step(ctx, yc, h_rk)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(5):
        rok.rk_step(ctx, yc, h_rk)
    e1.record(stream)
    barrier()
    rk_ms = e0.elapsed_time(e1) / 5
    yc = rok.state_tensor(y0)
    barrier()
    t0 = time.perf_counter()
    esd = rok.esdirk_step(ctx, yc, h, info=True)
    barrier()
    esd_ms = (time.perf_counter() - t0) * 1e3
    ros = {}
    for name, meth in (('ros4', rok.ROK_ROS_ROS4), ('row', rok.ROK_ROS_ROW)):
        yc = rok.state_tensor(y0)
        barrier()
        t0 = time.perf_counter()
        inf = rok.ros_step(ctx, yc, h, method=meth, info=True)
        barrier()
        ros[name] = ((time.perf_counter() - t0) * 1e3, inf)

    # the mixed-precision form (binary32 basis and Gram-Schmidt) on the same steps:
    # time per step and its difference from the binary64 form after the same steps
    forms = {}
    if args.forms:
        ctx32 = rok.rok_init(prob, krylov_max=KRYLOV, rounding=rounding, stream=stream, basis=rok.ROK_BASIS_FP32)
        if args.graph:
            rok.rok_set_graph(ctx32, True)
        ya, yb = rok.state_tensor(y0), rok.state_tensor(y0)
        for _ in range(args.warmup):
            rok.rok_step(ctx32, rok.state_tensor(y0), h, KRYLOV)
        barrier()
        ev32 = []
        for k in range(args.steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rok.rok_step(ctx32, ya, h, KRYLOV)
            b.record(stream)
            ev32.append((a, b))
            rok.rok_step(ctx, yb, h, KRYLOV)
        barrier()
        ms32 = sum(a.elapsed_time(b) for a, b in ev32) / args.steps
        diff = float((ya - yb).norm() / yb.norm())
        forms['mixed_fp32_basis'] = {'ms_per_step': round(ms32, 4), 'speedup_vs_fp64': round(ms_per_step / ms32, 3),
                                     'value': round(ws * cells * KRYLOV / (ms32 * 1e-3) / 1e6, 3),
                                     'rel_l2_vs_fp64_after_steps': diff, 'steps_compared': args.steps}
        # exact (dual-number) Jacobian-vector products inside the Arnoldi process
        ctxe = rok.rok_init(prob, krylov_max=KRYLOV, rounding=rounding, stream=stream, jvp=rok.ROK_JVP_EXACT)
        if args.graph:
            rok.rok_set_graph(ctxe, True)
        ye, yf = rok.state_tensor(y0), rok.state_tensor(y0)
        for _ in range(args.warmup):
            rok.rok_step(ctxe, rok.state_tensor(y0), h, KRYLOV)
        barrier()
        eve = []
        for k in range(args.steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rok.rok_step(ctxe, ye, h, KRYLOV)
            b.record(stream)
            eve.append((a, b))
            rok.rok_step(ctx, yf, h, KRYLOV)
        barrier()
        mse = sum(a.elapsed_time(b) for a, b in eve) / args.steps
        forms['exact_jvp'] = {'ms_per_step': round(mse, 4), 'speedup_vs_fd': round(ms_per_step / mse, 3),
                              'value': round(ws * cells * KRYLOV / (mse * 1e-3) / 1e6, 3),
                              'rel_l2_vs_fd_after_steps': float((ye - yf).norm() / yf.norm()),
                              'steps_compared': args.steps}
        forms['batched'] = batch_form(10)
        # the strict-rounding build (no contraction, IEEE division and square
        # root, the oracle's operation order): the build whose ten-step
        # trajectory equals the oracle's bit for bit
        ctxs = rok.rok_init(prob, krylov_max=KRYLOV, rounding=rok.ROK_ROUND_STRICT, stream=stream)
        if args.graph:
            rok.rok_set_graph(ctxs, True)
        ys = rok.state_tensor(y0)
        for _ in range(args.warmup):
            rok.rok_step(ctxs, ys, h, KRYLOV)
        barrier()
        evs = []
        for k in range(args.steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rok.rok_step(ctxs, ys, h, KRYLOV)
            b.record(stream)
            evs.append((a, b))
        barrier()
        mss = sum(a.elapsed_time(b) for a, b in evs) / args.steps
        forms['strict_rounding'] = {'ms_per_step': round(mss, 4), 'speedup_vs_fma': round(ms_per_step / mss, 3),
                                    'value': round(ws * cells * KRYLOV / (mss * 1e-3) / 1e6, 3),
                                    'parity': 'bit-exact against the oracle over 10 steps'}
    if rank != 0:
        return None
    peaks, src = _peaks()
    # FP64 roof from unit counts and clock: 152 SMs x 2 FP64 FMA lanes per SM per
    # clock (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on.peak_sustained =
    # 304 per clock per GPU) x 2 flops x the SM clock measured under load
    sm_mhz = clocks.get('sm_mhz') or 2070.0
    fp64_roof = 152 * 2 * 2 * sm_mhz * 1e6 / 1e12
    out = {
        'metric': METRIC, 'value': round(value, 3), 'unit': UNIT, 'n_gpus': ws, 'steps': args.steps,
        'warmup': args.warmup, 'ms_per_step': round(ms_per_step, 4), 'higher_is_better': True,
        'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic',
        'config': {'workload': WORKLOAD, 'cells': cells, 'krylov_m': KRYLOV, 'cfl': CFL, 'dt': h,
                   'rounding': args.rounding, 'l2': 'flushed between timed steps (256 MB write)',
                   'launch': 'CUDA-graph replay per step' if args.graph else 'kernel by kernel',
                   'parallelism': 'replicas' if ws > 1 else 'single-gpu'},
        'roofline': {'bound': 'alu', 'kernel': 'residual/JVP stencil (cart_kernel<NS>)',
                     'achieved': round(achieved, 4), 'peak': round(fp64_roof, 4), 'unit': 'TFLOP/s',
                     'frac': round(achieved / fp64_roof, 4),
                     'traffic': STENCIL_JVP_DRAM_BYTES_512 if N_GRID == 512 else None,
                     'traffic_unit': 'bytes per FD-JVP launch (ncu dram read+write)',
                     'algorithmic_bytes_per_launch': round(bytes_launch),
                     'peak_source': 'FP64 FMA roof = 152 SMs x 2 FMA/clk/SM x 2 flops x measured SM clock',
                     'fp64_fma_microbenchmark_tflops': round(fp64_peak, 4),
                     'flops_per_cell': {'residual': FLOPS_RESIDUAL_NS, 'jvp': FLOPS_JVP_NS},
                     'stencil_ms_per_launch': round(stencil_ms_per_launch, 5),
                     'hbm_frac_of_' + src: round(bytes_launch / (stencil_ms_per_launch * 1e-3) / 1e9 / peaks['hbm_gbs'], 5)},
        'clocks': clocks,
        'e2e': {'value': round(e2e_value, 3), 'unit': UNIT, 'h2d_bytes_per_step': int(y0.nbytes),
                'd2h_bytes_per_step': int(y0.nbytes)},
        'gpu_launches': int(cnt['launches']),
        'comparators': {'rk4_ms_per_step_cfl1': round(rk_ms, 4), 'rk4_dt': h_rk,
                        'esdirk3_ms_per_step_cfl8': round(esd_ms, 2), 'esdirk3_info': esd,
                        'ros4_ms_per_step_cfl8': round(ros['ros4'][0], 2), 'ros4_info': ros['ros4'][1],
                        'row_ms_per_step_cfl8': round(ros['row'][0], 2), 'row_info': ros['row'][1]},
        'wall_s_timed': round(wall, 3),
        'forms': forms,
    }
    if ws == 1:
        out['cpu_baseline'] = cpu_baseline(prob, y0, h)
    return out


def batch_form(steps, one_at_a_time=True):
    """The batched form: 64 independent Euler-vortex / Navier-Stokes Taylor-Green
    instances on periodic grids of sides 32..384 (per-instance seeds), ROK4
    M = 16, each at its own CFL-derived step; `steps` steps of all instances in
    one graph launch with autotuned launch shapes, against the same instances
    stepped one at a time through the single-problem entry point (graph replay
    per step).  Inputs are larger than L2 (flat vectors of ~110 MB, basis ~1.9 GB)."""
    import torch

    from paper_1607_06834_gb300 import rok
    from paper_1607_06834_gb300 import workloads as W
    M = 16
    inst = W.batched_instances()
    probs = [i.problem for i in inst]
    cells = sum(p.ncells for p in probs)
    stream = torch.cuda.current_stream()
    b = rok.rok_batch_init(probs, krylov_max=M, stream=stream)
    y0 = b.pack([i.y0 for i in inst])
    hs = []
    for i in inst:
        ctx = rok.rok_init(i.problem, krylov_max=1, stream=stream)
        hs.append(rok.rok_dt_from_cfl(ctx, rok.state_tensor(i.y0), i.cfl))
        del ctx
    tuning = rok.rok_batch_tune(b, y0)
    rok.rok_batch_set_graph(b, True)
    y = y0.clone()
    rok.rok_batch_step(b, y, hs, M, nsteps=steps)          # capture + first replay (warm-up)
    y = y0.clone()
    rok.rok_batch_get_launches(b, reset=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rok.rok_batch_step(b, y, hs, M, nsteps=steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = rok.rok_batch_get_launches(b)
    info = rok.rok_batch_step(b, y0.clone(), hs, M, nsteps=1, info=True)
    out = {'workload': 'batch-64-vortex-tgv-32..384-rok4-M16', 'instances': len(inst), 'cells': cells,
           'steps': steps, 'ms': round(ms, 3), 'ms_per_step': round(ms / steps, 4),
           'value': round(cells * M * steps / (ms * 1e-3) / 1e6, 3), 'unit': UNIT,
           'gpu_launches_per_graph': launches, 'tuning': tuning,
           'statuses_ok': all(i['status'] == 0 for i in info)}
    del b
    if one_at_a_time:
        total = 0.0
        for k, i in enumerate(inst):
            ctx = rok.rok_init(i.problem, krylov_max=M, stream=stream)
            rok.rok_set_graph(ctx, True)
            ys = rok.state_tensor(i.y0)
            rok.rok_step(ctx, ys, hs[k], M)
            ys = rok.state_tensor(i.y0)
            torch.cuda.synchronize()
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(steps):
                rok.rok_step(ctx, ys, hs[k], M)
            c.record(stream)
            torch.cuda.synchronize()
            total += a.elapsed_time(c)
            del ctx
        out['one_at_a_time_ms'] = round(total, 3)
        out['one_at_a_time_value'] = round(cells * M * steps / (total * 1e-3) / 1e6, 3)
        out['speedup_vs_one_at_a_time'] = round(total / ms, 3)
    return out


def run_batch(args):
    """--mode batch: the batched form alone, as one JSON line."""
    import torch
    torch.cuda.set_device(0)
    out = batch_form(args.steps)
    out.update({'metric': METRIC, 'mode': 'batch', 'dtype': 'f64', 'data': 'synthetic'})
    print(json.dumps(out))


def run_grad(args):
    """--mode grad: gradient of the final kinetic energy of the 256^2 Taylor-Green
    vortex (Re = 1000) after 100 ROK4 steps (M = 20, CFL 8) with respect to the
    initial state and the viscosity, through the reverse step with a checkpoint
    every 10 steps (segments re-run onto tapes of the step internals; the same
    gradient recomputing every step inside its reverse is timed beside it and
    compared bit for bit).  Reports forward and backward times, the derivatives along
    64 seeded random unit directions and central differences (h = 1e-6) of the
    GPU forward map along two directions.  (The checks of the reverse step
    against the oracle's adjoint and complex step are in tests/test_gpu_adjoint.py;
    on this low-Mach state the central differences are not a valid check.)"""
    import torch

    from paper_1607_06834_gb300 import autograd as G
    from paper_1607_06834_gb300 import rok
    from paper_1607_06834_gb300 import workloads as W
    torch.cuda.set_device(0)
    n, M, K, every = 256, 20, (args.steps if args.steps != 30 else 100), 10
    prob, y0 = W.taylor_green(n, mach=MACH, reynolds=1000.0)
    ctx = rok.rok_init(prob, krylov_max=M)
    yd0 = rok.state_tensor(y0)
    h = rok.rok_dt_from_cfl(ctx, yd0, CFL)
    stream = torch.cuda.current_stream()

    def grad(nsteps, tapes=True):
        y = yd0.clone().requires_grad_(True)
        mu = torch.tensor(prob.mu, dtype=torch.float64, requires_grad=True)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        J = G.kinetic_energy(G.integrate(ctx, y, mu, h, M, nsteps, checkpoint_every=every, tapes=tapes))
        e[1].record(stream)
        J.backward()
        e[2].record(stream)
        torch.cuda.synchronize()
        return y.grad.detach(), float(mu.grad), float(J), e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])

    grad(2)                                   # warm-up (allocations)
    grad(2, tapes=False)
    g, gmu, J, ms_f, ms_b = grad(K)
    gr, gmur, _, ms_fr, ms_br = grad(K, tapes=False)
    rng = np.random.default_rng(0)
    dirs = rng.standard_normal((64, y0.size))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    dd = dirs @ g.cpu().numpy().ravel()
    out = {'mode': 'grad', 'metric': METRIC, 'workload': 'ns2d-taylor-green-256x256-Re1000-rok4-M20-100steps',
           'steps': K, 'krylov_m': M, 'checkpoint_every': every, 'dt': h, 'J_final_ke': J,
           'forward_ms': round(ms_f, 2), 'backward_ms': round(ms_b, 2),
           'backward_ms_per_step': round(ms_b / K, 3),
           'tape_bytes_per_step': rok.rok_tape_bytes(ctx, M),
           'without_tapes': {'forward_ms': round(ms_fr, 2), 'backward_ms': round(ms_br, 2),
                             'gradient_bit_identical': bool(torch.equal(g, gr)) and gmu == gmur},
           'dJ_dmu': gmu,
           'grad_norm': float(g.norm()), 'directional_derivatives_64': {
               'min': float(dd.min()), 'max': float(dd.max()), 'rms': float(np.sqrt(np.mean(dd ** 2)))},
           'dtype': 'f64', 'data': 'synthetic'}
    # central differences of the GPU forward map (h = 1e-6) along two directions
    fd = []
    for k in range(2):
        dk = torch.from_numpy(dirs[k].reshape(y0.shape)).cuda()
        vals = []
        for sgn in (1.0, -1.0):
            y = yd0 + sgn * 1e-6 * dk
            for _ in range(K):
                rok.rok_step(ctx, y, h, M)
            vals.append(float(G.kinetic_energy(y)))
        fdv = (vals[0] - vals[1]) / 2e-6
        fd.append({'adjoint': float(dd[k]), 'central_fd': fdv, 'rel_diff': abs(fdv - dd[k]) / abs(dd[k])})
    out['central_fd_h1e-6'] = fd
    print(json.dumps(out))


def run_configs(args):
    """--mode configs: one line per workload of the method's configurations
    (vortex 64^2, Taylor-Green 512^2, cylinder O-grid with the binary64 and
    binary32 bases, 64-instance batch; the gradient workload has --mode grad):
    GPU time per step by CUDA events for the FMA and the strict build, the
    vortex's distance from its exact advected solution, and the CPU baseline
    (the oracle on a few steps of the same workload, one core).  The parity of
    every configuration against the oracle is asserted in tests/."""
    import torch

    from paper_1607_06834_gb300 import rok
    from paper_1607_06834_gb300 import workloads as W
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    out = {'mode': 'configs', 'metric': METRIC, 'dtype': 'f64', 'data': 'synthetic', 'configs': {}}

    def timed(ctx, y, h, M, steps):
        # warm-up step on the buffer that is timed (a graph is captured per buffer)
        yw = y.clone()
        rok.rok_step(ctx, yw, h, M)
        yw.copy_(y)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            rok.rok_step(ctx, yw, h, M)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    def both_builds(prob, y0, cfl, M, steps, basis=0):
        res = {}
        for name, rnd in (('fma', rok.ROK_ROUND_FAST), ('strict', rok.ROK_ROUND_STRICT)):
            ctx = rok.rok_init(prob, krylov_max=M, rounding=rnd, basis=basis)
            yd = rok.state_tensor(y0)
            h = rok.rok_dt_from_cfl(ctx, yd, cfl)
            rok.rok_set_graph(ctx, True)
            res[name] = (timed(ctx, yd, h, M, steps), ctx, h)
        return res

    # 1. Euler vortex 64^2, M = 12, 10 steps at CFL 5, exact advected solution
    prob, y0 = W.isentropic_vortex(64)
    r = both_builds(prob, y0, 5.0, 12, 10)
    ctx, h = r['fma'][1], r['fma'][2]
    yd = rok.state_tensor(y0)
    for _ in range(10):
        rok.rok_step(ctx, yd, h, 12)
    ex = W.vortex_exact(prob, 10 * h)
    yg = yd.cpu().numpy()
    out['configs']['1-vortex64-M12-cfl5-10steps'] = {
        'gpu_ms_per_step': round(r['fma'][0], 4), 'gpu_ms_per_step_strict': round(r['strict'][0], 4),
        'rel_l2_vs_exact_solution': float(np.linalg.norm(yg - ex) / np.linalg.norm(ex)),
        'cpu_baseline': cpu_baseline_steps(prob, y0, h, 12, 10)}
    # 2. Taylor-Green 512^2, M = 20, CFL 8
    prob, y0 = W.taylor_green(512, reynolds=1600.0)
    r = both_builds(prob, y0, 8.0, 20, 10)
    out['configs']['2-tgv512-M20-cfl8'] = {
        'gpu_ms_per_step': round(r['fma'][0], 4), 'gpu_ms_per_step_strict': round(r['strict'][0], 4),
        'cpu_baseline': cpu_baseline_steps(prob, y0, r['fma'][2], 20, 2)}
    # 3. cylinder O-grid 256 x 512, M = 30, CFL 10, binary64 and binary32 bases
    prob, y0, _ = W.cylinder_ogrid(256, 512)
    r64 = both_builds(prob, y0, 10.0, 30, 5)
    r32 = both_builds(prob, y0, 10.0, 30, 5, basis=rok.ROK_BASIS_FP32)
    c64, c32, h = r64['fma'][1], r32['fma'][1], r64['fma'][2]
    yd = rok.state_tensor(y0)
    ya, yb = yd.clone(), yd.clone()
    for _ in range(5):
        rok.rok_step(c64, ya, h, 30)
        rok.rok_step(c32, yb, h, 30)
    big = {}
    for cfl in (100.0, 1000.0):
        yy = yd.clone()
        try:
            rok.rok_step(c64, yy, rok.rok_dt_from_cfl(c64, yd, cfl), 30, info=True)
            big[str(cfl)] = 'ok'
        except rok.RokError as e:
            big[str(cfl)] = rok.rok_status_string(e.status)
    out['configs']['3-cylinder256x512-M30-cfl10'] = {
        'gpu_ms_per_step_fp64_basis': round(r64['fma'][0], 3), 'gpu_ms_per_step_fp32_basis': round(r32['fma'][0], 3),
        'gpu_ms_per_step_strict_fp64_basis': round(r64['strict'][0], 3),
        'gpu_ms_per_step_strict_fp32_basis': round(r32['strict'][0], 3),
        'fp32_speedup': round(r64['fma'][0] / r32['fma'][0], 3),
        'rel_l2_fp32_vs_fp64_after_5_steps': float((ya - yb).norm() / ya.norm()),
        'first_step_at_cfl_from_impulsive_start': big,
        'cpu_baseline': cpu_baseline_steps(prob, y0, h, 30, 2)}
    # 4. the batch
    out['configs']['4-batch64'] = batch_form(10)
    print(json.dumps(out))


def cpu_baseline_steps(prob, y0, h, M, steps):
    """CPU baseline of one configuration: the oracle, as it stands, for `steps`
    ROK4 steps on one core; milliseconds per step."""
    from oracle import core
    from oracle import integrators as I
    sys_ = core.System(prob)
    t0 = time.perf_counter()
    y = y0
    for _ in range(steps):
        y = I.rok_step(sys_, y, h, M)
    return {'ms_per_step': round((time.perf_counter() - t0) / steps * 1e3, 2), 'cores': 1, 'kind': 'oracle',
            'sample': '%d ROK4 step(s)' % steps}


def cpu_baseline(prob, y0, h, steps=8):
    """The CPU oracle, as it stands, on a bounded sample: `steps` ROK4 steps of the
    same workload, first single-threaded (the plain oracle), then with its
    residual and FD-JVP loops on every host core (the OpenMP build of the same
    C source, same bits; the NumPy parts of the integrator stay on one core)."""
    from oracle import core
    from oracle import integrators as I
    cores = len(os.sched_getaffinity(0))

    def run(n):
        sys_ = core.System(prob)
        t0 = time.perf_counter()
        y = y0
        for _ in range(n):
            y = I.rok_step(sys_, y, h, KRYLOV)
        return time.perf_counter() - t0

    dt1 = run(steps)
    try:
        core.use_parallel_build(cores)
        run(1)                                   # thread pool start-up
        dtn = run(steps)
    finally:
        core.use_parallel_build(None)
    v1 = prob.ncells * KRYLOV * steps / dt1 / 1e6
    vn = prob.ncells * KRYLOV * steps / dtn / 1e6
    return {'value': round(vn, 5), 'unit': UNIT, 'cores': cores, 'kind': 'oracle',
            'sample': '%d ROK4 step(s) of the 512x512 Taylor-Green workload (M=20), %.1f s on %d cores '
                      '(OpenMP residual, NumPy integrator on one core)' % (steps, dtn, cores),
            'single_thread': {'value': round(v1, 5), 'unit': UNIT, 'cores': 1,
                              'sample': '%d ROK4 step(s), %.1f s' % (steps, dt1)}}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return None
    from paper_1607_06834_gb300 import workloads as W
    from oracle import core
    from oracle import integrators as I
    prob, y0 = W.taylor_green(N_GRID, mach=MACH, reynolds=RE)
    h = I.dt_from_cfl(prob, y0, CFL)
    cores = len(os.sched_getaffinity(0))
    core.use_parallel_build(cores)          # residual loops on every host core, same bits
    sys_ = core.System(prob)
    y = y0
    for _ in range(args.warmup):
        y = I.rok_step(sys_, y, h, KRYLOV)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        y = I.rok_step(sys_, y, h, KRYLOV)
    dt = time.perf_counter() - t0
    value = prob.ncells * KRYLOV * args.steps / dt / 1e6
    return {'impl': 'reference', 'metric': METRIC, 'value': round(value, 5), 'unit': UNIT, 'n_gpus': ws,
            'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': round(dt / args.steps * 1e3, 2),
            'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic',
            'config': {'workload': WORKLOAD, 'cells': prob.ncells, 'krylov_m': KRYLOV, 'cfl': CFL},
            'cpu_baseline': {'value': round(value, 5), 'unit': UNIT, 'cores': cores, 'kind': 'oracle',
                             'sample': '%d timed ROK4 steps of the same workload (OpenMP residual on %d cores, '
                                       'NumPy integrator on one)' % (args.steps, cores)},
            'e2e': {'value': round(value, 5), 'unit': UNIT, 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0}}


def run_stencil_only(args):
    """Kernel-only mode (profiling): W + K FD-JVP stencil launches on an n x n
    Taylor-Green state (or, with --case cylinder, the 256 x 512 O-grid);
    prints the mean launch time."""
    import torch

    from paper_1607_06834_gb300 import rok
    from paper_1607_06834_gb300 import workloads as W
    if args.case == 'cylinder':
        prob, y0, _ = W.cylinder_ogrid(256, 512)
    else:
        prob, y0 = W.taylor_green(args.n, mach=MACH, reynolds=RE)
    rounding = rok.ROK_ROUND_STRICT if args.rounding == 'strict' else rok.ROK_ROUND_FAST
    ctx = rok.rok_init(prob, krylov_max=1, rounding=rounding)
    y = rok.state_tensor(y0)
    f0 = rok.rok_residual(ctx, y)
    g = torch.Generator(device='cuda').manual_seed(0)
    v = torch.randn(y.shape, dtype=torch.float64, device='cuda', generator=g)
    v /= v.norm()
    w = torch.empty_like(y)
    for _ in range(args.warmup):
        rok.rok_jvp(ctx, y, v, fy=f0, eps=2.0 ** -20, out=w)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        rok.rok_jvp(ctx, y, v, fy=f0, eps=2.0 ** -20, out=w)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({'mode': 'stencil', 'case': args.case, 'n': args.n, 'rounding': args.rounding, 'ms_per_launch': ms,
                      'tflops_alg': prob.ncells * FLOPS_JVP_NS / (ms * 1e-3) / 1e12}))


def _interp_time(points, target):
    """log-log interpolation of (error, seconds) points to a target error: the
    time a method needs to reach `target` (None if it never does in the range)."""
    pts = sorted((e, t) for e, t in points if e > 0)
    if not pts:
        return None
    if pts[0][0] > target:
        return None
    if pts[-1][0] <= target:
        return min(t for e, t in pts if e <= target)
    for (e0, t0), (e1, t1) in zip(pts, pts[1:]):
        if e0 <= target <= e1:
            a = (np.log(target) - np.log(e0)) / (np.log(e1) - np.log(e0))
            return float(np.exp(np.log(t0) + a * (np.log(t1) - np.log(t0))))
    return None


def run_wp(args):
    """Work-precision with adaptive steps (the paper's comparison, Sec. 4.2):
    ROK4 with its embedded estimate vs DOPRI5 vs fixed-step RK4 at CFL 1 over
    the same horizon as the time-to-error study, tolerances 1e-4, 1e-6, 1e-8
    (atol = rtol = tol); GPU time by CUDA events, error against an RK4
    reference at a 16x finer step."""
    import torch

    from paper_1607_06834_gb300 import rok
    from paper_1607_06834_gb300 import workloads as W
    torch.cuda.set_device(0)
    if args.case == 'tgv':
        prob, y0 = W.taylor_green(args.n, mach=MACH, reynolds=RE)
        krylov, base_cfl = KRYLOV, 8.0
    else:
        prob, y0, _ = W.cylinder_ogrid(256, 512)
        krylov, base_cfl = 30, 1.0
    ctx = rok.rok_init(prob, krylov_max=krylov)
    yd0 = rok.state_tensor(y0)
    dt1 = rok.rok_dt_from_cfl(ctx, yd0, 1.0)
    T = args.horizon * dt1 * base_cfl
    stream = torch.cuda.current_stream()

    def timed(fn):
        y = yd0.clone()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        info = fn(y)
        b.record(stream)
        torch.cuda.synchronize()
        return y, a.elapsed_time(b) / 1e3, info

    nref = int(round(T / (dt1 / 16)))
    yref, tref, _ = timed(lambda y: [rok.rk_step(ctx, y, T / nref) for _ in range(nref)])
    nrm = float(yref.norm())
    out = {'study': 'work-precision-adaptive', 'case': prob.name, 'T': T, 'dt_cfl1': dt1, 'reference_rk4_steps': nref,
           'methods': {}}
    nrk = int(round(T / dt1))
    y, s, _ = timed(lambda y: [rok.rk_step(ctx, y, T / nrk) for _ in range(nrk)])
    out['methods']['RK4 fixed CFL 1'] = [{'steps': nrk, 'gpu_s': s, 'rel_err': float((y - yref).norm()) / nrm}]
    for tol in (1e-4, 1e-6, 1e-8):
        for name, fn in (('ROK4 adaptive', lambda y: rok.rok_integrate(ctx, y, T, krylov, tol, tol, base_cfl * dt1)),
                         ('DOPRI5 adaptive', lambda y: rok.dopri5_integrate(ctx, y, T, tol, tol, dt1))):
            try:
                y, s, info = timed(fn)
                out['methods'].setdefault(name, []).append(
                    {'tol': tol, 'accepted': info['accepted'], 'rejected': info['rejected'], 'gpu_s': s,
                     'rel_err': float((y - yref).norm()) / nrm})
            except rok.RokError as err:
                out['methods'].setdefault(name, []).append({'tol': tol, 'failed': str(err)})
    print(json.dumps(out))


def run_tte(args):
    """Time to a fixed L2 error (the paper's work-precision measure, Sec. 4.2):
    ROK4 vs RK4 vs ESDIRK3 Newton-GMRES on one problem, fixed step sizes,
    error against an RK4 reference at a 16x finer step, GPU time of the whole
    integration by CUDA events."""
    import torch

    from paper_1607_06834_gb300 import rok
    from paper_1607_06834_gb300 import workloads as W
    torch.cuda.set_device(0)
    if args.case == 'tgv':
        prob, y0 = W.taylor_green(args.n, mach=MACH, reynolds=RE)
        krylov, cfls, cfl_rk = KRYLOV, [8.0, 4.0, 2.0], [1.0, 0.5]
        base_cfl = 8.0
    else:
        prob, y0, _ = W.cylinder_ogrid(256, 512)
        krylov, cfls, cfl_rk = 30, [1000.0, 300.0, 100.0, 30.0, 10.0], [1.0]
        base_cfl = 1.0
    if args.cfls:
        cfls = [float(x) for x in args.cfls.split(',')]
    ctx = rok.rok_init(prob, krylov_max=max(krylov, 30), rounding=rok.ROK_ROUND_FAST)
    yd = rok.state_tensor(y0)
    dt_unit = rok.rok_dt_from_cfl(ctx, yd, 1.0)
    start = 'closed-form initial condition'
    if args.developed > 0:
        # start from the state after `developed` RK4 steps at CFL 1 (past the
        # start-up transient of the impulsive start)
        for _ in range(args.developed):
            rok.rk_step(ctx, yd, dt_unit)
        y0 = yd.cpu().numpy()
        start = 'after %d RK4 steps at CFL 1 (t = %.4g)' % (args.developed, args.developed * dt_unit)
    T = args.horizon * dt_unit * base_cfl
    out = {'study': 'time-to-fixed-L2-error', 'case': prob.name, 'start': start, 'T': T, 'dt_cfl1': dt_unit,
           'methods': {}}

    def integrate(step_fn, dt, cap_s=None):
        n = max(1, int(round(T / dt)))
        h = T / n
        y = rok.state_tensor(y0)
        torch.cuda.synchronize()
        if cap_s is not None:
            # estimate the run from one step; skip runs that would exceed the cap
            t1 = time.perf_counter()
            step_fn(rok.state_tensor(y0), h)
            torch.cuda.synchronize()
            est = (time.perf_counter() - t1) * n
            if est > cap_s:
                raise TimeoutError('estimated %.0f s for %d steps' % (est, n))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record()
        infos = []
        for _ in range(n):
            r = step_fn(y, h)
            if r is not None:
                infos.append(r)
        e1.record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        return y, n, h, e0.elapsed_time(e1) / 1e3, wall, infos

    ref_dt = min(min(cfls), min(cfl_rk)) * dt_unit / args.ref_factor
    yref, nref, _, tref, _, _ = integrate(lambda y, h: rok.rk_step(ctx, y, h), ref_dt)
    yref_h = yref.cpu().numpy()
    out['reference'] = {'method': 'RK4', 'steps': nref, 'gpu_s': tref}
    nrm = float(np.linalg.norm(yref_h))

    def record(name, y, n, h, gs, ws, extra=None):
        e = float(np.linalg.norm(y.cpu().numpy() - yref_h))
        d = {'steps': n, 'h': h, 'gpu_s': gs, 'wall_s': ws, 'abs_err': e, 'rel_err': e / nrm}
        if extra:
            d.update(extra)
        out['methods'].setdefault(name, []).append(d)

    for c in cfls:
        try:
            y, n, h, gs, ws, _ = integrate(lambda y, h: rok.rok_step(ctx, y, h, krylov, info=True), c * dt_unit)
            record('ROK4', y, n, h, gs, ws, {'cfl': c, 'M': krylov})
        except rok.RokError as err:
            out['methods'].setdefault('ROK4', []).append({'cfl': c, 'failed': str(err)})
    for c in cfl_rk:
        y, n, h, gs, ws, _ = integrate(lambda y, h: rok.rk_step(ctx, y, h), c * dt_unit)
        record('RK4', y, n, h, gs, ws, {'cfl': c})
    for c in cfls:
        try:
            y, n, h, gs, ws, infos = integrate(lambda y, h: rok.esdirk_step(ctx, y, h, info=True), c * dt_unit,
                                               cap_s=args.esdirk_cap)
            record('ESDIRK3', y, n, h, gs, ws, {'cfl': c, 'gmres_iters': sum(i['gmres_iters'] for i in infos),
                                                'newton_iters': sum(i['newton_iters'] for i in infos)})
        except (rok.RokError, TimeoutError) as err:
            out['methods'].setdefault('ESDIRK3', []).append({'cfl': c, 'failed': str(err)})
    for name, meth in (('ROS4', rok.ROK_ROS_ROS4), ('ROW', rok.ROK_ROS_ROW)):
        for c in cfls:
            try:
                y, n, h, gs, ws, infos = integrate(lambda y, h: rok.ros_step(ctx, y, h, method=meth, info=True),
                                                   c * dt_unit, cap_s=args.esdirk_cap)
                record(name, y, n, h, gs, ws, {'cfl': c, 'gmres_iters': sum(i['gmres_iters'] for i in infos)})
            except (rok.RokError, TimeoutError) as err:
                out['methods'].setdefault(name, []).append({'cfl': c, 'failed': str(err)})
    out['time_to_error'] = {}
    for tgt in (1e-4, 1e-6, 1e-8, 1e-10):
        row = {}
        for m, pts in out['methods'].items():
            row[m] = _interp_time([(p['rel_err'], p['gpu_s']) for p in pts if 'rel_err' in p], tgt)
        out['time_to_error']['%g' % tgt] = row
    print(json.dumps(out))


def run_stability(args):
    """Largest stable CFL of ROK4 on the cylinder O-grid for several Krylov
    dimensions (the paper: ROK is conditionally stable, Sec. 3.1 table of
    methods; its Krylov size study, Sec. 4.4).  For each M, CFL numbers are
    tried in increasing order over the same physical time T = horizon x the
    CFL-1 step; a CFL counts as stable when every step stays finite and the
    state norm stays within 2x its start.  The scan per M stops at the first
    unstable CFL.  Start: the impulsive free stream, or with --developed K a
    state after K RK4 steps at CFL 1 from it (the start-up transient past)."""
    import torch

    from paper_1607_06834_gb300 import rok
    from paper_1607_06834_gb300 import workloads as W
    torch.cuda.set_device(0)
    prob, y0, _ = W.cylinder_ogrid(256, 512)
    ms = [int(x) for x in args.krylov_list.split(',')]
    cfls = [float(x) for x in (args.cfls or '1,2,3,5,7,10,15,20,30,50,100,300,1000').split(',')]
    ctx = rok.rok_init(prob, krylov_max=max(ms))
    y = rok.state_tensor(y0)
    dt1 = rok.rok_dt_from_cfl(ctx, y, 1.0)
    start = 'impulsive'
    if args.developed > 0:
        for _ in range(args.developed):
            rok.rk_step(ctx, y, dt1)
        torch.cuda.synchronize()
        start = 'after %d RK4 steps at CFL 1 (t = %.4g)' % (args.developed, args.developed * dt1)
    ys = y.clone()
    n0 = float(ys.norm())
    T = args.horizon * dt1
    out = {'study': 'stable-cfl-vs-krylov-dimension', 'case': prob.name, 'start': start, 'T': T, 'dt_cfl1': dt1,
           'scan': {}}
    for M in ms:
        rows, largest = [], None
        for c in cfls:
            n = max(1, int(round(T / (c * dt1))))
            h = T / n
            yy = ys.clone()
            ok, why = True, ''
            t0 = time.perf_counter()
            for k in range(n):
                try:
                    rok.rok_step(ctx, yy, h, M, info=(k % 10 == 9 or k == n - 1))
                except rok.RokError as e:
                    ok, why = False, 'step %d: %s' % (k + 1, rok.rok_status_string(e.status))
                    break
            if ok:
                nr = float(yy.norm())
                if not (nr <= 2.0 * n0):
                    ok, why = False, 'norm grew %.3g x' % (nr / n0)
            rows.append({'cfl': c, 'steps': n, 'stable': ok, 'why': why, 'wall_s': round(time.perf_counter() - t0, 2)})
            if not ok:
                break
            largest = c
        out['scan'][str(M)] = {'largest_stable_cfl': largest, 'runs': rows}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--study', default=None, choices=[None, 'tte', 'wp', 'stability'])
    ap.add_argument('--krylov-list', default='4,8,12,20,30', help='Krylov dimensions (stability study)')
    ap.add_argument('--developed', type=int, default=0, help='RK4 steps before the stability scan')
    ap.add_argument('--case', default='tgv', choices=['tgv', 'cylinder'])
    ap.add_argument('--horizon', type=float, default=50.0, help='T in units of the base-CFL step')
    ap.add_argument('--ref-factor', type=float, default=16.0)
    ap.add_argument('--esdirk-cap', type=float, default=150.0, help='skip ESDIRK runs estimated above this (s)')
    ap.add_argument('--cfls', default=None, help='comma-separated ROK/ESDIRK CFL numbers (study)')
    ap.add_argument('--mode', default='step', choices=['step', 'stencil', 'batch', 'grad', 'configs'])
    ap.add_argument('--n', type=int, default=N_GRID)
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=30)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--rounding', default='fast', choices=['fast', 'strict'])
    ap.add_argument('--graph', type=int, default=1, help='replay each ROK4 step as a captured CUDA graph (0: launch kernel by kernel)')
    ap.add_argument('--forms', type=int, default=1, help='also time the mixed-precision form')
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.mode == 'stencil':
        run_stencil_only(args)
        return
    if args.mode == 'batch':
        run_batch(args)
        return
    if args.mode == 'grad':
        run_grad(args)
        return
    if args.mode == 'configs':
        run_configs(args)
        return
    if args.study == 'tte':
        run_tte(args)
        return
    if args.study == 'wp':
        run_wp(args)
        return
    if args.study == 'stability':
        run_stability(args)
        return
    out = run_reference(args) if args.impl == 'reference' else run_ours(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == '__main__':
    main()
