"""Benchmark: constrained Brownian mid-point steps per second of the stresslet PSE method.

Workload (synthetic, seeded): N = 1,048,576 hard spheres of radius a = 1 at
volume fraction phi = 0.3 by random sequential addition in a cubic periodic
box L = (4 pi N / (3 phi))^{1/3}; eta = kT = 1; PSE tolerance eps = 1e-3;
mixed precision (FP32 grids, FFTs, pair sums and vectors; FP64 Krylov and
Lanczos scalars).  One step = one full constrained mid-point step: Brownian
slip by Lanczos + wave-space noise, mid-point move, GMRES stresslet solve,
final product and position update (no work skipped).  Inputs (grids 0.9 GB,
Krylov basis, particle data) exceed the 129 MB L2 between steps.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the host cores instead (a bounded sample of the same workload).  The default
line also carries a short serving measurement (`serving`: Poisson arrivals of
mobility / sample / step requests through the serving loop).

Other workloads (their own JSON line each):
  --workload batch256  256 independent suspensions (N log-uniform in [500, 20000],
                       phi uniform in [0.05, 0.45]) advanced by one batched
                       constrained step per iteration;
  --workload serve     the serving stream: Poisson arrivals of mobility / sample /
                       step requests, N log-uniform in [1000, 200000], phi in
                       {0.1, 0.25, 0.4}, eps in {1e-3, 1e-4}, state resident,
                       admission by device-memory footprint; the arrival rate is
                       swept until the completion rate saturates.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = 'Brownian steps/s, N=1M phi=0.3 eps=1e-3, mixed vs FP64; served p50/p99 latency'
FP32_PEAK_TFLOPS_AT_MAX = 152 * 128 * 2 * 2.070e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz
SMEM_PEAK_GBS_AT_MAX = 152 * 128 * 2.070e9 / 1e9          # 152 SMs x 128 B/clk shared-memory bandwidth x 2.07 GHz


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=10)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--N', type=int, default=1048576)
    ap.add_argument('--phi', type=float, default=0.3)
    ap.add_argument('--tol', type=float, default=1e-3)
    ap.add_argument('--xi', type=float, default=0.5)
    ap.add_argument('--dt', type=float, default=1e-3)
    ap.add_argument('--fp64-steps', type=int, default=2)
    ap.add_argument('--e2e-steps', type=int, default=3)
    ap.add_argument('--cpu-N', type=int, default=1000)
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--workload', default='step', choices=['step', 'batch256', 'serve'])
    ap.add_argument('--serve-seconds', type=float, default=12.0, help='per arrival rate')
    ap.add_argument('--serve-slots', type=int, default=4)
    ap.add_argument('--serve-pool', type=int, default=8, help='distinct resident suspensions')
    ap.add_argument('--serve-rates', default='', help='comma-separated arrival rates (req/s)')
    ap.add_argument('--no-serving', action='store_true', help='omit the serving block of the default line')
    ap.add_argument('--compare-sequential', action='store_true', help='batch256: also time one handle per suspension')
    ap.add_argument('--graph', type=int, default=1, help='1: time the graph-captured step (default)')
    ap.add_argument('--profile-steps', type=int, default=3, help='host-launched steps timed per stage')
    ap.add_argument('--no-accuracy', action='store_true', help='omit the mixed-vs-FP64 error per output')
    return ap.parse_args()


def max_over_ranks(x, pg, device):
    """Largest x over the ranks (x itself on one process)."""
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def replica_rate(world, steps, elapsed_max):
    """Whole-job rate of independent replicas: the steps of all ranks over the slowest rank's time."""
    return world * steps / elapsed_max


def dist_setup(args):
    world = int(os.environ.get('WORLD_SIZE', '1'))
    rank = int(os.environ.get('RANK', '0'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        os.environ.setdefault('MASTER_ADDR', '127.0.0.1')
        backend = 'nccl' if args.impl == 'ours' and torch.cuda.is_available() else 'gloo'
        if backend == 'nccl':
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    Q = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
         'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
         'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(['nvidia-smi', '-i', str(self.index), '--query-gpu=' + self.Q,
                                          '--format=csv,noheader,nounits', '-lms', '200'],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {'sm_mhz': None, 'sm_max_mhz': None, 'reasons': ['nvidia-smi unavailable']}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        for ln in self.lines:
            f = [x.strip() for x in ln.split(',')]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith('active'):
                    reasons.add(nm)
        return {'sm_mhz': float(np.median(sm)) if sm else None, 'sm_max_mhz': smax, 'reasons': sorted(reasons),
                'samples': len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, 'MEASURED_PEAKS.json')) as f:
            return json.load(f)
    except OSError:
        return {}


def oracle_step_rate(N_s, phi, tol, xi, dt, seed=1):
    """Seconds for one oracle constrained step at N_s particles (same phi, tol, xi)."""
    import pse_inputs
    from oracle import params, philox, pse as opse
    pos, L = pse_inputs.rsa_positions(N_s, phi, seed=seed)
    p = params.choose(N_s, L, 1.0, 1.0, 1.0, xi, tol)
    w1 = philox.lanczos_noise(seed, 0, N_s)
    w2 = philox.wave_noise(seed, 0, p.Ng)
    t0 = time.perf_counter()
    opse.constrained_step(pos, None, dt, w1, w2, p)
    return time.perf_counter() - t0


def cpu_baseline(args):
    dt_s = oracle_step_rate(args.cpu_N, args.phi, args.tol, args.xi, args.dt)
    value = (args.cpu_N / args.N) / dt_s          # linear-in-N scaling (PTPS constant, Sec. 4)
    return {'value': value, 'unit': 'steps/s', 'cores': 1, 'kind': 'oracle',
            'sample': 'one FP64 oracle constrained step at N=%d (phi=%g, eps=%g, xi=%g) took %.2f s; '
                      'scaled to N=%d by particle count' % (args.cpu_N, args.phi, args.tol, args.xi, dt_s, args.N)}


def run_reference(args, world, rank, pg):
    if rank != 0:
        return
    steps = max(1, args.steps)
    times = []
    for k in range(args.warmup + steps):
        t = oracle_step_rate(args.cpu_N, args.phi, args.tol, args.xi, args.dt, seed=1 + k)
        if k >= args.warmup:
            times.append(t)
    per = float(np.mean(times))
    value = (args.cpu_N / args.N) / per
    line = {'metric': METRIC, 'value': value, 'unit': 'steps/s', 'n_gpus': args.gpus, 'steps': steps,
            'warmup': args.warmup, 'ms_per_step': 1000.0 / value, 'higher_is_better': True, 'scaling': 'weak',
            'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic', 'impl': 'reference',
            'config': {'workload': 'N=%d hard spheres phi=%g eps=%g constrained mid-point step' % (args.N, args.phi, args.tol),
                       'N': args.N, 'phi': args.phi, 'tol': args.tol, 'xi': args.xi},
            'cpu_baseline': {'value': value, 'unit': 'steps/s', 'cores': 1, 'kind': 'oracle',
                             'sample': 'FP64 oracle constrained steps at N=%d, scaled to N=%d by particle count'
                                       % (args.cpu_N, args.N)},
            'e2e': {'value': value, 'unit': 'steps/s', 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0}}
    print(json.dumps(line), flush=True)


def accuracy_vs_fp64(pkg, torch, dev, args, pos_np, L, h64):
    """Relative L2 error of the mixed form against the all-FP64 form on the same
    seeded inputs and the same external noise: mobility U and E, Brownian U^B and
    E^B, one constrained step's displacement and stresslets; GMRES residuals."""
    hm = pkg.PSE(args.N, L, xi=args.xi, tol=args.tol, precision='mixed')
    N, Ng = args.N, hm.info['Ng']
    g = torch.Generator(device=dev).manual_seed(3)
    F = torch.randn((N, 3), generator=g, device=dev, dtype=torch.float64)
    S = torch.randn((N, 5), generator=g, device=dev, dtype=torch.float64)
    w1 = torch.randn((N, 8), generator=g, device=dev, dtype=torch.float64)
    w2 = torch.randn((6 * Ng * Ng * (Ng // 2 + 1),), generator=g, device=dev, dtype=torch.float64)
    x = torch.tensor(pos_np, device=dev, dtype=torch.float64)

    def rel(a, b):
        return float(torch.linalg.norm(a.double() - b) / torch.linalg.norm(b))
    out = {}
    U64, E64 = h64.mobility(x, F, S)
    U32, E32 = hm.mobility(x, F.float(), S.float())
    out['mobility_U'], out['mobility_E'] = rel(U32, U64), rel(E32, E64)
    U64, E64, _ = h64.brownian(x, args.dt, w1=w1, w2=w2)
    U32, E32, _ = hm.brownian(x, args.dt, w1=w1.float(), w2=w2.float())
    out['brownian_U'], out['brownian_E'] = rel(U32, U64), rel(E32, E64)
    x64, x32 = x.clone(), x.clone()
    S64, st64 = h64.step(x64, args.dt, w1=w1, w2=w2, want_S=True)
    S32, st32 = hm.step(x32, args.dt, w1=w1.float(), w2=w2.float(), want_S=True)
    d64 = x64 - x
    d32 = x32 - x
    d64 -= L * torch.round(d64 / L)
    d32 -= L * torch.round(d32 / L)
    out['step_displacement'] = rel(d32, d64)
    out['step_stresslet'] = rel(S32, S64)
    out['gmres_relres'] = {'mixed': st32['krylov_relres'], 'fp64': st64['krylov_relres'],
                           'iterations_mixed': st32['krylov_iters'], 'iterations_fp64': st64['krylov_iters']}
    out['note'] = 'relative L2 over all particles, N=%d, same positions, moments and external noise' % N
    hm.close()
    return out


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of the
# first launch of each kernel on the benchmark workload (N = 1048576, phi = 0.3, eps = 1e-3,
# xi = 0.5, N_g = 256, P = 6); reported only for that workload, and to be retaken whenever the
# kernel changes: 5-component spread and interpolation (16^3 tiles), full-product pair sum.
NCU_TRAFFIC_WORKLOAD = (1048576, 0.3, 1e-3, 0.5, 256, 6)
NCU_TRAFFIC = {'spread': 351.2e6, 'interp': 435.1e6, 'real': 1900.0e6}


def real_flops_per_pair():
    # FP32 operations of the pair kernel per neighbour, counted from its formulas (FMA = 2):
    # separation and 1/r 10; table interpolation 2 + 3 per function (7, 3 or 4 functions);
    # S r^ 26; r^.S r^ 5; r^.F 5; U terms 22 (13 without F); E terms 87 (78 without F, two
    # Y-basis products of 24 each).  Full 8->8 product (Lanczos), S->E (GMRES), [F;S]->U and
    # S->U (final velocity with and without an external force).
    return {'full': 178, 'se': 130, 'fsu': 82, 'su': 68}


def run_ours(args, world, rank, local, pg):
    import torch
    import pse_inputs
    import paper_1709_06946_gb300 as pkg

    pkg.load()
    dev = torch.device('cuda', local)
    torch.cuda.set_device(dev)
    pos_np, L = pse_inputs.rsa_positions(args.N, args.phi, seed=1 + rank)
    h = pkg.PSE(args.N, L, xi=args.xi, tol=args.tol, precision='mixed', use_graph=args.graph)
    inf = h.info
    x = torch.tensor(pos_np, device=dev, dtype=torch.float64)
    stream = torch.cuda.current_stream(dev)
    for k in range(args.warmup):
        h.step(x, args.dt, seed=1234 + rank, step=k)
    torch.cuda.synchronize(dev)
    graph_used = h.graph_ready()
    if pg is not None:
        pg.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize(dev)
    if pg is not None:
        pg.barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    lat = []
    iters = []
    ev0.record(stream)
    for k in range(args.steps):
        t0 = time.perf_counter()
        _, st = h.step(x, args.dt, seed=1234 + rank, step=args.warmup + k)
        lat.append((time.perf_counter() - t0) * 1000.0)
        iters.append((st['lanczos_iters'], st['krylov_iters'], st['neighbor_pairs']))
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if pg is not None:
        pg.barrier()
    elapsed = max_over_ranks(ev0.elapsed_time(ev1) / 1000.0, pg, dev)
    clk = clocks.stop()
    value = replica_rate(world, args.steps, elapsed)

    # per-stage device times: the same steps launched from the host with stage events
    # (a captured graph cannot hold the events); also gives the kernel count per step
    KP = max(1, args.profile_steps)
    h.set_profiling(True)
    pe0 = torch.cuda.Event(enable_timing=True)
    pe1 = torch.cuda.Event(enable_timing=True)
    piters = []
    pe0.record(stream)
    for k in range(KP):
        _, st = h.step(x, args.dt, seed=1234 + rank, step=args.warmup + args.steps + k)
        piters.append((st['lanczos_iters'], st['krylov_iters'], st['neighbor_pairs']))
    pe1.record(stream)
    torch.cuda.synchronize(dev)
    prof_elapsed = pe0.elapsed_time(pe1) / 1000.0
    prof = h.profile()
    h.set_profiling(False)

    # roofline of the dominant stage (device time per stage from CUDA events on the launching stream)
    peaks = measured_peaks()
    stage_ms = prof['ms']
    Li = sum(i[0] for i in piters)
    Ki = sum(i[1] for i in piters)
    npairs = float(np.mean([i[2] for i in piters]))
    Ng, N = inf['Ng'], args.N
    n3 = Ng ** 3
    nkh = Ng * Ng * (Ng // 2 + 1)
    K = KP
    # per step: GMRES products (5 -> 5) Ki/K times, one final S -> U product (no external
    # force), one noise pass
    spread_comps = [5] * Ki + [5] * K
    interp_comps = [5] * Ki + [3] * K + [8] * K
    algo = {
        'spread': sum(N * (32 + 4 * c) + c * n3 * 4 for c in spread_comps),
        'interp': sum(c * n3 * 4 + N * (32 + 4 * c) for c in interp_comps),
        'scale': sum((ci + co) * nkh * 8 for ci, co in [(5, 5)] * Ki + [(5, 3)] * K),
        'noise': K * 8 * nkh * 8,
    }
    dom = max(('real', 'spread', 'interp', 'scale', 'noise', 'fft'), key=lambda s: stage_ms[s])
    traffic_ok = (args.N, args.phi, args.tol, args.xi, Ng, inf['P']) == NCU_TRAFFIC_WORKLOAD
    fl = real_flops_per_pair()
    if dom == 'real' or dom == 'fft':
        flops = npairs * (fl['full'] * Li + fl['se'] * Ki + fl['su'] * K)
        achieved = flops / (stage_ms['real'] / 1000.0) / 1e12
        peak = FP32_PEAK_TFLOPS_AT_MAX
        roof = {'bound': 'alu', 'kernel': 'k_real (real-space pair sum)', 'achieved': achieved, 'peak': peak,
                'unit': 'TFLOP/s', 'frac': achieved / peak,
                'traffic': NCU_TRAFFIC['real'] if traffic_ok else None,
                'peak_note': 'derived FP32 peak: 152 SMs x 128 lanes x 2 flop x 2070 MHz',
                'launches': prof['calls']['real'], 'flops_per_pair': fl}
    else:
        hbm = peaks.get('hbm_gbs', 6800.0)
        achieved = algo[dom] / (stage_ms[dom] / 1000.0) / 1e9
        roof = {'bound': 'hbm', 'kernel': dom, 'achieved': achieved, 'peak': hbm, 'unit': 'GB/s',
                'frac': achieved / hbm, 'traffic': NCU_TRAFFIC.get(dom) if traffic_ok else None,
                'traffic_note': 'DRAM bytes per launch of the 5-component (GMRES) launch, one ncu capture',
                'peak_note': 'measured hbm_gbs (MEASURED_PEAKS.json)'}
    # the pair sum's FP32 rate is reported beside the dominant stage's roofline in any case
    real_flops = npairs * (fl['full'] * Li + fl['se'] * Ki + fl['su'] * K)
    real_rate = real_flops / (stage_ms['real'] / 1000.0) / 1e12 if stage_ms['real'] > 0 else None
    roof_real = {'bound': 'alu', 'kernel': 'k_real (real-space pair sum)', 'achieved': real_rate,
                 'peak': FP32_PEAK_TFLOPS_AT_MAX, 'unit': 'TFLOP/s',
                 'frac': real_rate / FP32_PEAK_TFLOPS_AT_MAX if real_rate else None,
                 'traffic': NCU_TRAFFIC['real'] if traffic_ok else None,
                 'traffic_note': 'DRAM bytes per full-product launch (neighbour records, 16 B per ordered pair)',
                 'peak_note': 'derived FP32 peak: 152 SMs x 128 lanes x 2 flop x 2070 MHz',
                 'flops_per_pair': fl}
    # the ceiling that binds spreading and interpolation: each particle's P^3 footprint x C
    # components in the shared tile, read and written (spread) or read (interpolation)
    P3 = inf['P'] ** 3
    smem_algo = {'spread': sum(N * P3 * c * 4 * 2 for c in spread_comps),
                 'interp': sum(N * P3 * c * 4 for c in interp_comps)}
    smem_rates = {k: {'GB/s': smem_algo[k] / (stage_ms[k] / 1000.0) / 1e9 if stage_ms[k] > 0 else None,
                      'peak_GB/s': SMEM_PEAK_GBS_AT_MAX,
                      'frac': (smem_algo[k] / (stage_ms[k] / 1000.0) / 1e9) / SMEM_PEAK_GBS_AT_MAX
                      if stage_ms[k] > 0 else None,
                      'note': 'shared-memory bytes of the footprint updates (N P^3 C x 4 B, x2 when read and '
                              'written) against the derived 152 SMs x 128 B/clk x 2070 MHz'} for k in smem_algo}
    wave_rates = {k: {'GB/s': algo[k] / (stage_ms[k] / 1000.0) / 1e9 if stage_ms[k] > 0 else None,
                      'frac_of_measured_hbm': (algo[k] / (stage_ms[k] / 1000.0) / 1e9) / peaks.get('hbm_gbs', 6800.0)
                      if stage_ms[k] > 0 else None} for k in algo}

    result = {'metric': METRIC, 'value': value, 'unit': 'steps/s', 'n_gpus': world, 'steps': args.steps,
              'warmup': args.warmup, 'ms_per_step': 1000.0 * elapsed / args.steps, 'higher_is_better': True,
              'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f32', 'data': 'synthetic',
              'config': {'workload': 'N=%d hard spheres (RSA) phi=%g eps=%g constrained mid-point step, mixed '
                                     'precision' % (args.N, args.phi, args.tol),
                         'N': args.N, 'phi': args.phi, 'tol': args.tol, 'xi': args.xi, 'L': L,
                         'Ng': Ng, 'P': inf['P'], 'rcut': inf['rcut'], 'tile': list(inf['tile']),
                         'precision': 'mixed (FP32 grids/pairs/vectors, FP64 Krylov scalars)',
                         'parallelism': 'replicas' if world > 1 else 'single GPU',
                         'l2': 'inputs larger than L2 (FFT grids %.2f GB)' % (8 * n3 * 4 * 2 / 1e9)},
              'ptps': value * args.N / world,
              'iterations': {'lanczos_mean': float(np.mean([i[0] for i in iters])),
                             'krylov_mean': float(np.mean([i[1] for i in iters])),
                             'neighbor_pairs': float(np.mean([i[2] for i in iters]))},
              'latency_ms': {'p50': float(np.percentile(lat, 50)), 'p99': float(np.percentile(lat, 99)),
                             'note': 'per constrained-step call (single stream, no serving loop)'},
              'execution': {'graph': bool(graph_used[0]), 'graph_error': graph_used[1],
                            'host_launched_steps_per_s': KP / prof_elapsed,
                            'note': 'value: steps captured as one CUDA graph (Krylov loops as conditional while '
                                    'nodes); stage times and roofline: the same steps launched from the host with '
                                    'stage events'},
              'stage_ms_per_step': {k: v / K for k, v in stage_ms.items()},
              'wave_stage_hbm': wave_rates, 'wave_stage_smem': smem_rates,
              'roofline': roof, 'roofline_pair_sum': roof_real, 'clocks': clk,
              'gpu_launches': int(round(prof['launches'] / K * args.steps)),
              'gpu_launches_note': 'kernels of this library per step (counted on the host-launched path) x timed '
                                   'steps; cuFFT kernels excluded',
              'fft_execs': int(round(prof['fft_execs'] / K * args.steps))}

    # end-to-end through the C ABI with host arrays (H2D positions in, D2H positions out, every step)
    if args.e2e_steps > 0:
        pos_host = np.ascontiguousarray(pos_np.copy())
        h.step(pos_host, args.dt, seed=7, step=0)
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            h.step(pos_host, args.dt, seed=7, step=1 + k)
        e2e_t = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, pg, dev)
        result['e2e'] = {'value': world / e2e_t, 'unit': 'steps/s', 'h2d_bytes_per_step': 24 * args.N,
                         'd2h_bytes_per_step': 24 * args.N}
    h.close()

    # all-FP64 form on the same workload (comparison for the mixed-precision speed-up)
    if args.fp64_steps > 0:
        h64 = pkg.PSE(args.N, L, xi=args.xi, tol=args.tol, precision='fp64')
        x64 = torch.tensor(pos_np, device=dev, dtype=torch.float64)
        h64.step(x64, args.dt, seed=99, step=0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for k in range(args.fp64_steps):
            h64.step(x64, args.dt, seed=99, step=1 + k)
        torch.cuda.synchronize(dev)
        t64 = (time.perf_counter() - t0) / args.fp64_steps
        result['fp64'] = {'steps_per_s': 1.0 / t64, 'ms_per_step': 1000.0 * t64,
                          'mixed_speedup': t64 / (elapsed / args.steps)}
        if not args.no_accuracy:
            result['accuracy'] = accuracy_vs_fp64(pkg, torch, dev, args, pos_np, L, h64)
        h64.close()
    if rank == 0 and world == 1 and not args.no_serving:
        res, desc = serving_measure(pkg, args, [8.0], 6, 200000, 10.0)
        r = res[0]
        result['serving'] = {'p50_ms': r['p50_ms'], 'p99_ms': r['p99_ms'], 'req_per_s': r['req_per_s'],
                             'offered_rate': r['offered_rate'], 'requests': r['requests'],
                             'peak_running': r['peak_running'], 'stream': desc}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result['cpu_baseline'] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(result), flush=True)


# ----------------------------------------------------------------------------- serving
def serve_pool(M, seed, nmax=200000):
    """M distinct suspensions of the serving stream (N log-uniform in [1000, nmax],
    phi in {0.1, 0.25, 0.4}, eps in {1e-3, 1e-4}), with positions and moments."""
    import pse_inputs
    rng = np.random.default_rng(seed)
    pool = []
    for k in range(M):
        N = int(round(math.exp(rng.uniform(math.log(1000), math.log(nmax)))))
        phi = float(rng.choice([0.1, 0.25, 0.4]))
        tol = float(rng.choice([1e-3, 1e-4]))
        pos, L = pse_inputs.hard_sphere_positions(N, phi, seed=1000 + k)
        F, S = pse_inputs.moments(N, seed=2000 + k)
        pool.append({'N': N, 'phi': phi, 'tol': tol, 'L': L, 'pos': pos, 'F': F.astype(np.float32),
                     'S': S.astype(np.float32)})
    return pool


def serve_at_rate(pkg, srv, pool, rate, seconds, xi, dt, seed):
    """Poisson arrivals at `rate` req/s for `seconds`; kinds and suspensions uniform."""
    rng = np.random.default_rng(seed)
    kinds = ['mobility', 'sample', 'step']
    srv.reset_stats()
    tickets = []
    t_end = time.perf_counter() + seconds
    t_next = time.perf_counter()
    n = 0
    while True:
        t_next += rng.exponential(1.0 / rate)
        if t_next > t_end:
            break
        d = t_next - time.perf_counter()
        if d > 0:
            time.sleep(d)
        q = pool[int(rng.integers(len(pool)))]
        kind = kinds[int(rng.integers(3))]
        if kind == 'mobility':
            t, _ = srv.submit('mobility', q['pos'], q['L'], xi=xi, tol=q['tol'], F=q['F'], S=q['S'])
        elif kind == 'sample':
            t, _ = srv.submit('sample', q['pos'], q['L'], xi=xi, tol=q['tol'], dt=dt, seed=n)
        else:
            t, _ = srv.submit('step', q['pos'].copy(), q['L'], xi=xi, tol=q['tol'], dt=dt, seed=n, counter=n)
        tickets.append(t)
        n += 1
    for t in tickets:
        srv.wait(t)
    st = srv.stats()
    return {'offered_rate': rate, 'arrival_rate': len(tickets) / seconds, 'requests': len(tickets),
            'req_per_s': st['requests_per_s'],
            'p50_ms': st['p50_ms'], 'p99_ms': st['p99_ms'], 'wait_p50_ms': st['wait_p50_ms'],
            'wait_p99_ms': st['wait_p99_ms'], 'service_p50_ms': st['service_p50_ms'],
            'peak_running': st['peak_running'], 'peak_resident_gb': st['peak_resident_bytes'] / 1e9,
            'handles_created': st['handles_created'], 'handles_evicted': st['handles_evicted']}


def serving_measure(pkg, args, rates, pool_size, nmax, seconds):
    pool = serve_pool(pool_size, seed=77, nmax=nmax)
    budget = int(0.8 * 280e9)
    srv = pkg.Server(slots=args.serve_slots, budget_bytes=budget)
    # make every suspension resident once (tables, plans, grids); not timed
    warm = [srv.submit('mobility', q['pos'], q['L'], xi=args.xi, tol=q['tol'], F=q['F'], S=q['S'])[0] for q in pool]
    for t in warm:
        srv.wait(t)
    out = []
    for k, r in enumerate(rates):
        res = serve_at_rate(pkg, srv, pool, r, seconds, args.xi, args.dt, seed=k)
        out.append(res)
        if res['req_per_s'] < 0.85 * res['arrival_rate']:   # saturated: completions no longer track arrivals
            break
    srv.close()
    desc = ('%d resident suspensions, N log-uniform in [1000, %d] (N = %s), phi in {0.1, 0.25, 0.4}, '
            'eps in {1e-3, 1e-4}, kinds mobility/sample/step uniform, %d slots, budget %.0f GB'
            % (pool_size, nmax, sorted(q['N'] for q in pool), args.serve_slots, budget / 1e9))
    return out, desc


def run_serve(args):
    import paper_1709_06946_gb300 as pkg
    pkg.load()
    rates = ([float(r) for r in args.serve_rates.split(',')] if args.serve_rates
             else [2, 5, 10, 20, 40, 80, 160, 320, 640, 1280])
    clocks = ClockSampler(0)
    clocks.start()
    res, desc = serving_measure(pkg, args, rates, max(args.serve_pool, 1), 200000, args.serve_seconds)
    clk = clocks.stop()
    # the highest arrival rate the loop kept up with (completions tracking arrivals), its latency,
    # and the completion rate once saturated
    kept = [r for r in res if r['req_per_s'] >= 0.85 * r['arrival_rate']] or res[:1]
    best = max(kept, key=lambda r: r['req_per_s'])
    line = {'metric': 'served requests/s and p50/p99 latency (mobility/sample/step stream)',
            'value': best['req_per_s'], 'unit': 'requests/s', 'n_gpus': 1, 'steps': len(res), 'warmup': 1,
            'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f32', 'data': 'synthetic',
            'config': {'workload': 'serving stream: ' + desc, 'seconds_per_rate': args.serve_seconds},
            'p50_ms': best['p50_ms'], 'p99_ms': best['p99_ms'],
            'saturated_req_per_s': max(r['req_per_s'] for r in res), 'sweep': res, 'clocks': clk}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- batch of suspensions
def batch_suspensions(n, seed):
    import pse_inputs
    rng = np.random.default_rng(seed)
    Ns, phis, pos, Ls = [], [], [], []
    for k in range(n):
        N = int(round(math.exp(rng.uniform(math.log(500), math.log(20000)))))
        phi = float(rng.uniform(0.05, 0.45))
        x, L = pse_inputs.hard_sphere_positions(N, phi, seed=5000 + k)
        Ns.append(N)
        phis.append(phi)
        pos.append(x)
        Ls.append(L)
    return Ns, phis, pos, Ls


def run_batch(args):
    import torch
    import paper_1709_06946_gb300 as pkg
    pkg.load()
    dev = torch.device('cuda', 0)
    nsys = 256
    Ns, phis, pos, Ls = batch_suspensions(nsys, seed=4)
    h = pkg.PSE(Ns, Ls, xi=args.xi, tol=args.tol, precision='mixed', grid_ladder=1)
    x = torch.tensor(np.concatenate(pos), device=dev, dtype=torch.float64)
    stream = torch.cuda.current_stream(dev)
    for k in range(args.warmup):
        h.step(x, args.dt, seed=11, step=k)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(0)
    clocks.start()
    h.set_profiling(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    iters = []
    ev0.record(stream)
    for k in range(args.steps):
        _, st = h.step(x, args.dt, seed=11, step=args.warmup + k)
        iters.append([(h.system_stats(s)['lanczos_iters'], h.system_stats(s)['krylov_iters']) for s in range(nsys)])
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    elapsed = ev0.elapsed_time(ev1) / 1000.0
    clk = clocks.stop()
    prof = h.profile()
    grids = sorted({h.system_info(s)['Ng'] for s in range(nsys)})
    it = np.array(iters)
    value = args.steps / elapsed
    line = {'metric': 'batched constrained steps/s (256 suspensions, one handle)', 'value': value,
            'unit': 'batch steps/s', 'n_gpus': 1, 'steps': args.steps, 'warmup': args.warmup,
            'ms_per_step': 1000.0 * elapsed / args.steps, 'higher_is_better': True, 'scaling': 'weak',
            'vs_baseline': None, 'dtype': 'f32', 'data': 'synthetic',
            'config': {'workload': '256 suspensions, N log-uniform in [500, 20000] (total %d), phi uniform in '
                                   '[0.05, 0.45], eps=%g, xi=%g, grids rounded to 2^i 3^j (%d FFT groups)'
                                   % (sum(Ns), args.tol, args.xi, len(grids)),
                       'total_N': int(sum(Ns)), 'grids': grids},
            'suspension_steps_per_s': nsys * value, 'ptps': sum(Ns) * value,
            'iterations': {'lanczos_min': int(it[..., 0].min()), 'lanczos_max': int(it[..., 0].max()),
                           'krylov_min': int(it[..., 1].min()), 'krylov_max': int(it[..., 1].max())},
            'stage_ms_per_step': {k: v / args.steps for k, v in prof['ms'].items()},
            'gpu_launches_per_step': prof['launches'] / args.steps, 'fft_execs_per_step': prof['fft_execs'] / args.steps,
            'clocks': clk}
    h.set_profiling(False)
    h.close()
    if args.compare_sequential:
        hs = [pkg.PSE(Ns[s], Ls[s], xi=args.xi, tol=args.tol, precision='mixed') for s in range(nsys)]
        xs = [torch.tensor(pos[s], device=dev, dtype=torch.float64) for s in range(nsys)]
        for s in range(nsys):
            hs[s].step(xs[s], args.dt, seed=11, step=0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for s in range(nsys):
            hs[s].step(xs[s], args.dt, seed=11, step=1)
        torch.cuda.synchronize(dev)
        tseq = time.perf_counter() - t0
        line['sequential_handles'] = {'s_per_round': tseq, 'batch_speedup': tseq / (elapsed / args.steps)}
        for hh in hs:
            hh.close()
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload != 'step':
        if args.impl == 'reference':
            print(json.dumps({'impl': 'reference', 'unavailable': 'the oracle arm covers the N=1M step workload only'}))
            return
        run_batch(args) if args.workload == 'batch256' else run_serve(args)
        return
    world, rank, local, pg = dist_setup(args)
    if args.impl == 'reference':
        run_reference(args, world, rank, pg)
    else:
        run_ours(args, world, rank, local, pg)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()


if __name__ == '__main__':
    main()
