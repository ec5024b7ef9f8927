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
    ap.add_argument('--cpu-N', type=int, default=3000, help='oracle size of the cpu_baseline sample')
    ap.add_argument('--ref-N', type=int, default=1000, help='oracle size of each --impl reference step')
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--workload', default='step', choices=['step', 'batch256', 'serve', 'equilibrium'])
    ap.add_argument('--eq-pair-steps', type=int, default=100000, help='equilibrium: spring-pair steps (mid-point)')
    ap.add_argument('--eq-sq-N', type=int, default=64000, help='equilibrium: ideal spheres for S(q)')
    ap.add_argument('--eq-sq-steps', type=int, default=600, help='equilibrium: steps per S(q) run')
    ap.add_argument('--serve-seconds', type=float, default=12.0, help='per arrival rate (--workload serve)')
    ap.add_argument('--serve-seconds-default', type=float, default=4.0,
                    help='per arrival rate of the serving sweep in the default line')
    ap.add_argument('--torque-reps', type=int, default=5,
                    help='timed 11-moment (torque) products on the workload for the default line (0: omit)')
    ap.add_argument('--eps2', type=float, default=1e-4, help='second PSE tolerance of the default line (0: omit)')
    ap.add_argument('--shear-steps', type=int, default=5,
                    help='timed steps on the sheared cell (strain 0.5) for the default line (0: omit)')
    ap.add_argument('--rfd-steps', type=int, default=3, help='timed RFD + Euler-Maruyama steps (0: omit)')
    ap.add_argument('--batch-steps', type=int, default=3,
                    help='timed steps of the 256-suspension block of the default line (0: omit)')
    ap.add_argument('--serve-slots', type=int, default=4)
    ap.add_argument('--serve-pool', type=int, default=8, help='distinct resident suspensions')
    ap.add_argument('--serve-rates', default='', help='comma-separated arrival rates (req/s)')
    ap.add_argument('--no-serving', action='store_true', help='omit the serving block of the default line')
    ap.add_argument('--compare-sequential', action='store_true', help='batch256: also time one handle per suspension')
    ap.add_argument('--graph', type=int, default=1, help='1: time the graph-captured step (default)')
    ap.add_argument('--profile-steps', type=int, default=3, help='host-launched steps timed per stage')
    ap.add_argument('--no-accuracy', action='store_true', help='omit the mixed-vs-FP64 error per output')
    ap.add_argument('--wave-kernel', type=int, default=0,
                    help='16^3-tile kernels: 0 grid-column spreading and shared-tile interpolation; bit 0: '
                         'shared-tile spreading; bit 1: grid-column interpolation')
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


def host_description():
    """Host CPU model, logical cores and the BLAS thread setting the oracle runs with."""
    model = ''
    try:
        with open('/proc/cpuinfo') as f:
            for ln in f:
                k = ln.split(':')[0].strip().lower()
                if k in ('model name', 'cpu model', 'hardware'):
                    model = ln.split(':', 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    blas = {k: os.environ[k] for k in ('OMP_NUM_THREADS', 'OPENBLAS_NUM_THREADS', 'MKL_NUM_THREADS')
            if k in os.environ}
    try:
        from threadpoolctl import threadpool_info
        blas['threadpools'] = [(d.get('internal_api'), d.get('num_threads')) for d in threadpool_info()]
    except ImportError:
        blas.setdefault('threadpools', 'threadpoolctl not installed; library default (all cores)')
    return {'cpu_model': model, 'host_cores': os.cpu_count(), 'blas': blas}


def oracle_step_time(N_s, phi, tol, xi, dt, seed=1):
    """(wall s, CPU s, iterations) of one oracle constrained step at N_s particles (same phi, tol, xi)."""
    import pse_inputs
    from oracle import params, philox, pse as opse
    pos, L = pse_inputs.rsa_positions(N_s, phi, seed=seed)
    p = params.choose(N_s, L, 1.0, 1.0, 1.0, xi, tol)
    w1 = philox.lanczos_noise(seed, 0, N_s)
    w2 = philox.wave_noise(seed, 0, p.Ng)
    c0, t0 = time.process_time(), time.perf_counter()
    _, _, st = opse.constrained_step(pos, None, dt, w1, w2, p)
    wall = time.perf_counter() - t0
    return wall, time.process_time() - c0, st


def cpu_baseline(args):
    """The FP64 oracle's constrained step timed on the host cores at N = cpu_N (a bounded
    sample of the workload), reported in the metric's unit by linear scaling in N
    (PTPS independent of N, Sec. 4) beside the measured figures."""
    wall, cpu, st = oracle_step_time(args.cpu_N, args.phi, args.tol, args.xi, args.dt)
    value = (args.cpu_N / args.N) / wall
    out = {'value': value, 'unit': 'steps/s', 'cores': round(cpu / wall, 2), 'kind': 'oracle',
           'sample': 'one FP64 oracle constrained step at N=%d (phi=%g, eps=%g, xi=%g): %.2f s wall, %.2f s CPU; '
                     'value scaled to N=%d by particle count (PTPS constant in N)'
                     % (args.cpu_N, args.phi, args.tol, args.xi, wall, cpu, args.N),
           'measured': {'N': args.cpu_N, 's_per_step': wall, 'ptps': args.cpu_N / wall,
                        'lanczos_iters': int(st['lanczos_iters']), 'krylov_iters': int(st['krylov_iters'])},
           'cores_note': 'cores = CPU time / wall time of the timed step (threads the oracle actually used)'}
    out.update(host_description())
    return out


def run_reference(args, world, rank, pg):
    """The oracle arm: constrained steps of the FP64 oracle on the host cores at N = cpu_N
    (the largest size whose K + W steps end within a few minutes); the line names the N it
    ran and gives the linear-in-N extrapolation to the benchmark size beside it."""
    if rank != 0:
        return
    steps = max(1, args.steps)
    N_s = args.ref_N
    times, cpus = [], []
    for k in range(args.warmup + steps):
        wall, cpu, _ = oracle_step_time(N_s, args.phi, args.tol, args.xi, args.dt, seed=1 + k)
        if k >= args.warmup:
            times.append(wall)
            cpus.append(cpu)
    per = float(np.mean(times))
    value = 1.0 / per
    cores = round(float(np.sum(cpus) / np.sum(times)), 2)
    line = {'metric': METRIC, 'value': value, 'unit': 'steps/s', 'n_gpus': args.gpus, 'steps': steps,
            'warmup': args.warmup, 'ms_per_step': 1000.0 * per, 'higher_is_better': True, 'scaling': 'weak',
            'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic', 'impl': 'reference',
            'config': {'workload': 'N=%d hard spheres (RSA) phi=%g eps=%g constrained mid-point step, FP64 oracle on '
                                   'the host cores (a bounded sample of the N=%d workload)'
                                   % (N_s, args.phi, args.tol, args.N),
                       'N': N_s, 'phi': args.phi, 'tol': args.tol, 'xi': args.xi},
            'ptps': N_s * value,
            'extrapolated': {'N': args.N, 'steps_per_s': N_s * value / args.N,
                             'basis': 'linear in N (PTPS constant in N, Sec. 4); not measured'},
            'cpu_baseline': {'value': value, 'unit': 'steps/s', 'cores': cores, 'kind': 'oracle',
                             'sample': '%d FP64 oracle constrained steps at N=%d after %d warm-up steps'
                                       % (steps, N_s, args.warmup)},
            'e2e': {'value': value, 'unit': 'steps/s', 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0}}
    line['cpu_baseline'].update(host_description())
    print(json.dumps(line), flush=True)


def accuracy_vs_fp64(pkg, torch, dev, args, pos_np, L, h64):
    """Relative L2 error of the mixed form against the all-FP64 form on the same
    seeded inputs and the same external noise: mobility U and E, Brownian U^B and
    E^B, one constrained step's displacement and stresslets; GMRES residuals."""
    hm = pkg.PSE(args.N, L, xi=args.xi, tol=args.tol, precision='mixed', wave_kernel=args.wave_kernel)
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


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of kernel instances on the
# benchmark workload (N = 1048576, phi = 0.3, eps = 1e-3, xi = 0.5, N_g = 256, P = 6): ncu captures of
# the N = 524288 case of the same workload (profiles/dram_bytes_N524288_phi0.3_eps1e-3.md), scaled to a
# full launch by the ordered pairs (1.1017e8 / 5.5086e7): the pair sum's DRAM bytes are its neighbour
# records.  The wave-space kernels are left out (their grid bytes stay partly in L2 between launches,
# so they do not scale with N_g^3).  Reported only for that workload.
NCU_TRAFFIC_WORKLOAD = (1048576, 0.3, 1e-3, 0.5, 256, 6)
NCU_TRAFFIC = {'k_real<float,M_FULL>': 1.926e9, 'k_real<float,M_SE>': 1.926e9, 'k_real<float,M_SU>': 1.892e9}


def real_flops_per_pair():
    # FP32 operations of the pair kernel per neighbour, counted from its formulas (FMA = 2):
    # separation and 1/r 10; table interpolation 2 + 3 per function (7, 3 or 4 functions);
    # S r^ 26; r^.S r^ 5; r^.F 5; U terms 22 (13 without F); E terms 87 (78 without F, two
    # Y-basis products of 24 each).  Full 8->8 product (Lanczos), S->E (GMRES), [F;S]->U and
    # S->U (final velocity with and without an external force).
    return {'full': 178, 'se': 130, 'fsu': 82, 'su': 68}


EST_FLOPS_PER_PAIR = 250        # a-priori estimate of the full 8 x 8 block per pair direction


def kernel_instances(prof, N, Ng, P, npairs, cubic, wave_kernel=0):
    """Device time, launches and algorithmic rate of each kernel instance of this library in the
    profiled steps.  Algorithmic bytes per launch (C components): spreading N(16 + 4C) + 4C N_g^3,
    interpolation 4C N_g^3 + N(16 + 4C), kernel scaling (C_in + C_out) n_k 8, noise 8 n_k 8 written
    (n_k = N_g^2 (N_g/2 + 1)); pair sum: formula flops per ordered pair x pairs."""
    vm, vc = prof['variant_ms'], prof['variant_calls']
    n3 = Ng ** 3
    nkh = Ng * Ng * (Ng // 2 + 1)
    # kernel names: 16^3 tiles take the grid-column spreading with the CTA-wide candidate scan and
    # the staged-region interpolation by default (wave_kernel bit 0: shared-tile spreading; bit 2:
    # column spreading with a scan per warp; bit 1: column, bit 4: tile-owned interpolation), other
    # tiles the general kernels
    ts = ('16' if wave_kernel & 1 else ('_col' if wave_kernel & 4 else '_colq')) if cubic else ''
    ti = ('_col' if wave_kernel & 2 else ('16' if wave_kernel & 16 else '_halo')) if cubic else ''
    fl = real_flops_per_pair()
    spec = [('spread', 'k_spread%s<C=8,P=%d>' % (ts, P), ('full', 'fsu'), N * (16 + 32) + 32 * n3),
            ('spread', 'k_spread%s<C=5,P=%d>' % (ts, P), ('se', 'su'), N * (16 + 20) + 20 * n3),
            ('interp', 'k_interp%s<C=8,P=%d>' % (ti, P), ('full',), 32 * n3 + N * (16 + 32)),
            ('interp', 'k_interp%s<C=5,P=%d>' % (ti, P), ('se',), 20 * n3 + N * (16 + 20)),
            ('interp', 'k_interp%s<C=3,P=%d>' % (ti, P), ('fsu', 'su'), 12 * n3 + N * (16 + 12)),
            ('scale', 'k_scale<M_FULL>', ('full',), 16 * nkh * 8),
            ('scale', 'k_scale<M_SE>', ('se',), 10 * nkh * 8),
            ('scale', 'k_scale<M_FSU>', ('fsu',), 11 * nkh * 8),
            ('scale', 'k_scale<M_SU>', ('su',), 8 * nkh * 8),
            ('noise', 'k_noise', ('full',), 8 * nkh * 8)]
    out = []
    for stage, name, vs, bytes_per_launch in spec:
        ms = sum(vm[stage][v] for v in vs)
        calls = sum(vc[stage][v] for v in vs)
        if calls == 0 or ms <= 0:
            continue
        per = ms / calls / 1e3
        out.append({'kernel': name, 'stage': stage, 'bound': 'hbm', 'launches': calls, 'ms': ms,
                    'us_per_launch': per * 1e6, 'algorithmic_bytes_per_launch': bytes_per_launch,
                    'achieved': bytes_per_launch / per / 1e9, 'unit': 'GB/s'})
    for v, mode in (('full', 'M_FULL'), ('se', 'M_SE'), ('fsu', 'M_FSU'), ('su', 'M_SU')):
        ms, calls = vm['real'][v], vc['real'][v]
        if calls == 0 or ms <= 0:
            continue
        per = ms / calls / 1e3
        out.append({'kernel': 'k_real<float,%s>' % mode, 'stage': 'real', 'bound': 'alu', 'launches': calls,
                    'ms': ms, 'us_per_launch': per * 1e6, 'flops_per_pair': fl[v],
                    'algorithmic_flops_per_launch': npairs * fl[v],
                    'achieved': npairs * fl[v] / per / 1e12, 'unit': 'TFLOP/s'})
    return out


def run_ours(args, world, rank, local, pg):
    import torch
    import pse_inputs
    import paper_1709_06946_gb300 as pkg

    pkg.load()
    dev = torch.device('cuda', local)
    torch.cuda.set_device(dev)
    pos_np, L = pse_inputs.rsa_positions(args.N, args.phi, seed=1 + rank)
    h = pkg.PSE(args.N, L, xi=args.xi, tol=args.tol, precision='mixed', use_graph=args.graph,
                wave_kernel=args.wave_kernel)
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

    # roofline of the dominant kernel instance (device time per stage and product variant from
    # CUDA events on the launching stream; cuFFT excluded, it is library code)
    peaks = measured_peaks()
    hbm = peaks.get('hbm_gbs')
    hbm_note = 'of measured hbm_gbs (MEASURED_PEAKS.json)' if hbm else 'of fallback 6800 GB/s'
    hbm = hbm or 6800.0
    stage_ms = prof['ms']
    Li = sum(i[0] for i in piters)
    Ki = sum(i[1] for i in piters)
    npairs = float(np.mean([i[2] for i in piters]))
    Ng, N = inf['Ng'], args.N
    n3 = Ng ** 3
    K = KP
    cubic = tuple(inf['tile']) == (16, 16, 16)
    kernels = kernel_instances(prof, N, Ng, inf['P'], npairs, cubic, args.wave_kernel)
    traffic_ok = (args.N, args.phi, args.tol, args.xi, Ng, inf['P']) == NCU_TRAFFIC_WORKLOAD
    for k in kernels:
        k['share_of_step'] = k['ms'] / (1000.0 * prof_elapsed)
        if k['bound'] == 'hbm':
            k['peak'], k['frac'] = hbm, k['achieved'] / hbm
        else:
            k['peak'], k['frac'] = FP32_PEAK_TFLOPS_AT_MAX, k['achieved'] / FP32_PEAK_TFLOPS_AT_MAX
        k['traffic'] = NCU_TRAFFIC.get(k['kernel']) if traffic_ok else None
    dom = max(kernels, key=lambda k: k['ms'])
    roof = {'bound': dom['bound'], 'kernel': dom['kernel'], 'achieved': dom['achieved'], 'peak': dom['peak'],
            'unit': dom['unit'], 'frac': dom['frac'], 'traffic': dom['traffic'], 'launches': dom['launches'],
            'us_per_launch': dom['us_per_launch'],
            'peak_note': (hbm_note if dom['bound'] == 'hbm' else
                          'derived FP32 peak: 152 SMs x 128 lanes x 2 flop x 2070 MHz'),
            'per_launch': ('algorithmic bytes %.4g (per-particle and per-grid-point bytes x units)' %
                           dom['algorithmic_bytes_per_launch']) if dom['bound'] == 'hbm' else
                          ('flops %.4g (%d per ordered pair x %.4g pairs)' %
                           (dom['algorithmic_flops_per_launch'], dom['flops_per_pair'], npairs))}
    # the pair sum: all of its instances against the derived FP32 peak, with the formula flops per
    # pair and the a-priori ~250-flop estimate of the full block beside them
    fl = real_flops_per_pair()
    real_flops = npairs * (fl['full'] * Li + fl['se'] * Ki + fl['su'] * K)
    real_rate = real_flops / (stage_ms['real'] / 1000.0) / 1e12 if stage_ms['real'] > 0 else None
    roof_real = {'bound': 'alu', 'kernel': 'k_real (real-space pair sum, all instances)', 'achieved': real_rate,
                 'peak': FP32_PEAK_TFLOPS_AT_MAX, 'unit': 'TFLOP/s',
                 'frac': real_rate / FP32_PEAK_TFLOPS_AT_MAX if real_rate else None,
                 'peak_note': 'derived FP32 peak: 152 SMs x 128 lanes x 2 flop x 2070 MHz',
                 'flops_per_pair': fl, 'estimate_flops_per_pair_full': EST_FLOPS_PER_PAIR,
                 'achieved_at_estimate_flops': (npairs * EST_FLOPS_PER_PAIR * (Li + Ki + K)
                                              / (stage_ms['real'] / 1000.0) / 1e12) if stage_ms['real'] > 0 else None}
    # per-step algorithmic rates of the wave-space stages, and the ceiling that binds spreading and
    # interpolation: each particle's P^3 footprint x C components in the shared tile, read and
    # written (spread) or read (interpolation)
    spread_comps = [5] * Ki + [5] * K
    interp_comps = [5] * Ki + [3] * K + [8] * K
    nkh = Ng * Ng * (Ng // 2 + 1)
    algo = {
        'spread': sum(N * (16 + 4 * c) + c * n3 * 4 for c in spread_comps),
        'interp': sum(c * n3 * 4 + N * (16 + 4 * c) for c in interp_comps),
        'scale': sum((ci + co) * nkh * 8 for ci, co in [(5, 5)] * Ki + [(5, 3)] * K),
        'noise': K * 8 * nkh * 8,
    }
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
                      'frac_of_measured_hbm': (algo[k] / (stage_ms[k] / 1000.0) / 1e9) / hbm
                      if stage_ms[k] > 0 else None} for k in algo}

    result = {'metric': METRIC, 'value': value, 'unit': 'steps/s', 'n_gpus': world, 'steps': args.steps,
              'warmup': args.warmup, 'ms_per_step': 1000.0 * elapsed / args.steps, 'higher_is_better': True,
              'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f32', 'data': 'synthetic',
              'config': {'workload': 'N=%d hard spheres (RSA) phi=%g eps=%g constrained mid-point step, mixed '
                                     'precision' % (args.N, args.phi, args.tol),
                         'N': args.N, 'phi': args.phi, 'tol': args.tol, 'xi': args.xi, 'L': L,
                         'Ng': Ng, 'P': inf['P'], 'rcut': inf['rcut'], 'tile': list(inf['tile']),
                         'wave_kernel': args.wave_kernel,
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
              'roofline': roof, 'roofline_pair_sum': roof_real, 'kernels': kernels, 'clocks': clk,
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
    if rank == 0 and world == 1 and args.rfd_steps > 0:
        result['rfd'] = rfd_measure(pkg, torch, dev, args, pos_np, L, value)
    if rank == 0 and world == 1 and args.torque_reps > 0:
        result['torque'] = torque_measure(pkg, torch, dev, args, pos_np, L, args.torque_reps)
    if rank == 0 and world == 1 and args.shear_steps > 0:
        result['lattice'] = lattice_measure(pkg, torch, dev, args, pos_np, L, value, steps=args.shear_steps)
    if rank == 0 and world == 1 and args.eps2 > 0:
        result['eps_%g' % args.eps2] = eps_measure(pkg, torch, dev, args, pos_np, L, args.eps2)
    if rank == 0 and world == 1 and args.batch_steps > 0:
        result['batch256'] = batch_measure(pkg, torch, dev, args, args.batch_steps, 2)
    if rank == 0 and world == 1 and not args.no_serving:
        rates = [float(r) for r in args.serve_rates.split(',')] if args.serve_rates else [8, 32, 128, 512, 1024]
        res, desc = serving_measure(pkg, args, rates, 6, 200000, args.serve_seconds_default)
        kept = [r for r in res if r['req_per_s'] >= 0.85 * r['arrival_rate']] or res[:1]
        best = max(kept, key=lambda r: r['req_per_s'])
        result['serving'] = {'p50_ms': best['p50_ms'], 'p99_ms': best['p99_ms'], 'req_per_s': best['req_per_s'],
                             'offered_rate': best['offered_rate'], 'requests': best['requests'],
                             'peak_running': best['peak_running'],
                             'saturated_req_per_s': max(r['req_per_s'] for r in res),
                             'note': 'latency at the highest Poisson rate whose completions kept up with arrivals; '
                                     'the sweep stops at the first rate that saturated',
                             'sweep': [{k: r[k] for k in ('offered_rate', 'req_per_s', 'p50_ms', 'p99_ms',
                                                          'peak_running', 'requests')} for r in res],
                             'stream': desc}
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


def batch_measure(pkg, torch, dev, args, steps, warmup, compare_sequential=False):
    """Batched constrained steps of the 256-suspension workload through one handle: batch steps/s,
    suspension-steps/s, particle-steps/s, per-suspension iteration spread and stage times."""
    nsys = 256
    Ns, phis, pos, Ls = batch_suspensions(nsys, seed=4)
    h = pkg.PSE(Ns, Ls, xi=args.xi, tol=args.tol, precision='mixed', grid_ladder=1,
                wave_kernel=args.wave_kernel)
    x = torch.tensor(np.concatenate(pos), device=dev, dtype=torch.float64)
    stream = torch.cuda.current_stream(dev)
    for k in range(warmup):
        h.step(x, args.dt, seed=11, step=k)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    h.set_profiling(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    iters = []
    ev0.record(stream)
    for k in range(steps):
        _, st = h.step(x, args.dt, seed=11, step=warmup + k)
        iters.append([(h.system_stats(q)['lanczos_iters'], h.system_stats(q)['krylov_iters']) for q in range(nsys)])
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    elapsed = ev0.elapsed_time(ev1) / 1000.0
    clk = clocks.stop()
    prof = h.profile()
    grids = sorted({h.system_info(q)['Ng'] for q in range(nsys)})
    it = np.array(iters)
    value = steps / elapsed
    out = {'value': value, 'unit': 'batch steps/s', 'steps': steps, 'warmup': warmup,
           'ms_per_step': 1000.0 * elapsed / steps,
           'workload': '256 suspensions, N log-uniform in [500, 20000] (total %d), phi uniform in [0.05, 0.45], '
                       'eps=%g, xi=%g, grids rounded to 2^i 3^j (%d FFT groups)'
                       % (sum(Ns), args.tol, args.xi, len(grids)),
           'total_N': int(sum(Ns)), 'grids': grids,
           'suspension_steps_per_s': nsys * value, 'ptps': sum(Ns) * value,
           'iterations': {'lanczos_min': int(it[..., 0].min()), 'lanczos_max': int(it[..., 0].max()),
                          'krylov_min': int(it[..., 1].min()), 'krylov_max': int(it[..., 1].max())},
           'stage_ms_per_step': {k: v / steps for k, v in prof['ms'].items()},
           'gpu_launches_per_step': prof['launches'] / steps, 'fft_execs_per_step': prof['fft_execs'] / steps,
           'clocks': clk}
    h.set_profiling(False)
    h.close()
    if compare_sequential:
        hs = [pkg.PSE(Ns[q], Ls[q], xi=args.xi, tol=args.tol, precision='mixed') for q in range(nsys)]
        xs = [torch.tensor(pos[q], device=dev, dtype=torch.float64) for q in range(nsys)]
        for q in range(nsys):
            hs[q].step(xs[q], args.dt, seed=11, step=0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for q in range(nsys):
            hs[q].step(xs[q], args.dt, seed=11, step=1)
        torch.cuda.synchronize(dev)
        tseq = time.perf_counter() - t0
        out['sequential_handles'] = {'s_per_round': tseq, 'batch_speedup': tseq / (elapsed / steps)}
        for hh in hs:
            hh.close()
    return out


def run_batch(args):
    import torch
    import paper_1709_06946_gb300 as pkg
    pkg.load()
    dev = torch.device('cuda', 0)
    b = batch_measure(pkg, torch, dev, args, args.steps, args.warmup, args.compare_sequential)
    line = {'metric': 'batched constrained steps/s (256 suspensions, one handle)', 'value': b['value'],
            'unit': 'batch steps/s', 'n_gpus': 1, 'steps': args.steps, 'warmup': args.warmup,
            'ms_per_step': b['ms_per_step'], 'higher_is_better': True, 'scaling': 'weak',
            'vs_baseline': None, 'dtype': 'f32', 'data': 'synthetic',
            'config': {'workload': b['workload'], 'total_N': b['total_N'], 'grids': b['grids']}}
    line.update({k: v for k, v in b.items() if k not in ('value', 'unit', 'steps', 'warmup', 'ms_per_step',
                                                         'workload', 'total_N', 'grids')})
    print(json.dumps(line), flush=True)


def rfd_measure(pkg, torch, dev, args, pos_np, L, midpoint_rate):
    """The Euler-Maruyama step with a random-finite-difference drift (three stresslet solves per
    step, the alternative the paper weighs against the mid-point scheme) on the same workload,
    launched from the host; its rate beside the mid-point step's."""
    stream = torch.cuda.current_stream(dev)
    h = pkg.PSE(args.N, L, xi=args.xi, tol=args.tol, precision='mixed', wave_kernel=args.wave_kernel)
    x = torch.tensor(pos_np, device=dev, dtype=torch.float64)
    h.rfd_step(x, args.dt, seed=77, step=0)
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    its = []
    ev0.record(stream)
    for k in range(args.rfd_steps):
        _, st = h.rfd_step(x, args.dt, seed=77, step=1 + k)
        its.append(st['krylov_iters'])
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    t = ev0.elapsed_time(ev1) / 1000.0 / args.rfd_steps
    h.close()
    return {'steps_per_s': 1.0 / t, 'ms_per_step': 1000.0 * t, 'krylov_iters_total_mean': float(np.mean(its)),
            'midpoint_speedup': midpoint_rate * t,
            'note': 'Euler-Maruyama with random-finite-difference drift (3 stresslet solves per step, host-launched) '
                    'against the graph-captured mid-point step (1 solve)'}


def lattice_measure(pkg, torch, dev, args, pos_np, L, cubic_rate, gamma=0.5, steps=5, warmup=2):
    """The constrained step on a sheared cell (strain gamma, Sec. 2.3.3; the workload's particles
    mapped into the cell), mixed precision, graph-captured: with the support size from Eq. bound
    with lambda_max (the default) and with the orthorhombic rule lambda_max = 1 (fewer support
    points, but past the tolerance on this lattice)."""
    stream = torch.cuda.current_stream(dev)
    A = np.array([[1.0, gamma, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    out = {'strain': gamma, 'lambda_max': 1 + gamma * gamma / 2 + gamma * np.sqrt(1 + gamma * gamma / 4)}
    for key, aware in (('lambda_aware', 1), ('orthorhombic_rule', 0)):
        h = pkg.PSE(args.N, L, xi=args.xi, tol=args.tol, precision='mixed', use_graph=args.graph, deform=A,
                    lambda_support=aware)
        inf = h.info
        x = torch.tensor(pos_np @ A.T, device=dev, dtype=torch.float64)
        for k in range(warmup):
            h.step(x, args.dt, seed=2468, step=k)
        torch.cuda.synchronize(dev)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        its = []
        ev0.record(stream)
        for k in range(steps):
            _, st = h.step(x, args.dt, seed=2468, step=warmup + k)
            its.append((st['lanczos_iters'], st['krylov_iters']))
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        t = ev0.elapsed_time(ev1) / 1000.0 / steps
        h.close()
        out[key] = {'steps_per_s': 1.0 / t, 'ms_per_step': 1000.0 * t, 'P': inf['P'], 'Ng': inf['Ng'],
                    'rcut': inf['rcut'], 'cells_per_side': inf['cells_per_side'],
                    'lanczos_mean': float(np.mean([i[0] for i in its])),
                    'krylov_mean': float(np.mean([i[1] for i in its]))}
    out['cubic_over_sheared'] = cubic_rate / out['lambda_aware']['steps_per_s']
    out['note'] = ('sheared cell: the 16^3-tile spreading / interpolation kernels with x-y coupled Gaussian '
                   'weights (the 8-component interpolation in passes of 5 and 3 components), grid resolving '
                   'k_cut along the longest lattice column')
    return out


def torque_measure(pkg, torch, dev, args, pos_np, L, reps, warmup=2):
    """The 11-moment product [U; Omega; E] = M [F; L; S] (forces, torques, stresslets) on the
    workload's positions, mixed precision, against the 8-moment product [U; E] = M [F; S] of
    the same handle; each timed with CUDA events over `reps` calls."""
    stream = torch.cuda.current_stream(dev)
    h = pkg.PSE(args.N, L, xi=args.xi, tol=args.tol, precision='mixed', torque=1,
                wave_kernel=args.wave_kernel)
    x = torch.tensor(pos_np, device=dev, dtype=torch.float64)
    g = torch.Generator(device=dev).manual_seed(5)
    F = torch.randn((args.N, 3), device=dev, generator=g)
    Lt = torch.randn((args.N, 3), device=dev, generator=g)
    S = torch.randn((args.N, 5), device=dev, generator=g)
    out = {}
    for name, call in (('eleven', lambda: h.mobility11(x, F, Lt, S)), ('eight', lambda: h.mobility(x, F, S))):
        for _ in range(warmup):
            call()
        torch.cuda.synchronize(dev)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(reps):
            call()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        out[name] = ev0.elapsed_time(ev1) / reps
    h.close()
    return {'ms_per_product': out['eleven'], 'ms_per_product_8': out['eight'],
            'ratio_11_over_8': out['eleven'] / out['eight'], 'reps': reps,
            'note': '11-moment product (11 grids, rotation couplings in the pair sum) and the 8-moment '
                    'product of the same handle; each call includes the cell and neighbour lists'}


def eps_measure(pkg, torch, dev, args, pos_np, L, tol, steps=5, warmup=2, fp64_steps=1):
    """The constrained step at another PSE tolerance on the same positions: mixed (graph) rate,
    all-FP64 rate, and the mixed form's error per output against the FP64 form on identical
    inputs and external noise."""
    stream = torch.cuda.current_stream(dev)
    h = pkg.PSE(args.N, L, xi=args.xi, tol=tol, precision='mixed', use_graph=args.graph,
                wave_kernel=args.wave_kernel)
    inf = h.info
    x = torch.tensor(pos_np, device=dev, dtype=torch.float64)
    for k in range(warmup):
        h.step(x, args.dt, seed=4321, step=k)
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    its = []
    ev0.record(stream)
    for k in range(steps):
        _, st = h.step(x, args.dt, seed=4321, step=warmup + k)
        its.append((st['lanczos_iters'], st['krylov_iters']))
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    t_mixed = ev0.elapsed_time(ev1) / 1000.0 / steps
    h.close()
    out = {'tol': tol, 'Ng': inf['Ng'], 'P': inf['P'], 'rcut': inf['rcut'], 'steps_per_s': 1.0 / t_mixed,
           'ms_per_step': 1000.0 * t_mixed, 'ptps': args.N / t_mixed,
           'lanczos_mean': float(np.mean([i[0] for i in its])), 'krylov_mean': float(np.mean([i[1] for i in its]))}
    if fp64_steps > 0:
        h64 = pkg.PSE(args.N, L, xi=args.xi, tol=tol, precision='fp64')
        x64 = torch.tensor(pos_np, device=dev, dtype=torch.float64)
        h64.step(x64, args.dt, seed=99, step=0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for k in range(fp64_steps):
            h64.step(x64, args.dt, seed=99, step=1 + k)
        torch.cuda.synchronize(dev)
        t64 = (time.perf_counter() - t0) / fp64_steps
        out['fp64'] = {'steps_per_s': 1.0 / t64, 'ms_per_step': 1000.0 * t64, 'mixed_speedup': t64 / t_mixed}
        if not args.no_accuracy:
            a = argparse.Namespace(**vars(args))
            a.tol = tol
            out['accuracy'] = accuracy_vs_fp64(pkg, torch, dev, a, pos_np, L, h64)
        h64.close()
    return out


# ----------------------------------------------------------------------------- equilibrium runs
def run_equilibrium(args):
    """The validation runs of Sec. 4: the spring-pair distance distribution against its Boltzmann
    density (mid-point and RFD schemes), and S(q) of non-interacting spheres at several volume
    fractions; one JSON line with the statistics and the step rates of the runs."""
    import torch
    import pse_inputs
    import paper_1709_06946_gb300 as pkg
    from paper_1709_06946_gb300.equilibrium import (boltzmann_pair_reference, pair_distance_run,
                                                    ideal_structure_factor_run)
    pkg.load()
    dev = torch.device('cuda', 0)
    K, R0, L, dt = 5.0, 3.0, 10.0, 0.01
    rgrid, cdf, mean_ref = boltzmann_pair_reference(K, R0)
    dens = np.gradient(cdf, rgrid)
    pair = {}
    for scheme, steps in (('midpoint', args.eq_pair_steps), ('rfd', args.eq_pair_steps // 4)):
        h = pkg.PSE(2, L, xi=1.0, tol=1e-3, precision='mixed', use_graph=1)
        x = torch.tensor([[3.0, 5.0, 5.0], [3.0 + R0, 5.0, 5.0]], device=dev, dtype=torch.float64)
        t0 = time.perf_counter()
        r = pair_distance_run(h, x, L, K, R0, dt, steps, every=10, seed=21, scheme=scheme, delta=0.01, burn=500)
        wall = time.perf_counter() - t0
        h.close()
        rs = np.sort(r)
        ks = float(np.max(np.abs(np.arange(1, rs.size + 1) / rs.size - np.interp(rs, rgrid, cdf))))
        bm = np.array([b.mean() for b in np.array_split(r, 20)])
        hist, edges = np.histogram(r, bins=24, range=(R0 - 1.2, R0 + 1.2), density=True)
        mid = 0.5 * (edges[1:] + edges[:-1])
        pair[scheme] = {'steps': steps, 'samples': int(r.size), 'steps_per_s': (steps + 500) / wall,
                        'mean_r': float(r.mean()), 'mean_r_boltzmann': mean_ref,
                        'mean_r_se': float(bm.std(ddof=1) / np.sqrt(bm.size)), 'ks_distance': ks,
                        'histogram': {'r': mid.round(3).tolist(), 'sampled': hist.round(4).tolist(),
                                      'boltzmann': np.interp(mid, rgrid, dens).round(4).tolist()}}
    sq = {}
    for phi in (0.1, 0.3, 0.5):
        N = args.eq_sq_N
        Lb = pse_inputs.box_length(N, phi)
        h = pkg.PSE(N, Lb, xi=0.6, tol=1e-3, precision='mixed', use_graph=1)
        x = torch.tensor(pse_inputs.random_positions(N, Lb, seed=31), device=dev, dtype=torch.float64)
        t0 = time.perf_counter()
        qs, S, cnt = ideal_structure_factor_run(h, x, Lb, 0.05, args.eq_sq_steps, 20, 12, seed=4)
        wall = time.perf_counter() - t0
        h.close()
        grand = float(np.average(S, axis=1, weights=cnt).mean())
        sq['phi=%g' % phi] = {'N': N, 'L': Lb, 'steps': args.eq_sq_steps, 'snapshots': int(S.shape[0]),
                              'steps_per_s': args.eq_sq_steps / wall, 'S_mean': grand,
                              'S_mean_se_one_snapshot': float(1.0 / np.sqrt(cnt.sum())),
                              'q': qs.round(4).tolist(), 'S_shell': S.mean(0).round(4).tolist()}
    line = {'metric': 'equilibrium validation (Sec. 4): spring-pair distance distribution, S(q) of ideal spheres',
            'value': pair['midpoint']['ks_distance'], 'unit': 'Kolmogorov distance to the Boltzmann CDF',
            'higher_is_better': False, 'n_gpus': 1, 'dtype': 'f32', 'data': 'synthetic',
            'config': {'workload': 'two spheres, U = k|r - r0| (k = 5 kT, r0 = 3a), L = 10a, dt = 0.01; '
                                   'N = %d ideal spheres at phi 0.1/0.3/0.5, dt = 0.05' % args.eq_sq_N},
            'pair': pair, 'structure_factor': sq}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload != 'step':
        if args.impl == 'reference':
            print(json.dumps({'impl': 'reference', 'unavailable': 'the oracle arm covers the N=1M step workload only'}))
            return
        {'batch256': run_batch, 'serve': run_serve, 'equilibrium': run_equilibrium}[args.workload](args)
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
