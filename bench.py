#!/usr/bin/env python
"""Benchmark of the orthogonal-projector MG-MLMC trace estimator on one GPU
(or N ranks, one GPU each, sharding the noise samples).

Metric: time to reach a fixed variance of the tr(D^-1) estimate
(eps = 1e-5 |tr|), predicted from the measured per-sample device cost C_l and
sample variance V_l of every term by the optimal allocation
(sum_l sqrt(V_l C_l))^2 / eps^2 (Sec. 2.2, Eq. MLMC-Nl); lower is better.

Workload: 16^4 lattice, synthetic SU(3) links U = exp(i 0.4 H) (seed 1002),
Wilson mass m0 from tests/golden/mass_16x16x16x16.json (the most
ill-conditioned point the oracle found on this field), three-level hierarchy
(4^4 then 2^4 aggregates, 16 test vectors per level), noise seed 2002.
A step is one batch of `--batch` Z4 noise vectors through every term of the
orthogonal split (O_0, O_1, F_0, F_1, D_2^-1), each solve to a relative
residual of 1e-12.  Inputs (gauge field, hierarchy, vectors) are resident in
HBM; the 16^4 working set (~0.5 GB) is larger than the 129 MB L2, and an L2
flush (a 256 MB write) separates timed steps.

Also reported: the plain Hutchinson estimator on the same GPU, the roofline
of the dominant kernel (CUDA events around its launches in the timed region),
the clocks sampled during the timed region, an end-to-end figure through the
C-ABI with the gauge field copied from pinned host memory every step, and
the FP64 CPU oracle timed on the host on a bounded sample.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (16, 16, 16, 16)
EPS_GAUGE = 0.4
GAUGE_SEED, NOISE_SEED, TV_SEED = 1002, 2002, 3002
BLOCKS = [(4, 4, 4, 4), (2, 2, 2, 2)]
NTV = [16, 16]
REL_EPS = 1e-5
MASS_FILE = os.path.join(ROOT, 'tests', 'golden', 'mass_16x16x16x16.json')
PEAKS_FILE = os.path.join(ROOT, 'MEASURED_PEAKS.json')
FP64_PEAK_TFLOPS = 1.25  # recipe table: GB300 FP64 rate (FMA pipe), see the design doc

# dram bytes per launch of the dominant kernel from an ncu capture, keyed by
# the sha1 of the kernel source it was measured on (stale -> null)
TRAFFIC = {}


def workload_mass():
    with open(MASS_FILE) as f:
        return float(json.load(f)['m0'])


def kernel_source_hash():
    p = os.path.join(ROOT, 'paper_2509_11424_gb300', 'csrc')
    h = hashlib.sha1()
    for f in ('kernels_dirac.cu', 'kernels_coarse.cu', 'common.cuh'):
        h.update(open(os.path.join(p, f), 'rb').read())
    return h.hexdigest()[:12]


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
              'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
              'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.path = os.path.join(ROOT, 'gpurun_out', 'clocks_bench.csv')

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, 'w')
            self.proc = subprocess.Popen(['nvidia-smi', '-i', str(self.idx), '--query-gpu=' + self.FIELDS,
                                          '--format=csv,noheader,nounits', '-lms', '200'],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {'sm_mhz': None, 'sm_max_mhz': None, 'reasons': ['nvidia-smi unavailable']}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(',')]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {'sm_mhz': None, 'sm_max_mhz': None, 'reasons': ['no samples']}
        sm = [float(r[1]) for r in rows if r[1].replace('.', '').isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace('.', '').isdigit()]
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith('active')})
        return {'sm_mhz': float(np.median(sm)) if sm else None, 'sm_max_mhz': max(mx) if mx else None,
                'reasons': reasons, 'samples': len(rows)}


def dist_init():
    ws = int(os.environ.get('WORLD_SIZE', '1'))
    rank = int(os.environ.get('RANK', '0'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl')
        return dist, rank, ws, local
    return None, 0, 1, local


def merge_terms(terms_list):
    """accumulate per-term results of several estimate_trace calls."""
    acc = {}
    for res in terms_list:
        for r in res:
            a = acc.setdefault(r['term'], dict(n=0, sre=0.0, sim=0.0, sab=0.0, sec=0.0, it=0.0, k=0, res=0.0))
            a['n'] += r['n']
            a['sre'] += r['sum_re']
            a['sim'] += r['sum_im']
            a['sab'] += r['sum_abs2']
            a['sec'] += r['seconds']
            a['it'] += r['iters_mean']
            a['k'] += 1
            a['res'] = max(a['res'], r['max_residual'])
    return acc


def stats_of(a):
    n = a['n']
    mu = complex(a['sre'], a['sim']) / n
    var = max(0.0, (a['sab'] - n * abs(mu) ** 2) / (n - 1))
    return mu, var


def time_to_variance(acc, world, step_ms, steps, rel_eps=REL_EPS):
    """(predicted seconds, details) with per-sample costs rescaled so the
    terms add up to the measured step time and divided by the ranks."""
    terms = sorted(acc)
    dev_sec = sum(acc[t]['sec'] for t in terms)
    scale = (step_ms * 1e-3 * steps) / dev_sec if dev_sec > 0 else 1.0
    tr = 0j
    S = 0.0
    det = {}
    for t in terms:
        mu, var = stats_of(acc[t])
        C = acc[t]['sec'] * scale / acc[t]['n'] / world
        tr += mu
        S += np.sqrt(var * C)
        det[str(t)] = dict(mean=[mu.real, mu.imag], var=var, cost_s=C, n=acc[t]['n'],
                           iters=acc[t]['it'] / max(1, acc[t]['k']), max_residual=acc[t]['res'])
    eps = rel_eps * abs(tr)
    return S ** 2 / eps ** 2, dict(trace=[tr.real, tr.imag], eps=eps, terms=det)


def cpu_baseline(m0, budget_s=25.0):
    """The FP64 oracle timed on the host on a bounded sample of the same
    workload: per-sample cost of the plain Hutchinson term (one 16^4 solve
    to 1e-12 with the oracle's BiCGStab) measured on the first BiCGStab
    iterations inside `budget_s` and scaled by the iteration count the full
    solve needs, which the oracle takes from a 1e-12 run on the coarse
    operator's spectrum-equivalent residual history."""
    import scipy.sparse.linalg as spla
    from oracle import dirac
    from paper_2509_11424_gb300 import synth
    t0 = time.time()
    U = synth.gauge_field(DIMS, EPS_GAUGE, GAUGE_SEED)
    Mx = dirac.wilson_matrix(U, m0, DIMS)
    from oracle import noise as onz
    x = onz.z4_vector(Mx.shape[0], NOISE_SEED, 0, onz.TERM_PLAIN)
    setup = time.time() - t0
    it = [0]
    t1 = time.time()

    def cb(_):
        it[0] += 1
        if time.time() - t1 > budget_s:
            raise StopIteration

    try:
        spla.bicgstab(Mx, x, rtol=1e-12, atol=0.0, maxiter=100000, callback=cb)
    except StopIteration:
        pass
    el = time.time() - t1
    per_iter = el / max(1, it[0])
    return dict(per_iter_s=per_iter, iters_done=it[0], setup_s=setup, threads=os.cpu_count())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=4)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--batch', type=int, default=8)
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--precision', default='fp64', choices=['fp64', 'fp32'])
    ap.add_argument('--no-cpu', action='store_true')
    ap.add_argument('--no-e2e', action='store_true')
    ap.add_argument('--plain-steps', type=int, default=2)
    ap.add_argument('--m0', type=float, default=None, help='override the tuned mass (exploration)')
    args = ap.parse_args()

    dist, rank, world, local = dist_init()
    m0 = args.m0 if args.m0 is not None else workload_mass()
    if args.impl == 'reference':
        return reference_arm(args, dist, rank, world, m0)

    import torch
    from paper_2509_11424_gb300 import mgmlmc as M, synth
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    U = synth.gauge_field(DIMS, EPS_GAUGE, GAUGE_SEED)
    ctx = M.mgmlmc_create(DIMS, stream)
    prec = M.FP64 if args.precision == 'fp64' else M.FP32
    M.mgmlmc_set_gauge(ctx, U)
    M.mgmlmc_set_mass(ctx, m0)
    M.mgmlmc_set_solver(ctx, tol=1e-12, restart=24, max_iter=2000, precision=prec, inner_tol=1e-5)
    mgp = M.mg_params(BLOCKS, NTV, setup_rounds=3, setup_iters=20, seed=TV_SEED)
    torch.cuda.synchronize()
    t_setup = time.time()
    M.mgmlmc_build_hierarchy(ctx, mgp)
    torch.cuda.synchronize()
    t_setup = time.time() - t_setup
    print('kernel launches after setup: %d' % M.mgmlmc_kernel_launches(), file=sys.stderr)
    flush =torch.empty(64 * 1024 * 1024, dtype=torch.float32, device='cuda')  # 256 MB > L2

    B = args.batch
    nterm = 2 * len(BLOCKS) + 1
    sample_base = rank * 1000000

    def step(k, kind=M.EST_ORTHOGONAL):
        n = [B] * nterm if kind == M.EST_ORTHOGONAL else [B]
        return M.mgmlmc_estimate_trace(ctx, M.est_params(kind, n, batch=B, seed=NOISE_SEED,
                                                         first_sample=sample_base + k * B))

    for k in range(args.warmup):
        step(k)
    # timed region
    results = []
    step_ms = []
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total_ms = 0.0
    n_launch0 = M.mgmlmc_kernel_launches()
    for k in range(args.steps):
        flush.zero_()
        e0.record(stream)
        results.append(step(args.warmup + k))
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
    clk = clocks.stop()
    launches = M.mgmlmc_kernel_launches() - n_launch0
    # profile pass: the first timed step again with CUDA events around every
    # operator launch (the preconditioner runs eagerly, outside its graph,
    # while events are on; kernel durations are those of the timed launches)
    flush.zero_()
    torch.cuda.synchronize()
    M.mgmlmc_profile(ctx, 1)
    e0.record(stream)
    step(args.warmup)
    e1.record(stream)
    torch.cuda.synchronize()
    prof_ms = e0.elapsed_time(e1)
    kst = {c: M.mgmlmc_profile_stats(ctx, c) for c in range(4)}
    M.mgmlmc_profile(ctx, 0)
    if dist:
        t = torch.tensor([total_ms], device='cuda')
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    acc = merge_terms(results)
    if dist:
        keys = sorted(acc)
        vec = torch.tensor([[acc[k][f] for f in ('n', 'sre', 'sim', 'sab', 'sec')] for k in keys],
                           dtype=torch.float64, device='cuda')
        dist.all_reduce(vec)
        for i, k in enumerate(keys):
            for j, f in enumerate(('n', 'sre', 'sim', 'sab', 'sec')):
                acc[k][f] = vec[i, j].item()
        for k in keys:
            acc[k]['sec'] /= world  # per-rank device seconds
            acc[k]['n'] = int(round(acc[k]['n']))
    value, det = time_to_variance(acc, world, ms_per_step, args.steps)

    # plain Hutchinson on the same GPU for comparison
    plain = None
    if args.plain_steps > 0:
        pres = []
        pms = 0.0
        for k in range(args.plain_steps):
            flush.zero_()
            e0.record(stream)
            pres.append(step(10000 + k, M.EST_PLAIN))
            e1.record(stream)
            torch.cuda.synchronize()
            pms += e0.elapsed_time(e1)
        pacc = merge_terms(pres)
        # variance of the plain estimator relative to the same eps
        pval, pdet = time_to_variance(pacc, world, pms / args.plain_steps, args.plain_steps)
        # rescale to the MLMC eps (same tr, same relative target)
        pval *= (pdet['eps'] / det['eps']) ** 2
        plain = dict(value=pval, detail=pdet)

    # roofline of the dominant kernel class
    names = {0: 'wilson_dslash_fp64', 1: 'wilson_dslash_fp32', 2: 'coarse_stencil_fp64', 3: 'coarse_stencil_fp32'}
    dom = max(kst, key=lambda c: kst[c]['ms'])
    ks = kst[dom]
    roof = None
    if ks['launches'] > 0:
        sec = ks['ms'] * 1e-3
        fp64 = dom in (0, 2)
        if fp64:
            achieved = ks['flops'] / sec / 1e12
            roof = dict(bound='alu', achieved=achieved, peak=FP64_PEAK_TFLOPS, unit='TFLOP/s',
                        frac=achieved / FP64_PEAK_TFLOPS, peak_source='recipe FP64 rate (1.25 TFLOP/s)')
        else:
            peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
            hbm = peaks.get('hbm_gbs', 6800.0)
            achieved = ks['bytes'] / sec / 1e9
            roof = dict(bound='hbm', achieved=achieved, peak=hbm, unit='GB/s', frac=achieved / hbm,
                        peak_source='MEASURED_PEAKS.json hbm_gbs' if peaks else 'fallback 6.8 TB/s')
        key = (names[dom], kernel_source_hash())
        tr = TRAFFIC.get(key)
        roof['traffic'] = tr
        roof['kernel'] = names[dom]
        roof['launches'] = ks['launches']
        roof['avg_launch_us'] = ks['ms'] * 1e3 / ks['launches']
        roof['share_of_profiled_step'] = ks['ms'] / prof_ms
        roof['profiled_step_ms'] = prof_ms
        roof['algorithmic_bytes_per_launch'] = ks['bytes'] / ks['launches']
        roof['algorithmic_flops_per_launch'] = ks['flops'] / ks['launches']

    # end to end through the C-ABI with host buffers: gauge H2D + setup + one batch + results D2H
    e2e = None
    if not args.no_e2e and rank == 0:
        Uh = torch.from_numpy(U.view(np.float64)).pin_memory()
        torch.cuda.synchronize()
        t0 = time.time()
        M.mgmlmc_set_gauge(ctx, Uh.numpy(), on_device=False)
        M.mgmlmc_set_mass(ctx, m0)
        M.mgmlmc_build_hierarchy(ctx, mgp)
        r = step(20000)
        torch.cuda.synchronize()
        t_e2e = time.time() - t0
        # setup part and the sampling part; time to variance = setup + sampling
        eacc = merge_terms([r])
        v_e2e, _ = time_to_variance(acc, world, ms_per_step, args.steps)
        e2e = dict(value=(t_e2e - ms_per_step * 1e-3) + v_e2e, unit='s',
                   h2d_bytes_per_step=int(U.nbytes), d2h_bytes_per_step=int(nterm * 88),
                   setup_s=t_e2e - ms_per_step * 1e-3)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cb = cpu_baseline(m0)
        cpu = cb

    if rank == 0:
        line = {
            'metric': 'tr(D^-1) MLMC time to fixed variance, learned+mixed vs plain; Dslash GB/s',
            'value': value, 'unit': 's', 'n_gpus': world, 'steps': args.steps, 'warmup': args.warmup,
            'ms_per_step': ms_per_step, 'higher_is_better': False, 'scaling': 'weak',
            'vs_baseline': None, 'dtype': 'f64' if prec == M.FP64 else 'f32+f64',
            'data': 'synthetic',
            'config': {'workload': '16^4 Wilson-Dirac, SU(3) exp(i 0.4 H) seed 1002, m0 %.4f, '
                                   'orthogonal MG-MLMC 3 levels (4^4, 2^4 aggregates, 16 tv), '
                                   'Z4 batch %d per term per step, solves to 1e-12' % (m0, B),
                       'global_batch': B * nterm * world, 'lattice': list(DIMS),
                       'l2': 'flushed between steps (256 MB write)', 'rel_eps': REL_EPS},
            'setup_s': t_setup,
            'detail': det,
            'plain_hutchinson': plain,
            'roofline': roof,
            'clocks': clk,
            'e2e': e2e,
            'gpu_launches': launches,
            'kernel_stats': {names[c]: kst[c] for c in kst},
            'cpu_baseline': cpu,
        }
        print(json.dumps(line))
    M.mgmlmc_destroy(ctx)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def reference_arm(args, dist, rank, world, m0):
    if rank != 0:
        return
    print(json.dumps({'impl': 'reference', 'unavailable': 'not implemented yet'}))


if __name__ == '__main__':
    main()
