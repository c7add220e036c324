#!/usr/bin/env python
"""Benchmark of the orthogonal-projector MG-MLMC trace estimator on one GPU
(or N ranks, one GPU each, sharding the noise samples; `--impl reference`
times the FP64 CPU oracle instead).

Metric: time to reach a fixed standard error eps = 1e-5 |tr| of the
tr(D^-1) estimate, predicted from the measured per-sample device cost C_l
and sample variance V_l of every term with the optimal allocation
(sum_l sqrt(V_l C_l))^2 / eps^2 (Sec. 2.2, Eq. MLMC-Nl); lower is better.

Workload: 16^4 lattice, synthetic SU(3) links U = exp(i 0.4 H) (seed 1002),
Wilson mass m0 from tests/golden/mass_16x16x16x16.json (the most
ill-conditioned point of an oracle scan on this field), three-level
hierarchy (4^4 then 2^4 aggregates, 16 test vectors per level), noise seed
2002.  A step is one batch of `--batch` Z4 noise vectors through every term
of the orthogonal split (O_0, O_1, F_0, F_1, D_2^-1), every solve to a
relative residual of 1e-12 (FP32 MG-preconditioned FGMRES with SAP and a
one-channel learned post-smoothing step, inside FP64 defect correction, by
default; `--precision fp64` for all-FP64).  Inputs (gauge field, hierarchy,
vectors) are resident in HBM; a 256 MB write flushes the 129 MB L2 between
timed steps.

Also reported, on the same GPU and noise samples: plain Hutchinson with the
same solver, the oblique MG-MLMC split, inexact deflation (k = 128), SAP-only
MG-MLMC, all-FP64 MG-MLMC and plain Hutchinson in FP64, with the per-term
difference of the mixed-precision estimate against FP64; the FP32 and BF16
Wilson operator bandwidth at 32^4; the roofline of the dominant kernel class
(CUDA events around its launches in a profiled repeat of the first timed
step); the clocks sampled during the timed region; an end-to-end figure
through the C-ABI (gauge field copied from pinned host memory, hierarchy
setup, then the sampling to the same eps); and the FP64 CPU oracle timed on
the host on a bounded sample.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

# the CPU oracle runs one worker thread per host core, each with a
# single-threaded BLAS (set before numpy loads its BLAS)
for _var in ('OPENBLAS_NUM_THREADS', 'OMP_NUM_THREADS', 'MKL_NUM_THREADS'):
    os.environ.setdefault(_var, '1')

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = 'tr(D^-1) MLMC time to fixed variance, learned+mixed vs plain; Dslash GB/s'
DIMS = (16, 16, 16, 16)
EPS_GAUGE = 0.4
GAUGE_SEED, NOISE_SEED, TV_SEED = 1002, 2002, 3002
ARMS = ('plain', 'oblique', 'deflated', 'sap', 'fp64', 'refined', 'augmented')
# refined arm (Sec. 5): level-0 test vectors refined toward the low modes of
# Gamma5 D, a block of N_tv + 8 columns, eigen-residual target and the
# tolerance of the refinement's FP64 solves
REFINE_BLOCK_EXTRA, REFINE_EIG_TOL, REFINE_SOLVE_TOL = 8, 1e-3, 1e-6
BLOCKS = [(4, 4, 4, 4), (2, 2, 2, 2)]
NTV = [16, 16]
REL_EPS = 1e-5
MASS_FILE = os.path.join(ROOT, 'tests', 'golden', 'mass_16x16x16x16.json')
PEAKS_FILE = os.path.join(ROOT, 'MEASURED_PEAKS.json')
FP64_PEAK_TFLOPS = 1.25  # GB300 FP64 rate: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 80.0  # 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz
SOLVER = dict(tol=1e-12, restart=24, max_iter=2000, smoother=1, smoother_steps=1, sap_iters=4,
              coarse_iters=4, inner_tol=1e-6, coarse_smoother_steps=4)
KERNELS = {0: 'wilson_dslash_fp64', 1: 'wilson_dslash_fp32', 2: 'coarse_stencil_fp64',
           3: 'coarse_stencil_fp32', 4: 'sap_sweep_fp64', 5: 'sap_sweep_fp32'}
# further event-timed groups (breakdown only; no roofline)
GROUPS = {6: 'transfer_in_cycle', 7: 'gram_schmidt', 8: 'learned_step', 9: 'coarsest_dense'}
SHARD_STRIDE = 1000000  # Z4 sample counters per rank
# dram bytes per launch of a kernel from an ncu capture, keyed by (kernel,
# sha1 of the kernel sources it was measured on, right-hand sides per
# launch); a stale or missing key gives null
TRAFFIC = {
    # one level-1 launch (4^4 x 32 dof, 8 rhs), cold-cache capture (the TMA
    # kernel's code and the shared helpers are byte-identical to the capture)
    ('coarse_stencil_fp32', 'f3db7ca784d1', 8): 19.43e6,
    # one sweep (block + boundary kernel, both colours), 16^4 x 8 rhs
    ('sap_sweep_fp32', '9a67c5f9b503', 8): 578.0e6,
    # the same sweep at 32 rhs, scaled from the 8-rhs capture by the rhs
    # count: every right-hand side is its own row of the launch grid and
    # moves its own residual, correction and block solution
    ('sap_sweep_fp32', '9a67c5f9b503', 32): 4 * 578.0e6,
}


def workload():
    with open(MASS_FILE) as f:
        return json.load(f)


# the source a kernel class's recorded ncu figures depend on: its file, or
# the region of it between two marker lines, plus the shared helpers
KERNEL_SOURCES = {
    'wilson': ('kernels_dirac.cu', None),
    'coarse': ('kernels_coarse.cu', ('// ---- TMA bulk staging', '// AT[X][d][j][i] = A[X][d][i][j]')),
    'sap': ('kernels_sap.cu', None),
}


def kernel_source_hash(kernel):
    """sha1 of the code of a kernel class plus the shared helpers: a recorded
    ncu traffic figure only applies to this exact code."""
    p = os.path.join(ROOT, 'paper_2509_11424_gb300', 'csrc')
    src, region = KERNEL_SOURCES[kernel.split('_')[0]]
    code = open(os.path.join(p, src), 'rb').read()
    if region:
        text = code.decode()
        code = text[text.index(region[0]):text.index(region[1])].encode()
    h = hashlib.sha1()
    h.update(code)
    h.update(open(os.path.join(p, 'common.cuh'), 'rb').read())
    return h.hexdigest()[:12]


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
              'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
              'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        # raw samples (the line carries their summary); MGMLMC_CLOCKS_DIR keeps them
        self.path = os.path.join(os.environ.get('MGMLMC_CLOCKS_DIR', tempfile.gettempdir()),
                                 'clocks_bench_%d.csv' % device_index)

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
        rows = [[p.strip() for p in line.split(',')] for line in open(self.path)]
        rows = [r for r in rows if len(r) >= 9]
        if not rows:
            return {'sm_mhz': None, 'sm_max_mhz': None, 'reasons': ['no samples']}
        num = lambda v: v.replace('.', '', 1).isdigit()
        sm = [float(r[1]) for r in rows if num(r[1])]
        mx = [float(r[2]) for r in rows if num(r[2])]
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
        if not dist.is_initialized():
            dist.init_process_group('nccl')
        return dist, rank, ws, local
    return None, 0, 1, local


def merge_terms(results):
    acc = {}
    for res in results:
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


def allreduce_terms(dist, acc, world, device):
    """Merge the per-term accumulators of all ranks in place: sums of N, X,
    |X|^2, iteration counts and seconds (the seconds then averaged over the
    ranks, which run at the same time), maximum of the true residuals.  Every
    rank holds the same terms; the only exchange of the sharded path."""
    import torch
    keys = sorted(acc)
    fields = ('n', 'sre', 'sim', 'sab', 'sec', 'it', 'k')
    vec = torch.tensor([[float(acc[k][f]) for f in fields] for k in keys], dtype=torch.float64,
                       device=device)
    dist.all_reduce(vec)
    res = torch.tensor([float(acc[k]['res']) for k in keys], dtype=torch.float64, device=device)
    dist.all_reduce(res, op=dist.ReduceOp.MAX)
    for i, k in enumerate(keys):
        for j, f in enumerate(fields):
            acc[k][f] = vec[i, j].item()
        acc[k]['sec'] /= world
        acc[k]['n'] = int(round(acc[k]['n']))
        acc[k]['k'] = int(round(acc[k]['k']))
        acc[k]['res'] = res[i].item()
    return acc


def max_over_ranks(dist, x, device):
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def first_sample(rank, k, batch):
    """Counter of the first Z4 sample of step k on a rank: ranks draw from
    disjoint ranges of SHARD_STRIDE samples."""
    return rank * SHARD_STRIDE + k * batch


def stats_of(a):
    n = a['n']
    mu = complex(a['sre'], a['sim']) / n
    var = max(0.0, (a['sab'] - n * abs(mu) ** 2) / (n - 1))
    return mu, var


def time_to_variance(acc, world, step_ms, steps, rel_eps=REL_EPS, var_of=None, eps=None):
    """(predicted seconds, details): per-sample costs from the library's
    per-term device time, rescaled so the terms add up to the measured step
    time (host gaps included), divided by the number of ranks.  var_of
    (term -> variance) and eps replace this run's own estimates: arms that
    compute the same per-sample values (same estimator, same noise, solves to
    1e-12) share the variances of the run with the most samples, so they
    differ only in cost."""
    terms = sorted(acc)
    dev_sec = sum(acc[t]['sec'] for t in terms)
    scale = (step_ms * 1e-3 * steps) / dev_sec if dev_sec > 0 else 1.0
    tr, S, det = 0j, 0.0, {}
    for t in terms:
        mu, var = stats_of(acc[t])
        if var_of is not None:
            var = var_of[str(t)]
        C = acc[t]['sec'] * scale / acc[t]['n'] / world
        tr += mu
        S += np.sqrt(var * C)
        det[str(t)] = dict(mean=[mu.real, mu.imag], var=var, cost_s=C, n=acc[t]['n'],
                           iters=acc[t]['it'] / max(1, acc[t]['k']), max_residual=acc[t]['res'])
    if eps is None:
        eps = rel_eps * abs(tr)
    return S ** 2 / eps ** 2, dict(trace=[tr.real, tr.imag], eps=eps, terms=det)


# ---------------------------------------------------------------- CPU oracle
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def host_memory_available():
    """Bytes this process may still allocate: MemAvailable, capped by the
    cgroup's limit when one is set (None when neither can be read)."""
    avail = None
    try:
        with open('/proc/meminfo') as f:
            for line in f:
                if line.startswith('MemAvailable:'):
                    avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    try:
        with open('/sys/fs/cgroup/memory.max') as f:
            lim = f.read().strip()
        with open('/sys/fs/cgroup/memory.current') as f:
            cur = int(f.read().strip())
        if lim != 'max':
            left = int(lim) - cur
            avail = left if avail is None else min(avail, left)
    except (OSError, ValueError):
        pass
    return avail


# host bytes of one oracle worker: the GMRES(64) basis of 65 vectors of the
# 16^4 system (786,432 complex doubles each), with slack for temporaries
ORACLE_WORKER_BYTES = 1.2e9


def oracle_threads(requested):
    """Worker threads for the oracle timing: the requested count (0: every
    core), cut to what the host's free memory holds beside the shared
    matrix and its construction (~8 GB)."""
    t = requested or host_cores()
    avail = host_memory_available()
    if avail is not None:
        t = min(t, max(1, int((avail - 8e9) / ORACLE_WORKER_BYTES)))
    return t


_ORACLE_MATRIX = {}


def oracle_matrix(m0):
    """The oracle's sparse 16^4 Wilson matrix (built once per mass) and its
    build time."""
    if m0 not in _ORACLE_MATRIX:
        from oracle import dirac
        from paper_2509_11424_gb300 import synth
        t0 = time.time()
        U = synth.gauge_field(DIMS, EPS_GAUGE, GAUGE_SEED)
        _ORACLE_MATRIX[m0] = (dirac.wilson_matrix(U, m0, DIMS).tocsr(), time.time() - t0)
    return _ORACLE_MATRIX[m0]


def oracle_gmres_cycle(m0, threads=1, first=0):
    """Bounded samples of the workload with the FP64 oracle on the host: in
    each of `threads` concurrent threads one restart cycle (64 iterations) of
    the oracle's GMRES(64) on the 16^4 plain-Hutchinson system D z = x, x the
    Z4 sample first + thread.  The threads share one matrix (scipy's sparse
    products and numpy's vector operations release the GIL).  Returns the
    host's seconds per GMRES iteration (wall time over the iterations of all
    threads), the wall and CPU seconds and the setup time."""
    import scipy.sparse.linalg as spla
    from oracle import noise
    M, setup = oracle_matrix(m0)
    its = [0] * threads

    def run(i):
        x = noise.z4_vector(M.shape[0], NOISE_SEED, first + i, noise.TERM_PLAIN)

        def cb(_):
            its[i] += 1

        spla.gmres(M, x, rtol=1e-12, atol=0.0, restart=64, maxiter=1, callback=cb, callback_type='pr_norm')

    workers = [threading.Thread(target=run, args=(i,)) for i in range(threads)]
    c0, t1 = time.process_time(), time.time()
    for w in workers:
        w.start()
    for w in workers:
        w.join()
    el, cpu = time.time() - t1, time.process_time() - c0
    total = max(1, sum(its))
    return dict(sec_per_iter=el / total, iters=total, seconds=el, cpu_seconds=cpu, setup_s=setup,
                threads=threads)


def oracle_time_to_variance(sample, wl):
    """Time to the benchmark's eps for the oracle's plain Hutchinson estimator:
    V and the iterations per 1e-12 solve from the oracle run stored in the
    workload file (tests/golden/oracle_workload.py), seconds per iteration
    measured now on this host."""
    op = wl['oracle_plain']
    C = sample['sec_per_iter'] * float(np.mean(op['gmres_iters']))
    eps = REL_EPS * abs(complex(*op['mean']))
    return op['var'] * C / eps ** 2, C


E2E_STEPS = 2  # steady end-to-end steps timed after the first one


def e2e_time_to_variance(setup_s, first_step_s, step_s, value, device_step_s):
    """End-to-end time to the benchmark's eps: the setup, the first step's
    one-time extra (graph capture, autotuning) over a steady step, and the
    steps the device-timed estimate needs, each at its end-to-end cost."""
    return setup_s + max(0.0, first_step_s - step_s) + value * step_s / device_step_s


def cpu_baseline(m0, wl, threads):
    """The `cpu_baseline` object of the GPU arm's line: the oracle's plain
    Hutchinson estimator timed on `threads` host threads (one GMRES cycle
    each, concurrently), with the single-thread figure beside it."""
    s1 = oracle_gmres_cycle(m0)
    sT = oracle_gmres_cycle(m0, threads, 1) if threads > 1 else s1
    v1, C1 = oracle_time_to_variance(s1, wl)
    value, C = oracle_time_to_variance(sT, wl)
    return {'value': value, 'unit': 's', 'cores': threads, 'kind': 'oracle',
            'sample': 'plain Hutchinson, %d concurrent 64-iteration GMRES(64) cycles of the oracle on the 16^4 '
                      'system, one per thread (%.1f s wall), scaled by %.0f iterations per 1e-12 solve and the '
                      'oracle variance' % (threads, sT['seconds'], np.mean(wl['oracle_plain']['gmres_iters'])),
            'seconds_per_solve': C, 'cpu_utilisation': sT['cpu_seconds'] / sT['seconds'],
            'single_core': {'value': v1, 'seconds_per_solve': C1, 'cycle_s': s1['seconds'],
                            'cpu_utilisation': s1['cpu_seconds'] / s1['seconds']},
            'threads_available': host_cores()}


def reference_arm(args, rank, world):
    """The FP64 CPU oracle on this host's cores, same metric and workload:
    each step one bounded sample (a 64-iteration GMRES cycle of the plain
    Hutchinson solve), the value its time to the same variance."""
    if rank != 0:
        return
    wl = workload()
    T = oracle_threads(args.oracle_threads)
    for k in range(args.warmup):
        oracle_gmres_cycle(wl['m0'], T, k * T)
    t = []
    samples = []
    for k in range(args.steps):
        s = oracle_gmres_cycle(wl['m0'], T, (args.warmup + k) * T)
        samples.append(s)
        t.append(s['seconds'])
    spi = float(np.mean([s['sec_per_iter'] for s in samples]))
    value, C = oracle_time_to_variance(dict(sec_per_iter=spi), wl)
    sample = ('plain Hutchinson, 16^4 solve by the oracle GMRES(64): per step %d concurrent 64-iteration '
              'restart cycles (one per thread, samples of their own) timed, scaled by %.0f iterations '
              'per 1e-12 solve and the oracle variance %.4g (tests/golden/mass_16x16x16x16.json)'
              % (T, np.mean(wl['oracle_plain']['gmres_iters']), wl['oracle_plain']['var']))
    util = float(np.mean([s['cpu_seconds'] / s['seconds'] for s in samples]))
    line = {'impl': 'reference', 'metric': METRIC, 'value': value, 'unit': 's', 'n_gpus': world,
            'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': 1e3 * float(np.mean(t)),
            'higher_is_better': False, 'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64',
            'data': 'synthetic',
            'config': {'workload': '16^4 Wilson-Dirac, SU(3) exp(i 0.4 H) seed 1002, m0 %.4f, '
                                   'plain Hutchinson with the FP64 CPU oracle' % wl['m0']},
            'cpu_baseline': {'value': value, 'unit': 's', 'cores': T, 'kind': 'oracle', 'sample': sample,
                             'seconds_per_solve': C, 'cpu_utilisation': util,
                             'threads_available': host_cores()},
            'e2e': {'value': value, 'unit': 's', 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------- Dslash
def dslash_hbm(M, torch, U16, m0, reps=5):
    """FP32 Wilson Dslash on a 32^4 lattice (the 16^4 field tiled 2x2x2x2, a
    valid SU(3) field), 1 and 8 right-hand sides: CUDA events around 10
    back-to-back launches, median of 5; each launch touches >= 400 MB, far
    above the 129 MB L2, so no flush between launches.
    Algorithmic bytes per site: (24 nrhs + 36) x 8 B (spinors in and out, four
    links)."""
    dims = (32, 32, 32, 32)
    V = int(np.prod(dims))
    U = np.tile(U16.reshape(16, 16, 16, 16, 36), (2, 2, 2, 2, 1)).reshape(-1)
    ctx = M.mgmlmc_create(dims, torch.cuda.current_stream())
    out = {}
    try:
        M.mgmlmc_set_gauge(ctx, U)
        M.mgmlmc_set_mass(ctx, m0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
        hbm = peaks.get('hbm_gbs')

        op = M.OP_D | M.LAYOUT_INTERNAL

        def timed(x, y, nrhs):
            # back-to-back launches, the steady state of an iterative solver;
            # no flush: every launch touches >= 400 MB, three times the L2
            for _ in range(3):
                M.mgmlmc_apply(ctx, op, 0, M.FP32, x, y, nrhs)
            ts = []
            for _ in range(reps):
                e0.record()
                for _ in range(10):
                    M.mgmlmc_apply(ctx, op, 0, M.FP32, x, y, nrhs)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) / 10)
            return float(np.median(ts))

        for nrhs in (1, 8):
            # operands in the library's internal (structure-of-arrays) order,
            # so the timed call is the operator alone
            xc = torch.randn((nrhs, V * 12), dtype=torch.complex64, device='cuda')
            x = torch.empty_like(xc)
            M.mgmlmc_reorder(ctx, xc, x, nrhs, 1)
            del xc
            y = torch.empty_like(x)
            by = V * (24.0 * nrhs + 36.0) * 8
            per_variant = {}
            for v in range(M.mgmlmc_kernel_variants(M.VARIANT_DSLASH_FP32)):
                M.mgmlmc_set_kernel_variant(ctx, M.VARIANT_DSLASH_FP32, v)
                per_variant[str(v)] = round(by / (timed(x, y, nrhs) * 1e-3) / 1e9, 1)
            M.mgmlmc_set_kernel_variant(ctx, M.VARIANT_DSLASH_FP32, M.VARIANT_AUTOTUNE)
            ms = timed(x, y, nrhs)
            gbs = by / (ms * 1e-3) / 1e9
            out['nrhs%d' % nrhs] = dict(
                ms=ms, algorithmic_bytes=by, achieved_gbs=gbs,
                frac_of_measured_hbm=gbs / hbm if hbm else None,
                variant=M.mgmlmc_get_kernel_variant(ctx, M.VARIANT_DSLASH_FP32, nrhs),
                gbs_per_variant=per_variant)
        # BF16 storage, FP32 arithmetic: (24 nrhs + 36) x 4 B per site
        for nrhs in (1, 8):
            xc = torch.randn((nrhs, V * 24), dtype=torch.float32, device='cuda').to(torch.bfloat16)
            x = torch.empty_like(xc)
            M.mgmlmc_reorder_bf16(ctx, xc, x, nrhs, 1)
            del xc
            y = torch.empty_like(x)

            def run_bf16():
                M.mgmlmc_apply(ctx, op, 0, M.BF16, x, y, nrhs)

            for _ in range(3):
                run_bf16()
            ts = []
            for _ in range(reps):
                e0.record()
                for _ in range(10):
                    run_bf16()
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) / 10)
            ms = float(np.median(ts))
            by = V * (24.0 * nrhs + 36.0) * 4
            gbs = by / (ms * 1e-3) / 1e9
            out['bf16_nrhs%d' % nrhs] = dict(ms=ms, algorithmic_bytes=by, achieved_gbs=gbs,
                                             frac_of_measured_hbm=gbs / hbm if hbm else None,
                                             site_updates_per_s=V * nrhs / (ms * 1e-3))
        out['lattice'] = list(dims)
    finally:
        M.mgmlmc_destroy(ctx)
    return out


# ---------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=4)
    ap.add_argument('--warmup', type=int, default=3)
    # 32 rhs per launch: the per-sample cost of every term falls with the
    # batch (8 -> 16 -> 32: 91 -> 75 -> 66 s to the same variance)
    ap.add_argument('--batch', type=int, default=32)
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--precision', default='fp32', choices=['fp64', 'fp32'])
    ap.add_argument('--compare-steps', type=int, default=2)
    ap.add_argument('--no-cpu', action='store_true')
    ap.add_argument('--no-e2e', action='store_true')
    ap.add_argument('--m0', type=float, default=None, help='override the tuned mass (exploration)')
    ap.add_argument('--learned', type=int, default=1, help='channels of the learned smoother (0: off)')
    ap.add_argument('--train-steps', type=int, default=200)
    ap.add_argument('--dslash-only', action='store_true', help='only the 32^4 FP32 Dslash measurement')
    ap.add_argument('--arms', default=','.join(ARMS),
                    help='comparison arms to run (comma list of %s)' % ', '.join(ARMS))
    ap.add_argument('--oracle-threads', type=int, default=0,
                    help='host threads of the CPU oracle timing (0: every core of this host)')
    ap.add_argument('--refine-iters', type=int, default=30,
                    help='cap on the test-vector refinement steps of the "refined" arm')
    args = ap.parse_args()

    dist, rank, world, local = dist_init()
    if args.impl == 'reference':
        reference_arm(args, rank, world)
        if dist:
            dist.destroy_process_group()
        return
    wl = workload() if (args.m0 is None or os.path.exists(MASS_FILE)) else {}
    m0 = args.m0 if args.m0 is not None else wl['m0']

    import torch
    from paper_2509_11424_gb300 import mgmlmc as M, synth
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    U = synth.gauge_field(DIMS, EPS_GAUGE, GAUGE_SEED)
    if args.dslash_only:
        print(json.dumps({'dslash_hbm': dslash_hbm(M, torch, U, m0)}))
        return
    ctx = M.mgmlmc_create(DIMS, stream)
    prec = M.FP64 if args.precision == 'fp64' else M.FP32
    M.mgmlmc_set_gauge(ctx, U)
    M.mgmlmc_set_mass(ctx, m0)
    M.mgmlmc_set_solver(ctx, precision=prec, **SOLVER)
    mgp = M.mg_params(BLOCKS, NTV, setup_rounds=6, setup_iters=30, seed=TV_SEED)
    torch.cuda.synchronize()
    t_setup = time.time()
    M.mgmlmc_build_hierarchy(ctx, mgp)
    torch.cuda.synchronize()
    t_setup = time.time() - t_setup
    train = None
    main_solver = dict(SOLVER)
    if args.learned > 0:
        # gauge-covariant network trained on the solver's own post-SAP residuals
        train = M.mgmlmc_learned_train(ctx, channels=args.learned, steps=args.train_steps, batch=8,
                                       pool=2000, lr=1e-3, seed=5002)
        main_solver['smoother'] = M.SMOOTHER_LEARNED
        M.mgmlmc_set_solver(ctx, precision=prec, **main_solver)
    print('kernel launches after setup: %d' % M.mgmlmc_kernel_launches(), file=sys.stderr)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device='cuda')  # 256 MB > L2

    B = args.batch
    nterm = 2 * len(BLOCKS) + 1
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def step(k, kind=M.EST_ORTHOGONAL):
        n = {M.EST_ORTHOGONAL: [B] * nterm, M.EST_OBLIQUE: [B] * (len(BLOCKS) + 1)}.get(kind, [B])
        return M.mgmlmc_estimate_trace(ctx, M.est_params(kind, n, batch=B, seed=NOISE_SEED,
                                                         first_sample=first_sample(rank, k, B)))

    def timed(k0, K, kind=M.EST_ORTHOGONAL):
        res, ms = [], 0.0
        for k in range(K):
            flush.zero_()
            e0.record(stream)
            res.append(step(k0 + k, kind))
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        return res, ms

    for k in range(args.warmup):
        step(k)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    n_launch0 = M.mgmlmc_kernel_launches()
    # profiler range = the timed steps (ncu --profile-from-start off captures
    # exactly these launches; a no-op without a profiler)
    torch.cuda.profiler.start()
    results, total_ms = timed(args.warmup, args.steps)
    torch.cuda.profiler.stop()
    launches = M.mgmlmc_kernel_launches() - n_launch0
    clk = clocks.stop()
    if dist:
        total_ms = max_over_ranks(dist, total_ms, 'cuda')
    ms_per_step = total_ms / args.steps
    acc = merge_terms(results)
    if dist:
        allreduce_terms(dist, acc, world, 'cuda')
    value, det = time_to_variance(acc, world, ms_per_step, args.steps)

    # profiled repeat of the first timed step: per-launch events
    flush.zero_()
    torch.cuda.synchronize()
    M.mgmlmc_profile(ctx, 1)
    e0.record(stream)
    step(args.warmup)
    e1.record(stream)
    torch.cuda.synchronize()
    prof_ms = e0.elapsed_time(e1)
    kst = {c: M.mgmlmc_profile_stats(ctx, c) for c in KERNELS}
    gst = {GROUPS[c]: M.mgmlmc_profile_stats(ctx, c) for c in GROUPS}
    M.mgmlmc_profile(ctx, 0)
    dom = max(kst, key=lambda c: kst[c]['ms'])
    ks = kst[dom]
    roof = None
    if ks['launches'] > 0:
        sec = ks['ms'] * 1e-3
        peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
        hbm = peaks.get('hbm_gbs')
        if dom in (0, 2, 4):  # FP64 kernels are bound by the FP64 pipe on this part
            achieved = ks['flops'] / sec / 1e12
            roof = dict(bound='alu', achieved=achieved, peak=FP64_PEAK_TFLOPS, unit='TFLOP/s',
                        frac=achieved / FP64_PEAK_TFLOPS, peak_source='GB300 FP64 rate 1.25 TFLOP/s (table)')
        else:
            achieved = ks['bytes'] / sec / 1e9
            peak = hbm if hbm else 6800.0
            roof = dict(bound='hbm', achieved=achieved, peak=peak, unit='GB/s', frac=achieved / peak,
                        peak_source='of measured (MEASURED_PEAKS.json hbm_gbs)' if hbm else 'of fallback 6.8 TB/s')
        roof['traffic'] = TRAFFIC.get((KERNELS[dom], kernel_source_hash(KERNELS[dom]), B))
        roof.update(kernel=KERNELS[dom], launches=ks['launches'], avg_launch_us=ks['ms'] * 1e3 / ks['launches'],
                    share_of_profiled_step=ks['ms'] / prof_ms, profiled_step_ms=prof_ms,
                    algorithmic_bytes_per_launch=ks['bytes'] / ks['launches'],
                    algorithmic_flops_per_launch=ks['flops'] / ks['launches'])
    # FP32 Dslash on its own terms (the metric's 'Dslash GB/s')
    dslash = None
    ws = kst[1] if prec == M.FP32 else kst[0]
    if ws['launches'] > 0:
        peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
        gbs = ws['bytes'] / (ws['ms'] * 1e-3) / 1e9
        dslash = dict(kernel=KERNELS[1 if prec == M.FP32 else 0], achieved_gbs=gbs,
                      frac_of_measured_hbm=gbs / peaks['hbm_gbs'] if 'hbm_gbs' in peaks else None,
                      avg_launch_us=ws['ms'] * 1e3 / ws['launches'], nrhs=B,
                      note='16^4 x 8 rhs working set ~0.12 GB is L2-resident within a step')

    dslash_32 = dslash_hbm(M, torch, U, m0) if rank == 0 else None

    compare = {}
    arms = set(a for a in args.arms.split(',') if a)
    if arms - set(ARMS):
        raise SystemExit('unknown arms: %s' % ', '.join(sorted(arms - set(ARMS))))
    k0 = args.warmup  # the timed run's first sample batch: identical noise
    cs = args.compare_steps
    # one eps for every arm; arms with the same estimator share variances
    eps0 = det['eps']
    if rank == 0 and args.compare_steps > 0:
        mvar = {t: v['var'] for t, v in det['terms'].items()}
        pvar = None
        if arms & {'plain', 'fp64'}:
            pres, pms = timed(k0, cs, M.EST_PLAIN)
            pval, pdet = time_to_variance(merge_terms(pres), 1, pms / cs, cs, eps=eps0)
            if 'plain' in arms:
                compare['plain_hutchinson_same_solver'] = dict(value=pval, ms_per_step=pms / cs, detail=pdet)
            pvar = {t: v['var'] for t, v in pdet['terms'].items()}
        # the paper's earlier decomposition (Eq. oblique_multigrid-multilevel-monte-carlo)
        # with the same solver: its own terms, variances from its own samples
        if 'oblique' in arms:
            ores, oms = timed(k0, cs, M.EST_OBLIQUE)
            oval, odet = time_to_variance(merge_terms(ores), 1, oms / cs, cs, eps=eps0)
            compare['mlmc_oblique_same_solver'] = dict(value=oval, ms_per_step=oms / cs, detail=odet)
        # inexact deflation of plain Hutchinson (Sec. 2.1, the paper's setting of
        # Sec. 4.2: k = 128, five inverse block power steps, inner solves to
        # 1e-6); the exact part has no variance, its cost is the basis build
        if 'deflated' in arms:
            dex, dsec = M.mgmlmc_deflation_build(ctx, 128, 5, 1e-6, TV_SEED + 4000)
            dres, dms = timed(k0, cs, M.EST_DEFLATED)
            dacc = {t: a for t, a in merge_terms(dres).items() if t == M.TERM_DEFL}
            dval, ddet = time_to_variance(dacc, 1, dms / cs, cs, eps=eps0)
            compare['deflated_hutchinson_same_solver'] = dict(
                value=dval, ms_per_step=dms / cs, setup_s=dsec, exact_part=[dex.real, dex.imag],
                value_with_setup=dval + dsec, detail=ddet)
        if args.learned > 0 and 'sap' in arms:
            M.mgmlmc_set_solver(ctx, precision=prec, **SOLVER)
            step(k0)
            sres, sms = timed(k0, cs)
            sval, sdet = time_to_variance(merge_terms(sres), 1, sms / cs, cs, var_of=mvar, eps=eps0)
            compare['mlmc_same_precision_sap_only'] = dict(value=sval, ms_per_step=sms / cs, detail=sdet)
        if prec == M.FP32 and 'fp64' in arms:
            M.mgmlmc_set_solver(ctx, precision=M.FP64, **SOLVER)
            step(k0)
            fres, fms = timed(k0, cs)
            fval, fdet = time_to_variance(merge_terms(fres), 1, fms / cs, cs, var_of=mvar, eps=eps0)
            # error of the mixed-precision estimate against FP64, per term, on
            # the same samples (the first cs timed steps)
            am, af = merge_terms(results[:cs]), merge_terms(fres)
            rel = {}
            for t in sorted(af):
                mu_m, mu_f = stats_of(am[t])[0], stats_of(af[t])[0]
                rel[str(t)] = abs(mu_m - mu_f) / abs(mu_f) if mu_f != 0 else abs(mu_m)
            compare['mlmc_fp64'] = dict(value=fval, ms_per_step=fms / cs, detail=fdet,
                                        mixed_vs_fp64_rel_diff=rel)
            pres, pms = timed(k0, 1, M.EST_PLAIN)
            p64, p64d = time_to_variance(merge_terms(pres), 1, pms, 1, var_of=pvar, eps=eps0)
            compare['plain_hutchinson_fp64'] = dict(value=p64, ms_per_step=pms)
        M.mgmlmc_set_solver(ctx, precision=prec, **main_solver)

    e2e = None
    if not args.no_e2e and rank == 0:
        # the whole job through the ABI, wall clock: the gauge field from
        # pinned host memory, the hierarchy, then estimate_trace calls (each
        # returns its term results to the host)
        Uh = torch.from_numpy(U.view(np.float64)).pin_memory()
        torch.cuda.synchronize()
        t0 = time.time()
        M.mgmlmc_set_gauge(ctx, Uh.numpy(), on_device=False)
        M.mgmlmc_set_mass(ctx, m0)
        M.mgmlmc_build_hierarchy(ctx, mgp)
        torch.cuda.synchronize()
        t_build = time.time() - t0
        t1 = time.time()
        step(40000)
        t_first = time.time() - t1
        t1 = time.time()
        for k in range(E2E_STEPS):
            step(40001 + k)
        step_s = (time.time() - t1) / E2E_STEPS
        e2e = dict(value=e2e_time_to_variance(t_build, t_first, step_s, value, ms_per_step * 1e-3), unit='s',
                   h2d_bytes_per_step=0, d2h_bytes_per_step=int(nterm * 2 * B * 16),
                   setup_h2d_bytes=int(U.nbytes), setup_s=t_build, first_step_s=t_first, step_s=step_s,
                   steps=E2E_STEPS,
                   note='wall clock through the ABI: gauge field from pinned host memory and hierarchy setup, '
                        'then estimate_trace steps at their end-to-end cost to the same eps; a step takes '
                        'no input bytes (its Z4 noise is drawn on the device from counters) and reads '
                        'its per-sample values back')

    # Sec. 5: test vectors computed to a small eigen-residual.  Last, because
    # it replaces the level-0 test vectors of the context for good.
    if rank == 0 and args.compare_steps > 0 and 'refined' in arms and args.refine_iters > 0:
        rough_tv = M.mgmlmc_get_test_vectors(ctx, 0) if 'augmented' in arms else None
        torch.cuda.synchronize()
        t0 = time.time()
        th, rh, rsteps = M.mgmlmc_refine_test_vectors(ctx, 0, NTV[0] + REFINE_BLOCK_EXTRA, args.refine_iters,
                                                      REFINE_EIG_TOL, REFINE_SOLVE_TOL, TV_SEED + 5000)
        torch.cuda.synchronize()
        rsec = time.time() - t0
        M.mgmlmc_set_solver(ctx, precision=prec, **main_solver)
        step(k0)
        rres, rms = timed(k0, cs)
        rval, rdet = time_to_variance(merge_terms(rres), 1, rms / cs, cs, eps=eps0)
        compare['mlmc_refined_test_vectors'] = dict(
            value=rval, ms_per_step=rms / cs, setup_s=rsec, value_with_setup=rval + rsec, steps=rsteps,
            block=NTV[0] + REFINE_BLOCK_EXTRA, eig_tol=REFINE_EIG_TOL, solve_tol=REFINE_SOLVE_TOL,
            eig_res_max=float(rh.max()), eig_res=[float(x) for x in rh], theta=[float(x) for x in th],
            detail=rdet)
        # more test vectors as well as more accurate ones (Sec. 5 raises N_tv
        # too): the rough and the refined level-0 vectors together
        if rough_tv is not None:
            try:
                aug = np.ascontiguousarray(np.concatenate([rough_tv, M.mgmlmc_get_test_vectors(ctx, 0)]))
                torch.cuda.synchronize()
                t0 = time.time()
                M.mgmlmc_set_test_vectors(ctx, 0, aug, aug.shape[0], aug.shape[1], on_device=False)
                M.mgmlmc_build_hierarchy(ctx, M.mg_params(BLOCKS, [aug.shape[0]] + NTV[1:], setup_rounds=6,
                                                          setup_iters=30, seed=TV_SEED))
                torch.cuda.synchronize()
                asec = time.time() - t0
                M.mgmlmc_set_solver(ctx, precision=prec, **main_solver)
                step(k0)
                ares, ams = timed(k0, cs)
                aval, adet = time_to_variance(merge_terms(ares), 1, ams / cs, cs, eps=eps0)
                compare['mlmc_rough_plus_refined_test_vectors'] = dict(
                    value=aval, ms_per_step=ams / cs, setup_s=rsec + asec, value_with_setup=aval + rsec + asec,
                    n_tv=[aug.shape[0]] + NTV[1:], detail=adet)
            except Exception as exc:  # a comparison arm never costs the line
                compare['mlmc_rough_plus_refined_test_vectors'] = dict(error=str(exc)[:300])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and 'oracle_plain' in wl:
        cpu = cpu_baseline(m0, wl, oracle_threads(args.oracle_threads))

    if rank == 0:
        line = {
            'metric': METRIC, 'value': value, 'unit': 's', 'n_gpus': world, 'steps': args.steps,
            'warmup': args.warmup, 'ms_per_step': ms_per_step, 'higher_is_better': False,
            'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64' if prec == M.FP64 else 'f32+f64',
            'data': 'synthetic',
            'config': {'workload': '16^4 Wilson-Dirac, SU(3) exp(i 0.4 H) seed 1002, m0 %.4f, orthogonal '
                                   'MG-MLMC 3 levels (4^4, 2^4 aggregates, 16 tv), SAP%s-MG FGMRES, Z4 batch %d '
                                   'per term per step, solves to 1e-12'
                                   % (m0, ' + learned(%d ch)' % args.learned if args.learned else '', B),
                       'global_batch': B * nterm * world, 'lattice': list(DIMS), 'rel_eps': REL_EPS,
                       'l2': 'flushed between steps (256 MB write)', 'parallelism': 'samples sharded, dp%d' % world},
            'dslash_hbm': dslash_32, 'setup_s': t_setup, 'learned': train, 'learned_fallbacks': M.mgmlmc_learned_stats(ctx),
            'detail': det, 'compare': compare, 'roofline': roof, 'dslash': dslash,
            'clocks': clk, 'e2e': e2e, 'gpu_launches': launches,
            'kernel_stats': {KERNELS[c]: kst[c] for c in kst}, 'group_stats': gst, 'cpu_baseline': cpu,
        }
        print(json.dumps(line))
    M.mgmlmc_destroy(ctx)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == '__main__':
    main()
