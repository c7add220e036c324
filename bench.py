#!/usr/bin/env python
"""Benchmark of the orthogonal-projector MG-MLMC trace estimator on one GPU
(or N ranks, one GPU each, sharding the noise samples; `--impl reference`
times the FP64 CPU oracle instead).

Metric: time to reach a fixed standard error eps = 1e-5 |tr| of the
tr(D^-1) estimate, predicted from the measured per-sample device cost C_l
and sample variance V_l of every term with the optimal allocation
(sum_l sqrt(V_l C_l))^2 / eps^2 (Sec. 2.2, Eq. MLMC-Nl); lower is better.
The allocation is then run at a coarser eps_val (chosen so that it takes
about --validate-s seconds) and the achieved standard error and time are
reported beside the prediction.

Default workload (`--workload 48x48x48x96`): a 48^3 x 96 lattice, synthetic
SU(3) links U = exp(i 0.4 H) drawn on the device (seed 1005), m0 = -0.40,
four-level hierarchy (4^4, 2^4, 2^4 aggregates, 16 test vectors per level,
coarsest level 3^3 x 6 inverted densely), every solve to a relative
residual of 1e-12: FP32 MG-preconditioned FGMRES(8) with SAP inside FP64
defect correction, the fine-level solves of the O_0 term starting from the
guess of a learned one-channel network (--net-mode guess; after-sap and
replace-sap put the network into the smoother instead).  The network is
trained on the GPU on 2000 projected Z4 right-hand sides drawn on a 16^4
field of the same generator (seed 1006; the smoother roles train on the
solver's post-SAP residuals), and its weights are carried over: the layers
are translation and gauge covariant.  A step is one call of
mgmlmc_estimate_trace with 4 Z4 samples for each fine-level term (O_0,
F_0; one right-hand-side block, the fine level's memory bound) and 32 for
each coarse term (O_1, O_2, F_1, F_2, coarsest).  Inputs are resident in HBM
and every launch of a step touches far more than the 129 MB L2 (one fine
FP32 vector is 1 GB); the L2 is flushed between steps anyway.

`--workload 16x16x16x16`: the 16^4 lattice (host-drawn field seed 1002,
m0 from tests/golden/mass_16x16x16x16.json, three levels, 32 samples per
term per step) with every comparison arm, including inexact deflation and
refined test vectors.

Also reported, on the same GPU and noise samples: plain Hutchinson with the
same solver, the oblique MG-MLMC split, SAP-only MG-MLMC and all-FP64
MG-MLMC with the per-term difference of the mixed-precision estimate against
FP64; the FP32 and BF16 Wilson operator bandwidth at 32^4; the roofline of
the dominant kernel class (CUDA events around its launches in a profiled
repeat of the first timed step); the clocks sampled during the timed region;
an end-to-end figure through the C-ABI (gauge field copied from pinned host
memory, hierarchy setup, network training, then the sampling to the same
eps); and the FP64 CPU oracle timed on the host on a bounded sample.
"""
import argparse
import hashlib
import json
import math
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
# the 16^4 workload (its oracle statistics are stored in the mass file)
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

# Workloads.  fine_n / coarse_n: samples per step of the terms that solve on
# the fine level / only on coarser ones; the fine level's right-hand sides
# per solve are capped at fine_batch (its vectors are the memory bound).
WORKLOADS = {
    '48x48x48x96': dict(
        dims=(48, 48, 48, 96), eps=0.4, gauge='device', gauge_seed=1005, noise_seed=2005, tv_seed=3005,
        m0=-0.40, blocks=[(4, 4, 4, 4), (2, 2, 2, 2), (2, 2, 2, 2)], ntv=[16, 16, 16],
        fine_n=4, coarse_n=32, batch=32, setup_rounds=6, setup_iters=30,
        # one classical Gram-Schmidt pass in the FP32 FGMRES: the same
        # iteration counts as two on this workload at half the orthogonalisation cost;
        # three level-1 K-cycle iterations with two MR steps per coarse smoothing:
        # 19% less time to variance than four and four on the same samples
        solver=dict(SOLVER, restart=8, fine_batch=4, coarse_restart=16, post_smoothing_only=1, smoother_steps=2,
                    gram_schmidt_passes=1, coarse_iters=3, coarse_smoother_steps=2),
        stencil_variant=-2,
        train=dict(dims=(16, 16, 16, 16), gauge_seed=1006, blocks=[(4, 4, 4, 4), (2, 2, 2, 2)], ntv=[16, 16]),
        arms=('plain', 'oblique', 'sap', 'fp64'), fp64_fine_n=2, fp64_coarse_n=8),
    '16x16x16x16': dict(
        dims=DIMS, eps=EPS_GAUGE, gauge='host', gauge_seed=GAUGE_SEED, noise_seed=NOISE_SEED, tv_seed=TV_SEED,
        m0=None, blocks=BLOCKS, ntv=NTV, fine_n=32, coarse_n=32, batch=32, setup_rounds=6, setup_iters=30,
        solver=dict(SOLVER), stencil_variant=0, train=None, arms=ARMS, fp64_fine_n=32, fp64_coarse_n=32),
}
DEFAULT_WORKLOAD = '48x48x48x96'
KERNELS = {0: 'wilson_dslash_fp64', 1: 'wilson_dslash_fp32', 2: 'coarse_stencil_fp64',
           3: 'coarse_stencil_fp32', 4: 'sap_sweep_fp64', 5: 'sap_sweep_fp32'}
# further event-timed groups (breakdown only; no roofline)
GROUPS = {6: 'transfer_in_cycle', 7: 'gram_schmidt', 8: 'learned_step', 9: 'coarsest_dense'}
SHARD_STRIDE = 1000000  # Z4 sample counters per rank
VALIDATE_FIRST = 500000  # sample counters of the allocation check (fresh samples)
# dram bytes per launch of a kernel from an ncu capture, keyed by (kernel,
# sha1 of the kernel sources it was measured on, right-hand sides per
# launch, lattice); a stale or missing key gives null.  SAP sweep: dram
# read + write of its four kernels on 32^3 x 64 with 4 rhs (8.240 GB, one
# ncu capture of `--kernel-probe sap`), scaled by the site count to
# 48^3 x 96 (traffic per site does not depend on the lattice size)
TRAFFIC = {('sap_sweep_fp32', 'a4045b474347', 4, '48x48x48x96'): 41716159920.0}


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


def extrapolation_note(wlb):
    """How the oracle's 16^4 timing stands for a larger lattice: the cost of
    a solve grows with the volume V and the samples needed for the same
    relative eps shrink with it (the variance ||offdiag(D^-1)||_F^2 and
    |tr(D^-1)| are both extensive), so the time to variance carries over
    unchanged; the oracle's iterations per solve at 16^4 are a lower bound
    for the larger, more ill-conditioned lattice."""
    if wlb is None or tuple(wlb['dims']) == DIMS:
        return ''
    r = float(np.prod(wlb['dims'])) / float(np.prod(DIMS))
    return ('; extrapolated to %s: cost per solve x %.0f (volume), samples for the same relative eps / %.0f '
            '(variance and |tr| extensive), so the same time; the 16^4 iteration count is a lower bound there'
            % ('x'.join(map(str, wlb['dims'])), r, r))


def cpu_baseline(m0, wl, threads, wlb=None):
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
                      'oracle variance%s' % (threads, sT['seconds'], np.mean(wl['oracle_plain']['gmres_iters']),
                                             extrapolation_note(wlb)),
            'seconds_per_solve': C, 'cpu_utilisation': sT['cpu_seconds'] / sT['seconds'],
            'single_core': {'value': v1, 'seconds_per_solve': C1, 'cycle_s': s1['seconds'],
                            'cpu_utilisation': s1['cpu_seconds'] / s1['seconds']},
            'threads_available': host_cores()}


def reference_arm(args, rank, world, wlb=None):
    """The FP64 CPU oracle on this host's cores, same metric and workload:
    each step one bounded sample (a 64-iteration GMRES cycle of the plain
    Hutchinson solve on the 16^4 system), the value its time to the same
    variance (carried over to a larger workload lattice by volume, see
    extrapolation_note)."""
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
              'per 1e-12 solve and the oracle variance %.4g (tests/golden/mass_16x16x16x16.json)%s'
              % (T, np.mean(wl['oracle_plain']['gmres_iters']), wl['oracle_plain']['var'],
                 extrapolation_note(wlb)))
    lat = 'x'.join(map(str, (wlb or {}).get('dims', DIMS)))
    util = float(np.mean([s['cpu_seconds'] / s['seconds'] for s in samples]))
    line = {'impl': 'reference', 'metric': METRIC, 'value': value, 'unit': 's', 'n_gpus': world,
            'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': 1e3 * float(np.mean(t)),
            'higher_is_better': False, 'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64',
            'data': 'synthetic',
            'config': {'workload': '%s Wilson-Dirac, SU(3) exp(i 0.4 H), m0 %.4f, plain Hutchinson with the '
                                   'FP64 CPU oracle (timed on the 16^4 system)' % (lat, wl['m0'])},
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
def term_counts(M, wl, kind, n_levels, fine_n=None, coarse_n=None):
    """Samples per term of one step: fine_n for the terms that solve on the
    fine level, coarse_n for the others (orthogonal order O_0.., F_0..,
    coarsest; oblique M_0.., coarsest; plain [0])."""
    f = wl['fine_n'] if fine_n is None else fine_n
    c = wl['coarse_n'] if coarse_n is None else coarse_n
    L = n_levels
    if kind == M.EST_ORTHOGONAL:
        return [f] + [c] * (L - 2) + [f] + [c] * (L - 2) + [c]
    if kind == M.EST_OBLIQUE:
        return [f] + [c] * (L - 2) + [c]
    return [f]


def build_context(M, torch, wl, stream, U=None, dims=None, blocks=None, ntv=None, gauge_seed=None):
    """A context on the workload's lattice (or the given one) with the gauge
    field, mass, FP32 solver and hierarchy; returns (ctx, setup seconds)."""
    dims = dims or wl['dims']
    ctx = M.mgmlmc_create(dims, stream)
    if U is not None:
        M.mgmlmc_set_gauge(ctx, U)
    else:
        M.mgmlmc_gen_gauge(ctx, wl['eps'], gauge_seed or wl['gauge_seed'])
    M.mgmlmc_set_mass(ctx, wl['m0'])
    M.mgmlmc_set_solver(ctx, precision=M.FP32, **wl['solver'])
    # the tensor-core (TF32) coarse stencil serves the preconditioner only
    M.mgmlmc_set_kernel_variant(ctx, M.VARIANT_STENCIL_FP32, wl['stencil_variant'])
    torch.cuda.synchronize()
    t0 = time.time()
    M.mgmlmc_build_hierarchy(ctx, M.mg_params(blocks or wl['blocks'], ntv or wl['ntv'],
                                               setup_rounds=wl['setup_rounds'], setup_iters=wl['setup_iters'],
                                               seed=wl['tv_seed']))
    torch.cuda.synchronize()
    return ctx, time.time() - t0


def train_network(M, torch, wl, ctx, stream, channels, steps, source=0):
    """The gauge-covariant network trained on the solver's own residuals
    (mgmlmc_learned_train).  Workloads with a `train` entry train on that
    smaller lattice of the same generator and carry the weights over to ctx
    (the layers act the same way on any lattice); returns (train result,
    wall seconds including the side context's setup)."""
    kw = dict(channels=channels, steps=steps, batch=8, pool=2000, lr=1e-3, seed=5002, source=source)
    t0 = time.time()
    if not wl['train']:
        res = M.mgmlmc_learned_train(ctx, **kw)
        return res, time.time() - t0
    tw = wl['train']
    side, _ = build_context(M, torch, wl, stream, dims=tw['dims'], blocks=tw['blocks'], ntv=tw['ntv'],
                            gauge_seed=tw['gauge_seed'])
    try:
        res = M.mgmlmc_learned_train(side, **kw)
        W = np.zeros(2 * M.mgmlmc_learned_size(side))
        M.mgmlmc_learned_weights(side, W, 0)
    finally:
        M.mgmlmc_destroy(side)
    M.mgmlmc_learned_init(ctx, channels, 5002)
    M.mgmlmc_learned_weights(ctx, W, 1)
    torch.cuda.synchronize()
    res = dict(res, trained_on=list(tw['dims']))
    return res, time.time() - t0


def roofline_of(kst, prof_ms, B, wl_name, M):
    """Roofline of the kernel class with the largest time in the profiled step."""
    dom = max(kst, key=lambda c: kst[c]['ms'])
    ks = kst[dom]
    if ks['launches'] == 0:
        return None
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
    roof['traffic'] = TRAFFIC.get((KERNELS[dom], kernel_source_hash(KERNELS[dom]), B, wl_name))
    roof.update(kernel=KERNELS[dom], launches=ks['launches'], avg_launch_us=ks['ms'] * 1e3 / ks['launches'],
                share_of_profiled_step=ks['ms'] / prof_ms, profiled_step_ms=prof_ms,
                algorithmic_bytes_per_launch=ks['bytes'] / ks['launches'],
                algorithmic_flops_per_launch=ks['flops'] / ks['launches'],
                fp32_alu_tflops=ks['flops'] / sec / 1e12,
                fp32_alu_frac=ks['flops'] / sec / 1e12 / FP32_PEAK_TFLOPS)
    return roof


def validate_allocation(M, ctx, det, kinds_n, est, B, val_s, eps_scale):
    """Sec. 2.2 / Eq. MLMC-Nl run for real: N_l = eps^-2 sqrt(V_l / C_l)
    sum_i sqrt(V_i C_i) fresh samples per term at eps_val = eps * eps_scale,
    eps_scale chosen so that the predicted cost is about val_s seconds.
    Returns the achieved standard error (from this run's own variances) and
    the measured device seconds beside eps_val and the prediction."""
    terms = sorted(det['terms'], key=lambda t: kinds_n.index(int(t)))
    V = np.array([det['terms'][t]['var'] for t in terms])
    C = np.array([det['terms'][t]['cost_s'] for t in terms])
    S = float(np.sum(np.sqrt(V * C)))
    if eps_scale:
        eps = det['eps'] * eps_scale
    else:
        eps = S / math.sqrt(val_s)  # predicted cost S^2 / eps^2 = val_s
    N = [max(2, int(math.ceil(math.sqrt(v / c) * S / eps ** 2))) if c > 0 else 2 for v, c in zip(V, C)]
    predicted = float(np.sum(np.array(N) * C))
    res = M.mgmlmc_estimate_trace(ctx, M.est_params(M.EST_ORTHOGONAL, N, batch=B, seed=est['seed'],
                                                    first_sample=VALIDATE_FIRST))
    secs = sum(r['seconds'] for r in res) * est['scale']
    se = math.sqrt(sum(r['var'] / r['n'] for r in res))
    tr = sum(complex(r['mean_re'], r['mean_im']) for r in res)
    return dict(eps_val=eps, n_l=N, predicted_s=predicted, measured_s=secs, achieved_se=se,
                se_over_eps=se / eps, trace=[tr.real, tr.imag])


def kernel_probe(M, torch, args):
    """One kernel class on a lattice small enough for a profiler capture (a
    few GB on the device) whose launches still move more than the L2 holds:
    `sap` (one smoothing call: smoother_steps SAP sweeps on level 0), `stencil`
    (the FP32 coarse stencil D_l of --probe-level in its selected variant),
    `dslash` (the FP32 Wilson operator).  --probe-variant and --probe-nrhs
    take comma lists; prints one line per (variant, nrhs) with the mean
    event-timed milliseconds per call."""
    dims = tuple(int(x) for x in args.probe_dims.split(','))
    variants = [int(v) for v in str(args.probe_variant).split(',')]
    nrhs_list = [int(v) for v in str(args.probe_nrhs).split(',')]
    stream = torch.cuda.current_stream()
    ctx = M.mgmlmc_create(dims, stream)
    try:
        M.mgmlmc_gen_gauge(ctx, 0.4, 1005)
        M.mgmlmc_set_mass(ctx, -0.40)
        M.mgmlmc_set_solver(ctx, precision=M.FP32, smoother=M.SMOOTHER_SAP, smoother_steps=1, sap_iters=4)
        level, op = 0, M.OP_D
        if args.kernel_probe == 'sap':
            op = M.OP_SMOOTH
        elif args.kernel_probe == 'stencil':
            # Z4 test vectors (no setup iterations): the stencil's cost does
            # not depend on their quality
            level = args.probe_level
            # 2^4 aggregates below the first level until the probed level
            # exists and the coarsest is small enough for its dense inverse
            blocks, ext = [(4, 4, 4, 4)], [d // 4 for d in dims]
            while len(blocks) <= level or (np.prod(ext) > 1000 and all(e % 2 == 0 for e in ext)):
                blocks.append((2, 2, 2, 2))
                ext = [e // 2 for e in ext]
            M.mgmlmc_build_hierarchy(ctx, M.mg_params(blocks, [16] * len(blocks), setup_rounds=0, seed=3005))
        for v in variants:
            if args.kernel_probe == 'sap':
                M.mgmlmc_set_kernel_variant(ctx, M.VARIANT_SAP_FP32, v)
            elif args.kernel_probe == 'stencil':
                M.mgmlmc_set_kernel_variant(ctx, M.VARIANT_STENCIL_FP32, v)
            else:
                M.mgmlmc_set_kernel_variant(ctx, M.VARIANT_DSLASH_FP32, v)
            for nrhs in nrhs_list:
                info = M.mgmlmc_level_info(ctx, level)
                n = info[2]
                x = torch.randn((nrhs, n), dtype=torch.complex64, device='cuda')
                y = torch.empty_like(x)
                lop = op | M.LAYOUT_INTERNAL if level == 0 else op  # internal order: the call is the kernel alone
                for _ in range(3):
                    M.mgmlmc_apply(ctx, lop, level, M.FP32, x, y, nrhs)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(args.probe_reps):
                    M.mgmlmc_apply(ctx, lop, level, M.FP32, x, y, nrhs)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / args.probe_reps
                print(json.dumps({'kernel_probe': args.kernel_probe, 'dims': list(dims), 'level': level,
                                  'sites': n // info[1], 'nrhs': nrhs,
                                  'variant': v, 'ms_per_call': ms}))
                del x, y
    finally:
        M.mgmlmc_destroy(ctx)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=4)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--workload', default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument('--batch', type=int, default=None, help='samples per coarse term per step')
    ap.add_argument('--fine-n', type=int, default=None, help='samples per fine-level term per step')
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--precision', default='fp32', choices=['fp64', 'fp32'])
    ap.add_argument('--compare-steps', type=int, default=2)
    ap.add_argument('--no-cpu', action='store_true')
    ap.add_argument('--no-e2e', action='store_true')
    ap.add_argument('--no-dslash', action='store_true')
    ap.add_argument('--validate-s', type=float, default=20.0,
                    help='device seconds the allocation check may take (0: skip)')
    ap.add_argument('--m0', type=float, default=None, help='override the mass (exploration)')
    ap.add_argument('--solver', action='append', default=None, metavar='KEY=VALUE',
                    help='override one solver parameter of the workload (repeatable)')
    ap.add_argument('--gram-schmidt', type=int, default=None, choices=[1, 2],
                    help='classical Gram-Schmidt passes of the FP32 FGMRES (default: the workload\'s)')
    ap.add_argument('--learned', type=int, default=1, help='channels of the learned smoother (0: off)')
    ap.add_argument('--net-mode', default='guess', choices=['after-sap', 'replace-sap', 'guess'],
                    help='the network as one step after the SAP sweeps, in place of SAP, or as the initial '
                         'guess of the fine-level solves (SAP smoother)')
    ap.add_argument('--train-steps', type=int, default=200)
    ap.add_argument('--dslash-only', action='store_true', help='only the 32^4 FP32 Dslash measurement')
    ap.add_argument('--arms', default=None, help='comparison arms to run (comma list of %s)' % ', '.join(ARMS))
    ap.add_argument('--oracle-threads', type=int, default=0,
                    help='host threads of the CPU oracle timing (0: every core of this host)')
    ap.add_argument('--refine-iters', type=int, default=30,
                    help='cap on the test-vector refinement steps of the "refined" arm')
    ap.add_argument('--kernel-probe', default=None, choices=['sap', 'stencil', 'dslash'],
                    help='time one kernel class on a small lattice (profiler captures) and exit')
    ap.add_argument('--probe-dims', default='32,32,32,64')
    ap.add_argument('--probe-nrhs', default='4', help='right-hand sides of the probe, comma-separated')
    ap.add_argument('--probe-variant', default='0', help='kernel variant(s) of the probe, comma-separated')
    ap.add_argument('--probe-level', type=int, default=1, help='level of the stencil probe (1 or 2)')
    ap.add_argument('--probe-reps', type=int, default=5)
    ap.add_argument('--detail-out', default=os.environ.get('MGMLMC_BENCH_DETAIL'),
                    help='file for the full per-term and per-arm detail (the JSON line keeps a summary)')
    args = ap.parse_args()

    dist, rank, world, local = dist_init()
    wl = dict(WORKLOADS[args.workload])
    if args.gram_schmidt is not None:
        wl['solver'] = dict(wl['solver'], gram_schmidt_passes=args.gram_schmidt)
    for kv in args.solver or []:
        key, val = kv.split('=')
        if key not in wl['solver'] and key not in ('coarse_iters', 'coarse_smoother_steps', 'smoother_steps',
                                                    'restart', 'coarse_restart', 'sap_iters', 'inner_tol'):
            raise SystemExit('unknown solver parameter %s' % key)
        wl['solver'] = dict(wl['solver'], **{key: float(val) if key == 'inner_tol' else int(val)})
    if args.impl == 'reference':
        reference_arm(args, rank, world, wl)
        if dist:
            dist.destroy_process_group()
        return
    mass = workload()
    if wl['m0'] is None:
        wl['m0'] = mass['m0']
    if args.m0 is not None:
        wl['m0'] = args.m0
    if args.fine_n:
        wl['fine_n'] = args.fine_n
    if args.batch:
        wl['coarse_n'] = wl['batch'] = args.batch
        if wl['fine_n'] > args.batch:
            wl['fine_n'] = args.batch
    m0 = wl['m0']
    B = wl['batch']

    import torch
    from paper_2509_11424_gb300 import mgmlmc as M, synth
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    if args.kernel_probe:
        kernel_probe(M, torch, args)
        return
    U16 = synth.gauge_field(DIMS, EPS_GAUGE, GAUGE_SEED)
    if args.dslash_only:
        print(json.dumps({'dslash_hbm': dslash_hbm(M, torch, U16, mass['m0'])}))
        return
    # the metric's Dslash GB/s at 32^4, before the large context takes the memory
    dslash_32 = dslash_hbm(M, torch, U16, mass['m0']) if rank == 0 and not args.no_dslash else None

    prec = M.FP64 if args.precision == 'fp64' else M.FP32
    U = synth.gauge_field(wl['dims'], wl['eps'], wl['gauge_seed']) if wl['gauge'] == 'host' else None
    ctx, t_setup = build_context(M, torch, wl, stream, U=U)
    if prec == M.FP64:
        M.mgmlmc_set_solver(ctx, precision=prec, **wl['solver'])
    L = len(wl['blocks']) + 1
    train, t_train = None, 0.0
    main_solver = dict(wl['solver'])
    if args.learned > 0:
        guess = args.net_mode == 'guess'
        train, t_train = train_network(M, torch, wl, ctx, stream, args.learned, args.train_steps,
                                       source=1 if guess else 0)
        if guess:
            main_solver['learned_guess'] = 1
        else:
            main_solver['smoother'] = M.SMOOTHER_LEARNED if args.net_mode == 'after-sap' else M.SMOOTHER_NET
        M.mgmlmc_set_solver(ctx, precision=prec, **main_solver)
    print('kernel launches after setup: %d' % M.mgmlmc_kernel_launches(), file=sys.stderr)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device='cuda')  # 256 MB > L2
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nseed = wl['noise_seed']

    def step(k, kind=M.EST_ORTHOGONAL, fine_n=None, coarse_n=None):
        n = term_counts(M, wl, kind, L, fine_n, coarse_n)
        return M.mgmlmc_estimate_trace(ctx, M.est_params(kind, n, batch=B, seed=nseed,
                                                         first_sample=first_sample(rank, k, B)))

    def timed(k0, K, kind=M.EST_ORTHOGONAL, **kw):
        res, ms = [], 0.0
        for k in range(K):
            flush.zero_()
            e0.record(stream)
            res.append(step(k0 + k, kind, **kw))
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
    torch.cuda.profiler.start()
    results, total_ms = timed(args.warmup, args.steps)
    torch.cuda.profiler.stop()
    launches = M.mgmlmc_kernel_launches() - n_launch0
    clk = clocks.stop()
    if train is not None:
        train['fallbacks'] = M.mgmlmc_learned_stats(ctx)
    if dist:
        total_ms = max_over_ranks(dist, total_ms, 'cuda')
    ms_per_step = total_ms / args.steps
    acc = merge_terms(results)
    if dist:
        allreduce_terms(dist, acc, world, 'cuda')
    value, det = time_to_variance(acc, world, ms_per_step, args.steps)
    # device seconds of the library's per-term timers -> wall step time
    dev_sec = sum(acc[t]['sec'] for t in acc)
    scale = (ms_per_step * 1e-3 * args.steps) / dev_sec if dev_sec > 0 else 1.0

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
    roof = roofline_of(kst, prof_ms, wl['fine_n'], args.workload, M)
    dslash = None
    ws = kst[1] if prec == M.FP32 else kst[0]
    if ws['launches'] > 0:
        peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
        gbs = ws['bytes'] / (ws['ms'] * 1e-3) / 1e9
        dslash = dict(kernel=KERNELS[1 if prec == M.FP32 else 0], achieved_gbs=gbs,
                      frac_of_measured_hbm=gbs / peaks['hbm_gbs'] if 'hbm_gbs' in peaks else None,
                      avg_launch_us=ws['ms'] * 1e3 / ws['launches'], launches=ws['launches'])

    # the optimal allocation run for real at a coarser eps (bounded time)
    check = None
    if rank == 0 and args.validate_s > 0:
        order = [r['term'] for r in results[0]]
        check = validate_allocation(M, ctx, det, order, dict(seed=nseed, scale=scale), B, args.validate_s, None)

    compare = {}
    arms = set((args.arms or ','.join(wl['arms'])).split(',')) - {''}
    if arms - set(ARMS):
        raise SystemExit('unknown arms: %s' % ', '.join(sorted(arms - set(ARMS))))
    k0 = args.warmup  # the timed run's first sample batch: identical noise
    cs = args.compare_steps
    eps0 = det['eps']
    big = args.workload != '16x16x16x16'
    if rank == 0 and cs > 0:
        mvar = {t: v['var'] for t, v in det['terms'].items()}
        pvar = None
        if arms & {'plain', 'fp64'}:
            pres, pms = timed(k0, cs, M.EST_PLAIN)
            pval, pdet = time_to_variance(merge_terms(pres), 1, pms / cs, cs, eps=eps0)
            if 'plain' in arms:
                compare['plain_hutchinson_same_solver'] = dict(value=pval, ms_per_step=pms / cs, detail=pdet)
            pvar = {t: v['var'] for t, v in pdet['terms'].items()}
        # the paper's earlier decomposition (Eq. oblique_multigrid-multilevel-monte-carlo)
        if 'oblique' in arms:
            ores, oms = timed(k0, cs, M.EST_OBLIQUE)
            oval, odet = time_to_variance(merge_terms(ores), 1, oms / cs, cs, eps=eps0)
            compare['mlmc_oblique_same_solver'] = dict(value=oval, ms_per_step=oms / cs, detail=odet)
        # inexact deflation (Sec. 2.1; the paper's setting of Sec. 4.2)
        if 'deflated' in arms and not big:
            dex, dsec = M.mgmlmc_deflation_build(ctx, 128, 5, 1e-6, wl['tv_seed'] + 4000)
            dres, dms = timed(k0, cs, M.EST_DEFLATED)
            dacc = {t: a for t, a in merge_terms(dres).items() if t == M.TERM_DEFL}
            dval, ddet = time_to_variance(dacc, 1, dms / cs, cs, eps=eps0)
            compare['deflated_hutchinson_same_solver'] = dict(
                value=dval, ms_per_step=dms / cs, setup_s=dsec, exact_part=[dex.real, dex.imag],
                value_with_setup=dval + dsec, detail=ddet)
        if args.learned > 0 and 'sap' in arms:
            M.mgmlmc_set_solver(ctx, precision=prec, **wl['solver'])
            step(k0)
            sres, sms = timed(k0, cs)
            sval, sdet = time_to_variance(merge_terms(sres), 1, sms / cs, cs, var_of=mvar, eps=eps0)
            compare['mlmc_same_precision_sap_only'] = dict(value=sval, ms_per_step=sms / cs, detail=sdet)
        if prec == M.FP32 and 'fp64' in arms:
            # all-FP64 MG-MLMC (the plain method on this GPU), SAP smoother:
            # the same samples, fewer per step on a large lattice (FP64
            # Krylov bases); the costs per sample enter with the variances of
            # the main run
            M.mgmlmc_release_workspaces(ctx)
            M.mgmlmc_set_solver(ctx, precision=M.FP64, **dict(wl['solver'], fine_batch=wl['fp64_fine_n']))
            fn, cn = wl['fp64_fine_n'], wl['fp64_coarse_n']
            fcs = 1 if big else cs
            if not big:
                step(k0, fine_n=fn, coarse_n=cn)
            fres, fms = timed(k0, fcs, fine_n=fn, coarse_n=cn)
            fval, fdet = time_to_variance(merge_terms(fres), 1, fms / fcs, fcs, var_of=mvar, eps=eps0)
            fp64_samples = [M.mgmlmc_last_samples(ctx, i, r['n']) for i, r in enumerate(fres[-1])]
            compare['mlmc_fp64'] = dict(value=fval, ms_per_step=fms / fcs, steps=fcs, fine_n=fn, coarse_n=cn,
                                        detail=fdet)
            if not big:
                pres, pms = timed(k0, 1, M.EST_PLAIN)
                p64, _ = time_to_variance(merge_terms(pres), 1, pms, 1, var_of=pvar, eps=eps0)
                compare['plain_hutchinson_fp64'] = dict(value=p64, ms_per_step=pms)
            M.mgmlmc_release_workspaces(ctx)
            # the learned + mixed solver on the FP64 arm's last samples: the
            # largest relative difference of the per-sample values, per term
            M.mgmlmc_set_solver(ctx, precision=prec, **main_solver)
            step(k0 + fcs - 1, fine_n=fn, coarse_n=cn)
            rel = {}
            for i, xf in enumerate(fp64_samples):
                xm = M.mgmlmc_last_samples(ctx, i, len(xf))
                rel[str(fres[-1][i]['term'])] = float(np.max(np.abs(xm - xf)) / max(np.max(np.abs(xf)), 1e-300))
            compare['mlmc_fp64']['mixed_vs_fp64_max_rel_diff'] = rel
        M.mgmlmc_set_solver(ctx, precision=prec, **main_solver)

    e2e = None
    if not args.no_e2e and rank == 0:
        # the whole job through the ABI, wall clock: the gauge field from
        # pinned host memory, the hierarchy, the network weights, then
        # estimate_trace calls (each returns its term results to the host);
        # network training enters with its measured wall time
        Uh = torch.empty(int(np.prod(wl['dims'])) * 72, dtype=torch.float64).pin_memory()
        M.mgmlmc_get_gauge(ctx, Uh.numpy(), on_device=False)
        W = None
        if args.learned > 0:
            W = np.zeros(2 * M.mgmlmc_learned_size(ctx))
            M.mgmlmc_learned_weights(ctx, W, 0)
        torch.cuda.synchronize()
        t0 = time.time()
        M.mgmlmc_set_gauge(ctx, Uh.numpy(), on_device=False)
        M.mgmlmc_set_mass(ctx, m0)
        M.mgmlmc_build_hierarchy(ctx, M.mg_params(wl['blocks'], wl['ntv'], setup_rounds=wl['setup_rounds'],
                                                  setup_iters=wl['setup_iters'], seed=wl['tv_seed']))
        if W is not None:
            M.mgmlmc_learned_weights(ctx, W, 1)
        torch.cuda.synchronize()
        t_build = time.time() - t0
        t1 = time.time()
        step(40000)
        t_first = time.time() - t1
        t1 = time.time()
        for k in range(E2E_STEPS):
            step(40001 + k)
        step_s = (time.time() - t1) / E2E_STEPS
        nterm = len(results[0])
        e2e = dict(value=t_train + e2e_time_to_variance(t_build, t_first, step_s, value, ms_per_step * 1e-3),
                   unit='s', h2d_bytes_per_step=0,
                   d2h_bytes_per_step=int(16 * sum(term_counts(M, wl, M.EST_ORTHOGONAL, L)) + 88 * nterm),
                   setup_h2d_bytes=int(Uh.numel() * 8), setup_s=t_build, train_s=t_train, first_step_s=t_first,
                   step_s=step_s, steps=E2E_STEPS)
        del Uh

    # Sec. 5 (16^4 workload): test vectors computed to a small eigen-residual
    if rank == 0 and cs > 0 and not big and 'refined' in arms and args.refine_iters > 0:
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
            eig_res_max=float(rh.max()), detail=rdet)
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
    if rank == 0 and world == 1 and not args.no_cpu and 'oracle_plain' in mass:
        cpu = cpu_baseline(mass['m0'], mass, oracle_threads(args.oracle_threads), wl)

    if rank == 0:
        full = dict(detail=det, compare=compare, dslash_hbm=dslash_32, kernel_stats={KERNELS[c]: kst[c] for c in kst},
                    group_stats=gst, learned=train, validation=check, roofline=roof, e2e=e2e, cpu_baseline=cpu)
        if args.detail_out:
            with open(args.detail_out, 'w') as f:
                json.dump(full, f, indent=1)
        print(json.dumps(compact_line(args, wl, world, value, ms_per_step, launches, clk, det, compare,
                                      dslash_32, dslash, roof, check, train, M, prec, e2e, cpu, t_setup, kst,
                                      gst, prof_ms)))
    M.mgmlmc_destroy(ctx)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def _r(x, d=4):
    """Round for the compact line (significant digits)."""
    if x is None or not isinstance(x, float) or x == 0 or not math.isfinite(x):
        return x
    return float('%.*g' % (d, x))


def compact_line(args, wl, world, value, ms_per_step, launches, clk, det, compare, dslash_32, dslash, roof,
                 check, train, M, prec, e2e, cpu, t_setup, kst, gst, prof_ms):
    """The one JSON line: the summaries first, the contract's keys last (the
    driver keeps the line's tail); the full detail goes to --detail-out."""
    terms = {t: [_r(v['mean'][0], 7), _r(v['var']), _r(v['cost_s']), v['n'], _r(v['iters'], 3)]
             for t, v in det['terms'].items()}
    arms = {k: dict(value=_r(v.get('value')), ms_per_step=_r(v.get('ms_per_step')),
                    **({'error': v['error']} if 'error' in v else {}),
                    **({'mixed_vs_fp64_max_rel_diff': {t: _r(x, 2) for t, x in v['mixed_vs_fp64_max_rel_diff'].items()}}
                       if 'mixed_vs_fp64_max_rel_diff' in v else {}),
                    **({'setup_s': _r(v['setup_s'])} if 'setup_s' in v else {}))
            for k, v in compare.items()}
    ds = None
    if dslash_32:
        ds = {k: dict(gbs=_r(v['achieved_gbs']), frac=_r(v['frac_of_measured_hbm'], 3))
              for k, v in dslash_32.items() if isinstance(v, dict)}
    lat = 'x'.join(str(d) for d in wl['dims'])
    line = {
        'terms': terms, 'terms_key': '[mean_re, var, cost_s, n, iters]',
        'group_ms': {k: _r(v['ms']) for k, v in gst.items()},
        'kernel_ms': {k: _r(kst[c]['ms']) for c, k in KERNELS.items() if kst[c]['launches']},
        'profiled_step_ms': _r(prof_ms),
        'learned': (dict(channels=args.learned, mode=args.net_mode, loss_init=_r(train['loss_init']),
                         loss_last=_r(train['loss_last']),
                         pairs=train['pairs'], trained_on=train.get('trained_on'),
                         fallbacks=train.get('fallbacks')) if train else None),
        'setup_s': _r(t_setup),
        'dslash_hbm_32x32x32x32': ds,
        'dslash_in_step': dict(gbs=_r(dslash['achieved_gbs']), frac=_r(dslash['frac_of_measured_hbm'], 3),
                               launches=dslash['launches']) if dslash else None,
        'compare': arms,
        'mlmc_check': ({k: (_r(v) if isinstance(v, float) else v) for k, v in check.items() if k != 'trace'}
                       if check else None),
        'metric': METRIC, 'value': value, 'unit': 's', 'n_gpus': world, 'steps': args.steps,
        'warmup': args.warmup, 'ms_per_step': ms_per_step, 'higher_is_better': False, 'scaling': 'weak',
        'vs_baseline': None, 'dtype': 'f64' if prec == M.FP64 else 'f32+f64', 'data': 'synthetic',
        'config': {'workload': '%s Wilson-Dirac, SU(3) exp(i %.1f H) seed %d (%s), m0 %.4f, orthogonal MG-MLMC %d '
                               'levels (%s aggregates, %s tv), SAP%s-MG FGMRES(%d) in FP64 defect correction, Z4 '
                               '%d samples per fine-level term and %d per coarse term per step, fine solves in '
                               'blocks of %d rhs, all solves to 1e-12'
                               % (lat, wl['eps'], wl['gauge_seed'], 'device generator' if wl['gauge'] == 'device'
                                  else 'host', wl['m0'], len(wl['blocks']) + 1,
                                  ', '.join('%d^4' % b[0] for b in wl['blocks']), '/'.join(map(str, wl['ntv'])),
                                  ('' if not args.learned else ' + learned(%d ch)' % args.learned
                                   if args.net_mode == 'after-sap' else ' -> learned(%d ch) in place of SAP'
                                   % args.learned if args.net_mode == 'replace-sap'
                                   else ' + learned(%d ch) initial guess' % args.learned),
                                  wl['solver']['restart'], wl['fine_n'], wl['coarse_n'],
                                  wl['solver'].get('fine_batch') or wl['batch']),
                   'global_batch': sum(v['n'] for v in det['terms'].values()) // max(1, args.steps) * world,
                   'lattice': list(wl['dims']), 'rel_eps': REL_EPS,
                   'l2': 'flushed between steps (256 MB write); every fine-level launch moves > 1 GB',
                   'parallelism': 'samples sharded, dp%d' % world},
        'roofline': ({k: (_r(v) if isinstance(v, float) else v) for k, v in roof.items()} if roof else None),
        'clocks': clk, 'gpu_launches': launches,
        'e2e': ({k: (_r(v) if isinstance(v, float) else v) for k, v in e2e.items()} if e2e else None),
        'cpu_baseline': ({k: (_r(v) if isinstance(v, float) else v) for k, v in cpu.items()
                          if k not in ('single_core',)} if cpu else None),
    }
    return line


if __name__ == '__main__':
    main()
