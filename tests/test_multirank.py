"""The sharded multi-rank path of bench.py on the CPU: two gloo ranks.

Noise samples are independent, so ranks draw disjoint sample counters and
the only exchange is one all-reduce of the per-term accumulators (sums of N,
X, |X|^2, iterations and seconds; maximum of the residuals) plus the maximum
of the timed region.  Each rank here merges its own synthetic per-batch
results, the ranks reduce over gloo, and the merged statistics must equal
those of all batches merged on one process.
"""
import json
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip('torch')
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

TERMS = (16, 17, 32, 33, 48)


def batches(rank, steps=3):
    """Per-batch term results of one rank, as mgmlmc_estimate_trace returns
    them (seeded by rank so the ranks differ)."""
    rng = np.random.default_rng(100 + rank)
    out = []
    for _ in range(steps):
        res = []
        for t in TERMS:
            x = rng.normal(size=8) + 1j * rng.normal(size=8)
            res.append(dict(term=t, n=8, sum_re=float(x.real.sum()), sum_im=float(x.imag.sum()),
                            sum_abs2=float((abs(x) ** 2).sum()), seconds=float(rng.uniform(0.01, 0.02)),
                            iters_mean=float(rng.integers(10, 30)), max_residual=float(rng.uniform(1e-13, 9e-13))))
        out.append(res)
    return out


def worker(rank, world, port, outdir):
    os.environ['MASTER_ADDR'] = '127.0.0.1'
    os.environ['MASTER_PORT'] = str(port)
    dist.init_process_group('gloo', rank=rank, world_size=world)
    try:
        acc = bench.merge_terms(batches(rank))
        bench.allreduce_terms(dist, acc, world, 'cpu')
        t = bench.max_over_ranks(dist, 10.0 + rank, 'cpu')
        with open(os.path.join(outdir, 'rank%d.json' % rank), 'w') as f:
            json.dump(dict(acc={str(k): v for k, v in acc.items()}, t=t), f)
    finally:
        dist.destroy_process_group()


def free_port():
    s = socket.socket()
    s.bind(('127.0.0.1', 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_rank_reduction_equals_serial_merge(tmp_path):
    world = 2
    mp.start_processes(worker, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method='spawn')
    ranks = [json.load(open(tmp_path / ('rank%d.json' % r))) for r in range(world)]
    # every rank ends with the same merged accumulators and the maximum time
    assert ranks[0]['acc'] == ranks[1]['acc']
    assert ranks[0]['t'] == ranks[1]['t'] == 11.0
    serial = bench.merge_terms(batches(0) + batches(1))
    for t in TERMS:
        got, want = ranks[0]['acc'][str(t)], serial[t]
        assert got['n'] == want['n'] == 48
        for f in ('sre', 'sim', 'sab', 'it'):
            assert got[f] == pytest.approx(want[f], rel=1e-14)
        assert got['k'] == want['k']
        assert got['sec'] == pytest.approx(want['sec'] / world, rel=1e-14)
        assert got['res'] == want['res']
        mu_g, var_g = bench.stats_of(got)
        mu_w, var_w = bench.stats_of(want)
        assert mu_g == pytest.approx(mu_w, rel=1e-13) and var_g == pytest.approx(var_w, rel=1e-13)


def test_sample_counters_disjoint_across_ranks():
    B, steps = 8, 50
    seen = set()
    for rank in range(8):
        for k in range(steps):
            s0 = bench.first_sample(rank, k, B)
            block = set(range(s0, s0 + B))
            assert not (block & seen)
            seen |= block
    assert steps * B <= bench.SHARD_STRIDE
