"""`bench.py --impl reference` (the oracle timed on the host) prints one JSON
line with the contract's keys, on the workload and metric of the GPU arm."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    env = dict(os.environ, OMP_NUM_THREADS='1')
    out = subprocess.run([sys.executable, os.path.join(ROOT, 'bench.py'), '--impl', 'reference',
                          '--steps', '1', '--warmup', '0', '--oracle-threads', '2'], capture_output=True,
                         text=True, env=env,
                         cwd=ROOT, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith('{')]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ('impl', 'metric', 'value', 'unit', 'n_gpus', 'steps', 'warmup', 'ms_per_step',
                'higher_is_better', 'scaling', 'vs_baseline', 'dtype', 'data', 'config', 'cpu_baseline',
                'e2e'):
        assert key in d, key
    assert d['impl'] == 'reference' and d['higher_is_better'] is False and d['value'] > 0
    assert d['cpu_baseline']['kind'] == 'oracle' and d['cpu_baseline']['value'] == d['value']
    assert d['cpu_baseline']['cores'] == 2
    assert d['e2e'] == {'value': d['value'], 'unit': d['unit'], 'h2d_bytes_per_step': 0,
                        'd2h_bytes_per_step': 0}
    import bench
    assert d['metric'] == bench.METRIC


def test_gpu_arm_cpu_baseline_object():
    """the GPU arm's cpu_baseline: the oracle on several host threads, with
    the single-thread figure beside it; more threads give more throughput."""
    import bench
    wl = bench.workload()
    c = bench.cpu_baseline(wl['m0'], wl, 2)
    assert c['kind'] == 'oracle' and c['cores'] == 2 and c['unit'] == 's'
    assert c['value'] > 0 and c['single_core']['value'] > 0
    assert c['value'] < c['single_core']['value']
    # (no upper bound here: inside pytest numpy's BLAS may already run
    # several threads; bench.py as a program pins it to one)
    assert c['cpu_utilisation'] > 0.5
