"""bench.py's time-to-variance (the headline metric) against the oracle's
MLMC allocation (Sec. 2.2, Eq. MLMC-Nl): for per-term accumulators with
known sample variances and costs, (sum_l sqrt(V_l C_l))^2 / eps^2 equals the
total cost of the optimal allocation, and the shared-variance option replaces
a run's variances and target exactly."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from oracle import estimators as oest  # noqa: E402


def _acc(X, sec):
    X = np.asarray(X)
    return dict(n=X.size, sre=X.real.sum(), sim=X.imag.sum(), sab=np.sum(np.abs(X) ** 2), sec=sec,
                it=10.0 * X.size, k=X.size, res=1e-13)


def test_time_to_variance_equals_optimal_allocation_cost():
    rng = np.random.default_rng(5)
    acc, V, C = {}, [], []
    for t, (mu, sd, sec) in enumerate([(100.0, 3.0, 0.8), (5.0, 1.0, 0.3), (-2.0, 0.4, 0.05)]):
        X = mu + sd * (rng.standard_normal(40) + 1j * rng.standard_normal(40))
        acc[t] = _acc(X, sec)
        V.append(oest.sample_stats(X)[1])
        C.append(sec / 40)
    step_ms = 1e3 * sum(a['sec'] for a in acc.values())  # measured time = device time
    val, det = bench.time_to_variance(acc, 1, step_ms, 1, rel_eps=1e-3)
    eps = det['eps']
    tr = sum(complex(a['sre'], a['sim']) / a['n'] for a in acc.values())
    assert abs(eps - 1e-3 * abs(tr)) < 1e-12 * eps
    _, cost = oest.mlmc_allocation(V, C, eps)
    assert abs(val - cost) < 1e-10 * cost
    # host gaps: a measured step twice the device time doubles every C_l
    val2, _ = bench.time_to_variance(acc, 1, 2 * step_ms, 1, rel_eps=1e-3)
    assert abs(val2 - 2 * val) < 1e-10 * val
    # shared variances and target
    var_of = {str(t): 4.0 * V[t] for t in acc}
    val3, det3 = bench.time_to_variance(acc, 1, step_ms, 1, var_of=var_of, eps=2 * eps)
    assert abs(val3 - cost) < 1e-10 * cost  # 4x variance, 2x eps
    assert det3['eps'] == 2 * eps


def test_e2e_time_to_variance():
    """end-to-end time = setup + the first step's one-time extra + the
    device-timed estimate rescaled to the end-to-end step cost."""
    import bench
    # steps at exactly the device cost: setup + first-step extra + value
    assert bench.e2e_time_to_variance(2.0, 0.5, 0.4, 70.0, 0.4) == 2.0 + 0.1 + 70.0
    # end-to-end steps 10% dearer than on the device
    assert abs(bench.e2e_time_to_variance(1.0, 0.44, 0.44, 50.0, 0.4) - (1.0 + 55.0)) < 1e-12
    # a first step faster than the steady ones adds nothing
    assert bench.e2e_time_to_variance(0.0, 0.1, 0.4, 10.0, 0.4) == 10.0


def test_oracle_threads_bounded_by_memory(monkeypatch):
    """the CPU oracle's worker count: every core by default, an explicit
    request as given, and never more than the free memory holds."""
    import bench
    monkeypatch.setattr(bench, 'host_cores', lambda: 16)
    monkeypatch.setattr(bench, 'host_memory_available', lambda: None)
    assert bench.oracle_threads(0) == 16 and bench.oracle_threads(3) == 3
    monkeypatch.setattr(bench, 'host_memory_available', lambda: 8e9 + 4.5 * bench.ORACLE_WORKER_BYTES)
    assert bench.oracle_threads(0) == 4
    monkeypatch.setattr(bench, 'host_memory_available', lambda: 1e9)
    assert bench.oracle_threads(0) == 1
    assert bench.host_cores() == 16


def test_roofline_class_and_traffic_lookup():
    """The roofline object: the class with the largest event time is the
    dominant kernel; achieved = algorithmic bytes / event seconds against the
    HBM peak; traffic is the recorded ncu figure only while the kernel's
    source hash and the workload match (null otherwise)."""
    names = {v: k for k, v in bench.KERNELS.items()}
    kst = {c: dict(launches=0, ms=0.0, bytes=0.0, flops=0.0) for c in bench.KERNELS}
    kst[names['sap_sweep_fp32']] = dict(launches=10, ms=150.0, bytes=10 * 35.67e9, flops=10 * 2.614e11)
    kst[names['coarse_stencil_fp32']] = dict(launches=100, ms=100.0, bytes=100 * 1.5e9, flops=1e12)
    roof = bench.roofline_of(kst, 600.0, 4, '48x48x48x96', None)
    assert roof['kernel'] == 'sap_sweep_fp32' and roof['bound'] == 'hbm'
    assert abs(roof['achieved'] - 35.67e9 / 15e-3 / 1e9) < 1e-6 * roof['achieved']
    assert abs(roof['frac'] - roof['achieved'] / roof['peak']) < 1e-12
    assert abs(roof['share_of_profiled_step'] - 0.25) < 1e-12
    key = ('sap_sweep_fp32', bench.kernel_source_hash('sap_sweep_fp32'), 4, '48x48x48x96')
    assert roof['traffic'] == bench.TRAFFIC.get(key)
    # another lattice or batch has no recorded traffic
    assert bench.roofline_of(kst, 600.0, 4, '16x16x16x16', None)['traffic'] is None
    assert bench.roofline_of(kst, 600.0, 8, '48x48x48x96', None)['traffic'] is None
