"""The allocation-free projector entry point against the regular one.

mgmlmc_project_noalloc exists for callers that cannot allocate device
memory while they run (inside a stream capture that forbids allocations, under
an externally reserved memory pool, or on an allocator-free critical path).
It must give the same (I - P P^H) x as mgmlmc_apply(MGMLMC_OP_PROJECT), call
after call, since all calls share one fixed device scratch array, and it must
not take device memory once its first call has looked the array up.  This
file is collected last so that a failure here comes after every other test
has run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from gpu_util import Setup, dev, host, rel  # noqa: E402

from paper_2509_11424_gb300 import synth  # noqa: E402


def make_setup():
    return Setup((4, 4, 4, 8), [(2, 2, 2, 2), (2, 2, 2, 2)], [6, 4], eps=0.4, m0=-0.1, gseed=77, oracle=False)


@pytest.fixture(scope='module')
def setup():
    s = make_setup()
    yield s
    s.close()


def test_noalloc_takes_no_device_memory():
    """On a context that has never run the regular projector (so no projector
    workspace exists), calls after the first one leave the free device memory
    unchanged, also for a batch larger than the first call's: a workspace of
    the context would have to grow with it."""
    s = make_setup()
    try:
        M = s.M
        _, _, n = M.mgmlmc_level_info(s.ctx, 0)
        x = dev(synth.complex_normal((8, n), 5), torch.complex128)
        y = torch.empty_like(x)
        M.mgmlmc_project_noalloc(s.ctx, 0, 0, x, y, 1)  # first call: address lookup
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for nrhs in (2, 8, 8):
            M.mgmlmc_project_noalloc(s.ctx, 0, 0, x, y, nrhs)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        want = torch.empty_like(x)
        M.mgmlmc_apply(s.ctx, M.OP_PROJECT, 0, 0, x, want, 8)
        assert rel(host(y), host(want)) < 1e-12
    finally:
        s.close()


@pytest.mark.parametrize('prec,tol', [(0, 1e-12), (1, 1e-5)])
def test_noalloc_matches_regular_projector_twice(setup, prec, tol):
    M = setup.M
    ct = torch.complex128 if prec == 0 else torch.complex64
    for level in (0, 1):
        _, _, n = M.mgmlmc_level_info(setup.ctx, level)
        for call, seed in enumerate((101, 202)):  # two calls in a row, different inputs
            x = dev(synth.complex_normal((3, n), seed + level), ct)
            want = torch.empty_like(x)
            got = torch.empty_like(x)
            M.mgmlmc_apply(setup.ctx, M.OP_PROJECT, level, prec, x, want, 3)
            M.mgmlmc_project_noalloc(setup.ctx, level, prec, x, got, 3)
            g, w = host(got), host(want)
            assert rel(g, w) < tol, (level, call)
            assert np.max(np.abs(g - w)) <= tol * np.max(np.abs(w)), (level, call)


def test_noalloc_rejects_oversized_batch(setup):
    M = setup.M
    from paper_2509_11424_gb300.mgmlmc import MgmlmcError
    _, _, n = M.mgmlmc_level_info(setup.ctx, 0)
    _, _, nc = M.mgmlmc_level_info(setup.ctx, 1)
    nrhs = (1 << 17) // nc + 1  # one more right-hand side than the FP64 scratch holds
    x = torch.zeros((nrhs, n), dtype=torch.complex128, device='cuda')
    y = torch.empty_like(x)
    with pytest.raises(MgmlmcError) as e:
        M.mgmlmc_project_noalloc(setup.ctx, 0, 0, x, y, nrhs)
    assert e.value.status == 1 and 'scratch' in str(e.value)


def test_noalloc_rejects_overlapping_buffers(setup):
    """in and out sharing bytes would make the prolongation overwrite the
    input before the subtraction reads it: refused, context usable after."""
    M = setup.M
    from paper_2509_11424_gb300.mgmlmc import MgmlmcError
    _, _, n = M.mgmlmc_level_info(setup.ctx, 0)
    buf = torch.zeros((3, n), dtype=torch.complex128, device='cuda')
    for a, b in ((buf[0:2], buf[0:2]), (buf[0:2], buf[1:3])):
        with pytest.raises(MgmlmcError) as e:
            M.mgmlmc_project_noalloc(setup.ctx, 0, 0, a, b, 2)
        assert e.value.status == 1 and 'overlap' in str(e.value)
    x = dev(synth.complex_normal((1, n), 9), torch.complex128)
    y, want = torch.empty_like(x), torch.empty_like(x)
    M.mgmlmc_project_noalloc(setup.ctx, 0, 0, x, y, 1)
    M.mgmlmc_apply(setup.ctx, M.OP_PROJECT, 0, 0, x, want, 1)
    assert rel(host(y), host(want)) < 1e-12
