"""ctypes binding of libmgmlmc.so (include/mgmlmc.h): the same entry points
under the same names, argument marshalling only.

Buffers may be torch tensors (host or CUDA; their data_ptr() is passed),
numpy arrays (host) or raw integer addresses.  Every call raises
MgmlmcError carrying the library's status and last error message when the
status is not MGMLMC_OK.  There is no fallback: if the shared library is not
built the first call raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, 'libmgmlmc.so')

MAX_LEVELS = 4
FP64, FP32, BF16 = 0, 1, 2
EST_PLAIN, EST_ORTHOGONAL, EST_OBLIQUE, EST_DEFLATED = 0, 1, 2, 3
OP_D, OP_RESTRICT, OP_PROLONG, OP_PROJECT, OP_SOLVE, OP_GAMMA5, OP_SMOOTH, OP_NET = range(8)
TERM_PLAIN, TERM_O, TERM_F, TERM_COARSEST, TERM_M = 0, 16, 32, 48, 144
TERM_DEFL, TERM_DEFL_EXACT, TERM_DEFL_START = 160, 161, 176
TERM_TV_EXTRA = 192
STATUS = {0: 'OK', 1: 'ERR_ARG', 2: 'ERR_STATE', 3: 'ERR_OOM', 4: 'ERR_CUDA',
          5: 'ERR_NOT_CONVERGED', 6: 'ERR_NUMERIC'}


class MgParams(ctypes.Structure):
    _fields_ = [('n_levels', ctypes.c_int),
                ('block', (ctypes.c_int * 4) * (MAX_LEVELS - 1)),
                ('n_tv', ctypes.c_int * (MAX_LEVELS - 1)),
                ('setup_rounds', ctypes.c_int),
                ('setup_iters', ctypes.c_int),
                ('seed', ctypes.c_uint64)]


class SolverParams(ctypes.Structure):
    _fields_ = [('tol', ctypes.c_double),
                ('max_iter', ctypes.c_int),
                ('restart', ctypes.c_int),
                ('smoother_steps', ctypes.c_int),
                ('coarse_iters', ctypes.c_int),
                ('precision', ctypes.c_int),
                ('inner_tol', ctypes.c_double),
                ('smoother', ctypes.c_int),
                ('sap_iters', ctypes.c_int),
                ('coarse_smoother_steps', ctypes.c_int),
                ('coarse_restart', ctypes.c_int),
                ('post_smoothing_only', ctypes.c_int),
                ('gram_schmidt_passes', ctypes.c_int),
                ('fine_batch', ctypes.c_int),
                ('learned_guess', ctypes.c_int)]


class EstParams(ctypes.Structure):
    _fields_ = [('kind', ctypes.c_int),
                ('n_samples', ctypes.c_int * (2 * MAX_LEVELS)),
                ('batch', ctypes.c_int),
                ('seed', ctypes.c_uint64),
                ('first_sample', ctypes.c_uint64)]


class TermResult(ctypes.Structure):
    _fields_ = [('term', ctypes.c_int), ('n', ctypes.c_int),
                ('mean_re', ctypes.c_double), ('mean_im', ctypes.c_double),
                ('var', ctypes.c_double),
                ('sum_re', ctypes.c_double), ('sum_im', ctypes.c_double),
                ('sum_abs2', ctypes.c_double),
                ('seconds', ctypes.c_double), ('iters_mean', ctypes.c_double),
                ('max_residual', ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class TrainParams(ctypes.Structure):
    _fields_ = [('channels', ctypes.c_int), ('steps', ctypes.c_int), ('batch', ctypes.c_int),
                ('pool', ctypes.c_int), ('lr', ctypes.c_double), ('seed', ctypes.c_uint64),
                ('source', ctypes.c_int)]


class TrainResult(ctypes.Structure):
    _fields_ = [('steps', ctypes.c_int), ('pairs', ctypes.c_int), ('loss_init', ctypes.c_double),
                ('loss_first', ctypes.c_double), ('loss_last', ctypes.c_double),
                ('seconds', ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class MgmlmcError(RuntimeError):
    def __init__(self, status, message):
        super().__init__('%s: %s' % (STATUS.get(status, status), message))
        self.status = status


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_U64 = ctypes.c_uint64
_I64 = ctypes.c_int64
_D = ctypes.c_double

_SIGNATURES = {
    'mgmlmc_create': [ctypes.POINTER(_I), _P, ctypes.POINTER(_P)],
    'mgmlmc_destroy': [_P],
    'mgmlmc_last_error': [_P],
    'mgmlmc_set_gauge': [_P, _P, _I],
    'mgmlmc_set_mass': [_P, _D],
    'mgmlmc_set_solver': [_P, ctypes.POINTER(SolverParams)],
    'mgmlmc_set_test_vectors': [_P, _I, _P, _I, _I64, _I],
    'mgmlmc_build_hierarchy': [_P, ctypes.POINTER(MgParams)],
    'mgmlmc_level_info': [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I64)],
    'mgmlmc_estimate_trace': [_P, ctypes.POINTER(EstParams), ctypes.POINTER(TermResult), _I,
                              ctypes.POINTER(_I)],
    'mgmlmc_coarsest_trace': [_P, ctypes.POINTER(_D), ctypes.POINTER(_D)],
    'mgmlmc_last_samples': [_P, _I, _P, _I, ctypes.POINTER(_I)],
    'mgmlmc_release_workspaces': [_P],
    'mgmlmc_get_gauge': [_P, _P, _I],
    'mgmlmc_test_staging_extra': [_P, _I],
    'mgmlmc_connected_correlator': [_P, _I, _I, _U64, _U64, _P, _P, ctypes.POINTER(_I)],
    'mgmlmc_disconnected_loop': [_P, _I, _I, _I, _U64, _U64, _P, _P, ctypes.POINTER(_I)],
    'mgmlmc_apply': [_P, _I, _I, _I, _P, _P, _I],
    'mgmlmc_noise': [_P, _I, _U64, _U64, _U64, _U64, _I, _P, _I],
    'mgmlmc_get_prolongator': [_P, _I, _P],
    'mgmlmc_get_test_vectors': [_P, _I, _P],
    'mgmlmc_get_coarse_op': [_P, _I, _P],
    'mgmlmc_last_solve_stats': [_P, ctypes.POINTER(_I), ctypes.POINTER(_D)],
    'mgmlmc_profile': [_P, _I],
    'mgmlmc_kernel_launches': [],
    'mgmlmc_project_noalloc': [_P, _I, _I, _P, _P, _I],
    'mgmlmc_learned_init': [_P, _I, _U64],
    'mgmlmc_learned_size': [_P, ctypes.POINTER(_I64)],
    'mgmlmc_learned_weights': [_P, _P, _I],
    'mgmlmc_learned_loss_grad': [_P, _P, _I, ctypes.POINTER(_D), _P],
    'mgmlmc_learned_train': [_P, ctypes.POINTER(TrainParams), ctypes.POINTER(TrainResult)],
    'mgmlmc_learned_stats': [_P, ctypes.POINTER(_I64)],
    'mgmlmc_profile_stats': [_P, _I, ctypes.POINTER(_I64), ctypes.POINTER(_D), ctypes.POINTER(_D),
                             ctypes.POINTER(_D)],
    'mgmlmc_set_kernel_variant': [_P, _I, _I],
    'mgmlmc_gen_gauge': [_P, _D, _U64],
    'mgmlmc_deflation_build': [_P, _I, _I, _D, _U64, _P, ctypes.POINTER(_D)],
    'mgmlmc_refine_test_vectors': [_P, _I, _I, _I, _D, _D, _U64, _P, _P, ctypes.POINTER(_I)],
    'mgmlmc_reorder': [_P, _P, _P, _I, _I],
    'mgmlmc_reorder_bf16': [_P, _P, _P, _I, _I],
    'mgmlmc_kernel_variants': [_I],
    'mgmlmc_get_kernel_variant': [_P, _I, _I, ctypes.POINTER(_I)],
}


def lib():
    """The loaded shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError('libmgmlmc.so is not built (run paper_2509_11424_gb300.build.build())')
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = None if name == 'mgmlmc_destroy' else (
                ctypes.c_char_p if name == 'mgmlmc_last_error' else (
                    ctypes.c_int64 if name == 'mgmlmc_kernel_launches' else ctypes.c_int))
        _lib = L
    return _lib


def ptr(buf):
    """Address of a torch tensor, numpy array or integer."""
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    if hasattr(buf, 'data_ptr'):
        return buf.data_ptr()
    if isinstance(buf, np.ndarray):
        if not buf.flags['C_CONTIGUOUS']:
            raise ValueError('numpy buffers must be C-contiguous')
        return buf.ctypes.data
    raise TypeError('unsupported buffer type %r' % type(buf))


def _check(ctx, status):
    if status != 0:
        msg = lib().mgmlmc_last_error(ctx)
        raise MgmlmcError(status, msg.decode() if msg else '')


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


# ---------------------------------------------------------------- entry points
def mgmlmc_create(dims, stream=None):
    d = (_I * 4)(*[int(v) for v in dims])
    out = _P()
    st = lib().mgmlmc_create(d, _stream_handle(stream), ctypes.byref(out))
    if st != 0:
        raise MgmlmcError(st, lib().mgmlmc_last_error(None).decode())
    return out.value


def mgmlmc_destroy(ctx):
    lib().mgmlmc_destroy(ctx)


def mgmlmc_last_error(ctx):
    return lib().mgmlmc_last_error(ctx).decode()


def mgmlmc_set_gauge(ctx, U, on_device=None):
    if on_device is None:
        on_device = bool(getattr(U, 'is_cuda', False))
    _check(ctx, lib().mgmlmc_set_gauge(ctx, ptr(U), int(on_device)))


def mgmlmc_set_mass(ctx, m0):
    _check(ctx, lib().mgmlmc_set_mass(ctx, float(m0)))


SMOOTHER_MR, SMOOTHER_SAP, SMOOTHER_LEARNED, SMOOTHER_NET = 0, 1, 2, 3


def solver_params(tol=1e-12, max_iter=2000, restart=16, smoother_steps=4, coarse_iters=8,
                  precision=FP64, inner_tol=1e-6, smoother=SMOOTHER_MR, sap_iters=4,
                  coarse_smoother_steps=4, coarse_restart=0, post_smoothing_only=0, gram_schmidt_passes=0,
                  fine_batch=0, learned_guess=0):
    return SolverParams(tol, max_iter, restart, smoother_steps, coarse_iters, precision, inner_tol,
                        smoother, sap_iters, coarse_smoother_steps, coarse_restart, post_smoothing_only,
                        gram_schmidt_passes, fine_batch, learned_guess)


def mgmlmc_set_solver(ctx, params=None, **kw):
    p = params if params is not None else solver_params(**kw)
    _check(ctx, lib().mgmlmc_set_solver(ctx, ctypes.byref(p)))


def mgmlmc_set_test_vectors(ctx, level, V, n_tv, n, on_device=None):
    if on_device is None:
        on_device = bool(getattr(V, 'is_cuda', False))
    _check(ctx, lib().mgmlmc_set_test_vectors(ctx, level, ptr(V), n_tv, n, int(on_device)))


def mg_params(blocks, n_tv, setup_rounds=3, setup_iters=20, seed=3000):
    p = MgParams()
    p.n_levels = len(blocks) + 1
    for l, b in enumerate(blocks):
        for i in range(4):
            p.block[l][i] = int(b[i])
        p.n_tv[l] = int(n_tv[l])
    p.setup_rounds = setup_rounds
    p.setup_iters = setup_iters
    p.seed = seed
    return p


def mgmlmc_build_hierarchy(ctx, params):
    _check(ctx, lib().mgmlmc_build_hierarchy(ctx, ctypes.byref(params)))


def mgmlmc_level_info(ctx, level):
    d = (_I * 4)()
    dof = _I()
    n = _I64()
    _check(ctx, lib().mgmlmc_level_info(ctx, level, d, ctypes.byref(dof), ctypes.byref(n)))
    return tuple(d), dof.value, n.value


def est_params(kind, n_samples, batch=8, seed=2000, first_sample=0):
    p = EstParams()
    p.kind = kind
    for i, v in enumerate(n_samples):
        p.n_samples[i] = int(v)
    p.batch = batch
    p.seed = seed
    p.first_sample = first_sample
    return p


def mgmlmc_estimate_trace(ctx, params):
    out = (TermResult * (2 * MAX_LEVELS))()
    nt = _I()
    _check(ctx, lib().mgmlmc_estimate_trace(ctx, ctypes.byref(params), out, 2 * MAX_LEVELS,
                                            ctypes.byref(nt)))
    return [out[i].as_dict() for i in range(nt.value)]


def mgmlmc_last_samples(ctx, index, max_samples):
    out = np.zeros(2 * max(1, max_samples))
    n = _I()
    _check(ctx, lib().mgmlmc_last_samples(ctx, index, ptr(out), max_samples, ctypes.byref(n)))
    return out[:2 * n.value].view(np.complex128).copy()


def mgmlmc_get_gauge(ctx, U, on_device=None):
    if on_device is None:
        on_device = bool(getattr(U, 'is_cuda', False))
    _check(ctx, lib().mgmlmc_get_gauge(ctx, ptr(U), int(on_device)))


def mgmlmc_test_staging_extra(ctx, extra_bytes):
    _check(ctx, lib().mgmlmc_test_staging_extra(ctx, extra_bytes))


def mgmlmc_release_workspaces(ctx):
    _check(ctx, lib().mgmlmc_release_workspaces(ctx))


def mgmlmc_coarsest_trace(ctx):
    re, im = _D(), _D()
    _check(ctx, lib().mgmlmc_coarsest_trace(ctx, ctypes.byref(re), ctypes.byref(im)))
    return complex(re.value, im.value)


def mgmlmc_connected_correlator(ctx, kind, n_samples, seed, first_sample, T, R_max):
    mean = np.zeros(2 * R_max * R_max * T)
    var = np.zeros(R_max * R_max * T)
    R = _I()
    _check(ctx, lib().mgmlmc_connected_correlator(ctx, kind, n_samples, seed, first_sample,
                                                  ptr(mean), ptr(var), ctypes.byref(R)))
    r = R.value
    m = mean[:2 * r * r * T].view(np.complex128).reshape(r, r, T)
    return m, var[:r * r * T].reshape(r, r, T)


def mgmlmc_disconnected_loop(ctx, kind, t, n_samples, seed, first_sample, R_max):
    mean = np.zeros(2 * R_max)
    var = np.zeros(R_max)
    R = _I()
    _check(ctx, lib().mgmlmc_disconnected_loop(ctx, kind, t, n_samples, seed, first_sample,
                                               ptr(mean), ptr(var), ctypes.byref(R)))
    r = R.value
    return mean[:2 * r].view(np.complex128), var[:r]


def mgmlmc_apply(ctx, op, level, precision, inp, out, nrhs=1):
    _check(ctx, lib().mgmlmc_apply(ctx, op, level, precision, ptr(inp), ptr(out), nrhs))


def mgmlmc_noise(ctx, level, seed, first_sample, term, aux, slice_, out, nrhs=1):
    _check(ctx, lib().mgmlmc_noise(ctx, level, seed, first_sample, term, aux, slice_, ptr(out), nrhs))


def mgmlmc_get_prolongator(ctx, level, out):
    _check(ctx, lib().mgmlmc_get_prolongator(ctx, level, ptr(out)))


def mgmlmc_get_test_vectors(ctx, level):
    """(N_tv, n) complex array: the test vectors P_level was built from."""
    _, dof, _ = mgmlmc_level_info(ctx, level + 1)
    n = mgmlmc_level_info(ctx, level)[2]
    out = np.zeros((dof // 2, n), dtype=np.complex128)
    _check(ctx, lib().mgmlmc_get_test_vectors(ctx, level, ptr(out)))
    return out


def mgmlmc_get_coarse_op(ctx, level, out):
    _check(ctx, lib().mgmlmc_get_coarse_op(ctx, level, ptr(out)))


def mgmlmc_last_solve_stats(ctx):
    it = _I()
    res = _D()
    _check(ctx, lib().mgmlmc_last_solve_stats(ctx, ctypes.byref(it), ctypes.byref(res)))
    return it.value, res.value


KERNEL_WILSON_FP64, KERNEL_WILSON_FP32, KERNEL_STENCIL_FP64, KERNEL_STENCIL_FP32 = 0, 1, 2, 3


def mgmlmc_profile(ctx, enable):
    _check(ctx, lib().mgmlmc_profile(ctx, int(bool(enable))))


def mgmlmc_profile_stats(ctx, kernel_class):
    n = _I64()
    ms, by, fl = _D(), _D(), _D()
    _check(ctx, lib().mgmlmc_profile_stats(ctx, kernel_class, ctypes.byref(n), ctypes.byref(ms),
                                           ctypes.byref(by), ctypes.byref(fl)))
    return {'launches': n.value, 'ms': ms.value, 'bytes': by.value, 'flops': fl.value}


def mgmlmc_kernel_launches():
    return int(lib().mgmlmc_kernel_launches())


VARIANT_DSLASH_FP32 = 0
VARIANT_STENCIL_FP32 = 1
VARIANT_SAP_FP32 = 2
VARIANT_TRANSFER_FP32 = 3
VARIANT_AUTOTUNE = -2
LAYOUT_INTERNAL = 0x100


def mgmlmc_reorder(ctx, inp, out, nrhs, to_internal):
    """Level-0 complex-float vectors: canonical <-> the library's internal
    structure-of-arrays order."""
    _check(ctx, lib().mgmlmc_reorder(ctx, ptr(inp), ptr(out), nrhs, int(bool(to_internal))))


def mgmlmc_reorder_bf16(ctx, inp, out, nrhs, to_internal):
    """Level-0 complex-bfloat16 vectors: canonical <-> internal chunked order."""
    _check(ctx, lib().mgmlmc_reorder_bf16(ctx, ptr(inp), ptr(out), nrhs, int(bool(to_internal))))


def mgmlmc_deflation_build(ctx, k, iters, tol, seed):
    """Inexact deflation basis (see include/mgmlmc.h); returns (exact part
    tr(V^H D^-1 V) as a complex, device seconds of the build)."""
    ex = np.zeros(2)
    sec = _D()
    _check(ctx, lib().mgmlmc_deflation_build(ctx, int(k), int(iters), float(tol), int(seed), ptr(ex),
                                             ctypes.byref(sec)))
    return complex(ex[0], ex[1]), sec.value


def mgmlmc_refine_test_vectors(ctx, level, n_vec, max_iters, eig_tol, solve_tol, seed):
    """Refine the test vectors of `level` toward low eigenvectors of
    Gamma5 D_l and rebuild the hierarchy (see include/mgmlmc.h); returns
    (theta, eigen-residuals, steps) of the N_tv refined vectors."""
    ntv = mgmlmc_level_info(ctx, level + 1)[1] // 2
    th = np.zeros(ntv)
    rh = np.zeros(ntv)
    st = _I()
    _check(ctx, lib().mgmlmc_refine_test_vectors(ctx, int(level), int(n_vec), int(max_iters), float(eig_tol),
                                                 float(solve_tol), int(seed), ptr(th), ptr(rh),
                                                 ctypes.byref(st)))
    return th, rh, st.value


def mgmlmc_gen_gauge(ctx, eps, seed):
    """Synthetic SU(3) gauge field U = exp(i eps H) generated on the device
    (counter-based draw, see include/mgmlmc.h)."""
    _check(ctx, lib().mgmlmc_gen_gauge(ctx, float(eps), int(seed)))


def mgmlmc_kernel_variants(kernel):
    return int(lib().mgmlmc_kernel_variants(kernel))


def mgmlmc_set_kernel_variant(ctx, kernel, variant):
    _check(ctx, lib().mgmlmc_set_kernel_variant(ctx, kernel, variant))


def mgmlmc_get_kernel_variant(ctx, kernel, nrhs):
    v = _I()
    _check(ctx, lib().mgmlmc_get_kernel_variant(ctx, kernel, nrhs, ctypes.byref(v)))
    return v.value


def mgmlmc_project_noalloc(ctx, level, precision, inp, out, nrhs=1):
    _check(ctx, lib().mgmlmc_project_noalloc(ctx, level, precision, ptr(inp), ptr(out), nrhs))


def mgmlmc_learned_init(ctx, channels=16, seed=5000):
    _check(ctx, lib().mgmlmc_learned_init(ctx, channels, seed))


def mgmlmc_learned_size(ctx):
    n = _I64()
    _check(ctx, lib().mgmlmc_learned_size(ctx, ctypes.byref(n)))
    return n.value


def mgmlmc_learned_weights(ctx, host, set_):
    _check(ctx, lib().mgmlmc_learned_weights(ctx, ptr(host), int(set_)))


def mgmlmc_learned_loss_grad(ctx, r, nrhs, grad_host):
    loss = _D()
    _check(ctx, lib().mgmlmc_learned_loss_grad(ctx, ptr(r), nrhs, ctypes.byref(loss), ptr(grad_host)))
    return loss.value


def mgmlmc_learned_train(ctx, channels=16, steps=200, batch=8, pool=2000, lr=1e-3, seed=5000, source=0):
    p = TrainParams(channels, steps, batch, pool, lr, seed, source)
    out = TrainResult()
    _check(ctx, lib().mgmlmc_learned_train(ctx, ctypes.byref(p), ctypes.byref(out)))
    return out.as_dict()


def mgmlmc_learned_stats(ctx):
    n = _I64()
    _check(ctx, lib().mgmlmc_learned_stats(ctx, ctypes.byref(n)))
    return n.value
