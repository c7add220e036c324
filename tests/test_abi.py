"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads,
exports every entry point include/mgmlmc.h declares, and the ctypes mirrors
of its structs have the C layout (no GPU call is made)."""
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, 'include', 'mgmlmc.h')


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r'/\*.*?\*/', '', text, flags=re.S)
    return sorted(set(re.findall(r'\b(mgmlmc_[a-z0-9_]+)\s*\(', text)))


@pytest.fixture(scope='module')
def lib():
    from paper_2509_11424_gb300 import build, mgmlmc
    if not os.path.exists(build.LIB) or any(os.path.getmtime(s) > os.path.getmtime(build.LIB)
                                            for s in build.sources()):
        build.build()
    return mgmlmc.lib()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_2509_11424_gb300 import mgmlmc
    for n in declared_functions():
        assert n in mgmlmc._SIGNATURES, n
        assert callable(getattr(mgmlmc, n)), n


def test_struct_layouts_match_c():
    from paper_2509_11424_gb300 import mgmlmc as M
    structs = {'mgmlmc_mg_params': M.MgParams, 'mgmlmc_solver_params': M.SolverParams,
               'mgmlmc_est_params': M.EstParams, 'mgmlmc_term_result': M.TermResult,
               'mgmlmc_train_params': M.TrainParams, 'mgmlmc_train_result': M.TrainResult}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mgmlmc.h"', 'int main(void){']
    for cname, py in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append('return 0;}')
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, 'l.c')
        exe = os.path.join(d, 'l')
        open(src, 'w').write('\n'.join(lines))
        subprocess.run(['gcc', '-I' + os.path.join(ROOT, 'include'), src, '-o', exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    got = dict(l.split() for l in out.strip().splitlines())
    import ctypes
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got['%s.%s' % (cname, f)]) == getattr(py, f).offset, (cname, f)


def _prototypes():
    text = open(HEADER).read()
    text = re.sub(r'/\*.*?\*/', '', text, flags=re.S)
    protos = {}
    for name, params in re.findall(r'\b(mgmlmc_[a-z0-9_]+)\s*\(([^)]*)\)\s*;', text):
        params = params.strip()
        protos[name] = [] if params in ('', 'void') else [p.strip() for p in params.split(',')]
    return protos


def _c_class(param):
    if '*' in param or '[' in param:
        return 'ptr'
    for key, cls in (('uint64_t', 'u64'), ('int64_t', 'i64'), ('double', 'f64'), ('int', 'i32')):
        if re.search(r'\b%s\b' % key, param):
            return cls
    raise AssertionError('unclassified parameter: ' + param)


def test_binding_signatures_match_prototypes():
    """every ctypes argument list has the prototype's length and, position by
    position, the same kind of argument (pointer, int, int64, uint64, double)."""
    import ctypes
    from paper_2509_11424_gb300 import mgmlmc
    protos = _prototypes()
    assert set(protos) == set(declared_functions())

    def py_class(t):
        if t is ctypes.c_void_p or isinstance(t, type) and issubclass(t, ctypes._Pointer):
            return 'ptr'
        return {ctypes.c_int: 'i32', ctypes.c_int64: 'i64', ctypes.c_uint64: 'u64',
                ctypes.c_double: 'f64', ctypes.c_char_p: 'ptr'}[t]

    for name, params in protos.items():
        args = mgmlmc._SIGNATURES[name]
        assert len(args) == len(params), (name, len(args), len(params))
        for i, (t, p) in enumerate(zip(args, params)):
            assert py_class(t) == _c_class(p), (name, i, p)
