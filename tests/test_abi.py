"""The C-ABI library builds, loads without a GPU, and exports every entry point
that include/rok.h declares; the binding exposes the same names."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, 'include', 'rok.h')).read()
    src = re.sub(r'/\*.*?\*/', '', src, flags=re.S)
    names = re.findall(r'^\s*(?:const\s+)?\w+\s*\*?\s*(rok_\w+|rk_step|esdirk_step|ros_step|dopri5_integrate)\s*\(', src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ('rok_init', 'rok_residual', 'rok_jvp', 'rok_step', 'rk_step', 'esdirk_step',
                     'rok_dt_from_cfl', 'rok_destroy', 'rok_status_string'):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1607_06834_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    lib.rok_status_string.restype = ctypes.c_char_p
    assert lib.rok_status_string(3).decode().startswith('non-finite')


def test_binding_names_match_header():
    from paper_1607_06834_gb300 import _build
    _build.build()
    from paper_1607_06834_gb300 import rok
    assert sorted(rok.EXPORTED) == _declared()
    for n in _declared():
        assert callable(getattr(rok, n))


def test_init_without_gpu_reports_an_error_not_a_crash():
    import torch
    if torch.cuda.is_available():
        return
    from paper_1607_06834_gb300 import _build
    lib = ctypes.CDLL(_build.build())
    lib.rok_init.restype = ctypes.c_int
    # a NULL description is rejected before any CUDA call
    assert lib.rok_init(None, None, None) == 1


def test_batch_init_validates_descriptions_before_any_cuda_call():
    from paper_1607_06834_gb300 import _build
    _build.build()
    from paper_1607_06834_gb300 import rok
    from paper_1607_06834_gb300 import workloads as W
    a, _ = W.isentropic_vortex(32)
    b, _ = W.taylor_green(40, reynolds=500.0)
    descs = (rok.ProblemDesc * 2)()
    descs[0], _ = rok._desc(a, 8, rok.ROK_ROUND_STRICT)
    descs[1], _ = rok._desc(b, 8, rok.ROK_ROUND_FAST)     # rounding differs
    h = ctypes.c_void_p()
    assert rok._lib.rok_batch_init(ctypes.byref(h), descs, 2, None) == rok.ROK_ERR_INVALID_ARG
    descs[1], _ = rok._desc(b, 8, rok.ROK_ROUND_STRICT, basis=rok.ROK_BASIS_FP32)
    assert rok._lib.rok_batch_init(ctypes.byref(h), descs, 2, None) == rok.ROK_ERR_UNSUPPORTED
    assert rok._lib.rok_batch_init(ctypes.byref(h), descs, 0, None) == rok.ROK_ERR_INVALID_ARG
    assert rok._lib.rok_batch_init(None, descs, 2, None) == rok.ROK_ERR_INVALID_ARG


def test_header_compiles_on_its_own_as_c_and_cxx():
    import shutil
    import subprocess

    import pytest
    hdr = os.path.join(ROOT, 'include', 'rok.h')
    for cc, args in (('gcc', ['-std=c99', '-x', 'c']), ('g++', ['-std=c++17', '-x', 'c++'])):
        if shutil.which(cc) is None:
            pytest.skip('%s not found' % cc)
        subprocess.run([cc, *args, '-Wall', '-Wextra', '-Werror', '-fsyntax-only', hdr], check=True)
