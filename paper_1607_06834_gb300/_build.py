"""Build ``librok.so`` in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel; the strict-rounding stencil
is compiled with ``--fmad=false``; host code never contracts multiply-adds
(``-ffp-contract=off``) so host-side metric precomputation is the IEEE result
of its written order.  The CUDA runtime is linked statically.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, 'csrc')
INCLUDE = os.path.join(ROOT, 'include')
OUT_DIR = os.path.join(HERE, '_lib')
LIB = os.path.join(OUT_DIR, 'librok.so')

ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']
SOURCES = {
    'api.cu': [],
    'linalg_common.cu': [],
    'linalg_fast.cu': [],
    'linalg_strict.cu': ['--fmad=false'],
    'stencil_fast.cu': [],
    'stencil_strict.cu': ['--fmad=false'],
    'peak.cu': [],
    'noalloc.cu': [],
    'selftest.cu': [],
    'batch.cu': [],
    'adjoint.cu': [],
    'adaptive.cu': [],
}


def _nvcc():
    for cand in (os.environ.get('NVCC'), '/usr/local/cuda/bin/nvcc', 'nvcc'):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return 'nvcc'


def _deps_newer(target):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, 'rok.h'), __file__]
    return any(os.path.getmtime(f) > t for f in files)


def build(force=False, verbose=False, ptxas_info=False):
    """Compile every translation unit and link librok.so; returns its path."""
    if not force and not _deps_newer(LIB):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = ['-O3', '-std=c++17', '-lineinfo', '-Xcompiler', '-fPIC,-ffp-contract=off,-O2',
              '-I', INCLUDE, '-I', CSRC] + ARCH
    if ptxas_info:
        common += ['-Xptxas', '-v']

    def compile_one(item):
        src, extra = item
        obj = os.path.join(OUT_DIR, src.replace('.cu', '.o'))
        cmd = [nvcc, '-c', os.path.join(CSRC, src), '-o', obj] + common + extra
        p = subprocess.run(cmd, capture_output=True, text=True)
        return obj, cmd, p

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES.items()))
    for obj, cmd, p in results:
        if verbose or ptxas_info:
            sys.stderr.write(p.stdout + p.stderr)
        if p.returncode != 0:
            raise RuntimeError('nvcc failed: %s\n%s%s' % (' '.join(cmd), p.stdout, p.stderr))
    tmp = LIB + '.tmp.%d' % os.getpid()
    link = [nvcc, '-shared', '-o', tmp] + [r[0] for r in results] + ARCH + ['-cudart', 'static']
    p = subprocess.run(link, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError('link failed: %s\n%s%s' % (' '.join(link), p.stdout, p.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == '__main__':
    print(build(force=True, verbose=True, ptxas_info='-v' in sys.argv))
