"""Compile ``oracle/residual.c`` into ``oracle/_build/liboracle.so``.

TEST INFRASTRUCTURE ONLY.  Plain gcc, no fused multiply-add contraction,
no fast-math, so every floating-point operation is the IEEE operation the
source spells out.

A second library, ``liboracle_omp.so``, is the same source compiled with
OpenMP (its independent row loops spread over threads; same bits), used only
to time the CPU baseline on every host core.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, 'residual.c')
OUT_DIR = os.path.join(HERE, '_build')
LIB = os.path.join(OUT_DIR, 'liboracle.so')


LIB_OMP = os.path.join(OUT_DIR, 'liboracle_omp.so')


def _compile(target, extra, tag):
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = target + '.tmp.%d' % os.getpid()
    flags = ['gcc', '-std=c11', '-ffp-contract=off', '-fno-fast-math', '-fPIC'] + extra
    o_real = os.path.join(OUT_DIR, 'residual_real%s.o' % tag)
    o_cplx = os.path.join(OUT_DIR, 'residual_cs%s.o' % tag)
    subprocess.check_call(flags + ['-c', SRC, '-o', o_real])
    subprocess.check_call(flags + ['-DORACLE_COMPLEX', '-c', SRC, '-o', o_cplx])
    link = ['gcc', '-shared', o_real, o_cplx, '-o', tmp, '-lm'] + (['-fopenmp'] if '-fopenmp' in extra else [])
    subprocess.check_call(link)
    os.replace(tmp, target)
    return target


def _stale(target):
    return not os.path.exists(target) or os.path.getmtime(target) < os.path.getmtime(SRC)


def build(force=False):
    """Build the oracle shared library if it is missing or older than its source."""
    if force or _stale(LIB):
        _compile(LIB, ['-O2'], '')
    return LIB


def build_parallel(force=False):
    """Build the OpenMP library of the CPU baseline (same source, same bits)."""
    if force or _stale(LIB_OMP):
        _compile(LIB_OMP, ['-O3', '-fopenmp'], '_omp')
    return LIB_OMP


if __name__ == '__main__':
    print(build(force=True))
    print(build_parallel(force=True))
