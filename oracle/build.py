"""Compile ``oracle/residual.c`` into ``oracle/_build/liboracle.so``.

TEST INFRASTRUCTURE ONLY.  Plain gcc, no fused multiply-add contraction,
no fast-math, so every floating-point operation is the IEEE operation the
source spells out.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, 'residual.c')
OUT_DIR = os.path.join(HERE, '_build')
LIB = os.path.join(OUT_DIR, 'liboracle.so')


def build(force=False):
    """Build the oracle shared library if it is missing or older than its source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + '.tmp.%d' % os.getpid()
    flags = ['gcc', '-std=c11', '-O2', '-ffp-contract=off', '-fno-fast-math', '-fPIC']
    o_real = os.path.join(OUT_DIR, 'residual_real.o')
    o_cplx = os.path.join(OUT_DIR, 'residual_cs.o')
    subprocess.check_call(flags + ['-c', SRC, '-o', o_real])
    subprocess.check_call(flags + ['-DORACLE_COMPLEX', '-c', SRC, '-o', o_cplx])
    subprocess.check_call(['gcc', '-shared', o_real, o_cplx, '-o', tmp, '-lm'])
    os.replace(tmp, LIB)
    return LIB


if __name__ == '__main__':
    print(build(force=True))
