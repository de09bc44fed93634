"""GB300-native Rosenbrock-Krylov (ROK) time stepping for compressible flow.

The compute path lives in ``librok.so`` (CUDA kernels for sm_103a behind a
C ABI, header ``include/rok.h``); ``paper_1607_06834_gb300.rok`` is the thin
ctypes binding with the same function names.  ``workloads`` builds the seeded
synthetic inputs.  Importing this package does not load the library; the
binding module raises if the library has not been built.
"""
__all__ = ['rok', 'workloads']
