// Vector kernels, FMA contraction allowed (default rounding mode).
#define ROK_NS fast
#include "linalg_impl.cuh"
