// Vector kernels, FMA contraction allowed (default rounding mode); the lanes'
// parts of the Gram-Schmidt and projection dot products are fused
// multiply-add chains.
#define ROK_NS fast
#define ROK_LINALG_FMA_DOT
#include "linalg_impl.cuh"
