// Vector kernels, FMA contraction allowed (default rounding mode); the lanes'
// parts of the Gram-Schmidt and projection dot products are fused
// multiply-add chains, the stage solves substitute column by column.
#define ROK_NS fast
#define ROK_LINALG_FAST
#include "linalg_impl.cuh"
