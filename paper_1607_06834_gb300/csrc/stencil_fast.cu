// Residual stencil, FMA contraction allowed (default rounding mode); the square
// roots of the Roe average and the speed of sound with 1/c^2 come from
// reciprocal square roots.
#define ROK_NS fast
#define ROK_STENCIL_RSQRT
#include "stencil_impl.cuh"
