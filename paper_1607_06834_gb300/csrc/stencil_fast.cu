// Residual stencil, FMA contraction allowed (default rounding mode); the speed of
// sound and 1/c^2 of the Roe average come from one reciprocal square root.
#define ROK_NS fast
#define ROK_STENCIL_RSQRT
#include "stencil_impl.cuh"
