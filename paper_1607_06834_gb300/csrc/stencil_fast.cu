// Residual stencil, FMA contraction allowed (default rounding mode).
#define ROK_NS fast
#include "stencil_impl.cuh"
