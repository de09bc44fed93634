// Residual stencil, FMA contraction allowed (default rounding mode): the
// uniform-grid faces use the restructured doubled-flux formulas, the Roe
// averages and the speed of sound come from reciprocal square roots.
#define ROK_NS fast
#define ROK_STENCIL_FAST
#include "stencil_impl.cuh"
