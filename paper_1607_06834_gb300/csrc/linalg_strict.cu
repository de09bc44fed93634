// Vector kernels compiled with --fmad=false: the IEEE result of the written-out
// formula order (bitwise reproducible against a plain CPU evaluation).
#define ROK_NS strict
#include "linalg_impl.cuh"
