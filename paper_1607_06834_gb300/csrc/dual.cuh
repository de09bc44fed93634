// Forward-mode dual numbers (value, tangent) for the exact Jacobian-vector
// product J(y) v = d/dt f(y + t v) at t = 0 (Sec. 2.3 mentions exact products
// as the alternative to Eq. matvecFD).  Each operation carries the tangent by
// the chain rule; branches (|x|, the entropy-fix switch) follow the value.
#pragma once
#include <math.h>

namespace rok {

// keep the binary64 overloads visible next to the dual ones
using ::fabs;
using ::rsqrt;
using ::sqrt;

struct Dual {
    double v, d;
};

__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b)
{
    double q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ Dual operator+(Dual a, double s) { return {a.v + s, a.d}; }
__device__ __forceinline__ Dual operator+(double s, Dual a) { return {s + a.v, a.d}; }
__device__ __forceinline__ Dual operator-(Dual a, double s) { return {a.v - s, a.d}; }
__device__ __forceinline__ Dual operator-(double s, Dual a) { return {s - a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, double s) { return {a.v * s, a.d * s}; }
__device__ __forceinline__ Dual operator*(double s, Dual a) { return {s * a.v, s * a.d}; }
__device__ __forceinline__ Dual operator/(Dual a, double s) { return {a.v / s, a.d / s}; }
__device__ __forceinline__ Dual operator/(double s, Dual b)
{
    double q = s / b.v;
    return {q, -(q * b.d) / b.v};
}
__device__ __forceinline__ Dual sqrt(Dual a)
{
    double s = ::sqrt(a.v);
    return {s, a.d / (2.0 * s)};
}
__device__ __forceinline__ Dual rsqrt(Dual a)
{
    double r = ::rsqrt(a.v);
    return {r, -0.5 * (r * r * r) * a.d};
}
__device__ __forceinline__ Dual fabs(Dual a) { return a.v < 0.0 ? -a : a; }

// value used for comparisons and branch decisions
__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ double val(Dual x) { return x.v; }
// the quantity a launch writes out: the value of a residual, the tangent of a JVP
__device__ __forceinline__ double result(double x) { return x; }
__device__ __forceinline__ double result(Dual x) { return x.d; }

}  // namespace rok
