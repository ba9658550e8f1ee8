// First-order dual numbers in FP64 for the tangent-linear (forward-mode)
// derivative of the time step: a value and its directional derivative.
#pragma once

#include <cuda_runtime.h>

namespace lbib {

struct dual {
    double v, d;
    __host__ __device__ dual() : v(0.0), d(0.0) {}
    __host__ __device__ dual(double value) : v(value), d(0.0) {}
    __host__ __device__ dual(double value, double deriv) : v(value), d(deriv) {}
};

__device__ __forceinline__ dual operator+(dual a, dual b) { return dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ dual operator-(dual a, dual b) { return dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ dual operator-(dual a) { return dual(-a.v, -a.d); }
__device__ __forceinline__ dual operator*(dual a, dual b) { return dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ dual operator/(dual a, dual b) {
    const double q = a.v / b.v;
    return dual(q, (a.d - q * b.d) / b.v);
}
__device__ __forceinline__ dual& operator+=(dual& a, dual b) { return a = a + b; }
__device__ __forceinline__ dual& operator-=(dual& a, dual b) { return a = a - b; }
__device__ __forceinline__ dual& operator*=(dual& a, dual b) { return a = a * b; }
__device__ __forceinline__ dual sqrt(dual a) {
    const double s = ::sqrt(a.v);
    return dual(s, s > 0.0 ? 0.5 * a.d / s : 0.0);
}
__device__ __forceinline__ dual recip(dual a) { return dual(1.0) / a; }
// |a| with the derivative of the branch taken (sign of the value)
__device__ __forceinline__ dual fabs(dual a) { return a.v < 0.0 ? -a : a; }
// d atan2(y, x) = (x dy - y dx) / (x^2 + y^2)
__device__ __forceinline__ dual atan2(dual y, dual x) {
    const double r2 = x.v * x.v + y.v * y.v;
    return dual(::atan2(y.v, x.v), (x.v * y.d - y.v * x.d) / r2);
}
__device__ __forceinline__ dual pow_m52(dual a) {  // a^(-5/2)
    const double p = 1.0 / (a.v * a.v * ::sqrt(a.v));
    return dual(p, -2.5 * p / a.v * a.d);
}

}  // namespace lbib
