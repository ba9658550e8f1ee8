// Extended-precision reals for the Lagrangian side.
//
// Marker positions need more than FP32 (x up to ~1e3 lattice units, per-step
// displacements down to ~1e-6, element-length and angle changes that cancel).
// In FP64 mode they are doubles.  In the FP32 modes they are float-float pairs
// (hi + lo, about 48 significant bits) handled with error-free transforms
// (Knuth's two-sum, Dekker's two-product via a fused multiply-add), so the
// Lagrangian kernels run on the FP32 pipes instead of the far slower FP64
// pipe.  Every operation is written with explicitly rounded intrinsics so the
// compiler cannot contract or reorder it: the rest shape then reproduces its
// stored products bit for bit.
#pragma once

#include <cuda_runtime.h>

namespace lbib {

struct ff {
    float hi, lo;
};

__host__ __device__ inline ff ff_from_double(double d) {
    const float h = (float)d;
    return ff{h, (float)(d - (double)h)};
}

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff{s, e};
}
__device__ __forceinline__ ff quick_two_sum(float a, float b) {  // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = two_sum(a.hi, b.hi);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_addf(ff a, float b) {
    const ff s = two_sum(a.hi, b);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return quick_two_sum(p, e);
}
__device__ __forceinline__ ff ff_mulf(ff a, float b) {
    const float p = __fmul_rn(a.hi, b);
    const float e = __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p));
    return quick_two_sum(p, e);
}
__device__ __forceinline__ float ff_to_float(ff a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }
// largest integer <= a, as a float (exact for |a| < 2^24)
__device__ __forceinline__ float ff_floor(ff a) {
    const float f = floorf(a.hi);
    return (f == a.hi && a.lo < 0.f) ? f - 1.f : f;
}

// ---- the extended type of each compute precision, with one set of names
template <typename C> struct Ext;
template <> struct Ext<double> { using E = double; };
template <> struct Ext<float> { using E = ff; };

__device__ __forceinline__ double eadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double esub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double emul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double emulc(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double eaddc(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double etoc(double a) { return a; }
__device__ __forceinline__ double etod(double a) { return a; }
__device__ __forceinline__ double efloor(double a) { return floor(a); }
__device__ __forceinline__ double ehi(double a) { return a; }

__device__ __forceinline__ ff eadd(ff a, ff b) { return ff_add(a, b); }
__device__ __forceinline__ ff esub(ff a, ff b) { return ff_sub(a, b); }
__device__ __forceinline__ ff emul(ff a, ff b) { return ff_mul(a, b); }
__device__ __forceinline__ ff emulc(ff a, float b) { return ff_mulf(a, b); }
__device__ __forceinline__ ff eaddc(ff a, float b) { return ff_addf(a, b); }
__device__ __forceinline__ float etoc(ff a) { return ff_to_float(a); }
__device__ __forceinline__ double etod(ff a) { return ff_to_double(a); }
__device__ __forceinline__ float efloor(ff a) { return ff_floor(a); }
__device__ __forceinline__ float ehi(ff a) { return a.hi; }

template <typename E> __device__ __forceinline__ E ezero();
template <> __device__ __forceinline__ double ezero<double>() { return 0.0; }
template <> __device__ __forceinline__ ff ezero<ff>() { return ff{0.f, 0.f}; }

// 2/3 in the extended type (the BDF2 factor of Eq. kinematicPos); the
// float-float split is folded at compile time
constexpr float kTwoThirdsHi = (float)(2.0 / 3.0);
constexpr float kTwoThirdsLo = (float)(2.0 / 3.0 - (double)kTwoThirdsHi);
template <typename E> __device__ __forceinline__ E two_thirds_e();
template <> __device__ __forceinline__ double two_thirds_e<double>() { return 2.0 / 3.0; }
template <> __device__ __forceinline__ ff two_thirds_e<ff>() { return ff{kTwoThirdsHi, kTwoThirdsLo}; }

template <typename C> __device__ __forceinline__ typename Ext<C>::E from_double_e(double d);
template <> __device__ __forceinline__ double from_double_e<double>(double d) { return d; }
template <> __device__ __forceinline__ ff from_double_e<float>(double d) { return ff_from_double(d); }

// periodic minimum image with an integer period L (|result| <= L/2 up to rounding)
__device__ __forceinline__ double ewrap(double d, double L, double invL) { return d - L * floor(d * invL + 0.5); }
__device__ __forceinline__ ff ewrap(ff d, float L, float invL) {
    const float k = floorf(__fmaf_rn(d.hi, invL, 0.5f));
    return k == 0.f ? d : ff_addf(d, -k * L);
}

// warp shuffle of an extended value from lane l (all lanes participate)
__device__ __forceinline__ void shfl_e(double& d, double s, int l) { d = __shfl_sync(0xffffffffu, s, l); }
__device__ __forceinline__ void shfl_e(ff& d, ff s, int l) {
    d.hi = __shfl_sync(0xffffffffu, s.hi, l);
    d.lo = __shfl_sync(0xffffffffu, s.lo, l);
}

// ---- marker positions: doubles (x, y) per vertex, or float-float pairs
// stored as float4 {x.hi, y.hi, x.lo, y.lo}
template <typename C> struct PosIO;
template <> struct PosIO<double> {
    __device__ static void load(const void* X, int v, double& x, double& y) {
        const double* p = static_cast<const double*>(X);
        x = p[2 * v];
        y = p[2 * v + 1];
    }
    __device__ static void store(void* X, int v, double x, double y) {
        double* p = static_cast<double*>(X);
        p[2 * v] = x;
        p[2 * v + 1] = y;
    }
};
template <> struct PosIO<float> {
    __device__ static void load(const void* X, int v, ff& x, ff& y) {
        const float4 q = static_cast<const float4*>(X)[v];
        x = ff{q.x, q.z};
        y = ff{q.y, q.w};
    }
    __device__ static void store(void* X, int v, ff x, ff y) {
        static_cast<float4*>(X)[v] = make_float4(x.hi, y.hi, x.lo, y.lo);
    }
};

// rest state of vertex v: squared length of element (v, v+1), the cross and dot
// products of the two edges at v, and the rest length
template <typename C>
struct Rest {
    typename Ext<C>::E lsq, cross, dot;
    C l0;
};
static_assert(sizeof(Rest<double>) <= 32 && sizeof(Rest<float>) <= 32, "rest record fits 32 bytes");

}  // namespace lbib
