// Device helpers shared by the Lagrangian kernels (forces / spreading and
// interpolation / advance / bonds).
#pragma once

#include <climits>

#include "bond_logic.cuh"
#include "ext_real.cuh"
#include "lbib_internal.cuh"

namespace lbib {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float wrap_half(float d, float L) {
    return d > 0.5f * L ? d - L : (d < -0.5f * L ? d + L : d);
}

// force value to the fixed-point grid of the spread field (scaled by 2^52)
template <typename C> __device__ __forceinline__ long long to_fix(C v);
template <> __device__ __forceinline__ long long to_fix<float>(float v) {
    // exact: t = v 2^52 is either below 2^23 in magnitude (round it with a 32-bit
    // conversion) or an integer whose mantissa is shifted into place
    const float t = v * 4503599627370496.0f;
    if (fabsf(t) < 8388608.0f) return (long long)__float2int_rn(t);
    const int bits = __float_as_int(t);
    const int e = ((bits >> 23) & 0xff) - 150;  // t = mant 2^e with e >= 0 here
    const long long mag = (long long)((bits & 0x7fffff) | 0x800000) << (e < 40 ? e : 40);
    return bits < 0 ? -mag : mag;
}
template <> __device__ __forceinline__ long long to_fix<double>(double v) {
    return __double2ll_rn(v * kFixScale);
}

// Range of the fixed-point conversions.  The spread field holds w F per
// (vertex, node) scaled by 2^52, the repulsion accumulators one magnitude per
// (vertex, segment) scaled by 2^60, in signed 64-bit integers.  A value at or
// beyond its bound, or not finite, is clamped to the bound (NaN to 0) and
// `bad` is set; the kernel then raises ST_FIXRANGE, which the host reads as
// LBIB_E_NONFINITE.  Bounds: 64 lu of force per (vertex, node), 2^58 in the
// field, so 32 such terms fit in one node's int64; repulsion 1 per
// (vertex, segment), 2^60 in an accumulator that holds 8 (Eq. repFor reaches
// 1 at d = 9.4e-3 lu, i.e. membranes that overlap).
constexpr double kFixLimit = 64.0;
constexpr double kFix60Limit = 1.0;
template <typename C>
__device__ __forceinline__ C clamp_fix(C v, C lim, bool& bad) {
    if (fabs(v) < lim) return v;  // false for NaN
    bad = true;
    return v > C(0) ? lim : (v < C(0) ? -lim : C(0));
}

// value scaled by 2^60 to a 64-bit integer (repulsion accumulators: magnitudes
// stay below 8, resolution 2^-60), exact for the float case
template <typename C> __device__ __forceinline__ long long to_fix60(C v);
template <> __device__ __forceinline__ long long to_fix60<float>(float v) {
    const float t = v * 1.152921504606846976e18f;  // 2^60
    if (fabsf(t) < 8388608.0f) return (long long)__float2int_rn(t);
    const int bits = __float_as_int(t);
    const int e = ((bits >> 23) & 0xff) - 150;
    const long long mag = (long long)((bits & 0x7fffff) | 0x800000) << (e < 39 ? e : 39);
    return bits < 0 ? -mag : mag;
}
template <> __device__ __forceinline__ long long to_fix60<double>(double v) {
    return __double2ll_rn(v * 1.152921504606846976e18);
}
template <typename C> __device__ __forceinline__ C fix60_to_c(long long v);
template <> __device__ __forceinline__ float fix60_to_c<float>(long long v) {
    const int hi = (int)(v >> 32);
    const unsigned lo = (unsigned)(v & 0xffffffffll);
    return fmaf((float)hi, 3.7252902984619141e-09f, (float)lo * 8.6736173798840355e-19f);
}
template <> __device__ __forceinline__ double fix60_to_c<double>(long long v) {
    return __ll2double_rn(v) * 8.6736173798840355e-19;
}

// fixed-point value (scaled by 2^52) back to the compute type
template <typename C> __device__ __forceinline__ C fix_to_c(long long v);
template <> __device__ __forceinline__ float fix_to_c<float>(long long v) {
    const int hi = (int)(v >> 32);
    const unsigned lo = (unsigned)(v & 0xffffffffll);
    return fmaf((float)hi, 9.5367431640625e-07f, (float)lo * 2.220446049250313e-16f);
}
template <> __device__ __forceinline__ double fix_to_c<double>(long long v) {
    return __ll2double_rn(v) * kFixInv;
}

// Roma, Peskin & Berger three-point regularised delta
template <typename C>
__device__ __forceinline__ C roma(C r) {
    const C a = fabs(r);
    if (a <= C(0.5)) return (C(1) + sqrt(C(1) - C(3) * a * a)) / C(3);
    if (a <= C(1.5)) {
        const C b = C(1) - a;
        return (C(5) - C(3) * a - sqrt(C(1) - C(3) * b * b)) / C(6);
    }
    return C(0);
}

template <typename C>
__device__ __forceinline__ void load_pos(const MarkerArgs& a, int v, typename Ext<C>::E& x,
                                         typename Ext<C>::E& y) {
    PosIO<C>::load(a.X, v, x, y);
}

// Edge products at a vertex in the extended type from the positions of L, v, R:
// squared length of e_R = x_R - x_v, and the cross and dot products of
// e_L = x_v - x_L with e_R (their rotation from the rest pair gives theta - theta_0).
template <typename C>
struct EdgeProducts {
    typename Ext<C>::E lsqR, cross, dot;
};
template <typename E, typename C>
__device__ __forceinline__ EdgeProducts<C> edge_products(E xL, E yL, E xv, E yv, E xR, E yR) {
    const E eLx = esub(xv, xL), eLy = esub(yv, yL), eRx = esub(xR, xv), eRy = esub(yR, yv);
    EdgeProducts<C> p;
    p.lsqR = eadd(emul(eRx, eRx), emul(eRy, eRy));
    p.cross = esub(emul(eLx, eRy), emul(eLy, eRx));
    p.dot = eadd(emul(eLx, eRx), emul(eLy, eRy));
    return p;
}

// Enclosed area of membrane m by the shoelace formula about vertex 0, summed
// by kAreaWarps warps in a fixed order (thread t of the group takes terms t,
// t + 32 kAreaWarps, ...; each warp reduces its lanes by a fixed tree; the warp
// partials are added in warp order), so every caller gets the same bits.  Call
// from the kAreaWarps consecutive warps starting at `w0` (all their lanes);
// `red` holds 32 kAreaWarps values; returns the area in every caller after the
// named barrier `bar` (kAreaWarps * 32 threads).  off, n: the membrane's first
// vertex and vertex count.
constexpr int kAreaWarps = 4;
template <typename C>
__device__ typename Ext<C>::E ring_area_group(const MarkerArgs& a, int off, int n, int w0,
                                              typename Ext<C>::E* red, int bar) {
    using E = typename Ext<C>::E;
    const int t = threadIdx.x - 32 * w0;  // 0 .. 32 kAreaWarps - 1
    const int lane = t & 31, w = t >> 5;
    E xr, yr;
    load_pos<C>(a, off, xr, yr);
    E acc = ezero<E>();
    // kBatch terms per pass with all their loads issued first (long rings:
    // one round trip per pass instead of one per term); same summation order
    constexpr int kBatch = 4;
    constexpr int stride = 32 * kAreaWarps;
    for (int k0 = t; k0 < n; k0 += kBatch * stride) {
        E xv[kBatch], yv[kBatch], xR[kBatch], yR[kBatch];
#pragma unroll
        for (int b = 0; b < kBatch; ++b) {
            const int k = k0 + b * stride;
            const int kk = k < n ? k : 0;
            const int R = kk == n - 1 ? 0 : kk + 1;
            load_pos<C>(a, off + kk, xv[b], yv[b]);
            load_pos<C>(a, off + R, xR[b], yR[b]);
        }
#pragma unroll
        for (int b = 0; b < kBatch; ++b) {
            if (k0 + b * stride >= n) break;
            const E term = esub(emul(esub(xv[b], xr), esub(yR[b], yr)), emul(esub(xR[b], xr), esub(yv[b], yr)));
            acc = eadd(acc, term);
        }
    }
    E* r = red + 32 * w;
    r[lane] = acc;
    __syncwarp();
    for (int o = 16; o > 0; o >>= 1) {
        if (lane < o) r[lane] = eadd(r[lane], r[lane + o]);
        __syncwarp();
    }
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(32 * kAreaWarps) : "memory");
    E s = red[0];
#pragma unroll
    for (int q = 1; q < kAreaWarps; ++q) s = eadd(s, red[32 * q]);
    return emulc(s, C(0.5));
}

// four block-wide sums in the compute type at once (every thread gets all four
// in its arguments); each by a fixed shuffle tree per warp, then over the warps
template <typename C>
__device__ void block_sum4_c(C& v0, C& v1, C& v2, C& v3, C* red) {
    C v[4] = {v0, v1, v2, v3};
#pragma unroll
    for (int q = 0; q < 4; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(kFull, v[q], o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) red[33 * q + w] = v[q];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            C t = threadIdx.x < nw ? red[33 * q + threadIdx.x] : C(0);
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(kFull, t, o);
            if (threadIdx.x == 0) red[33 * q + 32] = t;
        }
    }
    __syncthreads();
    v0 = red[32];
    v1 = red[33 + 32];
    v2 = red[66 + 32];
    v3 = red[99 + 32];
}

// Last-block epilogue: every block of a context's launch counts itself in once
// it is done; the block that arrives last (it sees all other blocks' writes
// after the fences) runs the epilogue and resets the counter.  No block ever
// waits for another.  nblocks: the context's blocks in the launch.
__device__ __forceinline__ bool arrive_last(unsigned int* counter, bool* flag, unsigned nblocks) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        *flag = atomicAdd(counter, 1u) == nblocks - 1;
    }
    __syncthreads();
    const bool last = *flag;
    if (last) __threadfence();
    return last;
}

// Box of one segment from positions held by a group of kSegV consecutive lanes
// (lane g of the group holds vertex v0 + g; lanes past the segment end hold a
// copy of the first vertex).  FP32 offsets from the first vertex; centre x
// wrapped into [0, nx).  All 32 lanes call it.
template <typename C>
__device__ __forceinline__ void seg_box_regs(const MarkerArgs& a, int sg, int lane, typename Ext<C>::E x,
                                             typename Ext<C>::E y) {
    using E = typename Ext<C>::E;
    const int g0 = lane & ~(kSegV - 1);
    // first vertex of the group, broadcast in its (hi, lo) parts
    E ax, ay;
    shfl_e(ax, x, g0);
    shfl_e(ay, y, g0);
    const float ox = float(etoc(esub(x, ax))), oy = float(etoc(esub(y, ay)));
    float lo_x = ox, hi_x = ox, lo_y = oy, hi_y = oy;
    for (int o = kSegV / 2; o > 0; o >>= 1) {
        lo_x = fminf(lo_x, __shfl_xor_sync(kFull, lo_x, o));
        hi_x = fmaxf(hi_x, __shfl_xor_sync(kFull, hi_x, o));
        lo_y = fminf(lo_y, __shfl_xor_sync(kFull, lo_y, o));
        hi_y = fmaxf(hi_y, __shfl_xor_sync(kFull, hi_y, o));
    }
    if (sg >= 0 && lane == g0) {
        const float Lx = a.f.nx;
        const float cx = float(ehi(ax)) + 0.5f * (lo_x + hi_x);
        a.seg_box[sg] = make_float4(cx - Lx * floorf(cx * a.f.inv_nx), float(ehi(ay)) + 0.5f * (lo_y + hi_y),
                                    0.5f * (hi_x - lo_x), 0.5f * (hi_y - lo_y));
    }
}

// interpolation U_v = sum_j phi_v(x_j) u(x_j) with the weights of this step
template <typename C>
__device__ __forceinline__ void interp_vertex(const MarkerArgs& a, int v, C& Ux, C& Uy) {
    const C* ux = static_cast<const C*>(a.ux);
    const C* uy = static_cast<const C*>(a.uy);
    const C* W = static_cast<const C*>(a.W);
    const int i0 = a.stencil[2 * v], j0 = a.stencil[2 * v + 1];
    C sx = C(0), sy = C(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        int j = j0 + b - 1;
        if (a.walls) {
            if (j < 0 || j >= a.ny) continue;
        } else {
            j = j < 0 ? j + a.ny : (j >= a.ny ? j - a.ny : j);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            int i = i0 + q - 1;
            i = i < 0 ? i + a.nx : (i >= a.nx ? i - a.nx : i);
            const C w = W[9 * (size_t)v + b * 3 + q];
            const size_t node = (size_t)j * a.nx + i;
            sx += w * ux[node];
            sy += w * uy[node];
        }
    }
    Ux = sx;
    Uy = sy;
}

// Eq. kinematicPos (BDF2): x^{n+1} = 2/3 (2 x^n - 1/2 x^{n-1} + U dt);
// forward Euler on the very first step
template <typename C>
__device__ __forceinline__ void bdf2(typename Ext<C>::E x, typename Ext<C>::E xp, C U, long long step,
                                     typename Ext<C>::E& xn) {
    using E = typename Ext<C>::E;
    if (step == 0) {
        xn = eaddc(x, U);
    } else {
        xn = emul(eaddc(esub(emulc(x, C(2)), emulc(xp, C(0.5))), U), two_thirds_e<E>());
    }
}

}  // namespace lbib
