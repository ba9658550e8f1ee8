// Per-node arithmetic of the fused collide-stream kernels: the fixed-point IB
// force back to the compute type, and the moments + Guo-forced BGK collision
// of one node in the shifted (deviation) form.  Both forms of the fused kernel
// (row tiles and the persistent bulk-copy pipeline) call the same functions,
// so they produce the same bits; for 16-bit storage the persistent form runs
// the collision on the stored (scaled) values (collide_node_scaled), whose
// results are the row tiles' times an exact power of two.
//
// Paper: Coclite, arXiv 1907.00080, Sec. 2.1 (Eqs. BGK, feq, GaussHermite),
// Sec. 2.2 (Eqs. forcedBGK, ForcingTerm; rho u = sum f e + G/2).
#pragma once

#include <type_traits>

#include "lbib_internal.cuh"

namespace lbib {

// fixed-point force value (scaled by 2^52) to the compute type
template <typename C> __device__ __forceinline__ C from_fix(long long v);
template <> __device__ __forceinline__ float from_fix<float>(long long v) {
    // two 32-bit conversions instead of a 64-bit one: hi 2^32 + lo, scaled by 2^-52
    const int hi = (int)(v >> 32);
    const unsigned lo = (unsigned)(v & 0xffffffffll);
    return fmaf((float)hi, 9.5367431640625e-07f, (float)lo * 2.220446049250313e-16f);
}
template <> __device__ __forceinline__ double from_fix<double>(long long v) {
    return __ll2double_rn(v) * kFixInv;
}

// momentum term of the lower (bottom = true) or upper moving wall in the compute type
template <typename C> __device__ __forceinline__ C wall_term(const LbArgs& a, bool bottom);
template <> __device__ __forceinline__ float wall_term<float>(const LbArgs& a, bool bottom) {
    return bottom ? a.bbf_bot : a.bbf_top;
}
template <> __device__ __forceinline__ double wall_term<double>(const LbArgs& a, bool bottom) {
    return bottom ? a.bb_bot : a.bb_top;
}

// Zou and He's known-velocity condition (Sec. 2.1) on a wall row, in the
// deviations d_i = f_i - w_i (the weights cancel): lower = true rebuilds
// d_2, d_5, d_6 of the row y = 0, else d_4, d_7, d_8 of the row y = NY - 1, from
// the known ones and the wall's velocity (uw, 0).  The populations' momentum
// is the wall velocity less the node's Guo half-force, j = rho (uw, 0) - G/2,
// so that the collision's velocity (sum f e + G/2) / rho is (uw, 0).
template <typename C>
__device__ __forceinline__ void zou_he(C (&d)[9], C Gx, C Gy, C uw, bool lower) {
    const C jy = C(-0.5) * Gy;
    const C s13 = d[1] - d[3];
    if (lower) {
        const C rho = C(1) + (d[0] + d[1] + d[3]) + C(2) * (d[4] + d[7] + d[8]) + jy;
        const C jx = rho * uw - C(0.5) * Gx;
        d[2] = d[4] + C(2.0 / 3.0) * jy;
        d[5] = d[7] - C(0.5) * s13 + C(0.5) * jx + C(1.0 / 6.0) * jy;
        d[6] = d[8] + C(0.5) * s13 - C(0.5) * jx + C(1.0 / 6.0) * jy;
    } else {
        const C rho = C(1) + (d[0] + d[1] + d[3]) + C(2) * (d[2] + d[5] + d[6]) - jy;
        const C jx = rho * uw - C(0.5) * Gx;
        d[4] = d[2] - C(2.0 / 3.0) * jy;
        d[7] = d[5] + C(0.5) * s13 - C(0.5) * jx - C(1.0 / 6.0) * jy;
        d[8] = d[6] - C(0.5) * s13 + C(0.5) * jx - C(1.0 / 6.0) * jy;
    }
}
template <typename C> __device__ __forceinline__ C zh_wall_u(const LbArgs& a, bool lower);
template <> __device__ __forceinline__ float zh_wall_u<float>(const LbArgs& a, bool lower) {
    return lower ? a.uwf_bot : a.uwf_top;
}
template <> __device__ __forceinline__ double zh_wall_u<double>(const LbArgs& a, bool lower) {
    return lower ? a.uw_bot : a.uw_top;
}

// omega, 3 omega and the body force in the compute type (the FP32 kernels
// read the copies rounded on the host: no FP64 conversion per node)
template <typename C> struct LbConst;
template <> struct LbConst<double> {
    __device__ static double om(const LbArgs& a) { return a.omega; }
    __device__ static double om3(const LbArgs& a) { return 3.0 * a.omega; }
    __device__ static double gx(const LbArgs& a) { return a.gx; }
    __device__ static double gy(const LbArgs& a) { return a.gy; }
};
template <> struct LbConst<float> {
    __device__ static float om(const LbArgs& a) { return a.omf; }
    __device__ static float om3(const LbArgs& a) { return a.om3f; }
    __device__ static float gx(const LbArgs& a) { return a.gxf; }
    __device__ static float gy(const LbArgs& a) { return a.gyf; }
};

__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }  // = 1.0f / x, correctly rounded
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
// 1 / rho in collide_node and collide_node_scaled.  In FP32 these serve only
// 16-bit storage, whose stored values are rounded to 2^-11 (FP16) or 2^-8
// (BF16) relative: there the hardware approximate reciprocal (PTX
// rcp.approx.ftz.f32, at most 1 ulp of error, 2^-23 relative) is used, which
// takes fewer instructions than the correctly rounded one.  Every form of a
// 16-bit run calls it, so the forms still give the same bits.
template <typename C> __device__ __forceinline__ C recip_node(C x) { return recip(x); }
template <> __device__ __forceinline__ float recip_node<float>(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// One node: f holds the pulled deviations d_i = f_i - w_i; G the total force
// (body force plus spread IB force).  Returns the post-collision deviations
//   d*_i = d_i - omega (d_i - deq_i) + (1 - omega/2) w_i [3(e_i - u) + 9 (e_i.u) e_i].G
// with deq_i = w_i (drho + rho (3 e.u + 4.5 (e.u)^2 - 1.5 u^2)) and the
// half-force velocity u = (sum d_i e_i + G/2) / rho, rho = 1 + sum d_i.
// Collecting terms, d*_i = (1 - omega) d_i + w_i [a + b eu + c eu^2 + g eG + h eu eG]
// with eu = e_i.u, eG = e_i.G and per-node constants
//   a = omega drho - 1.5 omega rho u^2 - 3 pre u.G,  b = 3 omega rho,
//   c = 4.5 omega rho,  g = 3 pre,  h = 9 pre   (pre = 1 - omega/2);
// opposite directions share the even part a + c eu^2 + h eu eG and flip the odd
// part b eu + g eG, so each of the four pairs costs one evaluation.
template <typename C>
__device__ __forceinline__ void collide_node(const C (&f)[9], C Gx, C Gy, C om, C pre, C (&out)[9],
                                             C& rho_o, C& ux_o, C& uy_o) {
    const C drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    const C jx = (f[1] - f[3]) + ((f[5] - f[7]) + (f[8] - f[6]));
    const C jy = (f[2] - f[4]) + ((f[5] - f[7]) + (f[6] - f[8]));
    const C rho = C(1) + drho;
    const C rinv = recip_node(rho);
    const C ux = (jx + C(0.5) * Gx) * rinv;
    const C uy = (jy + C(0.5) * Gy) * rinv;
    rho_o = rho;
    ux_o = ux;
    uy_o = uy;
    const C uu = ux * ux + uy * uy;
    const C uG = ux * Gx + uy * Gy;
    const C omr = om * rho;
    const C a = om * drho - C(1.5) * omr * uu - C(3) * pre * uG;
    const C b = C(3) * omr, c = C(4.5) * omr, g = C(3) * pre, h = C(9) * pre;
    const C omc = C(1) - om;
    out[0] = omc * f[0] + wgt<C>(0) * a;
    // pairs (i, opp(i)) with e_i = (1,0), (0,1), (1,1), (-1,1)
    const C eus[4] = {ux, uy, ux + uy, uy - ux};
    const C eGs[4] = {Gx, Gy, Gx + Gy, Gy - Gx};
    constexpr int ip[4] = {1, 2, 5, 6};
    constexpr int io[4] = {3, 4, 7, 8};
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const C eu = eus[p], eG = eGs[p];
        const C w = wgt<C>(ip[p]);
        const C even = a + eu * (c * eu + h * eG);
        const C odd = b * eu + g * eG;
        out[ip[p]] = omc * f[ip[p]] + w * (even + odd);
        out[io[p]] = omc * f[io[p]] + w * (even - odd);
    }
}

// The plain collision on the stored values of 16-bit storage, s_i = d_i 2^k,
// without scaling them first: the moments are summed from s and scaled by
// 2^-k once, and the relaxation runs on s with the weights scaled by 2^k, so
// that out_s = out 2^k goes to storage with no multiply.  Scaling by a power
// of two is exact (every intermediate stays a normal FP32 number: |s| is at
// most 65504 and at least 2^-24 where non-zero, k at most 40), so each
// rounded operation gives the unscaled one's result times 2^k and the stored
// bits equal those of collide_node on d = s 2^-k followed by out 2^k.
__device__ __forceinline__ void collide_node_scaled(const float (&s)[9], float Gx, float Gy, float om, float pre,
                                                    float inv, float scl, float (&out)[9], float& rho_o,
                                                    float& ux_o, float& uy_o) {
    const float drho = (((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7])) + s[8]) * inv;
    const float jx = ((s[1] - s[3]) + ((s[5] - s[7]) + (s[8] - s[6]))) * inv;
    const float jy = ((s[2] - s[4]) + ((s[5] - s[7]) + (s[6] - s[8]))) * inv;
    const float rho = 1.0f + drho;
    const float rinv = recip_node(rho);
    const float ux = (jx + 0.5f * Gx) * rinv;
    const float uy = (jy + 0.5f * Gy) * rinv;
    rho_o = rho;
    ux_o = ux;
    uy_o = uy;
    const float uu = ux * ux + uy * uy;
    const float uG = ux * Gx + uy * Gy;
    const float omr = om * rho;
    const float a = om * drho - 1.5f * omr * uu - 3.0f * pre * uG;
    const float b = 3.0f * omr, c = 4.5f * omr, g = 3.0f * pre, h = 9.0f * pre;
    const float omc = 1.0f - om;
    out[0] = omc * s[0] + (wgt<float>(0) * scl) * a;
    const float eus[4] = {ux, uy, ux + uy, uy - ux};
    const float eGs[4] = {Gx, Gy, Gx + Gy, Gy - Gx};
    constexpr int ip[4] = {1, 2, 5, 6};
    constexpr int io[4] = {3, 4, 7, 8};
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const float eu = eus[p], eG = eGs[p];
        const float w = wgt<float>(ip[p]) * scl;
        const float even = a + eu * (c * eu + h * eG);
        const float odd = b * eu + g * eG;
        out[ip[p]] = omc * s[ip[p]] + w * (even + odd);
        out[io[p]] = omc * s[io[p]] + w * (even - odd);
    }
}

// The same collision for FP32 storage, arranged so that the momentum it hands
// on carries no systematic rounding error.  In FP32 the per-node rounding of
// the momentum (about 1e-9 of populations near 0.01) is coherent across a
// slowly varying flow: with every operation rounded to nearest, double
// roundings (a sum rounded to one grid, then added to a term and rounded to a
// coarser one) leave a bias of a fraction of an ulp per node and step.  The
// flow integrates such a bias over its viscous time like a spurious body force
// (2.2e-4 lu of marker drift over 1000 steps of the 128x32 capsule at
// u_max = 0.02).  Three changes remove it:
//  * the momentum sums are exact: every pulled deviation is split into a part
//    on the 2^-20 grid (d + 12 - 12, exact for |d| < 4) and a remainder below
//    2^-21; the grid parts add without rounding, the remainders with errors
//    below 2^-42;
//  * the odd part of each direction pair, 3 omega (e.t) + 3 pre (e.G) with
//    t = rho u = j + G/2, is formed from those two parts by fused
//    multiply-adds with one final rounding (instead of from a rounded rho and
//    u, whose product re-rounds rho u);
//  * the weights are k/36 with k = 16, 4, 1 (exact multiples), and the
//    product by 1/36 is compensated: x/36 = x hi + x lo with hi + lo = 1/36
//    to 2^-48, so the weights carry no common relative error (the nearest
//    floats to 1/9, 1/36 and 4/9 are all 7.45e-9 too large, which would scale
//    the momentum of every collision by 1 + 7.45e-9).
// The remaining per-node momentum error is unbiased rounding: about 1e-11 of
// mean against 3e-10 of scatter at u = 0.015 (it was 7e-10 of mean).  At
// tau = 1 (omega = 1) every constant is exact.  At other tau, 3 omega and
// 1 - omega are rounded separately, which leaves a relative mismatch of at
// most 2^-24 between the odd moments and the relaxation.
// Mass (the even parts) keeps the plain arithmetic.
__device__ __forceinline__ void collide_node_exactj(const float (&f)[9], float Gx, float Gy, float om, float pre,
                                                    float om3, float (&out)[9], float& rho_o, float& ux_o,
                                                    float& uy_o) {
    const float drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    float hi[9], lo[9];
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        hi[i] = __fadd_rn(__fadd_rn(f[i], 12.0f), -12.0f);  // f[i] rounded to the 2^-20 grid
        lo[i] = __fadd_rn(f[i], -hi[i]);                     // exact remainder
    }
    const float Jxh = __fadd_rn(__fadd_rn(hi[1], -hi[3]), __fadd_rn(__fadd_rn(hi[5], -hi[7]), __fadd_rn(hi[8], -hi[6])));
    const float Jyh = __fadd_rn(__fadd_rn(hi[2], -hi[4]), __fadd_rn(__fadd_rn(hi[5], -hi[7]), __fadd_rn(hi[6], -hi[8])));
    const float Jxl = (lo[1] - lo[3]) + ((lo[5] - lo[7]) + (lo[8] - lo[6]));
    const float Jyl = (lo[2] - lo[4]) + ((lo[5] - lo[7]) + (lo[6] - lo[8]));
    const float Txl = fmaf(0.5f, Gx, Jxl), Tyl = fmaf(0.5f, Gy, Jyl);  // t = j + G/2 = (Jh) + (Tl)
    const float tx = Jxh + Txl, ty = Jyh + Tyl;
    const float rho = 1.0f + drho;
    const float rinv = recip(rho);
    const float ux = tx * rinv, uy = ty * rinv;
    rho_o = rho;
    ux_o = ux;
    uy_o = uy;
    const float tu = tx * ux + ty * uy;  // rho u^2
    const float uG = ux * Gx + uy * Gy;
    const float a = om * drho - 1.5f * om * tu - 3.0f * pre * uG;
    const float c45 = 4.5f * om, g = 3.0f * pre, h = 9.0f * pre;
    const float omc = 1.0f - om;
    constexpr float whi = 1.0f / 36.0f;
    constexpr float wlo = (float)(1.0 / 36.0 - (double)(1.0f / 36.0f));
    // k x / 36 + base with one final rounding of the weighted part; k is a
    // power of two, so k whi and k wlo are exact and x (k whi) = (k x) whi
    auto wmul = [&](float k, float x, float base) { return fmaf(x, k * whi, fmaf(x, k * wlo, base)); };
    out[0] = wmul(16.0f, a, omc * f[0]);
    const float eus[4] = {ux, uy, ux + uy, uy - ux};
    const float ets[4] = {tx, ty, tx + ty, ty - tx};
    const float eGs[4] = {Gx, Gy, Gx + Gy, Gy - Gx};
    const float eth[4] = {Jxh, Jyh, __fadd_rn(Jxh, Jyh), __fadd_rn(Jyh, -Jxh)};  // exact on the 2^-20 grid
    const float etl[4] = {Txl, Tyl, Txl + Tyl, Tyl - Txl};
    constexpr int ip[4] = {1, 2, 5, 6};
    constexpr int io[4] = {3, 4, 7, 8};
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const float k = p < 2 ? 4.0f : 1.0f;
        const float even = a + eus[p] * (c45 * ets[p] + h * eGs[p]);
        const float odd = fmaf(om3, eth[p], fmaf(om3, etl[p], g * eGs[p]));
        out[ip[p]] = wmul(k, even + odd, omc * f[ip[p]]);
        out[io[p]] = wmul(k, even - odd, omc * f[io[p]]);
    }
}

// the collision of storage type S: the exact-momentum form for FP32 storage,
// the plain form otherwise (FP64; 16-bit storage, whose own rounding is far
// coarser)
template <typename S, typename C>
__device__ __forceinline__ void collide(const C (&f)[9], C Gx, C Gy, C om, C pre, C om3, C (&out)[9], C& rho_o,
                                        C& ux_o, C& uy_o) {
    if constexpr (std::is_same<S, float>::value) {
        collide_node_exactj(f, Gx, Gy, om, pre, om3, out, rho_o, ux_o, uy_o);
    } else {
        collide_node<C>(f, Gx, Gy, om, pre, out, rho_o, ux_o, uy_o);
    }
}

}  // namespace lbib
