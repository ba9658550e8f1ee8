// Per-node arithmetic of the fused collide-stream kernels: the fixed-point IB
// force back to the compute type, and the moments + Guo-forced BGK collision
// of one node in the shifted (deviation) form.  Both forms of the fused kernel
// (row tiles and the persistent bulk-copy pipeline) call the same functions,
// so they produce the same bits.
//
// Paper: Coclite, arXiv 1907.00080, Sec. 2.1 (Eqs. BGK, feq, GaussHermite),
// Sec. 2.2 (Eqs. forcedBGK, ForcingTerm; rho u = sum f e + G/2).
#pragma once

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

__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }  // = 1.0f / x, correctly rounded
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

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
    const C rinv = recip(rho);
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

}  // namespace lbib
