// Ligand-receptor bond kinetics (device logic): rupture, then formation,
// decided with counter-based Philox draws so that the bond history is
// reproducible and independent of thread scheduling.
//
// Paper: Coclite, arXiv 1907.00080, Sec. 2.2 (wall-particle interaction: bonds
// form below a critical separation, a forward probability governs formation
// and a reverse probability governs rupture each step) and Sec. 3 (k_f/k_r0).
// Philox4x64-10: Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11 -- implemented here from that definition.
//
// Decisions are FP64 decisions: an FP32 estimate settles every test whose
// outcome is clear by a relative margin of 1e-5 (the estimates are accurate to
// ~1e-6), and anything closer is recomputed in FP64.
#pragma once

#include <climits>

#include "ext_real.cuh"
#include "lbib_internal.cuh"

namespace lbib {

// a scalar parameter in the compute precision (double field, or its FP32 copy)
template <typename C> __device__ __forceinline__ C par(double d, float f);
template <> __device__ __forceinline__ double par<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float par<float>(double, float f) { return f; }

__device__ __forceinline__ void philox4x64_10(unsigned long long c[4], unsigned long long k0,
                                              unsigned long long k1) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll 1
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const unsigned long long hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        const unsigned long long hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        const unsigned long long n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// uniform in [0,1) from the top 53 bits of the first output word
__device__ __forceinline__ double bond_uniform(const MarkerArgs& a, long long step, int lig, int rec,
                                               int tag) {
    unsigned long long c[4] = {(unsigned long long)step, (unsigned long long)lig,
                               (unsigned long long)rec, (unsigned long long)tag};
    philox4x64_10(c, a.seed, a.instance);
    return (double)(c[0] >> 11) * 0x1.0p-53;
}

// forward (formation) and reverse (rupture) probabilities per step, FP64
// (kept out of line: they run only for near ties, and scalars are passed so the
// argument block is never copied)
static __device__ __noinline__ double p_form_d(double d, double y_eq, double inv_y_eq, double kf_dt, double beta_f) {
    const double z = (d - y_eq) * inv_y_eq;
    return 1.0 - exp(-kf_dt * exp(-beta_f * z * z));
}
static __device__ __noinline__ double p_rupture_d(double d, double y_eq, double inv_y_eq, double kr0_dt, double beta_r) {
    const double z = (d - y_eq) * inv_y_eq;
    return 1.0 - exp(-kr0_dt * exp(beta_r * z * z));
}
__device__ __forceinline__ double p_form(const MarkerArgs& a, double d) {
    return p_form_d(d, a.y_eq, a.inv_y_eq, a.kf_dt, a.beta_f);
}
__device__ __forceinline__ double p_rupture(const MarkerArgs& a, double d) {
    return p_rupture_d(d, a.y_eq, a.inv_y_eq, a.kr0_dt, a.beta_r);
}
constexpr float kMargin = 1e-5f;
__device__ __forceinline__ float p_form_f(const MarkerArgs& a, float d) {
    const float z = (d - a.f.y_eq) * a.f.inv_y_eq;
    return 1.0f - expf(-a.f.kf_dt * expf(-a.f.beta_f * z * z));
}
__device__ __forceinline__ float p_rupture_f(const MarkerArgs& a, float d) {
    const float z = (d - a.f.y_eq) * a.f.inv_y_eq;
    return 1.0f - expf(-a.f.kr0_dt * expf(a.f.beta_r * z * z));
}

// ligand point to receptor (rx, ry) in FP64 (periodic minimum image in x, and
// in y without walls)
static __device__ __noinline__ double lig_rec_dist_d(double rx, double ry, double cxp, double cyp, double nx,
                                              double inv_nx, double ny, double inv_ny, int walls) {
    double dx = rx - cxp;
    dx -= nx * floor(dx * inv_nx + 0.5);
    double dy = ry - cyp;
    if (!walls) dy -= ny * floor(dy * inv_ny + 0.5);
    return sqrt(dx * dx + dy * dy);
}
__device__ __forceinline__ double lig_rec_dist(const MarkerArgs& a, double cxp, double cyp, int r) {
    return lig_rec_dist_d(a.rec_xy[2 * r], a.rec_xy[2 * r + 1], cxp, cyp, (double)a.nx, a.inv_nx,
                          (double)a.ny, a.inv_ny, a.walls);
}

// Ligand point (element centroid at X^{n+1}) and its distance to receptor r:
// the estimate in the compute precision, and the FP64 value on demand.
template <typename C>
struct LigandPoint {
    typename Ext<C>::E cx, cy;
    double cxd, cyd;
    bool have_d;
    __device__ void init(typename Ext<C>::E xa, typename Ext<C>::E ya, typename Ext<C>::E xb,
                         typename Ext<C>::E yb) {
        cx = emulc(eadd(xa, xb), C(0.5));
        cy = emulc(eadd(ya, yb), C(0.5));
        have_d = false;
    }
    __device__ bool finite() const { return isfinite(ehi(cx)) && isfinite(ehi(cy)); }
    __device__ C dist_est(const MarkerArgs& a, int r) const {
        typename Ext<C>::E rx, ry;
        PosIO<C>::load(a.rec_e, r, rx, ry);
        return dist_est_at(a, rx, ry);
    }
    __device__ C dist_est_at(const MarkerArgs& a, typename Ext<C>::E rx, typename Ext<C>::E ry) const {
        const C dx = etoc(ewrap(esub(rx, cx), par<C>(a.nx, a.f.nx), par<C>(a.inv_nx, a.f.inv_nx)));
        C dy = etoc(esub(ry, cy));
        if (!a.walls) dy = etoc(ewrap(esub(ry, cy), par<C>(a.ny, a.f.ny), par<C>(a.inv_ny, a.f.inv_ny)));
        return sqrt(dx * dx + dy * dy);
    }
    __device__ double dist(const MarkerArgs& a, int r) {
        if (!have_d) {
            cxd = etod(cx);
            cyd = etod(cy);
            have_d = true;
        }
        return lig_rec_dist(a, cxd, cyd, r);
    }
};

// formation test of ligand l with receptor r at (rx, ry) (tag 0): d < d_cut and u < P_f(d)
template <typename C>
__device__ __forceinline__ bool forms(const MarkerArgs& a, LigandPoint<C>& lp, long long step, int l, int r,
                                      typename Ext<C>::E rx, typename Ext<C>::E ry) {
    if (sizeof(C) == 8) {
        const double d = lp.dist(a, r);
        if (!(d < a.d_cut)) return false;
        return bond_uniform(a, step, l, r, 0) < p_form(a, d);
    }
    const float df = float(lp.dist_est_at(a, rx, ry));
    const float dc = a.f.d_cut;
    if (!(df < dc * (1.f + kMargin))) return false;  // surely beyond the cut-off
    double d = -1.0;
    if (!(df < dc * (1.f - kMargin))) {
        d = lp.dist(a, r);
        if (!(d < a.d_cut)) return false;
    }
    const double u = bond_uniform(a, step, l, r, 0);
    const float pf = p_form_f(a, df);
    if (u < (double)(pf - kMargin)) return true;
    if (u > (double)(pf + kMargin)) return false;
    if (d < 0.0) d = lp.dist(a, r);
    return u < p_form(a, d);
}

// rupture test of the bond (l, r) (tag 1): d >= d_break or u < P_r(d)
template <typename C>
__device__ __forceinline__ bool ruptures(const MarkerArgs& a, LigandPoint<C>& lp, long long step, int l, int r) {
    if (sizeof(C) == 8) {
        const double d = lp.dist(a, r);
        if (d >= a.d_break) return true;
        return bond_uniform(a, step, l, r, 1) < p_rupture(a, d);
    }
    const float df = float(lp.dist_est(a, r));
    const float db = a.f.d_break;
    double d = -1.0;
    if (df >= db * (1.f + kMargin)) return true;
    if (!(df < db * (1.f - kMargin))) {
        d = lp.dist(a, r);
        if (d >= a.d_break) return true;
    }
    const double u = bond_uniform(a, step, l, r, 1);
    const float pr = p_rupture_f(a, df);
    if (u < (double)(pr - kMargin)) return true;
    if (u > (double)(pr + kMargin)) return false;
    if (d < 0.0) d = lp.dist(a, r);
    return u < p_rupture(a, d);
}

// One ligand, one thread: rupture test of its bond, then (if free) the lowest
// receptor id that passes the formation test among the receptors of the 3x3
// grid cells around the ligand point (cells are at least d_cut wide), claimed
// with atomicMin so that the lowest ligand id wins.
template <typename C>
__device__ __forceinline__ void bond_decide(const MarkerArgs& a, int l, LigandPoint<C>& lp, long long step) {
    if (!lp.finite()) return;  // reported by the advance
    const int r = a.bond_of_lig[l];
    if (r >= 0) {
        if (!ruptures<C>(a, lp, step, l, r)) return;
        a.rupt[l] = r;
    }
    const float cxh = float(ehi(lp.cx)), cyh = float(ehi(lp.cy));
    const float xw = cxh - a.f.nx * floorf(cxh * a.f.inv_nx);
    int gx = (int)floorf(xw * a.f.inv_rc_w);
    gx = gx >= a.rc_nx ? a.rc_nx - 1 : (gx < 0 ? 0 : gx);
    const int gy = (int)fminf(fmaxf(floorf((cyh - a.f.rc_y0) * a.f.inv_rc_h), -4.f), float(a.rc_ny) + 4.f);
    // the three cell rows' ranges first (independent loads), then their receptors
    int p0[9], p1[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const int qy = gy - 1 + c / 3, qx = gx - 1 + c % 3;
        p0[c] = p1[c] = 0;
        if (qy >= 0 && qy < a.rc_ny) {
            const int cell = qy * a.rc_nx + ((qx % a.rc_nx) + a.rc_nx) % a.rc_nx;
            p0[c] = a.rcell_start[cell];
            p1[c] = a.rcell_start[cell + 1];
        }
    }
    int best = INT_MAX;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        for (int p = p0[c]; p < p1[c]; ++p) {
            const int rr = a.rcell_ids[p];
            typename Ext<C>::E rx, ry;
            PosIO<C>::load(a.rcell_pos, p, rx, ry);
            if (rr >= best || a.owner_cell[p] >= 0) continue;  // bound at the start of the step
            if (forms<C>(a, lp, step, l, rr, rx, ry)) best = rr;
        }
    }
    if (best != INT_MAX) {
        a.cand[l] = best;
        atomicMin(&a.claim[best], l);
    }
}

// 3x3 receptor-grid cells around a ligand point: the nine [p0, p1) ranges of
// the cell-ordered receptor arrays (empty outside the grid's rows)
template <typename C>
__device__ __forceinline__ void ligand_cells(const MarkerArgs& a, const LigandPoint<C>& lp, int p0[9], int p1[9]) {
    const float cxh = float(ehi(lp.cx)), cyh = float(ehi(lp.cy));
    const float xw = cxh - a.f.nx * floorf(cxh * a.f.inv_nx);
    int gx = (int)floorf(xw * a.f.inv_rc_w);
    gx = gx >= a.rc_nx ? a.rc_nx - 1 : (gx < 0 ? 0 : gx);
    const int gy = (int)fminf(fmaxf(floorf((cyh - a.f.rc_y0) * a.f.inv_rc_h), -4.f), float(a.rc_ny) + 4.f);
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const int qy = gy - 1 + c / 3, qx = gx - 1 + c % 3;
        p0[c] = p1[c] = 0;
        if (qy >= 0 && qy < a.rc_ny) {
            const int cell = qy * a.rc_nx + ((qx % a.rc_nx) + a.rc_nx) % a.rc_nx;
            p0[c] = a.rcell_start[cell];
            p1[c] = a.rcell_start[cell + 1];
        }
    }
}

// Epilogue run by one block after every ligand has been decided: apply the
// ruptures and the winning claims, clear the claims, advance the step counter.
// Data written by other blocks is read past L1.
static __device__ __forceinline__ void bond_apply_all(const MarkerArgs& a) {
    // ruptures free their receptor, won claims bind it; owner is kept both by
    // receptor id and in cell order (owner_cell, read by the formation tests)
    constexpr int kPer = 4;  // ligands per thread per pass, loads issued together
    const bool one_pass = a.nlig <= kPer * (int)blockDim.x;
    int keep_c[kPer];
    for (int base = 0; base < a.nlig; base += kPer * blockDim.x) {
        int q[kPer], r_old[kPer], c[kPer], cl[kPer], pr[kPer], pc[kPer];
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            q[i] = base + threadIdx.x + i * blockDim.x;
            r_old[i] = q[i] < a.nlig ? __ldcg(&a.rupt[q[i]]) : -1;
            c[i] = q[i] < a.nlig ? __ldcg(&a.cand[q[i]]) : -1;
            keep_c[i] = c[i];
        }
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            cl[i] = c[i] >= 0 ? __ldcg(&a.claim[c[i]]) : -1;
            pc[i] = c[i] >= 0 ? a.rcell_of_rec[c[i]] : -1;
            pr[i] = r_old[i] >= 0 ? a.rcell_of_rec[r_old[i]] : -1;
        }
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            if (r_old[i] >= 0) {
                a.owner[r_old[i]] = -1;
                a.owner_cell[pr[i]] = -1;
                a.bond_of_lig[q[i]] = -1;
                a.rupt[q[i]] = -1;
            }
            if (c[i] >= 0 && cl[i] == q[i]) {
                a.bond_of_lig[q[i]] = c[i];
                a.owner[c[i]] = q[i];
                a.owner_cell[pc[i]] = q[i];
            }
        }
    }
    __syncthreads();  // every claim has been read before any is cleared
    if (one_pass) {
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int q = threadIdx.x + i * blockDim.x;
            if (keep_c[i] >= 0) {
                a.claim[keep_c[i]] = INT_MAX;
                a.cand[q] = -1;
            }
        }
    } else {
        for (int q = threadIdx.x; q < a.nlig; q += blockDim.x) {
            const int c = __ldcg(&a.cand[q]);
            if (c >= 0) {
                a.claim[c] = INT_MAX;
                a.cand[q] = -1;
            }
        }
    }
}

}  // namespace lbib
