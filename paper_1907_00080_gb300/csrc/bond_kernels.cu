// Ligand-receptor bond kinetics: rupture, then formation, decided in FP64 with
// counter-based Philox draws so that the bond history is reproducible and
// independent of thread scheduling.
//
// Paper: Coclite, arXiv 1907.00080, Sec. 2.2 (wall-particle interaction: bonds
// form below a critical separation, a forward probability governs formation
// and a reverse probability governs rupture each step) and Sec. 3 (k_f/k_r0).
// Philox4x64-10: Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11 -- implemented here from that definition.
#include <climits>

#include "ext_real.cuh"
#include "lbib_internal.cuh"

namespace lbib {

__device__ __forceinline__ void philox4x64_10(unsigned long long c[4], unsigned long long k0,
                                              unsigned long long k1) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
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

__device__ __forceinline__ double p_form(const MarkerArgs& a, double d) {
    const double z = (d - a.y_eq) * a.inv_y_eq;
    return 1.0 - exp(-a.kf_dt * exp(-a.beta_f * z * z));
}
__device__ __forceinline__ double p_rupture(const MarkerArgs& a, double d) {
    const double z = (d - a.y_eq) * a.inv_y_eq;
    return 1.0 - exp(-a.kr0_dt * exp(a.beta_r * z * z));
}

// periodic minimum image (multiplication by 1/L: no FP64 division)
__device__ __forceinline__ double wrapd(double d, double L, double invL) { return d - L * floor(d * invL + 0.5); }

__device__ __forceinline__ double lig_rec_dist2(const MarkerArgs& a, double cxp, double cyp, int r) {
    const double dx = wrapd(a.rec_xy[2 * r] - cxp, (double)a.nx, a.inv_nx);
    double dy = a.rec_xy[2 * r + 1] - cyp;
    if (!a.walls) dy = wrapd(dy, (double)a.ny, a.inv_ny);
    return dx * dx + dy * dy;
}
__device__ __forceinline__ double lig_rec_dist(const MarkerArgs& a, double cxp, double cyp, int r) {
    return sqrt(lig_rec_dist2(a, cxp, cyp, r));
}

// FP32 estimates used to settle clear-cut decisions without the FP64 pipe;
// anything within kMargin of the threshold is decided again in FP64, so the
// outcome is the FP64 decision.  The estimates are accurate to ~1e-6.
constexpr float kMargin = 1e-5f;
__device__ __forceinline__ float p_form_f(const MarkerArgs& a, float d) {
    const float z = (d - float(a.y_eq)) * float(a.inv_y_eq);
    return 1.0f - expf(-float(a.kf_dt) * expf(-float(a.beta_f) * z * z));
}
__device__ __forceinline__ float p_rupture_f(const MarkerArgs& a, float d) {
    const float z = (d - float(a.y_eq)) * float(a.inv_y_eq);
    return 1.0f - expf(-float(a.kr0_dt) * expf(float(a.beta_r) * z * z));
}

// Ligand point (element centroid) and its distance to receptor r: the cheap
// estimate in the compute precision, and the FP64 value on demand.
template <typename C>
struct LigandPoint {
    typename Ext<C>::E cx, cy;
    double cxd, cyd;
    bool have_d;
    __device__ void init(const MarkerArgs& a, int l) {
        typename Ext<C>::E xa, ya, xb, yb;
        PosIO<C>::load(a.X, a.lig_a[l], xa, ya);
        PosIO<C>::load(a.X, a.lig_b[l], xb, yb);
        cx = emulc(eadd(xa, xb), C(0.5));
        cy = emulc(eadd(ya, yb), C(0.5));
        have_d = false;
    }
    __device__ bool finite() const { return isfinite(ehi(cx)) && isfinite(ehi(cy)); }
    __device__ C dist_est(const MarkerArgs& a, int r) const {
        typename Ext<C>::E rx, ry;
        PosIO<C>::load(a.rec_e, r, rx, ry);
        const C dx = etoc(ewrap(esub(rx, cx), C(a.nx), C(a.inv_nx)));
        C dy = etoc(esub(ry, cy));
        if (!a.walls) dy = etoc(ewrap(esub(ry, cy), C(a.ny), C(a.inv_ny)));
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

// Eq.-free decisions of the bond model: `below(u, P)` style tests with the FP32
// estimate first and FP64 where the estimate cannot settle it
template <typename C>
__device__ bool forms(const MarkerArgs& a, LigandPoint<C>& lp, long long step, int l, int r) {
    if (sizeof(C) == 8) {
        const double d = lp.dist(a, r);
        if (!(d < a.d_cut)) return false;
        return bond_uniform(a, step, l, r, 0) < p_form(a, d);
    }
    const float df = float(lp.dist_est(a, r));
    const float dc = float(a.d_cut);
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

template <typename C>
__device__ bool ruptures(const MarkerArgs& a, LigandPoint<C>& lp, long long step, int l, int r) {
    if (sizeof(C) == 8) {
        const double d = lp.dist(a, r);
        if (d >= a.d_break) return true;
        return bond_uniform(a, step, l, r, 1) < p_rupture(a, d);
    }
    const float df = float(lp.dist_est(a, r));
    const float db = float(a.d_break);
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

// Last-block epilogue: every block counts itself in once it is done; the block
// that arrives last (it sees all other blocks' writes after the fences) runs the
// epilogue and resets the counter.  No block ever waits for another.
__device__ bool arrive_last_b(unsigned int* counter) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// One warp per ligand: lane 0 tests the existing bond for rupture; then the
// lanes share the receptors of the 3x3 cell block around the ligand point, each
// keeps the lowest id that passes the formation test, a warp minimum gives the
// candidate (the first accepted receptor in ascending id), claimed with
// atomicMin so that the lowest ligand id wins.  The last block to finish applies
// ruptures and winning claims for all ligands, clears the claims and advances
// the step counter.
template <typename C>
__global__ void __launch_bounds__(128) k_bonds(const MarkerArgs a) {
    const int l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long step = *a.d_step;
    if (l < a.nlig) {  // warp-uniform
        LigandPoint<C> lp;
        lp.init(a, l);
        bool look = lp.finite();  // non-finite positions: reported by the advance
        const int r = a.bond_of_lig[l];
        if (look && r >= 0) {
            int rupture = 0;
            if (lane == 0) {
                rupture = ruptures<C>(a, lp, step, l, r);
                if (rupture) a.rupt[l] = r;
            }
            look = __shfl_sync(0xffffffffu, rupture, 0) != 0;
        }
        int best = INT_MAX;
        if (look) {
            // receptors within d_cut lie in the 3x3 block of grid cells around the ligand point
            const float cxh = float(ehi(lp.cx)), cyh = float(ehi(lp.cy));
            const float Lx = float(a.nx);
            const float xw = cxh - Lx * floorf(cxh / Lx);
            int gx = (int)floorf(xw * float(a.inv_rc_w));
            gx = gx >= a.rc_nx ? a.rc_nx - 1 : (gx < 0 ? 0 : gx);
            const int gy = (int)fminf(fmaxf(floorf((cyh - float(a.rc_y0)) * float(a.inv_rc_h)), -4.f),
                                      float(a.rc_ny) + 4.f);
            int t = 0;  // running index over the candidate receptors
            for (int qy = gy - 1; qy <= gy + 1; ++qy) {
                if (qy < 0 || qy >= a.rc_ny) continue;
                for (int qx = gx - 1; qx <= gx + 1; ++qx) {
                    const int cxc = ((qx % a.rc_nx) + a.rc_nx) % a.rc_nx;
                    const int cell = qy * a.rc_nx + cxc;
                    const int p0 = a.rcell_start[cell], p1 = a.rcell_start[cell + 1];
                    for (int p = p0 + ((lane - t) % 32 + 32) % 32; p < p1; p += 32) {
                        const int rr = a.rcell_ids[p];
                        if (rr >= best || a.owner[rr] >= 0) continue;  // bound at the start of the step
                        if (forms<C>(a, lp, step, l, rr)) best = rr;
                    }
                    t += p1 - p0;
                }
            }
            for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
        }
        if (lane == 0 && best != INT_MAX) {
            a.cand[l] = best;
            atomicMin(&a.claim[best], l);
        }
    }
    if (!arrive_last_b(&a.tickets[1])) return;
    // epilogue (last block): other blocks' writes are read past L1
    for (int q = threadIdx.x; q < a.nlig; q += blockDim.x) {
        const int r_old = __ldcg(&a.rupt[q]);
        if (r_old >= 0) {
            a.owner[r_old] = -1;
            a.bond_of_lig[q] = -1;
            a.rupt[q] = -1;
        }
        const int c = __ldcg(&a.cand[q]);
        if (c >= 0 && __ldcg(&a.claim[c]) == q) {
            a.bond_of_lig[q] = c;
            a.owner[c] = q;
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < a.nlig; q += blockDim.x) {
        const int c = __ldcg(&a.cand[q]);
        if (c >= 0) {
            a.claim[c] = INT_MAX;
            a.cand[q] = -1;
        }
    }
    if (threadIdx.x == 0) {
        *a.d_step += 1;
        a.tickets[1] = 0;
    }
}

cudaError_t launch_bonds(lbib_precision prec, const MarkerArgs& a, cudaStream_t s) {
    if (a.nlig > 0 && a.nrec > 0) {
        if (prec == LBIB_F64) k_bonds<double><<<(a.nlig + 3) / 4, 128, 0, s>>>(a);
        else k_bonds<float><<<(a.nlig + 3) / 4, 128, 0, s>>>(a);
    }
    return cudaGetLastError();
}

int bond_kernel_count(const MarkerArgs& a) { return (a.nlig > 0 && a.nrec > 0) ? 1 : 0; }

}  // namespace lbib
