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
__global__ void __launch_bounds__(128) k_bonds(const MarkerArgs a) {
    const int l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long step = *a.d_step;
    if (l < a.nlig) {  // warp-uniform
        const int va = a.lig_a[l], vb = a.lig_b[l];
        const double cxp = 0.5 * (a.X[2 * va] + a.X[2 * vb]);
        const double cyp = 0.5 * (a.X[2 * va + 1] + a.X[2 * vb + 1]);
        bool look = isfinite(cxp) && isfinite(cyp);  // non-finite positions: reported by the advance
        const int r = a.bond_of_lig[l];
        if (look && r >= 0) {
            int rupture = 0;
            if (lane == 0) {
                const double d = lig_rec_dist(a, cxp, cyp, r);
                rupture = d >= a.d_break;
                if (!rupture) rupture = bond_uniform(a, step, l, r, 1) < p_rupture(a, d);
                if (rupture) a.rupt[l] = r;
            }
            look = __shfl_sync(0xffffffffu, rupture, 0) != 0;
        }
        int best = INT_MAX;
        if (look) {
            // receptors within d_cut lie in the 3x3 block of grid cells around the ligand point
            const double xw = cxp - (double)a.nx * floor(cxp * a.inv_nx);
            int gx = (int)floor(xw * a.inv_rc_w);
            gx = gx >= a.rc_nx ? a.rc_nx - 1 : (gx < 0 ? 0 : gx);
            const int gy = (int)fmin(fmax(floor((cyp - a.rc_y0) * a.inv_rc_h), -4.0), (double)a.rc_ny + 4.0);
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
                        const double d2 = lig_rec_dist2(a, cxp, cyp, rr);
                        if (!(d2 < a.d_cut2)) continue;  // clearly beyond the cut-off
                        const double d = sqrt(d2);
                        if (!(d < a.d_cut)) continue;
                        if (bond_uniform(a, step, l, rr, 0) < p_form(a, d)) best = rr;
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

cudaError_t launch_bonds(const MarkerArgs& a, cudaStream_t s) {
    if (a.nlig > 0 && a.nrec > 0) k_bonds<<<(a.nlig + 3) / 4, 128, 0, s>>>(a);
    return cudaGetLastError();
}

int bond_kernel_count(const MarkerArgs& a) { return (a.nlig > 0 && a.nrec > 0) ? 1 : 0; }

}  // namespace lbib
