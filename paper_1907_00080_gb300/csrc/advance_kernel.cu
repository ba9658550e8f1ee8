// Interpolation, kinematic advance and bond kinetics in one kernel.
//
// One block of a.adv_threads (<= kAdvThreads) threads per unit: a chunk of up to kChunkV vertices
// of a kinematic membrane or a deformable dynamic particle, or a whole
// rigid-projected membrane or rigid dynamic particle (one vertex per thread;
// the velocities of the former are first projected on their least-squares
// rigid motion, the latter follows Newton-Euler).  Per vertex: interpolate
// u^n (Sec. 2.3), advance with Eq. kinematicPos (BDF2; forward Euler on the
// first step), refresh the repulsion boxes.  Then the ligands whose element
// lies inside the unit are decided at X^{n+1} (bond_logic.cuh); the last
// block to finish decides the few ligands whose element straddles two units,
// applies ruptures and formations for all ligands and advances the step
// counter.
#include "marker_common.cuh"

namespace lbib {

constexpr int kAdvThreads = 4 * kChunkV;  // most threads per unit: one vertex each of a rigid ring (<= 256)
constexpr int kMaxPairs = 512;  // (ligand, receptor) formation candidates staged per block

// receptor position p of the cell-ordered array
template <typename C>
__device__ __forceinline__ typename Ext<C>::E ehi_pos_x(const MarkerArgs& a, int p) {
    typename Ext<C>::E x, y;
    PosIO<C>::load(a.rcell_pos, p, x, y);
    return x;
}
template <typename C>
__device__ __forceinline__ typename Ext<C>::E ehi_pos_y(const MarkerArgs& a, int p) {
    typename Ext<C>::E x, y;
    PosIO<C>::load(a.rcell_pos, p, x, y);
    return y;
}

template <typename C>
__device__ __forceinline__ void load_pos_cg(const void* X, int v, typename Ext<C>::E& x,
                                            typename Ext<C>::E& y);
template <>
__device__ __forceinline__ void load_pos_cg<double>(const void* X, int v, double& x, double& y) {
    const double* p = static_cast<const double*>(X);
    x = __ldcg(p + 2 * v);
    y = __ldcg(p + 2 * v + 1);
}
template <>
__device__ __forceinline__ void load_pos_cg<float>(const void* X, int v, ff& x, ff& y) {
    const float4 q = __ldcg(static_cast<const float4*>(X) + v);
    x = ff{q.x, q.z};
    y = ff{q.y, q.w};
}

// Eqs. verletPos / verletVel of a deformable dynamic particle: the vertex moves
// by the interpolated velocity (the first tentative velocity) plus F / (2 m_v)
// (F the total force of this step, m_v = rho_P A_0 / n); its velocity is the
// backward difference 3/2 (x^{n+1} - x^n) - 1/2 (x^n - x^{n-1}) (first-order on
// the first step)
template <typename C>
__device__ __forceinline__ void verlet(const MarkerArgs& a, int m, int v, typename Ext<C>::E x,
                                       typename Ext<C>::E y, typename Ext<C>::E xp, typename Ext<C>::E yp,
                                       C Ux, C Uy, long long step, typename Ext<C>::E& xn,
                                       typename Ext<C>::E& yn) {
    const C* F = static_cast<const C*>(a.F);
    C* V = static_cast<C*>(a.V);
    const C mv = C(a.mem_dyn[3 * m + 2]);
    xn = eaddc(x, Ux + (C(0.5) * F[2 * (size_t)v]) / mv);
    yn = eaddc(y, Uy + (C(0.5) * F[2 * (size_t)v + 1]) / mv);
    if (step == 0) {
        V[2 * (size_t)v] = etoc(esub(xn, x));
        V[2 * (size_t)v + 1] = etoc(esub(yn, y));
    } else {
        V[2 * (size_t)v] = C(1.5) * etoc(esub(xn, x)) - C(0.5) * etoc(esub(x, xp));
        V[2 * (size_t)v + 1] = C(1.5) * etoc(esub(yn, y)) - C(0.5) * etoc(esub(y, yp));
    }
}

// repulsion boxes of a whole ring whose new positions are in shared memory:
// kSegV lanes per segment
template <typename C>
__device__ __forceinline__ void ring_boxes(const MarkerArgs& a, int m, int n, int tid, int lane,
                                           const typename Ext<C>::E* s_x, const typename Ext<C>::E* s_y) {
    const int per_pass = blockDim.x / kSegV;
    const int s0 = a.mem_seg_off[m], s1 = a.mem_seg_off[m + 1];
    for (int base = 0; base < s1 - s0; base += per_pass) {
        const int si = base + tid / kSegV;
        const int kfirst = si * kSegV;
        const int g = tid & (kSegV - 1);
        const bool ok = si < s1 - s0;
        const int kk = ok ? (kfirst + g < n ? kfirst + g : kfirst) : 0;
        seg_box_regs<C>(a, ok ? s0 + si : -1, lane, s_x[kk], s_y[kk]);
    }
}

// DYN: the context holds dynamic particles (without them their paths are not
// compiled into the kernel, which keeps its code small)
//
// advance_unit is the body for advance unit `u` of the context `a`, whose
// advance launch has `nblocks` blocks in all (the last of them to finish runs
// the epilogue): the single-context kernel runs unit blockIdx.x of gridDim.x,
// the batched kernel (ensembles) one unit of one member per block.
template <typename C, bool DYN>
__device__ __forceinline__ void advance_unit(const MarkerArgs& a, int u, unsigned nblocks) {
    using E = typename Ext<C>::E;
    const int4 u0 = a.au[2 * u], u1 = a.au[2 * u + 1];
    const int m = u0.x, k0 = u0.y, kn = u0.z, off = u0.w, n = u1.x, kind = u1.y;
    const int tid = threadIdx.x, lane = tid & 31;
    __shared__ E s_x[kAdvThreads], s_y[kAdvThreads];
    __shared__ C cred[4 * 33];
    __shared__ bool s_last;
    const long long step = *a.d_step;
    C* U = static_cast<C*>(a.U);
    // the unit's ligand records and current bonds, fetched now so that their
    // latency overlaps the marker advance (a unit has at most one ligand per thread)
    const int lq0 = u1.z;
    const int nlq = a.nrec > 0 ? u1.w : 0;
    int4 my_rec = make_int4(-1, 0, 0, 0);
    int my_bond = -1;
    if (tid < nlq) {
        my_rec = a.au_ligs[lq0 + tid];
        my_bond = a.bond_of_lig[my_rec.x];
    }

    if (kind == LBIB_MEMBRANE_KINEMATIC || (DYN && kind == LBIB_MEMBRANE_DYNAMIC)) {
        // ---- kinematic or deformable dynamic chunk: one vertex per thread
        const bool valid = tid < kn;
        const int v = off + k0 + (valid ? tid : 0);
        E x, y, xp, yp, xn, yn;
        load_pos<C>(a, v, x, y);
        PosIO<C>::load(a.Xp, v, xp, yp);
        if (valid) {
            C Ux, Uy;
            interp_vertex<C>(a, v, Ux, Uy);
            U[2 * v] = Ux;
            U[2 * v + 1] = Uy;
            if (DYN && kind == LBIB_MEMBRANE_DYNAMIC) {
                verlet<C>(a, m, v, x, y, xp, yp, Ux, Uy, step, xn, yn);
            } else {
                bdf2<C>(x, xp, Ux, step, xn);
                bdf2<C>(y, yp, Uy, step, yn);
            }
            if (!isfinite(ehi(xn)) || !isfinite(ehi(yn))) atomicOr(a.status, ST_NONFINITE);
            PosIO<C>::store(a.Xp, v, x, y);
            PosIO<C>::store(a.X, v, xn, yn);
            s_x[tid] = xn;
            s_y[tid] = yn;
        } else {
            xn = x;
            yn = y;
        }
        // boxes of the repulsion segments of this chunk (chunks are segment-aligned)
        const int gfirst = tid & ~(kSegV - 1);
        const int sg = gfirst < kn ? a.mem_seg_off[m] + (k0 + gfirst) / kSegV : -1;
        E gx, gy;
        shfl_e(gx, xn, lane & ~(kSegV - 1));
        shfl_e(gy, yn, lane & ~(kSegV - 1));
        seg_box_regs<C>(a, sg, lane, valid ? xn : gx, valid ? yn : gy);
    } else if (DYN && kind == LBIB_MEMBRANE_DYNAMIC_RIGID) {
        // ---- rigid dynamic particle, the whole ring in this block: Eqs.
        // linearVelRig / angularVelRig.  F and its moment M about the area
        // centroid give du/dt = F/m, domega/dt = M/I; the body translates by u
        // and turns by omega about its centroid (cos omega - 1 = -2 sin^2(omega/2))
        E xr, yr;
        load_pos<C>(a, off, xr, yr);
        const int k = tid;
        const bool valid = k < n;
        const C* F = static_cast<const C*>(a.F);
        E x, y;
        C Ux = 0, Uy = 0, ax = 0, ay = 0, bx = 0, by = 0, fx = 0, fy = 0;
        if (valid) {
            E xq, yq;
            load_pos<C>(a, off + k, x, y);
            load_pos<C>(a, off + (k + 1 == n ? 0 : k + 1), xq, yq);
            interp_vertex<C>(a, off + k, Ux, Uy);
            ax = etoc(esub(x, xr));
            ay = etoc(esub(y, yr));
            bx = etoc(esub(xq, xr));
            by = etoc(esub(yq, yr));
            fx = F[2 * (size_t)(off + k)];
            fy = F[2 * (size_t)(off + k) + 1];
        }
        // area centroid relative to vertex 0 from the triangles (vertex 0, k, k+1)
        const C cr = ax * by - ay * bx;
        C s2 = cr, gsx = cr * (ax + bx), gsy = cr * (ay + by), z0 = 0;
        block_sum4_c<C>(s2, gsx, gsy, z0, cred);
        const C gx = gsx / (C(3) * s2), gy = gsy / (C(3) * s2);
        const C rx = ax - gx, ry = ay - gy;
        // the rigid state is read by every thread before thread 0 rewrites it
        double* rb = a.rb + 6 * m;
        const double u0 = rb[0], v0 = rb[1], up = rb[2], vp = rb[3], w0 = rb[4], wp = rb[5];
        C Fx = fx, Fy = fy, Mz = valid ? rx * fy - ry * fx : C(0), z1 = 0;
        block_sum4_c<C>(Fx, Fy, Mz, z1, cred);
        const double mass = a.mem_dyn[3 * m], inertia = a.mem_dyn[3 * m + 1];
        const double axd = double(Fx) / mass, ayd = double(Fy) / mass, ald = double(Mz) / inertia;
        double un, vn, wn;
        if (step == 0) {
            un = u0 + axd;
            vn = v0 + ayd;
            wn = w0 + ald;
        } else {
            un = (2.0 / 3.0) * (2.0 * u0 - 0.5 * up + axd);
            vn = (2.0 / 3.0) * (2.0 * v0 - 0.5 * vp + ayd);
            wn = (2.0 / 3.0) * (2.0 * w0 - 0.5 * wp + ald);
        }
        if (tid == 0) {
            rb[2] = u0;
            rb[3] = v0;
            rb[5] = w0;
            rb[0] = un;
            rb[1] = vn;
            rb[4] = wn;
        }
        const C hs = sin(C(0.5) * C(wn));
        const C c1 = C(-2) * hs * hs, sn = sin(C(wn));
        if (valid) {
            const int v = off + k;
            const C drx = c1 * rx - sn * ry, dry = sn * rx + c1 * ry;
            C* V = static_cast<C*>(a.V);
            V[2 * (size_t)v] = C(un) - C(wn) * (ry + dry);
            V[2 * (size_t)v + 1] = C(vn) + C(wn) * (rx + drx);
            U[2 * v] = Ux;
            U[2 * v + 1] = Uy;
            const E xn = eaddc(x, C(un) + drx), yn = eaddc(y, C(vn) + dry);
            if (!isfinite(ehi(xn)) || !isfinite(ehi(yn))) atomicOr(a.status, ST_NONFINITE);
            PosIO<C>::store(a.Xp, v, x, y);
            PosIO<C>::store(a.X, v, xn, yn);
            s_x[k] = xn;
            s_y[k] = yn;
        }
        __syncthreads();
        ring_boxes<C>(a, m, n, tid, lane, s_x, s_y);
    } else {
        // ---- rigid-projected membrane: the whole ring in this block
        E xr, yr;
        load_pos<C>(a, off, xr, yr);
        const int k = tid;
        const bool valid = k < n;
        E x, y, xpv, ypv;
        C Ux = 0, Uy = 0;
        C sx = 0, sy = 0, su = 0, sv = 0;
        if (valid) {
            load_pos<C>(a, off + k, x, y);
            PosIO<C>::load(a.Xp, off + k, xpv, ypv);
            interp_vertex<C>(a, off + k, Ux, Uy);
            sx = etoc(esub(x, xr));
            sy = etoc(esub(y, yr));
            su = Ux;
            sv = Uy;
        }
        // least-squares rigid motion U_c + omega x (x - x_c), positions about vertex 0
        const C inv_n = C(1) / C(n);
        block_sum4_c<C>(sx, sy, su, sv, cred);
        const C mx = sx * inv_n, my = sy * inv_n, mu = su * inv_n, mv = sv * inv_n;
        C num = 0, den = 0;
        if (valid) {
            const C rx = etoc(esub(x, xr)) - mx, ry = etoc(esub(y, yr)) - my;
            num = rx * (Uy - mv) - ry * (Ux - mu);
            den = rx * rx + ry * ry;
        }
        C z0 = 0, z1 = 0;
        block_sum4_c<C>(num, den, z0, z1, cred);
        const C om = num / den;
        if (valid) {
            const int v = off + k;
            const C rx = etoc(esub(x, xr)) - mx, ry = etoc(esub(y, yr)) - my;
            const C px = mu - om * ry, py = mv + om * rx;
            U[2 * v] = px;
            U[2 * v + 1] = py;
            E xn, yn;
            bdf2<C>(x, xpv, px, step, xn);
            bdf2<C>(y, ypv, py, step, yn);
            if (!isfinite(ehi(xn)) || !isfinite(ehi(yn))) atomicOr(a.status, ST_NONFINITE);
            PosIO<C>::store(a.Xp, v, x, y);
            PosIO<C>::store(a.X, v, xn, yn);
            s_x[k] = xn;
            s_y[k] = yn;
        }
        __syncthreads();
        ring_boxes<C>(a, m, n, tid, lane, s_x, s_y);
    }
    __syncthreads();

    // ---- bond decisions for the ligands whose element lies inside this unit.
    // (a) per ligand: rupture test of its bond, and the receptors of the 3x3
    //     cells around it that were free at the start of the step, as
    //     (ligand, receptor) pairs;
    // (b) per pair: the formation test; each ligand keeps the lowest passing
    //     receptor id (a minimum: independent of evaluation order);
    // (c) per ligand that is free after (a): claim its receptor.
    if (nlq > 0) {
        __shared__ int s_pl[kMaxPairs], s_pr[kMaxPairs];
        __shared__ int s_best[kAdvThreads];
        __shared__ int s_look[kAdvThreads];
        __shared__ int s_lig[kAdvThreads], s_ka[kAdvThreads], s_kb[kAdvThreads];
        __shared__ int s_np;
        if (tid == 0) s_np = 0;
        __syncthreads();
        for (int q = tid; q < nlq; q += blockDim.x) {
            const int4 rec = my_rec;  // q == tid: a unit has no more ligands than threads
            const int l = rec.x, ka = rec.y, kb = rec.z;
            s_lig[q] = l;
            s_ka[q] = ka;
            s_kb[q] = kb;
            LigandPoint<C> lp;
            lp.init(s_x[ka], s_y[ka], s_x[kb], s_y[kb]);
            s_best[q] = INT_MAX;
            bool look = lp.finite();  // non-finite positions: reported above
            const int r = my_bond;
            if (look && r >= 0) {
                look = ruptures<C>(a, lp, step, l, r);
                if (look) a.rupt[l] = r;
            }
            s_look[q] = look;
            if (!look) continue;
            int p0[9], p1[9];
            ligand_cells<C>(a, lp, p0, p1);
            // every receptor of the cells becomes a pair; whether it was free at
            // the start of the step is checked per pair, in parallel
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                for (int p = p0[c]; p < p1[c]; ++p) {
                    const int slot = atomicAdd(&s_np, 1);
                    if (slot < kMaxPairs) {
                        s_pl[slot] = q;
                        s_pr[slot] = p;
                    } else {
                        // list full: decide in place
                        const int rr = a.rcell_ids[p];
                        if (a.owner_cell[p] < 0 && forms<C>(a, lp, step, l, rr, ehi_pos_x<C>(a, p), ehi_pos_y<C>(a, p)))
                            atomicMin(&s_best[q], rr);
                    }
                }
            }
        }
        __syncthreads();
        const int np = s_np < kMaxPairs ? s_np : kMaxPairs;
        for (int t = tid; t < np; t += blockDim.x) {
            const int q = s_pl[t], p = s_pr[t];
            const int rr = a.rcell_ids[p];
            typename Ext<C>::E rx, ry;
            PosIO<C>::load(a.rcell_pos, p, rx, ry);
            if (a.owner_cell[p] >= 0) continue;  // bound at the start of the step
            const int l = s_lig[q], ka = s_ka[q], kb = s_kb[q];
            LigandPoint<C> lp;
            lp.init(s_x[ka], s_y[ka], s_x[kb], s_y[kb]);
            if (forms<C>(a, lp, step, l, rr, rx, ry)) atomicMin(&s_best[q], rr);
        }
        __syncthreads();
        for (int q = tid; q < nlq; q += blockDim.x) {
            const int best = s_best[q];
            if (s_look[q] && best != INT_MAX) {
                const int l = s_lig[q];
                a.cand[l] = best;
                atomicMin(&a.claim[best], l);
            }
        }
    }

    // ---- epilogue of the last block: straddling ligands, apply, next step
    if (!arrive_last(&a.tickets[0], &s_last, nblocks)) return;
    for (int q = tid; q < (a.nrec > 0 ? a.nstrad : 0); q += blockDim.x) {
        const int l = a.strad_ligs[q];
        E xa, ya, xb, yb;
        load_pos_cg<C>(a.X, a.lig_a[l], xa, ya);
        load_pos_cg<C>(a.X, a.lig_b[l], xb, yb);
        LigandPoint<C> lp;
        lp.init(xa, ya, xb, yb);
        bond_decide<C>(a, l, lp, step);
    }
    __syncthreads();
    if (a.nlig > 0 && a.nrec > 0) bond_apply_all(a);
    __syncthreads();
    if (tid == 0) {
        *a.d_step += 1;
        a.tickets[0] = 0;
    }
}

template <typename C, bool DYN>
__global__ void __launch_bounds__(kAdvThreads) k_advance(const MarkerArgs a) {
    advance_unit<C, DYN>(a, blockIdx.x, gridDim.x);
}

// Batched form: the advance units of up to kBatchMax contexts (ensemble
// members) in one launch, one block per (member, unit); each member's last
// block runs its epilogue.  Blocks have the threads of the widest member (idle
// threads beyond a unit's vertices, as in the single-context kernel).
template <typename C, bool DYN>
__global__ void __launch_bounds__(kAdvThreads) k_advance_batch(const __grid_constant__ MarkerBatch b) {
    __shared__ MarkerArgs s_a;
    const int m = marker_member(b, blockIdx.x);
    stage_args(&s_a, b.args + m);
    advance_unit<C, DYN>(s_a, blockIdx.x - b.off[m], (unsigned)s_a.nau);
}

cudaError_t launch_advance(lbib_precision prec, const MarkerArgs& a, cudaStream_t s) {
    if (a.adv_threads < kChunkV || a.adv_threads > kAdvThreads || a.adv_threads % 32) return cudaErrorInvalidValue;
    if (prec == LBIB_F64) {
        if (a.has_dyn) k_advance<double, true><<<a.nau, a.adv_threads, 0, s>>>(a);
        else k_advance<double, false><<<a.nau, a.adv_threads, 0, s>>>(a);
    } else {
        if (a.has_dyn) k_advance<float, true><<<a.nau, a.adv_threads, 0, s>>>(a);
        else k_advance<float, false><<<a.nau, a.adv_threads, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_advance_batch(lbib_precision prec, bool dyn, const MarkerBatch& b, int threads, cudaStream_t s) {
    if (b.n < 1 || b.n > kBatchMax) return cudaErrorInvalidValue;
    const int nunits = b.off[b.n];
    if (nunits <= 0) return cudaSuccess;
    if (threads < kChunkV || threads > kAdvThreads || threads % 32) return cudaErrorInvalidValue;
    if (prec == LBIB_F64) {
        if (dyn) k_advance_batch<double, true><<<nunits, threads, 0, s>>>(b);
        else k_advance_batch<double, false><<<nunits, threads, 0, s>>>(b);
    } else {
        if (dyn) k_advance_batch<float, true><<<nunits, threads, 0, s>>>(b);
        else k_advance_batch<float, false><<<nunits, threads, 0, s>>>(b);
    }
    return cudaGetLastError();
}

}  // namespace lbib
