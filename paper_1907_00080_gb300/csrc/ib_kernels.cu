// Lagrangian-side kernels: membrane forces (stretching, bending, enclosed
// area, repulsion, bond springs), the IB shape functions and the spreading of
// the marker forces, and the interpolation + kinematic advance.
//
// Paper: Coclite, arXiv 1907.00080, Sec. 2.2 (Eqs. strainFor, bendFor,
// areaFor, repFor, adhFor; MLS exchange), Sec. 2.3 (nine Eulerian points per
// vertex, Eq. kinematicPos).
//
// Precision: the compute type C is double in FP64 mode and float otherwise;
// positions and every cancellation-prone product use the matching extended
// type E (double, or float-float) from ext_real.cuh.
#include <climits>

#include "ext_real.cuh"
#include "lbib_internal.cuh"

namespace lbib {

constexpr unsigned FULL = 0xffffffffu;

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

// Edge products at a vertex in the extended type: squared length of
// e_R = x_{v+1} - x_v, and the cross and dot products of e_L = x_v - x_{v-1}
// with e_R (their rotation from the rest pair gives theta - theta_0).
template <typename C>
struct EdgeProducts {
    typename Ext<C>::E lsqR, cross, dot;
};
template <typename C>
__device__ __forceinline__ EdgeProducts<C> edge_products(const MarkerArgs& a, int L, int v, int R) {
    using E = typename Ext<C>::E;
    E xL, yL, xv, yv, xR, yR;
    load_pos<C>(a, L, xL, yL);
    load_pos<C>(a, v, xv, yv);
    load_pos<C>(a, R, xR, yR);
    const E eLx = esub(xv, xL), eLy = esub(yv, yL), eRx = esub(xR, xv), eRy = esub(yR, yv);
    EdgeProducts<C> p;
    p.lsqR = eadd(emul(eRx, eRx), emul(eRy, eRy));
    p.cross = esub(emul(eLx, eRy), emul(eLy, eRx));
    p.dot = eadd(emul(eLx, eRx), emul(eLy, eRy));
    return p;
}

// Enclosed area of membrane m by the shoelace formula about vertex 0, summed by
// warp 0 of the calling block in a fixed order (lane l takes terms l, l+32, ...,
// then a fixed tree), so every caller gets the same bits.  The result is in
// red[32] after the call; all threads of the block must call it.
template <typename C>
__device__ void ring_area(const MarkerArgs& a, int m, typename Ext<C>::E* red) {
    using E = typename Ext<C>::E;
    const int off = a.mem_off[m], n = a.mem_n[m];
    if (threadIdx.x < 32) {
        E xr, yr;
        load_pos<C>(a, off, xr, yr);
        E acc = ezero<E>();
        for (int k = threadIdx.x; k < n; k += 32) {
            const int R = k == n - 1 ? 0 : k + 1;
            E xv, yv, xR, yR;
            load_pos<C>(a, off + k, xv, yv);
            load_pos<C>(a, off + R, xR, yR);
            const E t = esub(emul(esub(xv, xr), esub(yR, yr)), emul(esub(xR, xr), esub(yv, yr)));
            acc = eadd(acc, t);
        }
        red[threadIdx.x] = acc;
        __syncwarp();
        for (int o = 16; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] = eadd(red[threadIdx.x], red[threadIdx.x + o]);
            __syncwarp();
        }
        if (threadIdx.x == 0) red[32] = emulc(red[0], C(0.5));
    }
    __syncthreads();
}

// block-wide sum in the compute type (all threads get it)
template <typename C>
__device__ C block_sum_c(C v, C* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        C t = threadIdx.x < nw ? red[threadIdx.x] : C(0);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(FULL, t, o);
        if (threadIdx.x == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// ---------------------------------------------------------------- rest state
// Captures, per vertex, the squared and plain rest length of the element
// (v, v+1) and the rest cross/dot products of the two edges at v (which fix the
// rest turning angle theta_0), plus A_0 per membrane -- with the arithmetic the
// force kernel repeats, so the rest shape gives exactly zero force.
template <typename C>
__global__ void k_rest(const MarkerArgs a, void* rest_v, double* A0) {
    using E = typename Ext<C>::E;
    const int m = blockIdx.x;
    const int off = a.mem_off[m], n = a.mem_n[m];
    __shared__ E red[33];
    Rest<C>* rest = static_cast<Rest<C>*>(rest_v);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int v = off + k, L = off + (k == 0 ? n - 1 : k - 1), R = off + (k == n - 1 ? 0 : k + 1);
        const EdgeProducts<C> p = edge_products<C>(a, L, v, R);
        Rest<C> r;
        r.lsq = p.lsqR;
        r.cross = p.cross;
        r.dot = p.dot;
        r.l0 = sqrt(etoc(p.lsqR));
        rest[v] = r;
    }
    ring_area<C>(a, m, red);
    if (threadIdx.x == 0) A0[m] = etod(red[32]);
}

// ---------------------------------------------------------------- forces
// Eq. adhFor on element e (if its ligand is bonded), half to the vertex
template <typename C>
__device__ __forceinline__ void bond_on_element(const MarkerArgs& a, int e, C& Fx, C& Fy) {
    using E = typename Ext<C>::E;
    const int l = a.elem_lig[e];
    if (l < 0) return;
    const int r = a.bond_of_lig[l];
    if (r < 0) return;
    E xa, ya, xb, yb;
    load_pos<C>(a, a.lig_a[l], xa, ya);
    load_pos<C>(a, a.lig_b[l], xb, yb);
    E rx, ry;
    PosIO<C>::load(a.rec_e, r, rx, ry);
    // receptor minus ligand point (element centroid)
    const E cx = emulc(eadd(xa, xb), C(0.5)), cy = emulc(eadd(ya, yb), C(0.5));
    const C dx = etoc(ewrap(esub(rx, cx), C(a.nx), C(a.inv_nx)));
    C dy = etoc(esub(ry, cy));
    if (!a.walls) dy = etoc(ewrap(esub(ry, cy), C(a.ny), C(a.inv_ny)));
    const C d = sqrt(dx * dx + dy * dy);
    const C c = C(a.sigma) * (d - C(a.y_eq)) / d;
    Fx += C(0.5) * c * dx;
    Fy += C(0.5) * c * dy;
}

// One block per work unit (a chunk of up to kChunkV consecutive vertices of one
// membrane); one thread per vertex.  Computes F^n, the nine shape functions at
// X^n and spreads w_j F_v into the fixed-point force field.
template <typename C>
__global__ void __launch_bounds__(kChunkV) k_forces(const MarkerArgs a) {
    using E = typename Ext<C>::E;
    const int m = a.fu[3 * blockIdx.x], k0 = a.fu[3 * blockIdx.x + 1], kn = a.fu[3 * blockIdx.x + 2];
    const int off = a.mem_off[m], n = a.mem_n[m];
    __shared__ C s_mnx[kChunkV + 2], s_mny[kChunkV + 2], s_sL[kChunkV + 2], s_sR[kChunkV + 2];
    __shared__ C s_nx[kChunkV + 2], s_ny[kChunkV + 2];
    __shared__ E red[33];
    const Rest<C>* rest = static_cast<const Rest<C>*>(a.rest);
    const C kb = C(a.mem_kb[m]);

    // enclosed area (Eq. areaFor) with p_ref = 1/3: F_l = c_a (inward normal) l_l
    ring_area<C>(a, m, red);
    const C ca = C(-a.mem_ka[m] * (1.0 - etod(red[32]) / a.mem_A0[m]) * (1.0 / 3.0));
    const C ks = C(a.mem_ks[m]);

    // vertex geometry of local slots j = 0..kn+1 (vertex k0 - 1 + j, wrapped).
    // theta - theta_0 comes from the rotation between the rest and the current
    // edge pair, atan2(c d0 - c0 d, d d0 + c c0), free of the cancellation of
    // subtracting two nearly equal angles.
    for (int j = threadIdx.x; j < kn + 2; j += blockDim.x) {
        int k = k0 - 1 + j;
        k = k < 0 ? k + n : (k >= n ? k - n : k);
        const int v = off + k, L = off + (k == 0 ? n - 1 : k - 1), R = off + (k == n - 1 ? 0 : k + 1);
        const EdgeProducts<C> p = edge_products<C>(a, L, v, R);
        const Rest<C> r0 = rest[v];
        const E sn = esub(emul(p.cross, r0.dot), emul(r0.cross, p.dot));
        const E cs = eadd(emul(p.dot, r0.dot), emul(p.cross, r0.cross));
        const C dth = atan2(etoc(sn), etoc(cs));
        E xL, yL, xv, yv, xR, yR;
        load_pos<C>(a, L, xL, yL);
        load_pos<C>(a, v, xv, yv);
        load_pos<C>(a, R, xR, yR);
        const C eLx = etoc(esub(xv, xL)), eLy = etoc(esub(yv, yL));
        const C eRx = etoc(esub(xR, xv)), eRy = etoc(esub(yR, yv));
        const C lL = sqrt(eLx * eLx + eLy * eLy), lR = sqrt(eRx * eRx + eRy * eRy);
        // outward vertex normal: normalised sum of the outward edge normals (CCW ring)
        C nx_ = eLy / lL + eRy / lR;
        C ny_ = -eLx / lL - eRx / lR;
        const C nn = sqrt(nx_ * nx_ + ny_ * ny_);
        nx_ /= nn;
        ny_ /= nn;
        const C mb = kb * dth;
        s_mnx[j] = mb * nx_;
        s_mny[j] = mb * ny_;
        s_sL[j] = lL / (lL + lR);
        s_sR[j] = lR / (lL + lR);
        s_nx[j] = nx_;
        s_ny[j] = ny_;
    }

    // Eq. repFor screening, once per block: the segments of other membranes
    // whose box comes within d_rep of a box of this chunk's own segments, kept in
    // ascending segment order (ballot prefix per warp) so sums are reproducible
    constexpr int kMaxCand = 256;
    __shared__ int s_cand[kMaxCand];
    __shared__ int s_wcnt[kChunkV / 32];
    __shared__ int s_ncand;
    if (threadIdx.x == 0) s_ncand = 0;
    const bool repel = a.nmem > 1;
    const float Lxf = float(a.nx), Lyf = float(a.ny);
    if (repel) {
        const float reach = float(a.d_rep) + 2e-3f;
        const int sown0 = a.mem_seg_off[m] + k0 / kSegV;
        const int sown1 = a.mem_seg_off[m] + (k0 + kn + kSegV - 1) / kSegV;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int base = 0; base < a.nseg; base += blockDim.x) {
            const int sg = base + threadIdx.x;
            bool hit = false;
            if (sg < a.nseg && a.seg_mem[sg] != m) {
                const float4 b = a.seg_box[sg];
                for (int so = sown0; so < sown1 && !hit; ++so) {
                    const float4 o = a.seg_box[so];
                    const float dx = wrap_half(b.x - o.x, Lxf);
                    float dy = b.y - o.y;
                    if (!a.walls) dy = wrap_half(dy, Lyf);
                    hit = fabsf(dx) <= b.z + o.z + reach && fabsf(dy) <= b.w + o.w + reach;
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, hit);
            __syncthreads();  // s_ncand of the previous pass is final
            if (lane == 0) s_wcnt[wid] = __popc(bal);
            __syncthreads();
            int pos = s_ncand;
            for (int w = 0; w < wid; ++w) pos += s_wcnt[w];
            pos += __popc(bal & ((1u << lane) - 1u));
            if (hit && pos < kMaxCand) s_cand[pos] = sg;
            __syncthreads();
            if (threadIdx.x == 0) {
                int t = s_ncand;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_wcnt[w];
                s_ncand = t;
            }
        }
    }
    __syncthreads();
    // more candidates than the list holds: fall back to screening every segment
    const int ncand = s_ncand;
    const bool all_segs = ncand > kMaxCand;

    C* F = static_cast<C*>(a.F);
    C* W = static_cast<C*>(a.W);
    const C c_rep = C(1e-4 / (8.0 * 1.4142135623730951));
    for (int j = threadIdx.x; j < kn; j += blockDim.x) {
        const int k = k0 + j;
        const int kL = k == 0 ? n - 1 : k - 1, kR = k == n - 1 ? 0 : k + 1;
        const int v = off + k, L = off + kL, R = off + kR;
        const int sj = j + 1;  // shared-memory slot of vertex k
        E xv, yv, xl, yl, xR, yR;
        load_pos<C>(a, v, xv, yv);
        load_pos<C>(a, L, xl, yl);
        load_pos<C>(a, R, xR, yR);
        C Fx = C(0), Fy = C(0);
        // Eq. adhFor on the two elements sharing v, half each
        if (a.nlig > 0) {
            bond_on_element<C>(a, L, Fx, Fy);
            bond_on_element<C>(a, v, Fx, Fy);
        }
        // Eq. repFor against vertices of other membranes closer than d_rep:
        // candidate segments, then a per-vertex box test, then exact pairs
        if (repel && ncand > 0) {
            const float hx = float(ehi(xv));
            const float xvw = hx - Lxf * floorf(hx / Lxf);
            const float yvf = float(ehi(yv));
            const float reach = float(a.d_rep) + 2e-3f;
            const int nscan = all_segs ? a.nseg : ncand;
            for (int ci = 0; ci < nscan; ++ci) {
                const int sg = all_segs ? ci : s_cand[ci];
                if (a.seg_mem[sg] == m) continue;
                const float4 bx = a.seg_box[sg];
                const float ddx = wrap_half(xvw - bx.x, Lxf);
                float ddy = yvf - bx.y;
                if (!a.walls) ddy = wrap_half(ddy, Lyf);
                if (fabsf(ddx) > bx.z + reach || fabsf(ddy) > bx.w + reach) continue;
                const int b0 = a.seg_v0[sg], nb = a.seg_n[sg];
                for (int b = b0; b < b0 + nb; ++b) {
                    E xb, yb;
                    load_pos<C>(a, b, xb, yb);
                    const C dx = etoc(ewrap(esub(xv, xb), C(a.nx), C(a.inv_nx)));
                    C dy = etoc(esub(yv, yb));
                    if (!a.walls) dy = etoc(ewrap(esub(yv, yb), C(a.ny), C(a.inv_ny)));
                    const C d = sqrt(dx * dx + dy * dy);
                    if (d < C(a.d_rep)) {
                        const C mag = c_rep * sqrt(C(1) / (d * d * d * d * d));
                        Fx -= mag * s_nx[sj];
                        Fy -= mag * s_ny[sj];
                    }
                }
            }
        }
        // Eq. strainFor on elements (v, R) and (L, v); l - l_0 is formed as
        // (l^2 - l_0^2) / (l + l_0) with the squares in the extended type
        {
            const E ex = esub(xR, xv), ey = esub(yR, yv);
            const E lsq = eadd(emul(ex, ex), emul(ey, ey));
            const C l = sqrt(etoc(lsq));
            const Rest<C> rv = rest[v];
            const C c = ks * etoc(esub(lsq, rv.lsq)) / ((l + rv.l0) * l);
            Fx += c * etoc(ex);
            Fy += c * etoc(ey);
            const E gx = esub(xv, xl), gy = esub(yv, yl);
            const E lsq2 = eadd(emul(gx, gx), emul(gy, gy));
            const C l2 = sqrt(etoc(lsq2));
            const Rest<C> rl = rest[L];
            const C c2 = -ks * etoc(esub(lsq2, rl.lsq)) / ((l2 + rl.l0) * l2);
            Fx += c2 * etoc(gx);
            Fy += c2 * etoc(gy);
        }
        // Eq. bendFor gathered: own term plus the neighbours' shares
        Fx += -s_mnx[sj] + s_mnx[sj + 1] * s_sL[sj + 1] + s_mnx[sj - 1] * s_sR[sj - 1];
        Fy += -s_mny[sj] + s_mny[sj + 1] * s_sL[sj + 1] + s_mny[sj - 1] * s_sR[sj - 1];
        // Eq. areaFor, half of each adjacent element
        Fx += C(0.5) * ca * (-etoc(esub(yR, yl)));
        Fy += C(0.5) * ca * etoc(esub(xR, xl));
        F[2 * (size_t)v] = Fx;
        F[2 * (size_t)v + 1] = Fy;

        // ---- IB shape functions at X^n: nine nearest nodes, Roma weights,
        // MLS (basis 1, dx, dy) re-solved where wall rows drop out.  Node
        // indices are clamped so that a runaway position still stays in range;
        // the advance kernel flags non-finite positions.
        const C fi0 = fmin(fmax(C(efloor(eaddc(xv, C(0.5)))), C(-1.0e7)), C(1.0e7));
        const C fj0 = fmin(fmax(C(efloor(eaddc(yv, C(0.5)))), C(-1.0e6)), C(1.0e6));
        const int i0 = (int)fi0;
        const int j0 = (int)fj0;
        C rx[3], ry[3], wx[3], wy[3];
        bool rowok[3];
        bool all = true;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            // node minus marker, (i0 + q - 1) - x
            rx[q] = -etoc(eaddc(xv, -(fi0 + C(q - 1))));
            ry[q] = -etoc(eaddc(yv, -(fj0 + C(q - 1))));
            wx[q] = roma<C>(rx[q]);
            wy[q] = roma<C>(ry[q]);
            const int jj = j0 + q - 1;
            rowok[q] = a.walls ? (jj >= 0 && jj < a.ny) : true;
            all = all && rowok[q];
        }
        C w[9];
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int q = 0; q < 3; ++q) w[b * 3 + q] = rowok[b] ? wx[q] * wy[b] : C(0);
        if (!all) {
            C M00 = 0, M01 = 0, M02 = 0, M11 = 0, M12 = 0, M22 = 0, sw = 0;
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const C ww = w[b * 3 + q];
                    sw += ww;
                    M00 += ww;
                    M01 += ww * rx[q];
                    M02 += ww * ry[b];
                    M11 += ww * rx[q] * rx[q];
                    M12 += ww * rx[q] * ry[b];
                    M22 += ww * ry[b] * ry[b];
                }
            // first column of the inverse of the symmetric 3x3 moment matrix
            const C c0 = M11 * M22 - M12 * M12;
            const C c1 = -(M01 * M22 - M12 * M02);
            const C c2 = M01 * M12 - M11 * M02;
            const C det = M00 * c0 + M01 * c1 + M02 * c2;
            if (det > C(1e-10)) {
#pragma unroll
                for (int b = 0; b < 3; ++b)
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        w[b * 3 + q] = w[b * 3 + q] * (c0 + c1 * rx[q] + c2 * ry[b]) / det;
            } else if (sw > C(0)) {
#pragma unroll
                for (int q = 0; q < 9; ++q) w[q] = w[q] / sw;
            } else {
#pragma unroll
                for (int q = 0; q < 9; ++q) w[q] = C(0);
            }
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) W[9 * (size_t)v + q] = w[q];
        const int i0w = ((i0 % a.nx) + a.nx) % a.nx;
        const int j0s = a.walls ? j0 : (((j0 % a.ny) + a.ny) % a.ny);
        a.stencil[2 * (size_t)v] = i0w;
        a.stencil[2 * (size_t)v + 1] = j0s;

        // ---- spreading (Sec. 2.2, the transpose of the interpolation): w_j F_v
        // into the fixed-point force field, and flag the fused-kernel tiles hit
        int last_t = -1;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            int jj = j0 + b - 1;
            if (a.walls) {
                if (jj < 0 || jj >= a.ny) continue;
            } else {
                jj = jj < 0 ? jj + a.ny : (jj >= a.ny ? jj - a.ny : jj);
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                int ii = i0w + q - 1;
                ii = ii < 0 ? ii + a.nx : (ii >= a.nx ? ii - a.nx : ii);
                const size_t node = (size_t)jj * a.nx + ii;
                const C wq = w[b * 3 + q];
                unsigned long long* gp = reinterpret_cast<unsigned long long*>(a.gsum + node);
                atomicAdd(gp, (unsigned long long)to_fix<C>(wq * Fx));
                atomicAdd(gp + 1, (unsigned long long)to_fix<C>(wq * Fy));
                const int t = (jj / a.tile_h) * a.tiles_x + ii / a.tile_w;
                if (t != last_t) {
                    a.flags[t] = 1;
                    last_t = t;
                }
            }
        }
    }
}

// ---------------------------------------------------------------- segments
// One group of kSegV lanes per segment: bounding box of its vertices, in FP32
// offsets from the segment's first vertex, stored with the centre's x wrapped
// into [0, nx).  All 32 lanes of the warp call this; `sg` is this lane group's
// segment or -1.
template <typename C>
__device__ void seg_box_group(const MarkerArgs& a, int sg, int lane) {
    using E = typename Ext<C>::E;
    const int g = lane & (kSegV - 1);
    int v0 = 0, nb = 0;
    if (sg >= 0) {
        v0 = a.seg_v0[sg];
        nb = a.seg_n[sg];
    }
    float ox = 0.f, oy = 0.f;
    E ax = ezero<E>(), ay = ezero<E>();
    if (nb > 0) {
        load_pos<C>(a, v0, ax, ay);
        E px, py;
        load_pos<C>(a, v0 + (g < nb ? g : 0), px, py);
        ox = float(etoc(esub(px, ax)));
        oy = float(etoc(esub(py, ay)));
    }
    float lo_x = ox, hi_x = ox, lo_y = oy, hi_y = oy;
    for (int o = kSegV / 2; o > 0; o >>= 1) {
        lo_x = fminf(lo_x, __shfl_xor_sync(FULL, lo_x, o));
        hi_x = fmaxf(hi_x, __shfl_xor_sync(FULL, hi_x, o));
        lo_y = fminf(lo_y, __shfl_xor_sync(FULL, lo_y, o));
        hi_y = fmaxf(hi_y, __shfl_xor_sync(FULL, hi_y, o));
    }
    if (nb > 0 && g == 0) {
        const float Lx = float(a.nx);
        const float cx = float(ehi(ax)) + 0.5f * (lo_x + hi_x);
        a.seg_box[sg] = make_float4(cx - Lx * floorf(cx / Lx), float(ehi(ay)) + 0.5f * (lo_y + hi_y),
                                    0.5f * (hi_x - lo_x), 0.5f * (hi_y - lo_y));
    }
}

// boxes of segments [s0, s1) by the warps of a block, kSegV lanes per segment
template <typename C>
__device__ void seg_boxes_block(const MarkerArgs& a, int s0, int s1) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    constexpr int per_warp = 32 / kSegV;
    for (int base = s0 + wid * per_warp; base < s1; base += nw * per_warp) {
        const int sg = base + lane / kSegV;
        seg_box_group<C>(a, sg < s1 ? sg : -1, lane);
    }
}

// Last-block epilogue: every block counts itself in once it is done; the block
// that arrives last (it sees all other blocks' writes after the fences) runs the
// epilogue and resets the counter.  No block ever waits for another.
__device__ bool arrive_last(unsigned int* counter) {
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

// ---------------------------------------------------------------- advance
// interpolation U_v = sum_j phi_v(x_j) u(x_j) with the weights of this step
template <typename C>
__device__ __forceinline__ void interp_vertex(const MarkerArgs& a, int v) {
    const C* ux = static_cast<const C*>(a.ux);
    const C* uy = static_cast<const C*>(a.uy);
    const C* W = static_cast<const C*>(a.W);
    C* U = static_cast<C*>(a.U);
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
    U[2 * v] = sx;
    U[2 * v + 1] = sy;
}

// Eq. kinematicPos (BDF2): x^{n+1} = 2/3 (2 x^n - 1/2 x^{n-1} + U dt);
// forward Euler on the very first step
template <typename C>
__device__ __forceinline__ void advance_vertex(const MarkerArgs& a, int v, long long step) {
    using E = typename Ext<C>::E;
    const C* U = static_cast<const C*>(a.U);
    E x, y, xp, yp;
    load_pos<C>(a, v, x, y);
    PosIO<C>::load(a.Xp, v, xp, yp);
    E xn, yn;
    if (step == 0) {
        xn = eaddc(x, U[2 * v]);
        yn = eaddc(y, U[2 * v + 1]);
    } else {
        const E tt = two_thirds_e<E>();
        xn = emul(eaddc(esub(emulc(x, C(2)), emulc(xp, C(0.5))), U[2 * v]), tt);
        yn = emul(eaddc(esub(emulc(y, C(2)), emulc(yp, C(0.5))), U[2 * v + 1]), tt);
    }
    if (!isfinite(ehi(xn)) || !isfinite(ehi(yn))) atomicOr(a.status, ST_NONFINITE);
    PosIO<C>::store(a.Xp, v, x, y);
    PosIO<C>::store(a.X, v, xn, yn);
}

// One block per unit: a chunk of a kinematic membrane (independent vertices)
// or a whole rigid-projected membrane (needs its centroid and mean rotation).
template <typename C>
__global__ void __launch_bounds__(kChunkV) k_advance(const MarkerArgs a) {
    using E = typename Ext<C>::E;
    const int m = a.au[3 * blockIdx.x], k0 = a.au[3 * blockIdx.x + 1], kn = a.au[3 * blockIdx.x + 2];
    const int off = a.mem_off[m], n = a.mem_n[m];
    __shared__ C cred[33];
    const long long step = *a.d_step;
    if (a.mem_kind[m] != LBIB_MEMBRANE_RIGID_PROJECTED) {
        for (int j = threadIdx.x; j < kn; j += blockDim.x) {
            interp_vertex<C>(a, off + k0 + j);
            advance_vertex<C>(a, off + k0 + j, step);
        }
        __syncthreads();
        // boxes of the segments this chunk covers (chunks are segment-aligned)
        seg_boxes_block<C>(a, a.mem_seg_off[m] + k0 / kSegV, a.mem_seg_off[m] + (k0 + kn + kSegV - 1) / kSegV);
    } else {
        C* U = static_cast<C*>(a.U);
        for (int k = threadIdx.x; k < n; k += blockDim.x) interp_vertex<C>(a, off + k);
        __syncthreads();
        // least-squares rigid motion U_c + omega x (x - x_c) of the ring; the
        // sums run in the compute precision on positions taken about vertex 0
        E xr, yr;
        load_pos<C>(a, off, xr, yr);
        C sx = 0, sy = 0, su = 0, sv = 0;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int v = off + k;
            E x, y;
            load_pos<C>(a, v, x, y);
            sx += etoc(esub(x, xr));
            sy += etoc(esub(y, yr));
            su += U[2 * v];
            sv += U[2 * v + 1];
        }
        const C inv_n = C(1) / C(n);
        const C mx = block_sum_c<C>(sx, cred) * inv_n, my = block_sum_c<C>(sy, cred) * inv_n;
        const C mu = block_sum_c<C>(su, cred) * inv_n, mv = block_sum_c<C>(sv, cred) * inv_n;
        C num = 0, den = 0;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int v = off + k;
            E x, y;
            load_pos<C>(a, v, x, y);
            const C rx = etoc(esub(x, xr)) - mx, ry = etoc(esub(y, yr)) - my;
            num += rx * (U[2 * v + 1] - mv) - ry * (U[2 * v] - mu);
            den += rx * rx + ry * ry;
        }
        const C om = block_sum_c<C>(num, cred) / block_sum_c<C>(den, cred);
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int v = off + k;
            E x, y;
            load_pos<C>(a, v, x, y);
            const C rx = etoc(esub(x, xr)) - mx, ry = etoc(esub(y, yr)) - my;
            U[2 * v] = mu - om * ry;
            U[2 * v + 1] = mv + om * rx;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < n; k += blockDim.x) advance_vertex<C>(a, off + k, step);
        __syncthreads();
        seg_boxes_block<C>(a, a.mem_seg_off[m], a.mem_seg_off[m + 1]);
    }
    // without bond kinetics nothing later in the step reads the step counter
    if (a.bump_in_advance && arrive_last(&a.tickets[0])) {
        if (threadIdx.x == 0) {
            *a.d_step += 1;
            a.tickets[0] = 0;
        }
    }
}

// segment boxes alone (before the first step and after user-written markers)
template <typename C>
__global__ void k_seg_boxes(const MarkerArgs a) {
    constexpr int per_block = (256 / 32) * (32 / kSegV);
    const int s0 = blockIdx.x * per_block;
    seg_boxes_block<C>(a, s0, min(a.nseg, s0 + per_block));
}

template <typename C>
__global__ void k_areas(const MarkerArgs a, double* areas) {
    __shared__ typename Ext<C>::E red[33];
    ring_area<C>(a, blockIdx.x, red);
    if (threadIdx.x == 0) areas[blockIdx.x] = etod(red[32]);
}

// marker positions between doubles (x0, y0, x1, ...) and the device layout
template <typename C>
__global__ void k_pos_in(const double* xy, void* X, int nv) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    PosIO<C>::store(X, v, from_double_e<C>(xy[2 * v]), from_double_e<C>(xy[2 * v + 1]));
}
template <typename C>
__global__ void k_pos_out(const void* X, double* xy, int nv) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    typename Ext<C>::E x, y;
    PosIO<C>::load(X, v, x, y);
    xy[2 * v] = etod(x);
    xy[2 * v + 1] = etod(y);
}

// ---------------------------------------------------------------- launchers
static bool is_f64(lbib_precision p) { return p == LBIB_F64; }

cudaError_t launch_rest(lbib_precision prec, const MarkerArgs& a, void* rest, double* A0, cudaStream_t s) {
    if (is_f64(prec)) k_rest<double><<<a.nmem, 256, 0, s>>>(a, rest, A0);
    else k_rest<float><<<a.nmem, 256, 0, s>>>(a, rest, A0);
    return cudaGetLastError();
}

cudaError_t launch_forces(lbib_precision prec, const MarkerArgs& a, int, cudaStream_t s) {
    if (is_f64(prec)) k_forces<double><<<a.nfu, kChunkV, 0, s>>>(a);
    else k_forces<float><<<a.nfu, kChunkV, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_advance(lbib_precision prec, const MarkerArgs& a, cudaStream_t s) {
    if (is_f64(prec)) k_advance<double><<<a.nau, kChunkV, 0, s>>>(a);
    else k_advance<float><<<a.nau, kChunkV, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_seg_boxes(lbib_precision prec, const MarkerArgs& a, cudaStream_t s) {
    if (a.nseg == 0) return cudaSuccess;
    constexpr int per_block = (256 / 32) * (32 / kSegV);
    const int g = (a.nseg + per_block - 1) / per_block;
    if (is_f64(prec)) k_seg_boxes<double><<<g, 256, 0, s>>>(a);
    else k_seg_boxes<float><<<g, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_areas(lbib_precision prec, const MarkerArgs& a, double* areas, cudaStream_t s) {
    if (is_f64(prec)) k_areas<double><<<a.nmem, 32, 0, s>>>(a, areas);
    else k_areas<float><<<a.nmem, 32, 0, s>>>(a, areas);
    return cudaGetLastError();
}

cudaError_t launch_pos_in(lbib_precision prec, const double* xy, void* X, int nv, cudaStream_t s) {
    if (nv == 0) return cudaSuccess;
    if (is_f64(prec)) k_pos_in<double><<<(nv + 255) / 256, 256, 0, s>>>(xy, X, nv);
    else k_pos_in<float><<<(nv + 255) / 256, 256, 0, s>>>(xy, X, nv);
    return cudaGetLastError();
}

cudaError_t launch_pos_out(lbib_precision prec, const void* X, double* xy, int nv, cudaStream_t s) {
    if (nv == 0) return cudaSuccess;
    if (is_f64(prec)) k_pos_out<double><<<(nv + 255) / 256, 256, 0, s>>>(X, xy, nv);
    else k_pos_out<float><<<(nv + 255) / 256, 256, 0, s>>>(X, xy, nv);
    return cudaGetLastError();
}

}  // namespace lbib
