// Lagrangian-side kernels: membrane forces (stretching, bending, enclosed
// area, repulsion, bond springs), the IB shape functions and the spreading of
// the marker forces; rest state, segment boxes and position conversion.
//
// Paper: Coclite, arXiv 1907.00080, Sec. 2.2 (Eqs. strainFor, bendFor,
// areaFor, repFor, adhFor; MLS exchange), Sec. 2.3 (nine Eulerian points per
// vertex).
//
// Precision: the compute type C is double in FP64 mode and float otherwise;
// positions and every cancellation-prone product use the matching extended
// type E (double, or float-float) from ext_real.cuh.
#include "marker_common.cuh"

namespace lbib {

// ---------------------------------------------------------------- rest state
// Captures, per vertex, the squared and plain rest length of the element
// (v, v+1) and the rest cross/dot products of the two edges at v (which fix the
// rest turning angle theta_0), plus A_0 per membrane -- with the arithmetic the
// force kernel repeats, so the rest shape gives exactly zero force.
template <typename C>
__global__ void k_rest(const MarkerArgs a, void* rest_v, double* A0, double* qa) {
    using E = typename Ext<C>::E;
    const int m = blockIdx.x;
    const int off = a.mem_off[m], n = a.mem_n[m];
    __shared__ E red[32 * kAreaWarps];
    Rest<C>* rest = static_cast<Rest<C>*>(rest_v);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int v = off + k, L = off + (k == 0 ? n - 1 : k - 1), R = off + (k == n - 1 ? 0 : k + 1);
        E xL, yL, xv, yv, xR, yR;
        load_pos<C>(a, L, xL, yL);
        load_pos<C>(a, v, xv, yv);
        load_pos<C>(a, R, xR, yR);
        const EdgeProducts<C> p = edge_products<E, C>(xL, yL, xv, yv, xR, yR);
        Rest<C> r;
        r.lsq = p.lsqR;
        r.cross = p.cross;
        r.dot = p.dot;
        r.l0 = sqrt(etoc(p.lsqR));
        rest[v] = r;
    }
    if (threadIdx.x < 32 * kAreaWarps) {
        const E A = ring_area_group<C>(a, a.mem_off[m], a.mem_n[m], 0, red, 1);
        if (threadIdx.x == 0) {
            const double A0m = etod(A);
            A0[m] = A0m;
            qa[m] = a.mem_ka[m] * (1.0 / 3.0) / A0m;  // k_a p_ref / A_0 (p_ref = 1/3)
        }
    }
}

// ---------------------------------------------------------------- forces
// Eq. adhFor on element e (if its ligand is bonded), half to the vertex;
// positions of the element's two vertices are given
template <typename C, typename E>
__device__ __forceinline__ void bond_on_element(const MarkerArgs& a, int e, E xa, E ya, E xb, E yb, C& Fx,
                                                C& Fy) {
    const int l = a.elem_lig[e];
    if (l < 0) return;
    const int r = a.bond_of_lig[l];
    if (r < 0) return;
    E rx, ry;
    PosIO<C>::load(a.rec_e, r, rx, ry);
    // receptor minus ligand point (element centroid)
    const E cx = emulc(eadd(xa, xb), C(0.5)), cy = emulc(eadd(ya, yb), C(0.5));
    const C dx = etoc(ewrap(esub(rx, cx), par<C>(a.nx, a.f.nx), par<C>(a.inv_nx, a.f.inv_nx)));
    C dy = etoc(esub(ry, cy));
    if (!a.walls) dy = etoc(ewrap(esub(ry, cy), par<C>(a.ny, a.f.ny), par<C>(a.inv_ny, a.f.inv_ny)));
    const C d = sqrt(dx * dx + dy * dy);
    const C c = par<C>(a.sigma, a.f.sigma) * (d - par<C>(a.y_eq, a.f.y_eq)) / d;
    Fx += C(0.5) * c * dx;
    Fy += C(0.5) * c * dy;
}

constexpr int kForceWarps = 10;
constexpr int kScreenWarps = kForceWarps - 4 - kAreaWarps;  // phase 1: 2 bending, 2 weights, area, screening
static_assert(kScreenWarps == 2, "two screening warps");
constexpr int kForceThreads = 32 * kForceWarps;  // threads per force block
constexpr int kMaxCand = 256;                     // repulsion candidate segments per block
constexpr int kStageSeg = 48;                     // candidate segments staged in shared memory
constexpr int kScreenIter = 8;                    // segment boxes per lane loaded ahead of the screen

// One block per work unit (a chunk of up to kChunkV consecutive vertices of one
// membrane).  The warps split the work of a vertex:
//   phase 1  warps 0-1  bending geometry of the chunk plus one halo vertex each side
//            warps 2-3  IB shape functions (MLS / Roma) and stencil origins
//            warps 4-7  enclosed area of the whole membrane (fixed-order sum)
//            warps 8-9  repulsion candidate segments, one half of the segments
//                       each (ascending order)
//   phase 2  warps 0-1  stretching, bending, area and bond forces per vertex
//            warps 2-9  repulsion over (candidate segment, vertex) pairs,
//                       accumulated per vertex in fixed point (order-free)
//   phase 3  all        spreading: (vertex, node) pairs into the fixed-point field
//                       (of a dynamic particle: its forcing term, see dynamic_kernels.cu)
//
// forces_unit is the body for force unit `unit` of the context `a`: the
// single-context kernel runs unit blockIdx.x, the batched kernel (ensembles)
// one unit of one member per block.
template <typename C>
__device__ __forceinline__ void forces_unit(const MarkerArgs& a, int unit) {
    using E = typename Ext<C>::E;
    const int4 u0 = a.fu[2 * unit], u1 = a.fu[2 * unit + 1];
    const int m = u0.x, k0 = u0.y, kn = u0.z, off = u0.w, n = u1.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // positions of vertices k0-2 .. k0+kn+1 (slot p <-> vertex k0 - 2 + p)
    __shared__ E s_x[kChunkV + 4], s_y[kChunkV + 4];
    // bending geometry of vertices k0-1 .. k0+kn (slot j <-> vertex k0 - 1 + j)
    __shared__ C s_mnx[kChunkV + 2], s_mny[kChunkV + 2], s_sL[kChunkV + 2], s_sR[kChunkV + 2];
    __shared__ C s_nx[kChunkV + 2], s_ny[kChunkV + 2];
    __shared__ C s_w[kChunkV][9];
    __shared__ int s_i0[kChunkV], s_j0[kChunkV];
    __shared__ unsigned long long s_rep[kChunkV];
    __shared__ C s_F[kChunkV][2];
    __shared__ E red[32 * kAreaWarps];
    __shared__ C s_ca;
    __shared__ int s_cand[kScreenWarps][kMaxCand];  // each screening warp's hits, ascending
    __shared__ int s_ncw[kScreenWarps];
    __shared__ int s_ncand;
    // staged candidate segments: box, anchor (first vertex) and the offsets of
    // their vertices from the anchor in the compute type
    __shared__ float4 s_cbox[kStageSeg];
    __shared__ E s_cax[kStageSeg], s_cay[kStageSeg];
    __shared__ C s_cox[kStageSeg * kSegV], s_coy[kStageSeg * kSegV];
    __shared__ int s_cn[kStageSeg], s_cv0[kStageSeg];
    const Rest<C>* rest = static_cast<const Rest<C>*>(a.rest);

    // ---- phase 0: positions of the chunk and two halo vertices on each side
    for (int p = tid; p < kn + 4; p += blockDim.x) {
        int k = k0 - 2 + p;
        k = k < 0 ? k + n : (k >= n ? k - n : k);
        load_pos<C>(a, off + k, s_x[p], s_y[p]);
    }
    if (tid < kChunkV) s_rep[tid] = 0ull;
    // the screening warps fetch this chunk's own segment boxes now (the unit
    // record carries the membrane's first segment), behind the position loads
    const int sown0 = u1.z + k0 / kSegV;
    const int nown = (kn + kSegV - 1) / kSegV;  // <= kChunkV / kSegV <= 32
    float4 o0 = make_float4(0.f, 0.f, 0.f, 0.f), own = o0;
    if (wid >= 4 + kAreaWarps && a.nmem > 1) {
        o0 = a.seg_box[sown0];
        own = lane < nown ? a.seg_box[sown0 + lane] : o0;
    }
    __syncthreads();

    // ---- phase 1
    if (wid < 2) {
        // theta - theta_0 from the rotation between the rest and the current
        // edge pair, atan2(c d0 - c0 d, d d0 + c c0): no cancellation of two
        // nearly equal angles
        const C kb = par<C>(a.mem_kb[m], float(a.mem_kb[m]));
        for (int j = tid; j < kn + 2; j += 64) {
            int k = k0 - 1 + j;
            k = k < 0 ? k + n : (k >= n ? k - n : k);
            const E xL = s_x[j], yL = s_y[j], xv = s_x[j + 1], yv = s_y[j + 1], xR = s_x[j + 2], yR = s_y[j + 2];
            const EdgeProducts<C> p = edge_products<E, C>(xL, yL, xv, yv, xR, yR);
            const Rest<C> r0 = rest[off + k];
            const E sn = esub(emul(p.cross, r0.dot), emul(r0.cross, p.dot));
            const E cs = eadd(emul(p.dot, r0.dot), emul(p.cross, r0.cross));
            const C dth = atan2(etoc(sn), etoc(cs));
            const C eLx = etoc(esub(xv, xL)), eLy = etoc(esub(yv, yL));
            const C eRx = etoc(esub(xR, xv)), eRy = etoc(esub(yR, yv));
            const C lL = sqrt(eLx * eLx + eLy * eLy), lR = sqrt(eRx * eRx + eRy * eRy);
            const C iL = C(1) / lL, iR = C(1) / lR;
            // outward vertex normal: normalised sum of the outward edge normals (CCW ring)
            C nx_ = eLy * iL + eRy * iR;
            C ny_ = -eLx * iL - eRx * iR;
            const C inn = C(1) / sqrt(nx_ * nx_ + ny_ * ny_);
            nx_ *= inn;
            ny_ *= inn;
            const C mb = kb * dth;
            s_mnx[j] = mb * nx_;
            s_mny[j] = mb * ny_;
            const C isum = C(1) / (lL + lR);
            s_sL[j] = lL * isum;
            s_sR[j] = lR * isum;
            s_nx[j] = nx_;
            s_ny[j] = ny_;
        }
    } else if (wid < 4) {
        // IB shape functions at X^n: nine nearest nodes, Roma weights, MLS
        // (basis 1, dx, dy) re-solved where wall rows drop out.  Node indices are
        // clamped so that a runaway position still stays in range; the advance
        // kernel flags non-finite positions.
        const int j = tid - 64;
        if (j < kn) {
            const E xv = s_x[j + 2], yv = s_y[j + 2];
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
            const int v = off + k0 + j;
            C* W = static_cast<C*>(a.W);
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                W[9 * (size_t)v + q] = w[q];
                s_w[j][q] = w[q];
            }
            const int i0w = ((i0 % a.nx) + a.nx) % a.nx;
            const int j0s = a.walls ? j0 : (((j0 % a.ny) + a.ny) % a.ny);
            a.stencil[2 * (size_t)v] = i0w;
            a.stencil[2 * (size_t)v + 1] = j0s;
            s_i0[j] = i0w;
            s_j0[j] = j0;
        }
    } else if (wid < 4 + kAreaWarps) {
        // Eq. areaFor with p_ref = 1/3: F_l = c_a (inward normal) l_l
        // c_a = -k_a (1 - A/A_0) p_ref = q (A - A_0), q = k_a p_ref / A_0 from set-up
        const double A0 = a.mem_A0[m], q = a.mem_qa[m];
        // (off, n from the unit record: no dependent load before the ring's)
        const E A = ring_area_group<C>(a, off, n, 4, red, 1);
        if (tid == 32 * 4) s_ca = C(q * (etod(A) - A0));
    } else {
        // Eq. repFor screening, once per block: segments of other membranes whose
        // box comes within d_rep of this chunk's box (the union of its own
        // segments' boxes).  Screening warp sw takes the segments [lo, hi) of
        // its half and appends its hits in ascending order; the candidate list
        // is warp 0's hits, then warp 1's: ascending overall
        const int sw = wid - (4 + kAreaWarps);
        const int half = (a.nseg + 1) / 2;
        const int lo = sw == 0 ? 0 : half, hi = sw == 0 ? half : a.nseg;
        int cnt = 0;
        if (a.nmem > 1) {
            // the chunk box (from this chunk's own boxes) is formed once the
            // first batch of candidate boxes is in flight as well
            float cbx = 0.f, cby = 0.f, chx = 0.f, chy = 0.f;
            auto chunk_box = [&]() {
                float lo_x = 1e30f, hi_x = -1e30f, lo_y = 1e30f, hi_y = -1e30f;
                if (lane < nown) {
                    const float dx = wrap_half(own.x - o0.x, a.f.nx);
                    float dy = own.y - o0.y;
                    if (!a.walls) dy = wrap_half(dy, a.f.ny);
                    lo_x = dx - own.z;
                    hi_x = dx + own.z;
                    lo_y = dy - own.w;
                    hi_y = dy + own.w;
                }
                for (int o = 16; o > 0; o >>= 1) {
                    lo_x = fminf(lo_x, __shfl_xor_sync(kFull, lo_x, o));
                    hi_x = fmaxf(hi_x, __shfl_xor_sync(kFull, hi_x, o));
                    lo_y = fminf(lo_y, __shfl_xor_sync(kFull, lo_y, o));
                    hi_y = fmaxf(hi_y, __shfl_xor_sync(kFull, hi_y, o));
                }
                cbx = o0.x + 0.5f * (lo_x + hi_x);
                cby = o0.y + 0.5f * (lo_y + hi_y);
                chx = 0.5f * (hi_x - lo_x);
                chy = 0.5f * (hi_y - lo_y);
            };
            const float reach = a.f.d_rep + 2e-3f;
            auto screen = [&](int sg, int mem, const float4& b) {
                bool hit = false;
                if (sg < hi && mem != m) {
                    const float dx = wrap_half(b.x - cbx, a.f.nx);
                    float dy = b.y - cby;
                    if (!a.walls) dy = wrap_half(dy, a.f.ny);
                    hit = fabsf(dx) <= b.z + chx + reach && fabsf(dy) <= b.w + chy + reach;
                }
                const unsigned bal = __ballot_sync(kFull, hit);
                const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
                if (hit && pos < kMaxCand) s_cand[sw][pos] = sg;
                cnt += __popc(bal);
            };
            // batches of 32 kScreenIter segments: every box and owner of a batch in
            // flight at once, then the ordered screen
            for (int base = lo; base < hi; base += 32 * kScreenIter) {
                float4 bx[kScreenIter];
                int bm[kScreenIter];
#pragma unroll
                for (int it = 0; it < kScreenIter; ++it) {
                    const int sg = base + 32 * it + lane;
                    bm[it] = m;
                    if (sg < hi) {
                        bx[it] = a.seg_box[sg];
                        bm[it] = a.seg_mem[sg];
                    }
                }
                if (base == lo) chunk_box();
#pragma unroll
                for (int it = 0; it < kScreenIter; ++it)
                    if (base + 32 * it < hi) screen(base + 32 * it + lane, bm[it], bx[it]);
            }
            if (lane == 0) s_ncw[sw] = cnt;
            // both screening warps have their counts (named barrier 3)
            asm volatile("bar.sync 3, %0;" ::"r"(32 * kScreenWarps) : "memory");
            const int n0 = s_ncw[0], ntot = n0 + s_ncw[1];
            // the first kStageSeg candidates: box, vertex count and first vertex
            // (their positions are staged by the repulsion warps)
            const int nst = ntot < kStageSeg ? ntot : kStageSeg;
            for (int ci = tid - 32 * (4 + kAreaWarps); ci < nst; ci += 32 * kScreenWarps) {
                const int sg = ci < n0 ? s_cand[0][ci] : s_cand[1][ci - n0];
                s_cbox[ci] = a.seg_box[sg];
                s_cn[ci] = a.seg_n[sg];
                s_cv0[ci] = a.seg_v0[sg];
            }
            cnt = ntot;
        } else if (lane == 0) {
            s_ncw[sw] = 0;
        }
        if (sw == 0 && lane == 0) s_ncand = cnt;
    }
    __syncthreads();

    // ---- phase 2
    const int ncand = s_ncand;
    const bool all_segs = ncand > kMaxCand;  // list overflow: screen every segment
    C Fx = C(0), Fy = C(0);
    if (wid < 2) {
        const int j = tid;
        if (j < kn) {
            const int k = k0 + j;
            const int v = off + k, L = off + (k == 0 ? n - 1 : k - 1);
            const E xl = s_x[j + 1], yl = s_y[j + 1], xv = s_x[j + 2], yv = s_y[j + 2];
            const E xR = s_x[j + 3], yR = s_y[j + 3];
            const int sj = j + 1;  // geometry slot of vertex k
            // Eq. adhFor on the two elements sharing v, half each
            if (a.nlig > 0) {
                bond_on_element<C, E>(a, L, xl, yl, xv, yv, Fx, Fy);
                bond_on_element<C, E>(a, v, xv, yv, xR, yR, Fx, Fy);
            }
            // Eq. strainFor on elements (v, R) and (L, v); l - l_0 is formed as
            // (l^2 - l_0^2) / (l + l_0) with the squares in the extended type
            const C ks = par<C>(a.mem_ks[m], float(a.mem_ks[m]));
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
            const C ca = s_ca;
            Fx += C(0.5) * ca * (-etoc(esub(yR, yl)));
            Fy += C(0.5) * ca * etoc(esub(xR, xl));
        }
    } else if (a.nmem > 1 && ncand > 0) {
        // Eq. repFor against vertices of other membranes closer than d_rep, over
        // (candidate segment, vertex) pairs; the magnitudes of each vertex are
        // summed in fixed point (the direction is its own inward normal)
        // stage the candidates' vertices as offsets from their first vertex (the
        // anchor), then sync the repulsion warps (named barrier 2, warps 2-9)
        const int nst = all_segs ? 0 : (ncand < kStageSeg ? ncand : kStageSeg);
        for (int e = tid - 64; e < nst * kSegV; e += blockDim.x - 64) {
            const int ci = e / kSegV, g = e - ci * kSegV;
            if (g < s_cn[ci]) {
                E xa, ya, xb, yb;
                load_pos<C>(a, s_cv0[ci], xa, ya);
                load_pos<C>(a, s_cv0[ci] + g, xb, yb);
                s_cox[e] = etoc(esub(xb, xa));
                s_coy[e] = etoc(esub(yb, ya));
                if (g == 0) {
                    s_cax[ci] = xa;
                    s_cay[ci] = ya;
                }
            }
        }
        asm volatile("bar.sync 2, %0;" ::"r"(kForceThreads - 64) : "memory");
        const int nscan = all_segs ? a.nseg : ncand;
        const float reach = a.f.d_rep + 2e-3f;
        const C c_rep = C(1e-4 / (8.0 * 1.4142135623730951));
        const C drep = par<C>(a.d_rep, a.f.d_rep);
        for (int p = tid - 64; p < nscan * kn; p += blockDim.x - 64) {
            const int ci = p / kn, j = p - ci * kn;
            const bool staged = !all_segs && ci < kStageSeg;
            const int sg = all_segs ? ci : (ci < s_ncw[0] ? s_cand[0][ci] : s_cand[1][ci - s_ncw[0]]);
            if (all_segs && a.seg_mem[sg] == m) continue;
            const E xv = s_x[j + 2], yv = s_y[j + 2];
            const float hx = float(ehi(xv));
            const float xvw = hx - a.f.nx * floorf(hx * a.f.inv_nx);
            const float4 bx = staged ? s_cbox[ci] : a.seg_box[sg];
            const float ddx = wrap_half(xvw - bx.x, a.f.nx);
            float ddy = float(ehi(yv)) - bx.y;
            if (!a.walls) ddy = wrap_half(ddy, a.f.ny);
            if (fabsf(ddx) > bx.z + reach || fabsf(ddy) > bx.w + reach) continue;
            C mags = C(0);
            if (staged) {
                // vertex relative to the segment anchor once, then plain differences
                const int nb = s_cn[ci];
                const C dxa = etoc(ewrap(esub(xv, s_cax[ci]), par<C>(a.nx, a.f.nx), par<C>(a.inv_nx, a.f.inv_nx)));
                C dya = etoc(esub(yv, s_cay[ci]));
                if (!a.walls) dya = etoc(ewrap(esub(yv, s_cay[ci]), par<C>(a.ny, a.f.ny), par<C>(a.inv_ny, a.f.inv_ny)));
                for (int g = 0; g < nb; ++g) {
                    const C dx = dxa - s_cox[ci * kSegV + g], dy = dya - s_coy[ci * kSegV + g];
                    const C d = sqrt(dx * dx + dy * dy);
                    if (d < drep) mags += c_rep * sqrt(C(1) / (d * d * d * d * d));
                }
            } else {
                const int nb = a.seg_n[sg], b0 = a.seg_v0[sg];
                for (int g = 0; g < nb; ++g) {
                    E xb, yb;
                    load_pos<C>(a, b0 + g, xb, yb);
                    const C dx = etoc(ewrap(esub(xv, xb), par<C>(a.nx, a.f.nx), par<C>(a.inv_nx, a.f.inv_nx)));
                    C dy = etoc(esub(yv, yb));
                    if (!a.walls) dy = etoc(ewrap(esub(yv, yb), par<C>(a.ny, a.f.ny), par<C>(a.inv_ny, a.f.inv_ny)));
                    const C d = sqrt(dx * dx + dy * dy);
                    if (d < drep) mags += c_rep * sqrt(C(1) / (d * d * d * d * d));
                }
            }
            if (mags != C(0)) {
                bool bad = false;
                mags = clamp_fix(mags, C(kFix60Limit), bad);
                if (bad) atomicOr(a.status, ST_FIXRANGE);
                atomicAdd(&s_rep[j], (unsigned long long)to_fix60<C>(mags));
            }
        }
    }
    __syncthreads();
    if (wid < 2 && tid < kn) {
        const C mag = fix60_to_c<C>((long long)s_rep[tid]);
        Fx -= mag * s_nx[tid + 1];
        Fy -= mag * s_ny[tid + 1];
        C* F = static_cast<C*>(a.F);
        const int v = off + k0 + tid;
        C Sx = Fx, Sy = Fy;
        if (u1.y >= LBIB_MEMBRANE_DYNAMIC) {
            // dynamic particle (Sec. 2.4): the total force of Eq. newtonSoft adds
            // the hydrodynamic force; the fluid receives the forcing term instead
            const C* Hf = static_cast<const C*>(a.Hf);
            const C* D = static_cast<const C*>(a.Dib);
            Fx += Hf[2 * (size_t)v];
            Fy += Hf[2 * (size_t)v + 1];
            Sx = D[2 * (size_t)v];
            Sy = D[2 * (size_t)v + 1];
        }
        F[2 * (size_t)v] = Fx;
        F[2 * (size_t)v + 1] = Fy;
        s_F[tid][0] = Sx;
        s_F[tid][1] = Sy;
    }
    __syncthreads();

    // ---- phase 3: spreading (Sec. 2.2, the transpose of the interpolation):
    // w_j F_v into the fixed-point force field; flag the fused-kernel tiles hit
    for (int p = tid; p < 9 * kn; p += blockDim.x) {
        const int j = p / 9, q9 = p - 9 * j;
        const int b = q9 / 3, q = q9 - 3 * b;
        int jj = s_j0[j] + b - 1;
        if (a.walls) {
            if (jj < 0 || jj >= a.ny) continue;
        } else {
            jj = jj < 0 ? jj + a.ny : (jj >= a.ny ? jj - a.ny : jj);
        }
        int ii = s_i0[j] + q - 1;
        ii = ii < 0 ? ii + a.nx : (ii >= a.nx ? ii - a.nx : ii);
        const size_t node = (size_t)jj * a.nx + ii;
        const C wq = s_w[j][q9];
        bool bad = false;
        const C gx = clamp_fix(wq * s_F[j][0], C(kFixLimit), bad);
        const C gy = clamp_fix(wq * s_F[j][1], C(kFixLimit), bad);
        if (bad) atomicOr(a.status, ST_FIXRANGE);
        unsigned long long* gp = reinterpret_cast<unsigned long long*>(a.gsum + node);
        atomicAdd(gp, (unsigned long long)to_fix<C>(gx));
        atomicAdd(gp + 1, (unsigned long long)to_fix<C>(gy));
        a.flags[(jj / a.tile_h) * a.tiles_x + ii / a.tile_w] = 1;
    }
}

template <typename C>
__global__ void __launch_bounds__(kForceThreads) k_forces(const MarkerArgs a) {
    forces_unit<C>(a, blockIdx.x);
}

// Batched form: the force units of up to kBatchMax contexts (ensemble
// members) in one launch, one block per (member, unit).  The member's
// arguments are staged in shared memory.
// (three blocks per SM: the batch's thousands of blocks are limited by how
// many fit, not by one block's latency)
template <typename C>
__global__ void __launch_bounds__(kForceThreads, 3) k_forces_batch(const __grid_constant__ MarkerBatch b) {
    __shared__ MarkerArgs s_a;
    const int m = marker_member(b, blockIdx.x);
    stage_args(&s_a, b.args + m);
    forces_unit<C>(s_a, blockIdx.x - b.off[m]);
}

// ---------------------------------------------------------------- segments
// segment boxes alone (before the first step and after user-written markers):
// one group of kSegV lanes per segment
template <typename C>
__global__ void k_seg_boxes(const MarkerArgs a) {
    using E = typename Ext<C>::E;
    constexpr int per_block = (256 / 32) * (32 / kSegV);
    const int lane = threadIdx.x & 31;
    const int sg = blockIdx.x * per_block + (threadIdx.x >> 5) * (32 / kSegV) + lane / kSegV;
    const bool ok = sg < a.nseg;
    int v = 0;
    if (ok) {
        const int g = lane & (kSegV - 1);
        v = a.seg_v0[sg] + (g < a.seg_n[sg] ? g : 0);
    }
    E x, y;
    load_pos<C>(a, v, x, y);
    seg_box_regs<C>(a, ok ? sg : -1, lane, x, y);
}

template <typename C>
__global__ void k_areas(const MarkerArgs a, double* areas) {
    __shared__ typename Ext<C>::E red[32 * kAreaWarps];
    const typename Ext<C>::E A = ring_area_group<C>(a, a.mem_off[blockIdx.x], a.mem_n[blockIdx.x], 0, red, 1);
    if (threadIdx.x == 0) areas[blockIdx.x] = etod(A);
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

cudaError_t launch_rest(lbib_precision prec, const MarkerArgs& a, void* rest, double* A0, double* qa,
                        cudaStream_t s) {
    if (is_f64(prec)) k_rest<double><<<a.nmem, 256, 0, s>>>(a, rest, A0, qa);
    else k_rest<float><<<a.nmem, 256, 0, s>>>(a, rest, A0, qa);
    return cudaGetLastError();
}

cudaError_t launch_forces(lbib_precision prec, const MarkerArgs& a, int, cudaStream_t s) {
    if (is_f64(prec)) k_forces<double><<<a.nfu, kForceThreads, 0, s>>>(a);
    else k_forces<float><<<a.nfu, kForceThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_forces_batch(lbib_precision prec, const MarkerBatch& b, cudaStream_t s) {
    if (b.n < 1 || b.n > kBatchMax) return cudaErrorInvalidValue;
    const int nunits = b.off[b.n];
    if (nunits <= 0) return cudaSuccess;
    if (is_f64(prec)) k_forces_batch<double><<<nunits, kForceThreads, 0, s>>>(b);
    else k_forces_batch<float><<<nunits, kForceThreads, 0, s>>>(b);
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
    if (is_f64(prec)) k_areas<double><<<a.nmem, 32 * kAreaWarps, 0, s>>>(a, areas);
    else k_areas<float><<<a.nmem, 32 * kAreaWarps, 0, s>>>(a, areas);
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
