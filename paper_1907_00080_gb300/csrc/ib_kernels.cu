// Lagrangian-side kernels: membrane forces (stretching, bending, enclosed
// area, repulsion, bond springs), IB shape functions and tile binning, the
// deterministic tile lists, and the interpolation + kinematic advance.
//
// Paper: Coclite, arXiv 1907.00080, Sec. 2.2 (Eqs. strainFor, bendFor,
// areaFor, repFor, adhFor; MLS exchange), Sec. 2.3 (nine Eulerian points per
// vertex, Eq. kinematicPos).
#include <climits>

#include "lbib_internal.cuh"

namespace lbib {

constexpr unsigned FULL = 0xffffffffu;

// periodic minimum image, multiplying by 1/L (an FP64 division is a long
// instruction sequence on this part)
__device__ __forceinline__ double wrap_m(double d, double L, double invL) {
    return d - L * floor(d * invL + 0.5);
}
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

// Edge products at a vertex, in FP64 with every product and sum rounded as
// written (no contraction), so the rest shape reproduces them bit for bit:
// squared length of e_R = x_{v+1} - x_v, cross and dot of e_L = x_v - x_{v-1}
// with e_R.
struct EdgeProducts {
    double lsqR, cross, dot;
};
__device__ __forceinline__ EdgeProducts edge_products(double xL, double yL, double xv, double yv,
                                                      double xR, double yR) {
    const double eLx = __dsub_rn(xv, xL), eLy = __dsub_rn(yv, yL);
    const double eRx = __dsub_rn(xR, xv), eRy = __dsub_rn(yR, yv);
    EdgeProducts p;
    p.lsqR = __dadd_rn(__dmul_rn(eRx, eRx), __dmul_rn(eRy, eRy));
    p.cross = __dsub_rn(__dmul_rn(eLx, eRy), __dmul_rn(eLy, eRx));
    p.dot = __dadd_rn(__dmul_rn(eLx, eRx), __dmul_rn(eLy, eRy));
    return p;
}

// block-wide FP64 sum (blockDim multiple of 32, <= 1024); all threads get it
__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(FULL, t, o);
        if (threadIdx.x == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
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
__global__ void k_rest(const MarkerArgs a, double* rest, double* A0) {
    const int m = blockIdx.x;
    const int off = a.mem_off[m], n = a.mem_n[m];
    __shared__ double red[33];
    const double* X = a.X;
    const double xr = X[2 * off], yr = X[2 * off + 1];
    double ap = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int v = off + k, L = off + (k == 0 ? n - 1 : k - 1), R = off + (k == n - 1 ? 0 : k + 1);
        const EdgeProducts p = edge_products(X[2 * L], X[2 * L + 1], X[2 * v], X[2 * v + 1],
                                             X[2 * R], X[2 * R + 1]);
        rest[4 * (size_t)v + 0] = p.lsqR;
        rest[4 * (size_t)v + 1] = sqrt(p.lsqR);
        rest[4 * (size_t)v + 2] = p.cross;
        rest[4 * (size_t)v + 3] = p.dot;
        ap += (X[2 * v] - xr) * (X[2 * R + 1] - yr) - (X[2 * R] - xr) * (X[2 * v + 1] - yr);
    }
    const double s = block_sum(ap, red);
    if (threadIdx.x == 0) A0[m] = 0.5 * s;
}

// ---------------------------------------------------------------- forces
template <typename C>
__device__ __forceinline__ void bond_on_element(const MarkerArgs& a, int e, double nxd, double nyd,
                                                C& Fx, C& Fy) {
    const int l = a.elem_lig[e];
    if (l < 0) return;
    const int r = a.bond_of_lig[l];
    if (r < 0) return;
    const int va = a.lig_a[l], vb = a.lig_b[l];
    const double cxp = 0.5 * (a.X[2 * va] + a.X[2 * vb]);
    const double cyp = 0.5 * (a.X[2 * va + 1] + a.X[2 * vb + 1]);
    const double dx = wrap_m(a.rec_xy[2 * r] - cxp, nxd, a.inv_nx);
    double dy = a.rec_xy[2 * r + 1] - cyp;
    if (!a.walls) dy = wrap_m(dy, nyd, a.inv_ny);
    const double d = sqrt(dx * dx + dy * dy);
    const double c = a.sigma * (d - a.y_eq) / d;
    Fx += C(0.5 * c * dx);
    Fy += C(0.5 * c * dy);
}

// One block per work unit (a chunk of up to kChunkV consecutive vertices of one
// membrane); one thread per vertex.  The enclosed area of the whole membrane is
// summed by every unit of that membrane in the same fixed order (so all units
// agree bit for bit), and the bending geometry of the chunk plus one halo
// vertex on each side is staged in shared memory.
template <typename C>
__global__ void __launch_bounds__(kChunkV) k_forces(const MarkerArgs a) {
    const int m = a.fu[3 * blockIdx.x], k0 = a.fu[3 * blockIdx.x + 1], kn = a.fu[3 * blockIdx.x + 2];
    const int off = a.mem_off[m], n = a.mem_n[m];
    __shared__ C s_mnx[kChunkV + 2], s_mny[kChunkV + 2], s_sL[kChunkV + 2], s_sR[kChunkV + 2];
    __shared__ C s_nx[kChunkV + 2], s_ny[kChunkV + 2];
    __shared__ double red[33];
    const double* X = a.X;
    const double nxd = (double)a.nx, nyd = (double)a.ny;
    const double xr = X[2 * off], yr = X[2 * off + 1];
    const C kb = C(a.mem_kb[m]);

    // shoelace area about vertex 0 over the whole ring (FP64)
    double ap = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int v = off + k, R = off + (k == n - 1 ? 0 : k + 1);
        ap += (X[2 * v] - xr) * (X[2 * R + 1] - yr) - (X[2 * R] - xr) * (X[2 * v + 1] - yr);
    }
    const double A = 0.5 * block_sum(ap, red);
    // Eq. areaFor with p_ref = 1/3: F_l = c_a (inward normal) l_l
    const C ca = C(-a.mem_ka[m] * (1.0 - A / a.mem_A0[m]) * (1.0 / 3.0));
    const C ks = C(a.mem_ks[m]);

    // vertex geometry of local slots j = 0..kn+1 (vertex k0 - 1 + j, wrapped).
    // theta - theta_0 comes from the rotation between the rest and the current
    // edge pair, atan2(c d0 - d c0, d d0 + c c0), free of the cancellation of
    // subtracting two nearly equal angles.
    for (int j = threadIdx.x; j < kn + 2; j += blockDim.x) {
        int k = k0 - 1 + j;
        k = k < 0 ? k + n : (k >= n ? k - n : k);
        const int v = off + k, L = off + (k == 0 ? n - 1 : k - 1), R = off + (k == n - 1 ? 0 : k + 1);
        const double xL = X[2 * L], yL = X[2 * L + 1], xv = X[2 * v], yv = X[2 * v + 1];
        const double xR = X[2 * R], yR = X[2 * R + 1];
        const EdgeProducts p = edge_products(xL, yL, xv, yv, xR, yR);
        const double c0 = a.rest[4 * (size_t)v + 2], d0 = a.rest[4 * (size_t)v + 3];
        const double sn = __dsub_rn(__dmul_rn(p.cross, d0), __dmul_rn(p.dot, c0));
        const double cs = __dadd_rn(__dmul_rn(p.dot, d0), __dmul_rn(p.cross, c0));
        const C dth = atan2(C(sn), C(cs));
        const C eLx = C(xv - xL), eLy = C(yv - yL), eRx = C(xR - xv), eRy = C(yR - yv);
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
    if (repel) {
        const float Lx = float(a.nx), Ly = float(a.ny);
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
                    const float dx = wrap_half(b.x - o.x, Lx);
                    float dy = b.y - o.y;
                    if (!a.walls) dy = wrap_half(dy, Ly);
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
        const double xv = X[2 * v], yv = X[2 * v + 1];
        const double xl = X[2 * L], yl = X[2 * L + 1], xR = X[2 * R], yR = X[2 * R + 1];
        C Fx = C(0), Fy = C(0);
        // Eq. adhFor on the two elements sharing v, half each
        if (a.nlig > 0) {
            bond_on_element<C>(a, L, nxd, nyd, Fx, Fy);
            bond_on_element<C>(a, v, nxd, nyd, Fx, Fy);
        }
        // Eq. repFor against vertices of other membranes closer than d_rep:
        // segment boxes are screened in FP32 (wrapped x), close pairs in FP64
        if (repel && (ncand > 0)) {
            const float Lx = float(a.nx), Ly = float(a.ny);
            const float xvw = float(xv - nxd * floor(xv * a.inv_nx));
            const float yvf = float(yv);
            const float reach = float(a.d_rep) + 1e-3f;
            const int nscan = all_segs ? a.nseg : ncand;
            for (int ci = 0; ci < nscan; ++ci) {
                const int sg = all_segs ? ci : s_cand[ci];
                if (a.seg_mem[sg] == m) continue;
                const float4 bx = a.seg_box[sg];
                const float ddx = wrap_half(xvw - bx.x, Lx);
                float ddy = yvf - bx.y;
                if (!a.walls) ddy = wrap_half(ddy, Ly);
                if (fabsf(ddx) > bx.z + reach || fabsf(ddy) > bx.w + reach) continue;
                const int b0 = a.seg_v0[sg], nb = a.seg_n[sg];
                if (sizeof(C) == 4) {
                    // one FP64 offset to the segment anchor, then FP32 per vertex
                    const double2 an = a.seg_anchor[sg];
                    const float bxo = float(wrap_m(xv - an.x, nxd, a.inv_nx));
                    double byd = yv - an.y;
                    if (!a.walls) byd = wrap_m(byd, nyd, a.inv_ny);
                    const float byo = float(byd);
                    for (int b = b0; b < b0 + nb; ++b) {
                        const float2 o = a.xoff[b];
                        const C dx = C(bxo - o.x), dy = C(byo - o.y);
                        const C d = sqrt(dx * dx + dy * dy);
                        if (d < C(a.d_rep)) {
                            const C mag = c_rep * sqrt(C(1) / (d * d * d * d * d));
                            Fx -= mag * s_nx[sj];
                            Fy -= mag * s_ny[sj];
                        }
                    }
                } else {
                    for (int b = b0; b < b0 + nb; ++b) {
                        const C dx = C(wrap_m(xv - X[2 * b], nxd, a.inv_nx));
                        double dyd = yv - X[2 * b + 1];
                        if (!a.walls) dyd = wrap_m(dyd, nyd, a.inv_ny);
                        const C dy = C(dyd);
                        const C d = sqrt(dx * dx + dy * dy);
                        if (d < C(a.d_rep)) {
                            const C mag = c_rep * sqrt(C(1) / (d * d * d * d * d));
                            Fx -= mag * s_nx[sj];
                            Fy -= mag * s_ny[sj];
                        }
                    }
                }
            }
        }
        // Eq. strainFor on elements (v, R) and (L, v); l - l_0 is formed as
        // (l^2 - l_0^2) / (l + l_0) with the squares in FP64
        {
            const double ex = __dsub_rn(xR, xv), ey = __dsub_rn(yR, yv);
            const double lsq = __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey));
            const C l = sqrt(C(lsq));
            const C c = ks * C(__dsub_rn(lsq, a.rest[4 * (size_t)v])) / ((l + C(a.rest[4 * (size_t)v + 1])) * l);
            Fx += c * C(ex);
            Fy += c * C(ey);
            const double gx = __dsub_rn(xv, xl), gy = __dsub_rn(yv, yl);
            const double lsq2 = __dadd_rn(__dmul_rn(gx, gx), __dmul_rn(gy, gy));
            const C l2 = sqrt(C(lsq2));
            const C c2 = -ks * C(__dsub_rn(lsq2, a.rest[4 * (size_t)L])) / ((l2 + C(a.rest[4 * (size_t)L + 1])) * l2);
            Fx += c2 * C(gx);
            Fy += c2 * C(gy);
        }
        // Eq. bendFor gathered: own term plus the neighbours' shares
        Fx += -s_mnx[sj] + s_mnx[sj + 1] * s_sL[sj + 1] + s_mnx[sj - 1] * s_sR[sj - 1];
        Fy += -s_mny[sj] + s_mny[sj + 1] * s_sL[sj + 1] + s_mny[sj - 1] * s_sR[sj - 1];
        // Eq. areaFor, half of each adjacent element
        Fx += C(0.5) * ca * C(-(yR - yl));
        Fy += C(0.5) * ca * C(xR - xl);
        F[2 * (size_t)v] = Fx;
        F[2 * (size_t)v + 1] = Fy;

        // ---- IB shape functions at X^n: nine nearest nodes, Roma weights,
        // MLS (basis 1, dx, dy) re-solved where wall rows drop out
        // clamped so that a runaway (or NaN) position still yields in-range integers;
        // the advance kernel flags non-finite positions
        const double fi0 = fmin(fmax(floor(xv + 0.5), -1.0e9), 1.0e9);
        const double fj0 = fmin(fmax(floor(yv + 0.5), -1.0e6), 1.0e6);
        const long long i0 = (long long)fi0;
        const int j0 = (int)fj0;
        C rx[3], ry[3], wx[3], wy[3];
        bool rowok[3];
        bool all = true;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            rx[q] = C((fi0 + (q - 1)) - xv);
            ry[q] = C((fj0 + (q - 1)) - yv);
            wx[q] = roma<C>(rx[q]);
            wy[q] = roma<C>(ry[q]);
            const int j = j0 + q - 1;
            rowok[q] = a.walls ? (j >= 0 && j < a.ny) : true;
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
        const int i0w = (int)(((i0 % a.nx) + a.nx) % a.nx);
        const int j0s = a.walls ? j0 : (((j0 % a.ny) + a.ny) % a.ny);
        a.stencil[2 * (size_t)v] = i0w;
        a.stencil[2 * (size_t)v + 1] = j0s;

        // ---- spreading (Sec. 2.2, the transpose of the interpolation): w_j F_v
        // into the fixed-point force field, and flag the fused-kernel tiles hit
        int last_t = -1;
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
                int i = i0w + q - 1;
                i = i < 0 ? i + a.nx : (i >= a.nx ? i - a.nx : i);
                const size_t node = (size_t)j * a.nx + i;
                const C wq = w[b * 3 + q];
                unsigned long long* gp = reinterpret_cast<unsigned long long*>(a.gsum + node);
                atomicAdd(gp, (unsigned long long)to_fix<C>(wq * Fx));
                atomicAdd(gp + 1, (unsigned long long)to_fix<C>(wq * Fy));
                const int t = (j / a.tile_h) * a.tiles_x + i / a.tile_w;
                if (t != last_t) {
                    a.flags[t] = 1;
                    last_t = t;
                }
            }
        }
    }
}

// ---------------------------------------------------------------- advance
// one warp: bounding box of a 32-vertex segment, stored as FP32 with the
// centre's x wrapped into [0, nx)
// One group of kSegV lanes per segment: FP32 offsets of the vertices from the
// segment's first vertex (the anchor), their bounding box reduced within the
// group, stored with the centre's x wrapped into [0, nx).  All 32 lanes of the
// warp call this; `sg` is this lane group's segment or -1.
__device__ void seg_box_group(const MarkerArgs& a, int sg, int lane) {
    const int g = lane & (kSegV - 1);
    int v0 = 0, nb = 0;
    if (sg >= 0) {
        v0 = a.seg_v0[sg];
        nb = a.seg_n[sg];
    }
    float ox = 0.f, oy = 0.f;
    double ax = 0.0, ay = 0.0;
    if (nb > 0) {
        ax = a.X[2 * v0];
        ay = a.X[2 * v0 + 1];
        const int v = v0 + (g < nb ? g : 0);
        ox = float(a.X[2 * v] - ax);
        oy = float(a.X[2 * v + 1] - ay);
        if (g < nb) a.xoff[v] = make_float2(ox, oy);
    }
    float lo_x = ox, hi_x = ox, lo_y = oy, hi_y = oy;
    for (int o = kSegV / 2; o > 0; o >>= 1) {
        lo_x = fminf(lo_x, __shfl_xor_sync(FULL, lo_x, o));
        hi_x = fmaxf(hi_x, __shfl_xor_sync(FULL, hi_x, o));
        lo_y = fminf(lo_y, __shfl_xor_sync(FULL, lo_y, o));
        hi_y = fmaxf(hi_y, __shfl_xor_sync(FULL, hi_y, o));
    }
    if (nb > 0 && g == 0) {
        const double cxd = ax + 0.5 * (double)(lo_x + hi_x);
        const double cxw = cxd - (double)a.nx * floor(cxd * a.inv_nx);
        a.seg_box[sg] = make_float4(float(cxw), float(ay + 0.5 * (double)(lo_y + hi_y)),
                                    0.5f * (hi_x - lo_x), 0.5f * (hi_y - lo_y));
        a.seg_anchor[sg] = make_double2(ax, ay);
    }
}

// boxes of segments [s0, s1) by the warps of a block, kSegV lanes per segment
__device__ void seg_boxes_block(const MarkerArgs& a, int s0, int s1) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    constexpr int per_warp = 32 / kSegV;
    for (int base = s0 + wid * per_warp; base < s1; base += nw * per_warp) {
        const int sg = base + lane / kSegV;
        seg_box_group(a, sg < s1 ? sg : -1, lane);
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

// Eq. kinematicPos (BDF2); forward Euler on the very first step
template <typename C>
__device__ __forceinline__ void advance_vertex(const MarkerArgs& a, int v, long long step) {
    const C* U = static_cast<const C*>(a.U);
    double* X = a.X;
    double* Xp = a.Xp;
    const double Ux = (double)U[2 * v], Uy = (double)U[2 * v + 1];
    const double x = X[2 * v], y = X[2 * v + 1];
    double xn, yn;
    if (step == 0) {
        xn = x + Ux;
        yn = y + Uy;
    } else {
        xn = (2.0 / 3.0) * (2.0 * x - 0.5 * Xp[2 * v] + Ux);
        yn = (2.0 / 3.0) * (2.0 * y - 0.5 * Xp[2 * v + 1] + Uy);
    }
    if (!isfinite(xn) || !isfinite(yn)) atomicOr(a.status, ST_NONFINITE);
    Xp[2 * v] = x;
    Xp[2 * v + 1] = y;
    X[2 * v] = xn;
    X[2 * v + 1] = yn;
}

// One block per unit: a chunk of a kinematic membrane (independent vertices)
// or a whole rigid-projected membrane (needs its centroid and mean rotation).
template <typename C>
__global__ void __launch_bounds__(kChunkV) k_advance(const MarkerArgs a) {
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
        seg_boxes_block(a, a.mem_seg_off[m] + k0 / kSegV, a.mem_seg_off[m] + (k0 + kn + kSegV - 1) / kSegV);
    } else {
        C* U = static_cast<C*>(a.U);
        double* X = a.X;
        for (int k = threadIdx.x; k < n; k += blockDim.x) interp_vertex<C>(a, off + k);
        __syncthreads();
        // least-squares rigid motion U_c + omega x (x - x_c) of the ring; the
        // sums run in the compute precision on positions taken about vertex 0
        const double xr = X[2 * off], yr = X[2 * off + 1];
        C sx = 0, sy = 0, su = 0, sv = 0;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int v = off + k;
            sx += C(X[2 * v] - xr);
            sy += C(X[2 * v + 1] - yr);
            su += U[2 * v];
            sv += U[2 * v + 1];
        }
        const C inv_n = C(1) / C(n);
        const C mx = block_sum_c<C>(sx, cred) * inv_n, my = block_sum_c<C>(sy, cred) * inv_n;
        const C mu = block_sum_c<C>(su, cred) * inv_n, mv = block_sum_c<C>(sv, cred) * inv_n;
        C num = 0, den = 0;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int v = off + k;
            const C rx = C(X[2 * v] - xr) - mx, ry = C(X[2 * v + 1] - yr) - my;
            num += rx * (U[2 * v + 1] - mv) - ry * (U[2 * v] - mu);
            den += rx * rx + ry * ry;
        }
        const C om = block_sum_c<C>(num, cred) / block_sum_c<C>(den, cred);
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int v = off + k;
            const C rx = C(X[2 * v] - xr) - mx, ry = C(X[2 * v + 1] - yr) - my;
            U[2 * v] = mu - om * ry;
            U[2 * v + 1] = mv + om * rx;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < n; k += blockDim.x) advance_vertex<C>(a, off + k, step);
        __syncthreads();
        seg_boxes_block(a, a.mem_seg_off[m], a.mem_seg_off[m + 1]);
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
__global__ void k_seg_boxes(const MarkerArgs a) {
    constexpr int per_block = (256 / 32) * (32 / kSegV);
    const int s0 = blockIdx.x * per_block;
    seg_boxes_block(a, s0, min(a.nseg, s0 + per_block));
}

__global__ void k_areas(const MarkerArgs a, double* areas) {
    const int m = blockIdx.x;
    const int off = a.mem_off[m], n = a.mem_n[m];
    __shared__ double red[33];
    const double* X = a.X;
    const double xr = X[2 * off], yr = X[2 * off + 1];
    double ap = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int v = off + k, R = off + (k == n - 1 ? 0 : k + 1);
        ap += (X[2 * v] - xr) * (X[2 * R + 1] - yr) - (X[2 * R] - xr) * (X[2 * v + 1] - yr);
    }
    const double s = block_sum(ap, red);
    if (threadIdx.x == 0) areas[m] = 0.5 * s;
}

// ---------------------------------------------------------------- launchers
static bool is_f64(lbib_precision p) { return p == LBIB_F64; }

cudaError_t launch_rest(lbib_precision, const MarkerArgs& a, double* rest, double* A0, cudaStream_t s) {
    k_rest<<<a.nmem, 256, 0, s>>>(a, rest, A0);
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

cudaError_t launch_seg_boxes(const MarkerArgs& a, cudaStream_t s) {
    if (a.nseg == 0) return cudaSuccess;
    constexpr int per_block = (256 / 32) * (32 / kSegV);
    k_seg_boxes<<<(a.nseg + per_block - 1) / per_block, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_areas(const MarkerArgs& a, double* areas, cudaStream_t s) {
    k_areas<<<a.nmem, 256, 0, s>>>(a, areas);
    return cudaGetLastError();
}

}  // namespace lbib
