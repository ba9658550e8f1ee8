// Per-vertex pieces of the FP64 time step in dual numbers, shared by the
// forward-mode tangent (tangent_kernels.cu) and the reverse-mode adjoint
// (adjoint_kernels.cu).  A Seed says which input carries the derivative:
//   kTangent   the tangent direction of the TangentArgs (dX, dks, dkb, dsigma,
//              and the area tangents Ad);
//   kPos       marker coordinate `coord` (0 x, 1 y) of vertex `vtx`;
//   kArea      the enclosed area of membrane `mem` (taken as an input);
//   kKs, kKb   k_s, k_b of membrane `mem`;
//   kSigma     the bond stiffness.
// The adjoint forms local Jacobians column by column with one-hot seeds.
#pragma once

#include "dual.cuh"
#include "ext_real.cuh"
#include "tangent.cuh"

namespace lbib {

enum SeedKind { kTangent = 0, kPos = 1, kArea = 2, kKs = 3, kKb = 4, kSigma = 5 };
struct Seed {
    int kind, vtx, coord, mem;
};
__device__ __forceinline__ Seed tangent_seed() { return Seed{kTangent, -1, 0, -1}; }

constexpr double kPrefT = 1.0 / 3.0;  // p_ref = rho_0 c_s^2 (Eq. areaFor)
constexpr double kRepC0 = 1e-4 / (8.0 * 1.4142135623730951);  // repulsion prefactor (Eq. repFor)

__device__ __forceinline__ int t_mem_of(const TangentArgs& t, int v) {
    int lo = 0, hi = t.m.nmem - 1;
    while (lo < hi) {  // last membrane with mem_off <= v
        const int mid = (lo + hi + 1) >> 1;
        if (t.m.mem_off[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void t_pos(const TangentArgs& t, int v, const Seed& s, dual& x, dual& y) {
    const double* X = static_cast<const double*>(t.m.X);
    double dx = 0.0, dy = 0.0;
    if (s.kind == kTangent) {
        dx = t.dX[2 * v];
        dy = t.dX[2 * v + 1];
    } else if (s.kind == kPos && s.vtx == v) {
        dx = s.coord == 0 ? 1.0 : 0.0;
        dy = s.coord == 1 ? 1.0 : 0.0;
    }
    x = dual(X[2 * v], dx);
    y = dual(X[2 * v + 1], dy);
}
__device__ __forceinline__ dual t_ks(const TangentArgs& t, int m, const Seed& s) {
    return dual(t.m.mem_ks[m], s.kind == kTangent ? t.dks[m] : (s.kind == kKs && s.mem == m ? 1.0 : 0.0));
}
__device__ __forceinline__ dual t_kb(const TangentArgs& t, int m, const Seed& s) {
    return dual(t.m.mem_kb[m], s.kind == kTangent ? t.dkb[m] : (s.kind == kKb && s.mem == m ? 1.0 : 0.0));
}
__device__ __forceinline__ dual t_sigma(const TangentArgs& t, const Seed& s) {
    return dual(t.m.sigma, s.kind == kTangent ? t.dsigma : (s.kind == kSigma ? 1.0 : 0.0));
}
__device__ __forceinline__ dual t_area(const TangentArgs& t, int m, const Seed& s) {
    return dual(t.A[m], s.kind == kTangent ? t.Ad[m] : (s.kind == kArea && s.mem == m ? 1.0 : 0.0));
}

// vertex k of membrane (off, n), local index wrapped
__device__ __forceinline__ int t_ring(int off, int n, int k) { return off + ((k % n) + n) % n; }

__device__ __forceinline__ dual t_wrap_x(const TangentArgs& t, dual dx) {
    dx.v -= t.m.nx * floor(dx.v * t.m.inv_nx + 0.5);
    return dx;
}
__device__ __forceinline__ dual t_wrap_y(const TangentArgs& t, dual dy) {
    if (!t.m.walls) dy.v -= t.m.ny * floor(dy.v * t.m.inv_ny + 0.5);
    return dy;
}

// turning angle, outward vertex normal and adjacent edge lengths at vertex k
struct VGeo {
    dual th, nx, ny, lL, lR;
};
__device__ __forceinline__ VGeo t_vgeo(const TangentArgs& t, int off, int n, int k, const Seed& s) {
    dual xL, yL, xv, yv, xR, yR;
    t_pos(t, t_ring(off, n, k - 1), s, xL, yL);
    t_pos(t, t_ring(off, n, k), s, xv, yv);
    t_pos(t, t_ring(off, n, k + 1), s, xR, yR);
    const dual eLx = xv - xL, eLy = yv - yL, eRx = xR - xv, eRy = yR - yv;
    VGeo g;
    g.lL = sqrt(eLx * eLx + eLy * eLy);
    g.lR = sqrt(eRx * eRx + eRy * eRy);
    g.th = atan2(eLx * eRy - eLy * eRx, eLx * eRx + eLy * eRy);
    dual nx_ = eLy / g.lL + eRy / g.lR;
    dual ny_ = -eLx / g.lL - eRx / g.lR;
    const dual nn = sqrt(nx_ * nx_ + ny_ * ny_);
    g.nx = nx_ / nn;
    g.ny = ny_ / nn;
    return g;
}

// bond spring of the ligand on element e (if bonded), half on each end vertex
__device__ __forceinline__ void t_bond_half(const TangentArgs& t, int e, const Seed& s, dual& fx, dual& fy) {
    const int l = t.m.elem_lig[e];
    if (l < 0) return;
    const int r = t.m.bond_of_lig[l];
    if (r < 0) return;
    dual xa, ya, xb, yb;
    t_pos(t, t.m.lig_a[l], s, xa, ya);
    t_pos(t, t.m.lig_b[l], s, xb, yb);
    const dual cx = 0.5 * (xa + xb), cy = 0.5 * (ya + yb);
    const dual dx = t_wrap_x(t, dual(t.m.rec_xy[2 * r]) - cx);
    const dual dy = t_wrap_y(t, dual(t.m.rec_xy[2 * r + 1]) - cy);
    const dual d = sqrt(dx * dx + dy * dy);
    const dual c = t_sigma(t, s) * (d - dual(t.m.y_eq)) / d;
    fx += 0.5 * c * dx;
    fy += 0.5 * c * dy;
}

// true if vertex (x, y) can be within d_rep of membrane mb (its bounding box,
// periodic in x, grown by d_rep)
__device__ __forceinline__ bool t_near_box(const TangentArgs& t, int mb, double x, double y) {
    const double reach = t.m.d_rep + 1e-9;
    const double* bb = t.box + 4 * mb;
    double cxm = x - 0.5 * (bb[0] + bb[1]);
    cxm -= t.m.nx * floor(cxm * t.m.inv_nx + 0.5);
    double cym = y - 0.5 * (bb[2] + bb[3]);
    if (!t.m.walls) cym -= t.m.ny * floor(cym * t.m.inv_ny + 0.5);
    return ::fabs(cxm) <= 0.5 * (bb[1] - bb[0]) + reach && ::fabs(cym) <= 0.5 * (bb[3] - bb[2]) + reach;
}

// plain-value pre-check of a repulsion pair: false only where the pair is
// certainly farther apart than d_rep (the squared distance, with a margin far
// above its rounding), so the exact test d < d_rep after the square root keeps
// the same pairs
__device__ __forceinline__ bool t_rep_candidate(const TangentArgs& t, double xv, double yv, int b) {
    const double* X = static_cast<const double*>(t.m.X);
    const double dx = t_wrap_x(t, dual(xv - X[2 * b])).v;
    const double dy = t_wrap_y(t, dual(yv - X[2 * b + 1])).v;
    return dx * dx + dy * dy < t.m.d_rep * t.m.d_rep * (1.0 + 1e-10);
}

// Total Lagrangian force on vertex v (membrane m, local index k) at X^n:
// bond springs (Eq. adhFor) of the elements sharing v, repulsion (Eq. repFor)
// from the other membranes, stretching (Eq. strainFor), bending (Eq. bendFor:
// own term and the shares of both neighbours) and the area penalty (Eq.
// areaFor, half of each adjacent element, with the membrane's area t.A).
// `terms` selects the contributions (kTerm* bits); the adjoint evaluates only
// those that depend on its seed and takes the repulsion separately.
enum ForceTerm : unsigned {
    kTermBond = 1u,
    kTermRep = 2u,
    kTermStretch = 4u,
    kTermBendL = 8u,   // bending moment at vertex v - 1 (depends on X_{v-2} .. X_v)
    kTermBendV = 16u,  // at v (X_{v-1} .. X_{v+1})
    kTermBendR = 32u,  // at v + 1 (X_v .. X_{v+2})
    kTermArea = 64u,
    kTermAll = 127u
};
__device__ __forceinline__ void t_vertex_force(const TangentArgs& t, int v, int m, const Seed& s, dual& fx, dual& fy,
                                               unsigned terms = kTermAll) {
    const int off = t.m.mem_off[m], n = t.m.mem_n[m], k = v - off;
    const int L = t_ring(off, n, k - 1), R = t_ring(off, n, k + 1);
    fx = dual(0.0);
    fy = dual(0.0);
    dual xL, yL, xv, yv, xR, yR;
    t_pos(t, L, s, xL, yL);
    t_pos(t, v, s, xv, yv);
    t_pos(t, R, s, xR, yR);
    if ((terms & kTermBond) && t.m.nlig > 0) {
        t_bond_half(t, L, s, fx, fy);
        t_bond_half(t, v, s, fx, fy);
    }
    if ((terms & kTermRep) && t.m.nmem > 1) {
        const double c0 = kRepC0;
        bool have_g = false;
        VGeo g;
        for (int mb = 0; mb < t.m.nmem; ++mb) {
            if (mb == m || !t_near_box(t, mb, xv.v, yv.v)) continue;
            if (!have_g) {
                g = t_vgeo(t, off, n, k, s);
                have_g = true;
            }
            const int o2 = t.m.mem_off[mb], n2 = t.m.mem_n[mb];
            for (int b = o2; b < o2 + n2; ++b) {
                if (!t_rep_candidate(t, xv.v, yv.v, b)) continue;
                dual xb, yb;
                t_pos(t, b, s, xb, yb);
                const dual dx = t_wrap_x(t, xv - xb), dy = t_wrap_y(t, yv - yb);
                const dual d = sqrt(dx * dx + dy * dy);
                if (d.v < t.m.d_rep) {
                    const dual mag = c0 * pow_m52(d);
                    fx -= mag * g.nx;
                    fy -= mag * g.ny;
                }
            }
        }
    }
    if (terms & kTermStretch) {
        const dual ks = t_ks(t, m, s);
        const dual rx = xv - xR, ry = yv - yR;
        const dual l = sqrt(rx * rx + ry * ry);
        const dual c = -ks * (l - dual(t.l0[v])) / l;
        fx += c * rx;
        fy += c * ry;
        const dual qx = xL - xv, qy = yL - yv;
        const dual l2 = sqrt(qx * qx + qy * qy);
        const dual c2 = -ks * (l2 - dual(t.l0[L])) / l2;
        fx -= c2 * qx;
        fy -= c2 * qy;
    }
    if (terms & (kTermBendL | kTermBendV | kTermBendR)) {
        const dual kb = t_kb(t, m, s);
        if (terms & kTermBendL) {
            const VGeo gL = t_vgeo(t, off, n, k - 1, s);
            const dual mL = kb * (gL.th - dual(t.th0[L]));
            const dual sR_L = gL.lR / (gL.lL + gL.lR);
            fx += mL * sR_L * gL.nx;
            fy += mL * sR_L * gL.ny;
        }
        if (terms & kTermBendV) {
            const VGeo gv = t_vgeo(t, off, n, k, s);
            const dual mv = kb * (gv.th - dual(t.th0[v]));
            fx -= mv * gv.nx;
            fy -= mv * gv.ny;
        }
        if (terms & kTermBendR) {
            const VGeo gR = t_vgeo(t, off, n, k + 1, s);
            const dual mR = kb * (gR.th - dual(t.th0[R]));
            const dual sL_R = gR.lL / (gR.lL + gR.lR);
            fx += mR * sL_R * gR.nx;
            fy += mR * sL_R * gR.ny;
        }
    }
    if (terms & kTermArea) {
        const dual A = t_area(t, m, s);
        const dual c = -t.m.mem_ka[m] * (dual(1.0) - A / dual(t.m.mem_A0[m])) * kPrefT;
        fx += 0.5 * c * (-(yR - yv)) + 0.5 * c * (-(yv - yL));
        fy += 0.5 * c * (xR - xv) + 0.5 * c * (xv - xL);
    }
}

__device__ __forceinline__ dual t_roma(dual r) {
    const dual a = fabs(r);
    if (a.v <= 0.5) return (dual(1.0) + sqrt(dual(1.0) - 3.0 * a * a)) / dual(3.0);
    if (a.v <= 1.5) {
        const dual b = dual(1.0) - a;
        return (dual(5.0) - 3.0 * a - sqrt(dual(1.0) - 3.0 * b * b)) / dual(6.0);
    }
    return dual(0.0);
}

// Shape functions of vertex v (MLS with Roma weights on the nine nearest
// nodes, Sec. 2.2 / 2.3; out-of-fluid rows dropped and the 3x3 system re-solved):
// w[k] for node (i0 + k % 3 - 1, j0 + k / 3 - 1), in[k] false for dropped nodes.
__device__ __forceinline__ void t_vertex_weights(const TangentArgs& t, int v, const Seed& s, dual w[9], bool in[9],
                                                 int& i0, int& j0) {
    dual px, py;
    t_pos(t, v, s, px, py);
    i0 = (int)floor(px.v + 0.5);
    j0 = (int)floor(py.v + 0.5);
    // the Roma factors of the three columns and the three rows
    dual rxa[3], rya[3], phx[3], phy[3];
    for (int a = 0; a < 3; ++a) {
        rxa[a] = dual((double)(i0 + a - 1)) - px;
        rya[a] = dual((double)(j0 + a - 1)) - py;
        phx[a] = t_roma(rxa[a]);
        phy[a] = t_roma(rya[a]);
    }
    dual Wr[9], rx[9], ry[9];
    int nvalid = 0;
    for (int b = -1; b <= 1; ++b)
        for (int a = -1; a <= 1; ++a) {
            const int k = (b + 1) * 3 + (a + 1);
            rx[k] = rxa[a + 1];
            ry[k] = rya[b + 1];
            const int j = j0 + b;
            in[k] = t.m.walls ? (j >= 0 && j < t.m.ny) : true;
            Wr[k] = in[k] ? phx[a + 1] * phy[b + 1] : dual(0.0);
            nvalid += in[k];
        }
    for (int k = 0; k < 9; ++k) w[k] = dual(0.0);
    if (nvalid == 9) {
        for (int k = 0; k < 9; ++k) w[k] = Wr[k];
        return;
    }
    dual A00, A01, A02, A11, A12, A22, sw;
    for (int k = 0; k < 9; ++k) {
        sw += Wr[k];
        A00 += Wr[k];
        A01 += Wr[k] * rx[k];
        A02 += Wr[k] * ry[k];
        A11 += Wr[k] * rx[k] * rx[k];
        A12 += Wr[k] * rx[k] * ry[k];
        A22 += Wr[k] * ry[k] * ry[k];
    }
    const dual c00 = A11 * A22 - A12 * A12;
    const dual c10 = -(A01 * A22 - A12 * A02);
    const dual c20 = A01 * A12 - A11 * A02;
    const dual det = A00 * c00 + A01 * c10 + A02 * c20;
    if (det.v > 1e-10) {
        for (int k = 0; k < 9; ++k) w[k] = Wr[k] * (c00 / det + c10 / det * rx[k] + c20 / det * ry[k]);
    } else if (sw.v > 0.0) {
        for (int k = 0; k < 9; ++k) w[k] = Wr[k] / sw;
    }
}

// node index of stencil entry k (x periodic; y periodic without walls)
__device__ __forceinline__ size_t t_node(const TangentArgs& t, int i0, int j0, int k) {
    int i = (i0 + k % 3 - 1) % t.m.nx;
    i = i < 0 ? i + t.m.nx : i;
    int j = j0 + k / 3 - 1;
    if (!t.m.walls) j = ((j % t.m.ny) + t.m.ny) % t.m.ny;
    return (size_t)j * t.m.nx + i;
}

// storage index that population i of `node` is pulled from (half-way
// bounce-back where the source row is outside the walls); every index is the
// source of exactly one (node, i)
__device__ __forceinline__ size_t t_pull_src(size_t node, int i, int nx, int ny, int walls) {
    const size_t N = (size_t)nx * ny;
    const int y = (int)(node / nx), x = (int)(node % nx);
    int sy = y - cy(i), sx = x - cx(i);
    sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
    if (walls && (sy < 0 || sy >= ny)) return (size_t)opp(i) * N + node;
    sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
    return (size_t)i * N + (size_t)sy * nx + sx;
}

}  // namespace lbib
