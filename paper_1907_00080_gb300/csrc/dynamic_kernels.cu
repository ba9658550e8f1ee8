// Dynamic IB for particles (Sec. 2.4): the hydrodynamic stresses on the
// elements of each dynamic membrane and the forcing term its vertices exert
// on the fluid, at the start of a step (before the force kernel).
//
// Per element l = (v, v+1) of a CCW ring, Eqs. hydroForP / hydroForNu:
//   F_l = (-p n_l + tau . n_l) l_l,  tau = nu (grad u + grad u^T),
// with n_l the outward unit normal and p, grad u fitted by moving least
// squares (linear basis, Roma weights, the 3x3 nodes nearest to the probe
// c_l + 1.2 n_l that lie in the fluid).  The flow is that of the populations
// f^n the step starts from: rho = sum f, u = (sum f e + G_body / 2) / rho,
// p = (rho - 1) / 3.  Each vertex gets half of both adjacent element forces
// (added to its membrane force by the force kernel) and exerts on the fluid
//   D_v = 2 dV_v (u_p,v - U~_v),
// the direct-forcing reading of the paper's effective forcing term (Uhlmann
// 2005; MLS transfer of Vanella & Balaras 2009): U~ is the flow interpolated
// at the vertex with the IB shape functions, dV_v half the two adjacent
// element lengths, and the factor 2 accounts for the half force a node's
// velocity carries under Guo forcing.
//
// One block per chunk of 16 (FP32) or 4 (FP64) vertices of a dynamic
// membrane, one thread per (fit, stencil node) pair.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "marker_common.cuh"

namespace lbib {

template <typename C> __device__ __forceinline__ C hydro_wall(const HydroArgs& h, bool bottom);
template <> __device__ __forceinline__ float hydro_wall<float>(const HydroArgs& h, bool bottom) {
    return bottom ? h.bbf_bot : h.bbf_top;
}
template <> __device__ __forceinline__ double hydro_wall<double>(const HydroArgs& h, bool bottom) {
    return bottom ? h.bb_bot : h.bb_top;
}

// Division and square root of the FP32 path through the hardware's fast
// approximations (a few ulp: far inside the FP32 path's 1e-5 bar, and the
// kernel is bound by its dependent chain of these operations); the FP64 path
// keeps the correctly rounded ones.
__device__ __forceinline__ float hdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double hdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float hsqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
__device__ __forceinline__ double hsqrt(double x) { return sqrt(x); }

// Roma, Peskin & Berger three-point regularised delta with those operations
template <typename C>
__device__ __forceinline__ C roma_h(C r) {
    const C a = fabs(r);
    if (a <= C(0.5)) return hdiv(C(1) + hsqrt(C(1) - C(3) * a * a), C(3));
    if (a <= C(1.5)) {
        const C b = C(1) - a;
        return hdiv(C(5) - C(3) * a - hsqrt(C(1) - C(3) * b * b), C(6));
    }
    return C(0);
}

// p, u, v of node (i, j) (i in [0, nx), j a fluid row) from the pre-collision
// populations: the pull of the post-collision deviations, with the half-way
// bounce-back (plus the moving-wall term) where the source lies behind a wall
template <typename S>
__device__ __forceinline__ void node_flow(const MarkerArgs& a, const HydroArgs& h, int i, int j,
                                          typename Storage<S>::C& p, typename Storage<S>::C& u,
                                          typename Storage<S>::C& v) {
    using C = typename Storage<S>::C;
    const S* src = static_cast<const S*>(h.src);
    const int nx = a.nx, ny = a.ny;
    const size_t N = (size_t)nx * ny;
    const size_t node = (size_t)j * nx + i;
    C d[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        int sy = j - cy(q);
        if (a.walls && (sy < 0 || sy >= ny)) {
            d[q] = Storage<S>::load(src[(size_t)opp(q) * N + node], h.inv_scale);
            if (cx(q) != 0) d[q] += C(cx(q)) * hydro_wall<C>(h, cy(q) > 0);
        } else {
            sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
            int sx = i - cx(q);
            sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
            d[q] = Storage<S>::load(src[(size_t)q * N + (size_t)sy * nx + sx], h.inv_scale);
        }
    }
    const C drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    const C jx = (d[1] - d[3]) + ((d[5] - d[7]) + (d[8] - d[6]));
    const C jy = (d[2] - d[4]) + ((d[5] - d[7]) + (d[6] - d[8]));
    const C rho = C(1) + drho;
    u = hdiv(jx + C(0.5) * C(h.gx), rho);
    v = hdiv(jy + C(0.5) * C(h.gy), rho);
    p = hdiv(drho, C(3));
}

// nearest-node stencil of a point: origin, node-minus-point offsets, Roma
// factors and which rows are fluid
template <typename C>
struct Stencil {
    int i0, j0;
    C rx[3], ry[3], wx[3], wy[3];
    bool rowok[3];
    int nrow;
};

template <typename C, typename E>
__device__ __forceinline__ Stencil<C> stencil_at(const MarkerArgs& a, E px, E py) {
    Stencil<C> st;
    // clamped so that a runaway position still indexes in range (the advance
    // kernel reports non-finite positions)
    const C fi0 = fmin(fmax(C(efloor(eaddc(px, C(0.5)))), C(-1.0e7)), C(1.0e7));
    const C fj0 = fmin(fmax(C(efloor(eaddc(py, C(0.5)))), C(-1.0e6)), C(1.0e6));
    st.i0 = (int)fi0;
    st.j0 = (int)fj0;
    st.nrow = 0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        st.rx[q] = -etoc(eaddc(px, -(fi0 + C(q - 1))));
        st.ry[q] = -etoc(eaddc(py, -(fj0 + C(q - 1))));
        st.wx[q] = roma_h<C>(st.rx[q]);
        st.wy[q] = roma_h<C>(st.ry[q]);
        const int jj = st.j0 + q - 1;
        st.rowok[q] = a.walls ? (jj >= 0 && jj < a.ny) : true;
        st.nrow += st.rowok[q] ? 1 : 0;
    }
    return st;
}

// the stencil's values at row b, column q, picked with unrolled selects (no
// run-time indexing of the register arrays)
template <typename C>
struct NodeOf {
    C rx, ry, wx, wy;
    bool rowok;
};
template <typename C>
__device__ __forceinline__ NodeOf<C> node_of(const Stencil<C>& st, int b, int q) {
    NodeOf<C> o{C(0), C(0), C(0), C(0), false};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (k == q) {
            o.rx = st.rx[k];
            o.wx = st.wx[k];
        }
        if (k == b) {
            o.ry = st.ry[k];
            o.wy = st.wy[k];
            o.rowok = st.rowok[k];
        }
    }
    return o;
}

template <typename C>
__device__ __forceinline__ void stencil_node(const MarkerArgs& a, const Stencil<C>& st, int b, int q, int& i,
                                             int& j) {
    j = st.j0 + b - 1;
    if (!a.walls) j = ((j % a.ny) + a.ny) % a.ny;
    i = ((st.i0 + q - 1) % a.nx + a.nx) % a.nx;
}

// The work of a block: a chunk of up to V consecutive vertices of one
// dynamic membrane.  Its fits are the probes of the kv + 1 elements k0 - 1 ..
// k0 + kv - 1 (each vertex needs the elements on both sides) and the kv
// vertices; each (fit, stencil node) pair is one thread, so that the nine
// node flows of a fit are read in parallel and the fit's sums are formed
// afterwards in the fixed node order.
// Chunk sizes: 16 vertices (320 threads) in FP32; 4 vertices (96 threads) in
// FP64, where the work is bound by the FP64 pipe of the SMs it runs on, so
// more, smaller blocks spread it over more SMs.
template <int V>
struct HydroShape {
    static constexpr int fits = 2 * V + 1;
    static constexpr int threads = (9 * fits + 31) / 32 * 32;  // one thread per (fit, node)
};
constexpr int kHydroV32 = 16, kHydroV64 = 4;

// node-flow products of one (fit, node) pair: a probe's MLS rows times (p, u, u, v, v)
// (value of p, x and y derivatives of u and of v), or a vertex's shape
// function times (u, v)
template <typename S, typename E>
__device__ __forceinline__ void probe_part(const MarkerArgs& a, const HydroArgs& h, E qx, E qy, int b, int q,
                                           typename Storage<S>::C (&part)[5]) {
    using C = typename Storage<S>::C;
    const Stencil<C> st = stencil_at<C, E>(a, qx, qy);
    C M00 = 0, M01 = 0, M02 = 0, M11 = 0, M12 = 0, M22 = 0;
#pragma unroll
    for (int bb = 0; bb < 3; ++bb)
#pragma unroll
        for (int qq = 0; qq < 3; ++qq) {
            const C w = st.rowok[bb] ? st.wx[qq] * st.wy[bb] : C(0);
            M00 += w;
            M01 += w * st.rx[qq];
            M02 += w * st.ry[bb];
            M11 += w * st.rx[qq] * st.rx[qq];
            M12 += w * st.rx[qq] * st.ry[bb];
            M22 += w * st.ry[bb] * st.ry[bb];
        }
#pragma unroll
    for (int r = 0; r < 5; ++r) part[r] = C(0);
    const NodeOf<C> nd = node_of<C>(st, b, q);
    if (!nd.rowok) return;
    int i, j;
    stencil_node<C>(a, st, b, q, i, j);
    C pk, uk, vk;
    node_flow<S>(a, h, i, j, pk, uk, vk);
    const C w = nd.wx * nd.wy;
    // inverse of the symmetric moment matrix by its adjugate; with one fluid
    // row (or none) the y derivative is undetermined: the value falls back to
    // the normalised weights, the gradient to zero
    const C c00 = M11 * M22 - M12 * M12;
    const C c01 = -(M01 * M22 - M12 * M02);
    const C c02 = M01 * M12 - M11 * M02;
    const C det = M00 * c00 + M01 * c01 + M02 * c02;
    if (st.nrow >= 2 && det > C(1e-10)) {
        const C c11 = M00 * M22 - M02 * M02;
        const C c12 = -(M00 * M12 - M01 * M02);
        const C c22 = M00 * M11 - M01 * M01;
        const C f0 = hdiv(w * (c00 + c01 * nd.rx + c02 * nd.ry), det);
        const C f1 = hdiv(w * (c01 + c11 * nd.rx + c12 * nd.ry), det);
        const C f2 = hdiv(w * (c02 + c12 * nd.rx + c22 * nd.ry), det);
        part[0] = f0 * pk;
        part[1] = f1 * uk;
        part[2] = f2 * uk;
        part[3] = f1 * vk;
        part[4] = f2 * vk;
    } else {
        part[0] = (M00 > C(0) ? hdiv(w, M00) : C(0)) * pk;
    }
}

// the IB shape function of a vertex at one stencil node (Roma weights on the
// full stencil; near a wall the MLS value row, as in the force kernel) times
// the node's (u, v)
template <typename S, typename E>
__device__ __forceinline__ void vertex_part(const MarkerArgs& a, const HydroArgs& h, E xv, E yv, int b, int q,
                                            typename Storage<S>::C (&part)[5]) {
    using C = typename Storage<S>::C;
    const Stencil<C> st = stencil_at<C, E>(a, xv, yv);
#pragma unroll
    for (int r = 0; r < 5; ++r) part[r] = C(0);
    const NodeOf<C> nd = node_of<C>(st, b, q);
    if (!nd.rowok) return;
    C w = nd.wx * nd.wy;
    if (st.nrow < 3) {
        C M00 = 0, M01 = 0, M02 = 0, M11 = 0, M12 = 0, M22 = 0, sw = 0;
#pragma unroll
        for (int bb = 0; bb < 3; ++bb)
#pragma unroll
            for (int qq = 0; qq < 3; ++qq) {
                const C ww = st.rowok[bb] ? st.wx[qq] * st.wy[bb] : C(0);
                sw += ww;
                M00 += ww;
                M01 += ww * st.rx[qq];
                M02 += ww * st.ry[bb];
                M11 += ww * st.rx[qq] * st.rx[qq];
                M12 += ww * st.rx[qq] * st.ry[bb];
                M22 += ww * st.ry[bb] * st.ry[bb];
            }
        const C c0 = M11 * M22 - M12 * M12;
        const C c1 = -(M01 * M22 - M12 * M02);
        const C c2 = M01 * M12 - M11 * M02;
        const C det = M00 * c0 + M01 * c1 + M02 * c2;
        if (det > C(1e-10)) w = hdiv(w * (c0 + c1 * nd.rx + c2 * nd.ry), det);
        else w = sw > C(0) ? hdiv(w, sw) : C(0);
    }
    int i, j;
    stencil_node<C>(a, st, b, q, i, j);
    C pk, uk, vk;
    node_flow<S>(a, h, i, j, pk, uk, vk);
    part[0] = w * uk;
    part[1] = w * vk;
}

template <typename S, int kHydroV>
__global__ void __launch_bounds__(HydroShape<kHydroV>::threads) k_hydro(const MarkerArgs a, const HydroArgs h) {
    constexpr int kHydroFits = HydroShape<kHydroV>::fits;
    using C = typename Storage<S>::C;
    using E = typename Ext<C>::E;
    // the unit record carries the membrane's offset and size, so that no block
    // waits on a second table before its first position load
    const int4 u = h.units[blockIdx.x];
    const int k0 = u.x, kv = u.y, off = u.z, n = u.w;
    const int nel = kv + 1, nfit = 2 * kv + 1;
    // the particle velocities of the chunk, fetched now for the last stage
    C vpx = C(0), vpy = C(0);
    if (threadIdx.x < kv) {
        const C* V = static_cast<const C*>(a.V);
        vpx = V[2 * (size_t)(off + k0 + threadIdx.x)];
        vpy = V[2 * (size_t)(off + k0 + threadIdx.x) + 1];
    }
    __shared__ C s_part[kHydroFits][9][5];
    __shared__ C s_nx[kHydroV + 1], s_ny[kHydroV + 1], s_len[kHydroV + 1];
    __shared__ C s_fx[kHydroV + 1], s_fy[kHydroV + 1], s_ux[kHydroV], s_uy[kHydroV];
    const int t = threadIdx.x;
    const int fit = t / 9, node = t - 9 * (t / 9);
    const int b = node / 3, q = node - 3 * (node / 3);

    // ---- one (fit, node) pair per thread
    if (fit < nfit) {
        C part[5];
        if (fit < nel) {
            // element e = (k0 - 1 + fit) mod n between vertices e and e + 1:
            // outward normal, length, probe c_e + 1.2 n_e
            int e = k0 - 1 + fit;
            e = e < 0 ? e + n : (e >= n ? e - n : e);
            E x0, y0, x1, y1;
            load_pos<C>(a, off + e, x0, y0);
            load_pos<C>(a, off + (e + 1 == n ? 0 : e + 1), x1, y1);
            const C ex = etoc(esub(x1, x0)), ey = etoc(esub(y1, y0));
            const C len = hsqrt(ex * ex + ey * ey);
            const C nx = hdiv(ey, len), ny = hdiv(-ex, len);
            const E qx = eaddc(emulc(eadd(x0, x1), C(0.5)), C(1.2) * nx);
            const E qy = eaddc(emulc(eadd(y0, y1), C(0.5)), C(1.2) * ny);
            probe_part<S, E>(a, h, qx, qy, b, q, part);
            if (node == 0) {
                s_nx[fit] = nx;
                s_ny[fit] = ny;
                s_len[fit] = len;
            }
        } else {
            E xv, yv;
            load_pos<C>(a, off + k0 + fit - nel, xv, yv);
            vertex_part<S, E>(a, h, xv, yv, b, q, part);
        }
#pragma unroll
        for (int r = 0; r < 5; ++r) s_part[fit][node][r] = part[r];
    }
    __syncthreads();

    // ---- per fit: the sums over the nine nodes in node order
    if (t < nfit) {
        C sum[5] = {C(0), C(0), C(0), C(0), C(0)};
        for (int k = 0; k < 9; ++k)
#pragma unroll
            for (int r = 0; r < 5; ++r) sum[r] += s_part[t][k][r];
        if (t < nel) {
            // Eqs. hydroForP / hydroForNu: (-p n + tau . n) l, tau = nu (grad u + grad u^T)
            const C p = sum[0], dux = sum[1], duy = sum[2], dvx = sum[3], dvy = sum[4];
            const C nu = C(h.nu), nx = s_nx[t], ny = s_ny[t], len = s_len[t];
            const C txx = C(2) * nu * dux, tyy = C(2) * nu * dvy, txy = nu * (duy + dvx);
            s_fx[t] = (-p * nx + (txx * nx + txy * ny)) * len;
            s_fy[t] = (-p * ny + (txy * nx + tyy * ny)) * len;
        } else {
            s_ux[t - nel] = sum[0];
            s_uy[t - nel] = sum[1];
        }
    }
    __syncthreads();

    // ---- per vertex: half of both adjacent element forces, and the forcing term
    if (t < kv) {
        const int v = off + k0 + t;  // elements k0 + t - 1 and k0 + t are fits t and t + 1
        C* H = static_cast<C*>(a.Hf);
        C* D = static_cast<C*>(a.Dib);
        H[2 * (size_t)v] = C(0.5) * (s_fx[t] + s_fx[t + 1]);
        H[2 * (size_t)v + 1] = C(0.5) * (s_fy[t] + s_fy[t + 1]);
        const C dV = C(0.5) * (s_len[t] + s_len[t + 1]);
        D[2 * (size_t)v] = C(2) * dV * (vpx - s_ux[t]);
        D[2 * (size_t)v + 1] = C(2) * dV * (vpy - s_uy[t]);
    }
}

int hydro_chunk(lbib_precision prec) { return prec == LBIB_F64 ? kHydroV64 : kHydroV32; }

cudaError_t launch_hydro(lbib_precision prec, const MarkerArgs& a, const HydroArgs& h, cudaStream_t s) {
    if (h.nunits == 0) return cudaSuccess;
    switch (prec) {
        case LBIB_F64:
            k_hydro<double, kHydroV64><<<h.nunits, HydroShape<kHydroV64>::threads, 0, s>>>(a, h);
            break;
        case LBIB_F32:
            k_hydro<float, kHydroV32><<<h.nunits, HydroShape<kHydroV32>::threads, 0, s>>>(a, h);
            break;
        case LBIB_F32_STORE_F16:
            k_hydro<__half, kHydroV32><<<h.nunits, HydroShape<kHydroV32>::threads, 0, s>>>(a, h);
            break;
        case LBIB_F32_STORE_BF16:
            k_hydro<__nv_bfloat16, kHydroV32><<<h.nunits, HydroShape<kHydroV32>::threads, 0, s>>>(a, h);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace lbib
