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
// One block per dynamic membrane, one thread per vertex (<= 256 vertices).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "marker_common.cuh"

namespace lbib {

constexpr int kHydroThreads = 4 * kChunkV;  // most vertices of a dynamic membrane

template <typename C> __device__ __forceinline__ C hydro_wall(const HydroArgs& h, bool bottom);
template <> __device__ __forceinline__ float hydro_wall<float>(const HydroArgs& h, bool bottom) {
    return bottom ? h.bbf_bot : h.bbf_top;
}
template <> __device__ __forceinline__ double hydro_wall<double>(const HydroArgs& h, bool bottom) {
    return bottom ? h.bb_bot : h.bb_top;
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
    u = (jx + C(0.5) * C(h.gx)) / rho;
    v = (jy + C(0.5) * C(h.gy)) / rho;
    p = drho / C(3);
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
        st.wx[q] = roma<C>(st.rx[q]);
        st.wy[q] = roma<C>(st.ry[q]);
        const int jj = st.j0 + q - 1;
        st.rowok[q] = a.walls ? (jj >= 0 && jj < a.ny) : true;
        st.nrow += st.rowok[q] ? 1 : 0;
    }
    return st;
}

template <typename C>
__device__ __forceinline__ void stencil_node(const MarkerArgs& a, const Stencil<C>& st, int b, int q, int& i,
                                             int& j) {
    j = st.j0 + b - 1;
    if (!a.walls) j = ((j % a.ny) + a.ny) % a.ny;
    i = ((st.i0 + q - 1) % a.nx + a.nx) % a.nx;
}

// MLS fit at the probe: value of p and the gradient of (u, v)
template <typename S, typename E>
__device__ void probe_fit(const MarkerArgs& a, const HydroArgs& h, E qx, E qy, typename Storage<S>::C& p,
                          typename Storage<S>::C& dux, typename Storage<S>::C& duy,
                          typename Storage<S>::C& dvx, typename Storage<S>::C& dvy) {
    using C = typename Storage<S>::C;
    const Stencil<C> st = stencil_at<C, E>(a, qx, qy);
    C M00 = 0, M01 = 0, M02 = 0, M11 = 0, M12 = 0, M22 = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const C w = st.rowok[b] ? st.wx[q] * st.wy[b] : C(0);
            M00 += w;
            M01 += w * st.rx[q];
            M02 += w * st.ry[b];
            M11 += w * st.rx[q] * st.rx[q];
            M12 += w * st.rx[q] * st.ry[b];
            M22 += w * st.ry[b] * st.ry[b];
        }
    // inverse of the symmetric moment matrix by its adjugate
    const C c00 = M11 * M22 - M12 * M12;
    const C c01 = -(M01 * M22 - M12 * M02);
    const C c02 = M01 * M12 - M11 * M02;
    const C c11 = M00 * M22 - M02 * M02;
    const C c12 = -(M00 * M12 - M01 * M02);
    const C c22 = M00 * M11 - M01 * M01;
    const C det = M00 * c00 + M01 * c01 + M02 * c02;
    // one fluid row (or none) leaves the y derivative undetermined: the value
    // falls back to the normalised weights, the gradient to zero
    const bool solve = st.nrow >= 2 && det > C(1e-10);
    p = dux = duy = dvx = dvy = C(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        if (!st.rowok[b]) continue;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            int i, j;
            stencil_node<C>(a, st, b, q, i, j);
            C pk, uk, vk;
            node_flow<S>(a, h, i, j, pk, uk, vk);
            const C w = st.wx[q] * st.wy[b];
            if (solve) {
                const C f0 = w * (c00 + c01 * st.rx[q] + c02 * st.ry[b]) / det;
                const C f1 = w * (c01 + c11 * st.rx[q] + c12 * st.ry[b]) / det;
                const C f2 = w * (c02 + c12 * st.rx[q] + c22 * st.ry[b]) / det;
                p += f0 * pk;
                dux += f1 * uk;
                duy += f2 * uk;
                dvx += f1 * vk;
                dvy += f2 * vk;
            } else {
                p += (M00 > C(0) ? w / M00 : C(0)) * pk;
            }
        }
    }
}

// the flow interpolated at a vertex with the IB shape functions (Roma weights
// on the full stencil; near a wall the MLS value row, as in the force kernel)
template <typename S, typename E>
__device__ void vertex_flow(const MarkerArgs& a, const HydroArgs& h, E xv, E yv, typename Storage<S>::C& Ux,
                            typename Storage<S>::C& Uy) {
    using C = typename Storage<S>::C;
    const Stencil<C> st = stencil_at<C, E>(a, xv, yv);
    C w[9];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int q = 0; q < 3; ++q) w[b * 3 + q] = st.rowok[b] ? st.wx[q] * st.wy[b] : C(0);
    if (st.nrow < 3) {
        C M00 = 0, M01 = 0, M02 = 0, M11 = 0, M12 = 0, M22 = 0, sw = 0;
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const C ww = w[b * 3 + q];
                sw += ww;
                M00 += ww;
                M01 += ww * st.rx[q];
                M02 += ww * st.ry[b];
                M11 += ww * st.rx[q] * st.rx[q];
                M12 += ww * st.rx[q] * st.ry[b];
                M22 += ww * st.ry[b] * st.ry[b];
            }
        const C c0 = M11 * M22 - M12 * M12;
        const C c1 = -(M01 * M22 - M12 * M02);
        const C c2 = M01 * M12 - M11 * M02;
        const C det = M00 * c0 + M01 * c1 + M02 * c2;
        if (det > C(1e-10)) {
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    w[b * 3 + q] = w[b * 3 + q] * (c0 + c1 * st.rx[q] + c2 * st.ry[b]) / det;
        } else if (sw > C(0)) {
#pragma unroll
            for (int q = 0; q < 9; ++q) w[q] = w[q] / sw;
        } else {
#pragma unroll
            for (int q = 0; q < 9; ++q) w[q] = C(0);
        }
    }
    Ux = Uy = C(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        if (!st.rowok[b]) continue;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            int i, j;
            stencil_node<C>(a, st, b, q, i, j);
            C pk, uk, vk;
            node_flow<S>(a, h, i, j, pk, uk, vk);
            Ux += w[b * 3 + q] * uk;
            Uy += w[b * 3 + q] * vk;
        }
    }
}

template <typename S>
__global__ void __launch_bounds__(kHydroThreads) k_hydro(const MarkerArgs a, const HydroArgs h) {
    using C = typename Storage<S>::C;
    using E = typename Ext<C>::E;
    const int m = h.dyn_mem[blockIdx.x];
    const int off = a.mem_off[m], n = a.mem_n[m];
    const int k = threadIdx.x;
    const bool valid = k < n;
    __shared__ C s_fx[kHydroThreads], s_fy[kHydroThreads], s_len[kHydroThreads];
    E x, y;
    if (valid) {
        E xr, yr;
        load_pos<C>(a, off + k, x, y);
        load_pos<C>(a, off + (k + 1 == n ? 0 : k + 1), xr, yr);
        const C ex = etoc(esub(xr, x)), ey = etoc(esub(yr, y));
        const C len = sqrt(ex * ex + ey * ey);
        const C nx = ey / len, ny = -ex / len;
        // probe c_l + 1.2 n_l
        const E qx = eaddc(emulc(eadd(x, xr), C(0.5)), C(1.2) * nx);
        const E qy = eaddc(emulc(eadd(y, yr), C(0.5)), C(1.2) * ny);
        C p, dux, duy, dvx, dvy;
        probe_fit<S, E>(a, h, qx, qy, p, dux, duy, dvx, dvy);
        const C nu = C(h.nu);
        const C txx = C(2) * nu * dux, tyy = C(2) * nu * dvy, txy = nu * (duy + dvx);
        s_fx[k] = (-p * nx + (txx * nx + txy * ny)) * len;
        s_fy[k] = (-p * ny + (txy * nx + tyy * ny)) * len;
        s_len[k] = len;
    }
    __syncthreads();
    if (!valid) return;
    const int kl = k == 0 ? n - 1 : k - 1;
    const int v = off + k;
    C* H = static_cast<C*>(a.Hf);
    C* D = static_cast<C*>(a.Dib);
    const C* V = static_cast<const C*>(a.V);
    H[2 * (size_t)v] = C(0.5) * (s_fx[kl] + s_fx[k]);
    H[2 * (size_t)v + 1] = C(0.5) * (s_fy[kl] + s_fy[k]);
    C Ux, Uy;
    vertex_flow<S, E>(a, h, x, y, Ux, Uy);
    const C dV = C(0.5) * (s_len[kl] + s_len[k]);
    D[2 * (size_t)v] = C(2) * dV * (V[2 * (size_t)v] - Ux);
    D[2 * (size_t)v + 1] = C(2) * dV * (V[2 * (size_t)v + 1] - Uy);
}

cudaError_t launch_hydro(lbib_precision prec, const MarkerArgs& a, const HydroArgs& h, cudaStream_t s) {
    if (h.ndyn == 0) return cudaSuccess;
    if (h.threads < 32 || h.threads > kHydroThreads || h.threads % 32) return cudaErrorInvalidValue;
    switch (prec) {
        case LBIB_F64: k_hydro<double><<<h.ndyn, h.threads, 0, s>>>(a, h); break;
        case LBIB_F32: k_hydro<float><<<h.ndyn, h.threads, 0, s>>>(a, h); break;
        case LBIB_F32_STORE_F16: k_hydro<__half><<<h.ndyn, h.threads, 0, s>>>(a, h); break;
        case LBIB_F32_STORE_BF16: k_hydro<__nv_bfloat16><<<h.ndyn, h.threads, 0, s>>>(a, h); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace lbib
