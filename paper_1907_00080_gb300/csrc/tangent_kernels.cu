// Tangent-linear (forward-mode) derivative of one FP64 time step.
//
// For a direction (dk_s, dk_b per membrane, dsigma, and the tangent of the
// initial marker positions) these kernels carry, next to the state of step n,
// its directional derivative: dX^n, dX^{n-1} and the derivative of the stored
// post-collision deviations.  Every quantity of the step is recomputed from
// the FP64 state of the primal context in dual numbers (value + derivative),
// in the step's order:
//   forces at X^n (stretch Eq. strainFor, bend Eq. bendFor, area Eq. areaFor,
//   repulsion Eq. repFor, bond springs Eq. adhFor with the bonds of step n held
//   fixed) -> MLS / Roma shape functions -> spreading -> pull-stream + Guo BGK
//   (the same per-node arithmetic as the fused kernel, on duals) ->
//   interpolation -> BDF2 (Euler on the first step).
// Bond formation and rupture are discrete events: the tangent takes the bond
// set of every step as given (the primal run's), i.e. the derivative of the
// path with that topology.  Rigid-projected membranes are not supported.
// One thread per vertex or node: these kernels favour plain structure over
// speed (a tangent costs a few primal steps).
#include <climits>

#include "dual.cuh"
#include "ext_real.cuh"
#include "lb_node.cuh"
#include "tangent.cuh"

namespace lbib {
namespace {

constexpr double kPref = 1.0 / 3.0;  // p_ref = rho_0 c_s^2 (Eq. areaFor)

__device__ __forceinline__ int mem_of(const TangentArgs& t, int v) {
    int lo = 0, hi = t.m.nmem - 1;
    while (lo < hi) {  // last membrane with mem_off <= v
        const int mid = (lo + hi + 1) >> 1;
        if (t.m.mem_off[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void pos(const TangentArgs& t, int v, dual& x, dual& y) {
    const double* X = static_cast<const double*>(t.m.X);
    x = dual(X[2 * v], t.dX[2 * v]);
    y = dual(X[2 * v + 1], t.dX[2 * v + 1]);
}

// vertex k of membrane (off, n), local index wrapped
__device__ __forceinline__ int ring(int off, int n, int k) { return off + ((k % n) + n) % n; }

__device__ __forceinline__ dual wrap_x(const TangentArgs& t, dual dx) {
    dx.v -= t.m.nx * floor(dx.v * t.m.inv_nx + 0.5);
    return dx;
}
__device__ __forceinline__ dual wrap_y(const TangentArgs& t, dual dy) {
    if (!t.m.walls) dy.v -= t.m.ny * floor(dy.v * t.m.inv_ny + 0.5);
    return dy;
}

// turning angle, outward vertex normal and adjacent edge lengths at vertex k
struct VGeo {
    dual th, nx, ny, lL, lR;
};
__device__ VGeo vgeo(const TangentArgs& t, int off, int n, int k) {
    dual xL, yL, xv, yv, xR, yR;
    pos(t, ring(off, n, k - 1), xL, yL);
    pos(t, ring(off, n, k), xv, yv);
    pos(t, ring(off, n, k + 1), xR, yR);
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

// enclosed area of each membrane (shoelace about vertex 0), one block each
__global__ void k_t_area(const TangentArgs t) {
    const int m = blockIdx.x;
    const int off = t.m.mem_off[m], n = t.m.mem_n[m];
    dual x0, y0;
    pos(t, off, x0, y0);
    dual s;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        dual xa, ya, xb, yb;
        pos(t, off + k, xa, ya);
        pos(t, ring(off, n, k + 1), xb, yb);
        s += (xa - x0) * (yb - y0) - (xb - x0) * (ya - y0);
    }
    // bounding box of the membrane (unwrapped x), for the repulsion screen
    double bx0 = 1e300, bx1 = -1e300, by0 = 1e300, by1 = -1e300;
    const double* X = static_cast<const double*>(t.m.X);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double x = X[2 * (off + k)], y = X[2 * (off + k) + 1];
        bx0 = fmin(bx0, x);
        bx1 = fmax(bx1, x);
        by0 = fmin(by0, y);
        by1 = fmax(by1, y);
    }
    __shared__ double rv[256], rd[256], rb[4][256];
    rv[threadIdx.x] = s.v;
    rd[threadIdx.x] = s.d;
    rb[0][threadIdx.x] = bx0;
    rb[1][threadIdx.x] = bx1;
    rb[2][threadIdx.x] = by0;
    rb[3][threadIdx.x] = by1;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            rv[threadIdx.x] += rv[threadIdx.x + o];
            rd[threadIdx.x] += rd[threadIdx.x + o];
            rb[0][threadIdx.x] = fmin(rb[0][threadIdx.x], rb[0][threadIdx.x + o]);
            rb[1][threadIdx.x] = fmax(rb[1][threadIdx.x], rb[1][threadIdx.x + o]);
            rb[2][threadIdx.x] = fmin(rb[2][threadIdx.x], rb[2][threadIdx.x + o]);
            rb[3][threadIdx.x] = fmax(rb[3][threadIdx.x], rb[3][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        t.A[m] = 0.5 * rv[0];
        t.Ad[m] = 0.5 * rd[0];
        for (int q = 0; q < 4; ++q) t.box[4 * m + q] = rb[q][0];
    }
}

// bond spring of the ligand on element e (if bonded), half on each end vertex
__device__ void bond_half(const TangentArgs& t, int e, dual& fx, dual& fy) {
    const int l = t.m.elem_lig[e];
    if (l < 0) return;
    const int r = t.m.bond_of_lig[l];
    if (r < 0) return;
    dual xa, ya, xb, yb;
    pos(t, t.m.lig_a[l], xa, ya);
    pos(t, t.m.lig_b[l], xb, yb);
    const dual cx = 0.5 * (xa + xb), cy = 0.5 * (ya + yb);
    const dual dx = wrap_x(t, dual(t.m.rec_xy[2 * r]) - cx);
    const dual dy = wrap_y(t, dual(t.m.rec_xy[2 * r + 1]) - cy);
    const dual d = sqrt(dx * dx + dy * dy);
    const dual c = dual(t.m.sigma, t.dsigma) * (d - dual(t.m.y_eq)) / d;
    fx += 0.5 * c * dx;
    fy += 0.5 * c * dy;
}

__global__ void k_t_forces(const TangentArgs t) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= t.m.nv) return;
    const int m = mem_of(t, v);
    const int off = t.m.mem_off[m], n = t.m.mem_n[m], k = v - off;
    const int L = ring(off, n, k - 1), R = ring(off, n, k + 1);
    const Rest<double>* rest = static_cast<const Rest<double>*>(t.m.rest);
    dual fx, fy;
    dual xL, yL, xv, yv, xR, yR;
    pos(t, L, xL, yL);
    pos(t, v, xv, yv);
    pos(t, R, xR, yR);
    // Eq. adhFor on the two elements sharing v
    if (t.m.nlig > 0) {
        bond_half(t, L, fx, fy);
        bond_half(t, v, fx, fy);
    }
    // Eq. repFor against every vertex of the other membranes closer than d_rep
    if (t.m.nmem > 1) {
        const double c0 = 1e-4 / (8.0 * 1.4142135623730951);
        const double reach = t.m.d_rep + 1e-9;
        bool have_g = false;
        VGeo g;
        for (int mb = 0; mb < t.m.nmem; ++mb) {
            if (mb == m) continue;
            // skip membranes whose box (periodic in x) is out of reach of v
            const double* bb = t.box + 4 * mb;
            const double hx = 0.5 * (bb[1] - bb[0]);
            double cxm = xv.v - 0.5 * (bb[0] + bb[1]);
            cxm -= t.m.nx * floor(cxm * t.m.inv_nx + 0.5);
            double cym = yv.v - 0.5 * (bb[2] + bb[3]);
            if (!t.m.walls) cym -= t.m.ny * floor(cym * t.m.inv_ny + 0.5);
            if (::fabs(cxm) > hx + reach || ::fabs(cym) > 0.5 * (bb[3] - bb[2]) + reach) continue;
            if (!have_g) {
                g = vgeo(t, off, n, k);
                have_g = true;
            }
            const int o2 = t.m.mem_off[mb], n2 = t.m.mem_n[mb];
            for (int b = o2; b < o2 + n2; ++b) {
                dual xb, yb;
                pos(t, b, xb, yb);
                const dual dx = wrap_x(t, xv - xb), dy = wrap_y(t, yv - yb);
                const dual d = sqrt(dx * dx + dy * dy);
                if (d.v < t.m.d_rep) {
                    const dual mag = c0 * pow_m52(d);
                    fx -= mag * g.nx;
                    fy -= mag * g.ny;
                }
            }
        }
    }
    // Eq. strainFor on (v, R) and (L, v)
    const dual ks(t.m.mem_ks[m], t.dks[m]);
    {
        const dual rx = xv - xR, ry = yv - yR;
        const dual l = sqrt(rx * rx + ry * ry);
        const dual c = -ks * (l - dual(rest[v].l0)) / l;
        fx += c * rx;
        fy += c * ry;
        const dual qx = xL - xv, qy = yL - yv;
        const dual l2 = sqrt(qx * qx + qy * qy);
        const dual c2 = -ks * (l2 - dual(rest[L].l0)) / l2;
        fx -= c2 * qx;
        fy -= c2 * qy;
    }
    // Eq. bendFor: own term and the shares of the two neighbours
    const dual kb(t.m.mem_kb[m], t.dkb[m]);
    {
        const VGeo gL = vgeo(t, off, n, k - 1), gv = vgeo(t, off, n, k), gR = vgeo(t, off, n, k + 1);
        const dual mL = kb * (gL.th - dual(atan2(rest[L].cross, rest[L].dot)));
        const dual mv = kb * (gv.th - dual(atan2(rest[v].cross, rest[v].dot)));
        const dual mR = kb * (gR.th - dual(atan2(rest[R].cross, rest[R].dot)));
        const dual sR_L = gL.lR / (gL.lL + gL.lR), sL_R = gR.lL / (gR.lL + gR.lR);
        fx += mL * sR_L * gL.nx - mv * gv.nx + mR * sL_R * gR.nx;
        fy += mL * sR_L * gL.ny - mv * gv.ny + mR * sL_R * gR.ny;
    }
    // Eq. areaFor, half of each adjacent element
    {
        const dual A(t.A[m], t.Ad[m]);
        const dual c = -t.m.mem_ka[m] * (dual(1.0) - A / dual(t.m.mem_A0[m])) * kPref;
        fx += 0.5 * c * (-(yR - yv)) + 0.5 * c * (-(yv - yL));
        fy += 0.5 * c * (xR - xv) + 0.5 * c * (xv - xL);
    }
    t.Fv[2 * v] = fx.v;
    t.Fv[2 * v + 1] = fy.v;
    t.Fd[2 * v] = fx.d;
    t.Fd[2 * v + 1] = fy.d;
}

__device__ dual roma_d(dual r) {
    const dual a = fabs(r);
    if (a.v <= 0.5) return (dual(1.0) + sqrt(dual(1.0) - 3.0 * a * a)) / dual(3.0);
    if (a.v <= 1.5) {
        const dual b = dual(1.0) - a;
        return (dual(5.0) - 3.0 * a - sqrt(dual(1.0) - 3.0 * b * b)) / dual(6.0);
    }
    return dual(0.0);
}

// shape functions (MLS with Roma weights, Sec. 2.2 / 2.3) and their tangents,
// then the spreading of value and tangent of w_j F_v into the node fields
__global__ void k_t_weights_spread(const TangentArgs t) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= t.m.nv) return;
    dual px, py;
    pos(t, v, px, py);
    const int i0 = (int)floor(px.v + 0.5), j0 = (int)floor(py.v + 0.5);
    dual Wr[9], rx[9], ry[9];
    bool in[9];
    int nvalid = 0;
    for (int b = -1; b <= 1; ++b)
        for (int a = -1; a <= 1; ++a) {
            const int k = (b + 1) * 3 + (a + 1);
            rx[k] = dual((double)(i0 + a)) - px;
            ry[k] = dual((double)(j0 + b)) - py;
            const int j = j0 + b;
            in[k] = t.m.walls ? (j >= 0 && j < t.m.ny) : true;
            Wr[k] = in[k] ? roma_d(rx[k]) * roma_d(ry[k]) : dual(0.0);
            nvalid += in[k];
        }
    dual w[9];
    if (nvalid == 9) {
        for (int k = 0; k < 9; ++k) w[k] = Wr[k];
    } else {
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
    const dual Fx(t.Fv[2 * v], t.Fd[2 * v]), Fy(t.Fv[2 * v + 1], t.Fd[2 * v + 1]);
    for (int k = 0; k < 9; ++k) {
        t.Wv[9 * v + k] = in[k] ? w[k].v : 0.0;
        t.Wd[9 * v + k] = in[k] ? w[k].d : 0.0;
        if (!in[k]) continue;
        const int a = k % 3 - 1, b = k / 3 - 1;
        int i = (i0 + a) % t.m.nx;
        i = i < 0 ? i + t.m.nx : i;
        int j = j0 + b;
        if (!t.m.walls) j = ((j % t.m.ny) + t.m.ny) % t.m.ny;
        const size_t node = (size_t)j * t.m.nx + i;
        const dual gx = w[k] * Fx, gy = w[k] * Fy;
        atomicAdd(&t.Gv[2 * node], gx.v);
        atomicAdd(&t.Gv[2 * node + 1], gy.v);
        atomicAdd(&t.Gd[2 * node], gx.d);
        atomicAdd(&t.Gd[2 * node + 1], gy.d);
    }
    t.st[2 * v] = i0;
    t.st[2 * v + 1] = j0;
}

// pull-stream + Guo BGK of value and tangent at every node
__global__ void k_t_lb(const TangentArgs t) {
    const int nx = t.m.nx, ny = t.m.ny;
    const size_t N = (size_t)nx * ny;
    for (size_t node = blockIdx.x * (size_t)blockDim.x + threadIdx.x; node < N;
         node += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(node / nx), x = (int)(node % nx);
        dual f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            int sy = y - cy(i), sx = x - cx(i);
            sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
            size_t src;
            if (t.m.walls && (sy < 0 || sy >= ny)) {
                src = (size_t)opp(i) * N + node;
            } else {
                sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
                src = (size_t)i * N + (size_t)sy * nx + sx;
            }
            f[i] = dual(t.f[src], t.fd_src[src]);
        }
        const dual Gx(t.gx + t.Gv[2 * node], t.Gd[2 * node]);
        const dual Gy(t.gy + t.Gv[2 * node + 1], t.Gd[2 * node + 1]);
        dual out[9], rho, ux, uy;
        collide_node<dual>(f, Gx, Gy, dual(t.omega), dual(1.0 - 0.5 * t.omega), out, rho, ux, uy);
#pragma unroll
        for (int i = 0; i < 9; ++i) t.fd_dst[(size_t)i * N + node] = out[i].d;
        t.u[2 * node] = ux.v;
        t.u[2 * node + 1] = uy.v;
        t.ud[2 * node] = ux.d;
        t.ud[2 * node + 1] = uy.d;
    }
}

// interpolation and BDF2 (Euler on the first step) of the tangent
__global__ void k_t_advance(const TangentArgs t) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= t.m.nv) return;
    const int i0 = t.st[2 * v], j0 = t.st[2 * v + 1];
    dual Ux, Uy;
    for (int k = 0; k < 9; ++k) {
        const double wv = t.Wv[9 * v + k], wd = t.Wd[9 * v + k];
        if (wv == 0.0 && wd == 0.0) continue;
        const int a = k % 3 - 1, b = k / 3 - 1;
        int i = (i0 + a) % t.m.nx;
        i = i < 0 ? i + t.m.nx : i;
        int j = j0 + b;
        if (!t.m.walls) j = ((j % t.m.ny) + t.m.ny) % t.m.ny;
        if (j < 0 || j >= t.m.ny) continue;
        const size_t node = (size_t)j * t.m.nx + i;
        const dual w(wv, wd);
        Ux += w * dual(t.u[2 * node], t.ud[2 * node]);
        Uy += w * dual(t.u[2 * node + 1], t.ud[2 * node + 1]);
    }
    for (int c = 0; c < 2; ++c) {
        const double dU = c == 0 ? Ux.d : Uy.d;
        const double dx = t.dX[2 * v + c], dxp = t.dXp[2 * v + c];
        t.dXn[2 * v + c] = t.step == 0 ? dx + dU : (2.0 / 3.0) * (2.0 * dx - 0.5 * dxp + dU);
    }
}

}  // namespace

cudaError_t launch_tangent_step(const TangentArgs& t, cudaStream_t s) {
    cudaError_t e;
    const size_t N = (size_t)t.m.nx * t.m.ny;
    if ((e = cudaMemsetAsync(t.Gv, 0, 2 * N * sizeof(double), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(t.Gd, 0, 2 * N * sizeof(double), s)) != cudaSuccess) return e;
    // small blocks: these FP64 kernels have one thread per vertex, spread them over the SMs
    const int nvb = (t.m.nv + 31) / 32;
    if (t.m.nv > 0) {
        k_t_area<<<t.m.nmem, 256, 0, s>>>(t);
        k_t_forces<<<nvb, 32, 0, s>>>(t);
        k_t_weights_spread<<<nvb, 32, 0, s>>>(t);
    }
    const int g = (int)((N + 255) / 256 < 4096 ? (N + 255) / 256 : 4096);
    k_t_lb<<<g, 256, 0, s>>>(t);
    if (t.m.nv > 0) k_t_advance<<<nvb, 32, 0, s>>>(t);
    return cudaGetLastError();
}

}  // namespace lbib
