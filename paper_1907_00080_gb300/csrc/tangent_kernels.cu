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

#include "lb_node.cuh"
#include "tangent_ops.cuh"

namespace lbib {
namespace {

// enclosed area of each membrane (shoelace about vertex 0) with its tangent,
// and its bounding box (repulsion screen); one block of 256 threads each
__global__ void k_t_area(const TangentArgs t) {
    const int m = blockIdx.x;
    const int off = t.m.mem_off[m], n = t.m.mem_n[m];
    const Seed sd = tangent_seed();
    dual x0, y0;
    t_pos(t, off, sd, x0, y0);
    dual s;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        dual xa, ya, xb, yb;
        t_pos(t, off + k, sd, xa, ya);
        t_pos(t, t_ring(off, n, k + 1), sd, xb, yb);
        s += (xa - x0) * (yb - y0) - (xb - x0) * (ya - y0);
    }
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

__global__ void k_t_forces(const TangentArgs t) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= t.m.nv) return;
    dual fx, fy;
    t_vertex_force(t, v, t_mem_of(t, v), tangent_seed(), fx, fy);
    t.Fv[2 * v] = fx.v;
    t.Fv[2 * v + 1] = fy.v;
    t.Fd[2 * v] = fx.d;
    t.Fd[2 * v + 1] = fy.d;
}

// shape functions and their tangents, then the spreading of value and tangent
// of w_j F_v into the node fields
__global__ void k_t_weights_spread(const TangentArgs t) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= t.m.nv) return;
    dual w[9];
    bool in[9];
    int i0, j0;
    t_vertex_weights(t, v, tangent_seed(), w, in, i0, j0);
    const dual Fx(t.Fv[2 * v], t.Fd[2 * v]), Fy(t.Fv[2 * v + 1], t.Fd[2 * v + 1]);
    for (int k = 0; k < 9; ++k) {
        t.Wv[9 * v + k] = in[k] ? w[k].v : 0.0;
        t.Wd[9 * v + k] = in[k] ? w[k].d : 0.0;
        if (!in[k]) continue;
        const size_t node = t_node(t, i0, j0, k);
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
        dual f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const size_t src = t_pull_src(node, i, nx, ny, t.m.walls);
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
        if (t.m.walls && (j0 + k / 3 - 1 < 0 || j0 + k / 3 - 1 >= t.m.ny)) continue;
        const size_t node = t_node(t, i0, j0, k);
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

template <typename C>
__global__ void k_rest_fp64(const MarkerArgs m, double* l0, double* th0) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= m.nv) return;
    const Rest<C>* rest = static_cast<const Rest<C>*>(m.rest);
    l0[v] = (double)rest[v].l0;
    th0[v] = ::atan2(etod(rest[v].cross), etod(rest[v].dot));
}

}  // namespace

cudaError_t launch_rest_fp64(lbib_precision prec, const MarkerArgs& m, double* l0, double* th0, cudaStream_t s) {
    if (m.nv == 0) return cudaSuccess;
    const int g = (m.nv + 127) / 128;
    if (prec == LBIB_F64) k_rest_fp64<double><<<g, 128, 0, s>>>(m, l0, th0);
    else k_rest_fp64<float><<<g, 128, 0, s>>>(m, l0, th0);
    return cudaGetLastError();
}

cudaError_t launch_tangent_areas(const TangentArgs& t, cudaStream_t s) {
    if (t.m.nv > 0) k_t_area<<<t.m.nmem, 256, 0, s>>>(t);
    return cudaGetLastError();
}

cudaError_t launch_tangent_markers(const TangentArgs& t, cudaStream_t s) {
    // small blocks: these FP64 kernels have one thread per vertex, spread them over the SMs
    const int nvb = (t.m.nv + 31) / 32;
    if (t.m.nv > 0) {
        k_t_area<<<t.m.nmem, 256, 0, s>>>(t);
        k_t_forces<<<nvb, 32, 0, s>>>(t);
        k_t_weights_spread<<<nvb, 32, 0, s>>>(t);
    }
    return cudaGetLastError();
}

cudaError_t launch_tangent_step(const TangentArgs& t, cudaStream_t s) {
    cudaError_t e;
    const size_t N = (size_t)t.m.nx * t.m.ny;
    if ((e = cudaMemsetAsync(t.Gv, 0, 2 * N * sizeof(double), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(t.Gd, 0, 2 * N * sizeof(double), s)) != cudaSuccess) return e;
    if ((e = launch_tangent_markers(t, s)) != cudaSuccess) return e;
    const int g = (int)((N + 255) / 256 < 4096 ? (N + 255) / 256 : 4096);
    k_t_lb<<<g, 256, 0, s>>>(t);
    if (t.m.nv > 0) k_t_advance<<<(t.m.nv + 31) / 32, 32, 0, s>>>(t);
    return cudaGetLastError();
}

}  // namespace lbib
