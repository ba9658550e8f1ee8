// Reverse-mode (adjoint) step of the FP64 time step.
//
// Transposes, in reverse order, the parts of one step (Sec. 2.1 - 2.4):
//   BDF2 advance (Euler on step 0), interpolation      -> k_a_interp
//   moments + Guo-forced BGK collision and pull stream -> k_a_collide
//   spreading, membrane, bond and repulsion forces,
//   MLS/Roma shape functions                           -> k_a_forces
//   enclosed area                                      -> k_a_area
// (the areas and bounding boxes the force terms use are evaluated for a whole
// taped segment at once, k_tape_areas)
// The lattice part (every node, FP64) is written out by hand: the collision
// is (1 - omega) d_i plus a function of five scalars (drho, j, G), and its
// transpose costs about as much as the collision itself.  The per-vertex parts
// (a few thousand vertices) take local Jacobian columns from the dual-number
// functions of the tangent (one-hot seeds), so they share their arithmetic
// with the forward-mode derivative.
#include <algorithm>

#include "adjoint.cuh"
#include "lb_node.cuh"
#include "tangent_ops.cuh"

namespace lbib {
namespace {

// Transpose of collide_node<double> at one node.  d: pulled deviations, (Gx, Gy)
// total force; yb: adjoints of the nine outputs d*_i, (ubx, uby) adjoint of the
// velocity output.  Returns the adjoints of d and of G.  With eu_i = e_i.u and
// eG_i = e_i.G every output is
//   d*_i = (1 - omega) d_i + w_i [a + b eu_i + c eu_i^2 + g eG_i + h eu_i eG_i],
//   a = omega drho - 1.5 omega rho u.u - 3 pre u.G,  b = 3 omega rho,
//   c = 4.5 omega rho,  g = 3 pre,  h = 9 pre,
//   u = (j + G/2) / rho,  rho = 1 + drho,  drho = sum d_i,  j = sum e_i d_i.
__device__ __forceinline__ void collide_node_rev(const double (&d)[9], double Gx, double Gy, double om, double pre,
                                                 const double (&yb)[9], double ubx, double uby, double (&db)[9],
                                                 double& Gbx, double& Gby) {
    double drho = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        drho += d[i];
        jx += cx(i) * d[i];
        jy += cy(i) * d[i];
    }
    const double rho = 1.0 + drho, r = 1.0 / rho;
    const double px = jx + 0.5 * Gx, py = jy + 0.5 * Gy;
    const double ux = px * r, uy = py * r;
    const double uu = ux * ux + uy * uy;
    const double omr = om * rho;
    const double b = 3.0 * omr, c = 4.5 * omr, g = 3.0 * pre, h = 9.0 * pre;
    // adjoints of a, b, c and of u, G through eu_i, eG_i; opposite directions
    // (e_o = -e_i) share eu^2 and flip eu, eG, so each pair is summed once in its
    // even (y_i + y_o) and odd (y_i - y_o) parts
    double Sa = wgt<double>(0) * yb[0], Sb = 0.0, Sc = 0.0;
    double uxb = ubx, uyb = uby;
    Gbx = 0.0;
    Gby = 0.0;
    const double eus[4] = {ux, uy, ux + uy, uy - ux};
    const double eGs[4] = {Gx, Gy, Gx + Gy, Gy - Gx};
    constexpr int ip[4] = {1, 2, 5, 6};
    constexpr int io[4] = {3, 4, 7, 8};
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const double w = wgt<double>(ip[p]);
        const double eu = eus[p], eG = eGs[p];
        const double yE = w * (yb[ip[p]] + yb[io[p]]), yO = w * (yb[ip[p]] - yb[io[p]]);
        Sa += yE;
        Sb += eu * yO;
        Sc += eu * eu * yE;
        const double deu = b * yO + (2.0 * c * eu + h * eG) * yE;  // along e_ip
        const double deG = g * yO + h * eu * yE;
        uxb += cx(ip[p]) * deu;
        uyb += cy(ip[p]) * deu;
        Gbx += cx(ip[p]) * deG;
        Gby += cy(ip[p]) * deG;
    }
    // a, b, c -> drho, rho, u.u, u.G
    double drhob = om * Sa;
    double rhob = -1.5 * om * uu * Sa + 3.0 * om * Sb + 4.5 * om * Sc;
    const double uub = -1.5 * omr * Sa, uGb = -3.0 * pre * Sa;
    uxb += 2.0 * ux * uub + Gx * uGb;
    uyb += 2.0 * uy * uub + Gy * uGb;
    Gbx += ux * uGb;
    Gby += uy * uGb;
    // u = (j + G/2) r,  r = 1/rho,  rho = 1 + drho
    const double jxb = r * uxb, jyb = r * uyb;
    Gbx += 0.5 * r * uxb;
    Gby += 0.5 * r * uyb;
    rhob -= r * r * (px * uxb + py * uyb);
    drhob += rhob;
    const double omc = 1.0 - om;
#pragma unroll
    for (int i = 0; i < 9; ++i) db[i] = omc * yb[i] + drhob + cx(i) * jxb + cy(i) * jyb;
}

// velocity output of the collision at `node` (the field the markers interpolate)
__device__ __forceinline__ void node_velocity(const TangentArgs& t, const longlong2 g, size_t node, double& ux,
                                              double& uy) {
    const int nx = t.m.nx, ny = t.m.ny;
    double d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = t.f[t_pull_src(node, i, nx, ny, t.m.walls)];
    double out[9], rho;
    collide_node<double>(d, t.gx + from_fix<double>(g.x), t.gy + from_fix<double>(g.y), t.omega, 1.0 - 0.5 * t.omega,
                         out, rho, ux, uy);
}

// BDF2 coefficients of X^{n+1} = ca X^n + cb X^{n-1} + cu U^n (Euler on step 0)
struct Bdf2 {
    double ca, cb, cu;
};
__device__ __forceinline__ Bdf2 bdf2(long long step) {
    return step == 0 ? Bdf2{1.0, 0.0, 1.0} : Bdf2{4.0 / 3.0, -1.0 / 3.0, 2.0 / 3.0};
}

// Adjoint of the advance X^{n+1} = ca X^n + cb X^{n-1} + cu U^n and of the
// interpolation U_v = sum_k W_vk u(x_k): the velocity adjoint cu X_v^{n+1}-bar is
// scattered onto the nodes, and W_vk-bar = U_v-bar . u(x_k).  One thread per
// (vertex, stencil entry k = blockIdx.y); the k = 0 thread also starts X^n-bar.
__global__ void k_a_interp(const AdjointArgs a) {
    const TangentArgs& t = a.t;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (v == 0 && k == 0)
        for (int m = 0; m < t.m.nmem; ++m) a.Abar[m] = 0.0;
    if (v >= t.m.nv) return;
    const Bdf2 q = bdf2(t.step);
    const double Ubx = q.cu * a.XB[2 * v], Uby = q.cu * a.XB[2 * v + 1];
    if (k == 0) {
        // the BDF2 part: X^n-bar = X^n-slot-bar + ca X^{n+1}-bar, X^{n-1}-bar = cb X^{n+1}-bar
        for (int c = 0; c < 2; ++c) {
            const double xb = a.XB[2 * v + c];
            a.XB_out[2 * v + c] = a.XPB[2 * v + c] + q.ca * xb;
            a.XPB[2 * v + c] = q.cb * xb;
        }
    }
    const int i0 = t.st[2 * v], j0 = t.st[2 * v + 1];
    double wb = 0.0;
    if (!(t.m.walls && (j0 + k / 3 - 1 < 0 || j0 + k / 3 - 1 >= t.m.ny))) {
        const size_t node = t_node(t, i0, j0, k);
        const double w = t.Wv[9 * v + k];
        double ux, uy;
        node_velocity(t, a.gfix[node], node, ux, uy);
        atomicAdd(&a.ubar[2 * node], w * Ubx);
        atomicAdd(&a.ubar[2 * node + 1], w * Uby);
        wb = Ubx * ux + Uby * uy;
    }
    a.Wbar[9 * v + k] = wb;
}

// Adjoint of the collision and of the pull stream at every node.  The pull is a
// permutation of the stored values, so each adjoint entry has exactly one
// writer.  Also clears this step's u-bar for the next step.
__global__ void k_a_collide(const AdjointArgs a) {
    const TangentArgs& t = a.t;
    const int nx = t.m.nx, ny = t.m.ny;
    const size_t N = (size_t)nx * ny;
    const double om = t.omega, pre = 1.0 - 0.5 * t.omega;
    for (size_t node = blockIdx.x * (size_t)blockDim.x + threadIdx.x; node < N;
         node += (size_t)gridDim.x * blockDim.x) {
        size_t src[9];
        double d[9], yb[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            src[i] = t_pull_src(node, i, nx, ny, t.m.walls);
            d[i] = t.f[src[i]];
            yb[i] = a.fbar[(size_t)i * N + node];
        }
        const longlong2 gf = a.gfix[node];
        const double ubx = a.ubar[2 * node], uby = a.ubar[2 * node + 1];
        double db[9], Gbx, Gby;
        collide_node_rev(d, t.gx + from_fix<double>(gf.x), t.gy + from_fix<double>(gf.y), om, pre, yb, ubx, uby, db,
                         Gbx, Gby);
#pragma unroll
        for (int i = 0; i < 9; ++i) a.fbar_out[src[i]] = db[i];
        a.Gbar[2 * node] = Gbx;
        a.Gbar[2 * node + 1] = Gby;
        if (ubx != 0.0 || uby != 0.0) {
            a.ubar[2 * node] = 0.0;
            a.ubar[2 * node + 1] = 0.0;
        }
    }
}

// Tasks of k_a_forces (blockIdx.y): one dual evaluation each, of the force
// terms of vertex v that depend on one seed.  Position seeds X_{v+d}: the
// bending moment at v-1 depends on d in -2..0, the one at v on -1..1, the one
// at v+1 on 0..2; bonds, stretching and the area penalty on -1..1.
struct AdjTask {
    signed char kind, d, coord;  // kind: a SeedKind, or kRepTask / kWeightsTask
    unsigned char terms;
};
constexpr int kRepTask = 100, kWeightsTask = 101;
constexpr unsigned char kOther = kTermBond | kTermStretch | kTermArea;
constexpr int kNumTasks = 33;
__constant__ AdjTask c_tasks[kNumTasks] = {
    // x coordinate
    {kPos, -2, 0, kTermBendL},
    {kPos, -1, 0, kTermBendL}, {kPos, -1, 0, kTermBendV}, {kPos, -1, 0, kOther},
    {kPos, 0, 0, kTermBendL}, {kPos, 0, 0, kTermBendV}, {kPos, 0, 0, kTermBendR}, {kPos, 0, 0, kOther},
    {kPos, 1, 0, kTermBendV}, {kPos, 1, 0, kTermBendR}, {kPos, 1, 0, kOther},
    {kPos, 2, 0, kTermBendR},
    // y coordinate
    {kPos, -2, 1, kTermBendL},
    {kPos, -1, 1, kTermBendL}, {kPos, -1, 1, kTermBendV}, {kPos, -1, 1, kOther},
    {kPos, 0, 1, kTermBendL}, {kPos, 0, 1, kTermBendV}, {kPos, 0, 1, kTermBendR}, {kPos, 0, 1, kOther},
    {kPos, 1, 1, kTermBendV}, {kPos, 1, 1, kTermBendR}, {kPos, 1, 1, kOther},
    {kPos, 2, 1, kTermBendR},
    // parameters and the area
    {kArea, 0, 0, kTermArea}, {kKs, 0, 0, kTermStretch}, {kSigma, 0, 0, kTermBond},
    {kKb, 0, 0, kTermBendL}, {kKb, 0, 0, kTermBendV}, {kKb, 0, 0, kTermBendR},
    // repulsion pairs, shape functions against x_v and y_v
    {kRepTask, 0, 0, 0}, {kWeightsTask, 0, 0, 0}, {kWeightsTask, 0, 1, 0}};

// Adjoint of the total Lagrangian force on vertex v and of its shape functions.
// Bonds, stretching, bending and the area penalty depend on X_{v-2} .. X_{v+2},
// the membrane's area, k_s, k_b and sigma: one dual evaluation per (seed, term
// group) gives that part of the column dF_v/d(seed), and F_v-bar . column is
// added to the seed's adjoint.  The repulsion -sum_b c0 d_vb^{-5/2} n_v (Eq.
// repFor) is transposed pair by pair: through d_vb into X_v and X_b, and through
// the vertex normal n_v into X_{v-1}, X_v, X_{v+1}.  The shape functions of v
// depend on X_v alone (two seeds).  Each (vertex, task) is one thread: the FP64
// chains are long, and one thread per vertex would leave most SMs idle.
__global__ void k_a_forces(const AdjointArgs a) {
    const TangentArgs& t = a.t;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= t.m.nv) return;
    const AdjTask q = c_tasks[blockIdx.y];
    // the spreading G(x_k) += W_vk F_v transposed: F_v-bar = sum_k W_vk G-bar(x_k),
    // and the shape functions' share G-bar(x_k) . F_v
    const int i0 = t.st[2 * v], j0 = t.st[2 * v + 1];
    const double Fx = t.Fv[2 * v], Fy = t.Fv[2 * v + 1];
    double Fbx = 0.0, Fby = 0.0, gF[9];
    for (int k = 0; k < 9; ++k) {
        gF[k] = 0.0;
        if (t.m.walls && (j0 + k / 3 - 1 < 0 || j0 + k / 3 - 1 >= t.m.ny)) continue;
        const size_t node = t_node(t, i0, j0, k);
        const double w = t.Wv[9 * v + k];
        const double gbx = a.Gbar[2 * node], gby = a.Gbar[2 * node + 1];
        Fbx += w * gbx;
        Fby += w * gby;
        gF[k] = gbx * Fx + gby * Fy;
    }
    double* XB = a.XB_out;
    if (q.kind == kWeightsTask) {
        dual w[9];
        bool in[9];
        int si, sj;
        t_vertex_weights(t, v, Seed{kPos, v, q.coord, -1}, w, in, si, sj);
        double acc = 0.0;
        for (int k = 0; k < 9; ++k)
            if (in[k]) acc += (a.Wbar[9 * v + k] + gF[k]) * w[k].d;
        atomicAdd(&XB[2 * v + q.coord], acc);
        return;
    }
    if (Fbx == 0.0 && Fby == 0.0) return;
    const int m = t_mem_of(t, v);
    const int off = t.m.mem_off[m], n = t.m.mem_n[m], k = v - off;
    if (q.kind != kRepTask) {
        if (q.kind == kSigma && t.m.nlig == 0) return;
        const int u = q.kind == kPos ? t_ring(off, n, k + q.d) : -1;
        dual fx, fy;
        t_vertex_force(t, v, m, Seed{q.kind, u, q.coord, m}, fx, fy, q.terms);
        const double g = Fbx * fx.d + Fby * fy.d;
        double* dst = q.kind == kPos ? &XB[2 * u + q.coord]
                      : q.kind == kArea ? &a.Abar[m]
                      : q.kind == kKs   ? &a.ks_bar[m]
                      : q.kind == kKb   ? &a.kb_bar[m]
                                        : a.sigma_bar;
        atomicAdd(dst, g);
        return;
    }
    // the repulsion pairs of v
    if (t.m.nmem < 2) return;
    const double* X = static_cast<const double*>(t.m.X);
    const double xv = X[2 * v], yv = X[2 * v + 1];
    bool have_g = false;
    VGeo g;
    double nbx = 0.0, nby = 0.0, xvb = 0.0, yvb = 0.0;
    for (int mb = 0; mb < t.m.nmem; ++mb) {
        if (mb == m || !t_near_box(t, mb, xv, yv)) continue;
        if (!have_g) {
            g = t_vgeo(t, off, n, k, tangent_seed());
            have_g = true;
        }
        const double gnx = g.nx.v, gny = g.ny.v;
        const int o2 = t.m.mem_off[mb], n2 = t.m.mem_n[mb];
        for (int b = o2; b < o2 + n2; ++b) {
            if (!t_rep_candidate(t, xv, yv, b)) continue;
            const double dxv = t_wrap_x(t, dual(xv - X[2 * b])).v;
            const double dyv = t_wrap_y(t, dual(yv - X[2 * b + 1])).v;
            // magnitude and its two partials with respect to (dx, dy)
            const dual ddx = sqrt(dual(dxv, 1.0) * dual(dxv, 1.0) + dual(dyv) * dual(dyv));
            if (ddx.v >= t.m.d_rep) continue;
            const dual ddy = sqrt(dual(dxv) * dual(dxv) + dual(dyv, 1.0) * dual(dyv, 1.0));
            const dual mx = kRepC0 * pow_m52(ddx), my = kRepC0 * pow_m52(ddy);
            // F_v -= mag n_v
            nbx -= mx.v * Fbx;
            nby -= mx.v * Fby;
            const double magb = -(Fbx * gnx + Fby * gny);
            const double gx = magb * mx.d, gy = magb * my.d;
            xvb += gx;
            yvb += gy;
            atomicAdd(&XB[2 * b], -gx);
            atomicAdd(&XB[2 * b + 1], -gy);
        }
    }
    if (!have_g) return;
    atomicAdd(&XB[2 * v], xvb);
    atomicAdd(&XB[2 * v + 1], yvb);
    if (nbx == 0.0 && nby == 0.0) return;
    for (int dk = -1; dk <= 1; ++dk) {
        const int u = t_ring(off, n, k + dk);
        for (int c = 0; c < 2; ++c) {
            const VGeo gs = t_vgeo(t, off, n, k, Seed{kPos, u, c, -1});
            atomicAdd(&XB[2 * u + c], nbx * gs.nx.d + nby * gs.ny.d);
        }
    }
}

// Adjoint of the enclosed area (shoelace): dA/dx_v = (y_{v+1} - y_{v-1}) / 2,
// dA/dy_v = (x_{v-1} - x_{v+1}) / 2.
__global__ void k_a_area(const AdjointArgs a) {
    const TangentArgs& t = a.t;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= t.m.nv) return;
    const int m = t_mem_of(t, v);
    const double Ab = a.Abar[m];
    if (Ab == 0.0) return;
    const int off = t.m.mem_off[m], n = t.m.mem_n[m], k = v - off;
    const double* X = static_cast<const double*>(t.m.X);
    const int L = t_ring(off, n, k - 1), R = t_ring(off, n, k + 1);
    atomicAdd(&a.XB_out[2 * v], 0.5 * Ab * (X[2 * R + 1] - X[2 * L + 1]));
    atomicAdd(&a.XB_out[2 * v + 1], 0.5 * Ab * (X[2 * L] - X[2 * R]));
}

// areas (shoelace about vertex 0) and bounding boxes of the taped positions of
// step k = blockIdx.y, membrane m = blockIdx.x
__global__ void k_tape_areas(const MarkerArgs mg, const double* __restrict__ tape_X, double* A, double* box) {
    const int m = blockIdx.x, k = blockIdx.y;
    const int off = mg.mem_off[m], n = mg.mem_n[m];
    const double* X = tape_X + (size_t)k * 2 * (size_t)(mg.nv > 0 ? mg.nv : 1);
    const double x0 = X[2 * off], y0 = X[2 * off + 1];
    double s = 0.0, bx0 = 1e300, bx1 = -1e300, by0 = 1e300, by1 = -1e300;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int a = off + j, b = off + (j + 1) % n;
        s += (X[2 * a] - x0) * (X[2 * b + 1] - y0) - (X[2 * b] - x0) * (X[2 * a + 1] - y0);
        bx0 = fmin(bx0, X[2 * a]);
        bx1 = fmax(bx1, X[2 * a]);
        by0 = fmin(by0, X[2 * a + 1]);
        by1 = fmax(by1, X[2 * a + 1]);
    }
    __shared__ double r[5][256];
    r[0][threadIdx.x] = s;
    r[1][threadIdx.x] = bx0;
    r[2][threadIdx.x] = bx1;
    r[3][threadIdx.x] = by0;
    r[4][threadIdx.x] = by1;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            r[0][threadIdx.x] += r[0][threadIdx.x + o];
            r[1][threadIdx.x] = fmin(r[1][threadIdx.x], r[1][threadIdx.x + o]);
            r[2][threadIdx.x] = fmax(r[2][threadIdx.x], r[2][threadIdx.x + o]);
            r[3][threadIdx.x] = fmin(r[3][threadIdx.x], r[3][threadIdx.x + o]);
            r[4][threadIdx.x] = fmax(r[4][threadIdx.x], r[4][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const size_t q = (size_t)k * mg.nmem + m;
        A[q] = 0.5 * r[0][0];
        for (int c = 0; c < 4; ++c) box[4 * q + c] = r[1 + c][0];
    }
}

// read-back layout <-> stored deviations (a permutation; the constant w_i of the
// read-back has no adjoint)
__global__ void k_a_perm(const double* __restrict__ in, double* __restrict__ out, int nx, int ny, int walls,
                         int to_storage) {
    const size_t N = (size_t)nx * ny;
    for (size_t node = blockIdx.x * (size_t)blockDim.x + threadIdx.x; node < N;
         node += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const size_t src = t_pull_src(node, i, nx, ny, walls);
            if (to_storage) out[src] = in[(size_t)i * N + node];
            else out[(size_t)i * N + node] = in[src];
        }
    }
}

template <typename S>
__global__ void k_widen_storage(const S* __restrict__ src, double* __restrict__ dst, size_t n, float inv) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        dst[k] = (double)Storage<S>::load(src[k], inv);
}

template <typename C>
__global__ void k_widen_compute(const C* __restrict__ src, double* __restrict__ dst, size_t n) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        dst[k] = (double)src[k];
}

__global__ void k_copy_words(const CopyList l) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    for (int c = 0; c < l.n; ++c) {
        const uint32_t* __restrict__ src = static_cast<const uint32_t*>(l.src[c]);
        uint32_t* __restrict__ dst = static_cast<uint32_t*>(l.dst[c]);
        size_t head = 0;
        if ((((uintptr_t)src | (uintptr_t)dst) & 15) == 0) {
            // 16-byte vectors where both ends are aligned, then the remaining words
            head = l.words[c] & ~(size_t)3;
            const uint4* __restrict__ s4 = reinterpret_cast<const uint4*>(src);
            uint4* __restrict__ d4 = reinterpret_cast<uint4*>(dst);
            for (size_t k = t0; k < head / 4; k += stride) d4[k] = s4[k];
        }
        for (size_t k = head + t0; k < l.words[c]; k += stride) dst[k] = src[k];
    }
}

int node_grid(size_t N) { return (int)((N + 255) / 256 < 4096 ? (N + 255) / 256 : 4096); }

}  // namespace

cudaError_t launch_adjoint_step(const AdjointArgs& a, cudaStream_t s) {
    const TangentArgs& t = a.t;
    const size_t N = (size_t)t.m.nx * t.m.ny;
    const int nvb = (t.m.nv + 31) / 32;
    if (t.m.nv > 0) k_a_interp<<<dim3(nvb, 9), 32, 0, s>>>(a);
    // FP64-bound: 128-thread blocks, up to 16 per SM
    k_a_collide<<<(int)std::min<size_t>((N + 127) / 128, 152 * 16), 128, 0, s>>>(a);
    if (t.m.nv > 0) {
        k_a_forces<<<dim3(nvb, kNumTasks), 32, 0, s>>>(a);
        k_a_area<<<nvb, 32, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_copy_words(const CopyList& l, cudaStream_t s) {
    size_t most = 0;
    for (int c = 0; c < l.n; ++c) most = l.words[c] > most ? l.words[c] : most;
    if (most == 0) return cudaSuccess;
    k_copy_words<<<std::min<size_t>((most / 4 + 255) / 256 + 1, 152 * 8), 256, 0, s>>>(l);
    return cudaGetLastError();
}

cudaError_t launch_widen_storage(lbib_precision prec, const void* src, double* dst, size_t n, float inv_scale,
                                 cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int g = node_grid(n);
    switch (prec) {
        case LBIB_F64: k_widen_storage<double><<<g, 256, 0, s>>>(static_cast<const double*>(src), dst, n, inv_scale); break;
        case LBIB_F32: k_widen_storage<float><<<g, 256, 0, s>>>(static_cast<const float*>(src), dst, n, inv_scale); break;
        case LBIB_F32_STORE_F16:
            k_widen_storage<__half><<<g, 256, 0, s>>>(static_cast<const __half*>(src), dst, n, inv_scale);
            break;
        default:
            k_widen_storage<__nv_bfloat16><<<g, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(src), dst, n,
                                                             inv_scale);
    }
    return cudaGetLastError();
}

cudaError_t launch_widen_compute(lbib_precision prec, const void* src, double* dst, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int g = node_grid(n);
    if (prec == LBIB_F64) k_widen_compute<double><<<g, 256, 0, s>>>(static_cast<const double*>(src), dst, n);
    else k_widen_compute<float><<<g, 256, 0, s>>>(static_cast<const float*>(src), dst, n);
    return cudaGetLastError();
}

cudaError_t launch_tape_areas(const MarkerArgs& m, const double* tape_X, int len, double* A, double* box,
                              cudaStream_t s) {
    if (m.nv == 0 || len == 0) return cudaSuccess;
    k_tape_areas<<<dim3(m.nmem, len), 256, 0, s>>>(m, tape_X, A, box);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_perm(const double* in, double* out, int nx, int ny, int walls, int to_storage,
                                cudaStream_t s) {
    k_a_perm<<<node_grid((size_t)nx * ny), 256, 0, s>>>(in, out, nx, ny, walls, to_storage);
    return cudaGetLastError();
}

}  // namespace lbib
