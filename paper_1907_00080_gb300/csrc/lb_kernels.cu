// Lattice-Boltzmann kernels: the fused pull-stream + bounce-back + moments +
// Guo-forced BGK collision with the spread IB force read per flagged tile (the
// hot kernel), and the small helpers that convert between the stored
// post-collision deviations and user-facing populations.
//
// Paper: Coclite, arXiv 1907.00080, Sec. 2.1 (Eqs. BGK, feq, GaussHermite),
// Sec. 2.2 (Eqs. forcedBGK, ForcingTerm; momentum with the half-force),
// Sec. 3 (periodic x, no-slip walls in y).
#include "lb_node.cuh"

namespace lbib {

constexpr unsigned FULL = 0xffffffffu;

template <typename S, int VEC>
struct alignas(sizeof(S) * VEC) Pack {
    S v[VEC];
};

template <typename S, int VEC>
__device__ __forceinline__ void load_pack(const S* __restrict__ row, int x0, bool ok, float inv,
                                          typename Storage<S>::C (&out)[VEC]) {
    using C = typename Storage<S>::C;
    if (ok) {
        const Pack<S, VEC> p = *reinterpret_cast<const Pack<S, VEC>*>(row + x0);
#pragma unroll
        for (int k = 0; k < VEC; ++k) out[k] = Storage<S>::load(p.v[k], inv);
    } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) out[k] = C(0);
    }
}

// Fused step over one tile of (32*VEC) x blockDim.y nodes.  One warp covers
// 32*VEC consecutive x of one row, so every row predicate is warp-uniform; the
// x-shifted pulls load aligned vectors and take the single off-vector element
// from the neighbouring lane (or, at the warp edge, with one scalar load).
// IB: 0 no markers; 1 the spread force read in the tiles the spreading
// flagged; 2 the same, with every node's force read up front (see below)
// The tile (bx, by) of the lattice `a`: the body of the single-lattice kernel
// (bx, by = blockIdx) and of the batched kernel (one block per (lattice, tile)).
template <typename S, int VEC, bool WALLS, int IB>
__device__ __forceinline__ void lb_tile(const LbArgs& a, int bx, int by) {
    constexpr bool HAS_IB = IB > 0;
    using C = typename Storage<S>::C;
    const int lane = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const int y = by * blockDim.y + threadIdx.y;
    const int x0 = (bx * 32 + lane) * VEC;
    const bool ok = (y < ny) && (x0 < nx);
    const size_t N = (size_t)nx * ny;
    const S* __restrict__ src = static_cast<const S*>(a.src);
    const float inv = a.inv_scale;

    // ---- on lattices that stay in L2, the spread force of every node is read
    // up front (the field is zero outside the tiles this step's spreading
    // touched), so that its latency overlaps the population loads instead of
    // following the tile flag
    longlong2 gpre[VEC];
    const bool pre_g = IB == 2 && a.g_prefetch && ok;
    if (pre_g) {
#pragma unroll
        for (int k = 0; k < VEC; ++k) gpre[k] = a.gsum[(size_t)y * nx + x0 + k];
    }
    // this thread's force tile and its flags, read before the populations so
    // that the flag (an L2 hit) is back while the population loads are still
    // in flight and the force load that depends on it overlaps them: during a
    // step the row-tile form flags segments of 32 nodes of one row (tile_w =
    // 32, tile_h = 1), so the threads that share a flag are lanes of one warp;
    // in the fields-only read-back the tiles may be those of the persistent form
    int t = 0, flag = 0, flag_o = 0;
    if (HAS_IB) {
        t = (min(y, ny - 1) / a.tile_h) * a.tiles_x + min(x0, nx - 1) / a.tile_w;
        flag = a.flags[t];
        if (a.clear_other) flag_o = a.flags_other[t];
    }

    // ---- pull streaming (Eq. BGK left side) with half-way bounce-back
    C f[9][VEC];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int sy = y - cy(i);
        bool bb = false;
        if (WALLS) {
            bb = (sy < 0) || (sy >= ny);
        } else {
            sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
        }
        if (bb) {
            // the population that left this node toward the wall comes back
            // reversed, plus the momentum of a moving wall (diagonals only)
            const S* row = src + (size_t)opp(i) * N + (size_t)y * nx;
            load_pack<S, VEC>(row, x0, ok, inv, f[i]);
            if (cx(i) != 0) {
                const C t = C(cx(i)) * wall_term<C>(a, cy(i) > 0);
#pragma unroll
                for (int k = 0; k < VEC; ++k) f[i][k] += t;
            }
            continue;
        }
        const S* row = src + (size_t)i * N + (size_t)sy * nx;
        C v[VEC];
        load_pack<S, VEC>(row, x0, ok, inv, v);
        if (cx(i) == 0) {
#pragma unroll
            for (int k = 0; k < VEC; ++k) f[i][k] = v[k];
        } else if (cx(i) == 1) {
            // needs x0-1 .. x0+VEC-2
            C prev = __shfl_up_sync(FULL, v[VEC - 1], 1);
            if (lane == 0 && ok) prev = Storage<S>::load(row[x0 == 0 ? nx - 1 : x0 - 1], inv);
            f[i][0] = prev;
#pragma unroll
            for (int k = 1; k < VEC; ++k) f[i][k] = v[k - 1];
        } else {
            // needs x0+1 .. x0+VEC
            C next = __shfl_down_sync(FULL, v[0], 1);
            if (ok && (lane == 31 || x0 + VEC >= nx))
                next = Storage<S>::load(row[x0 + VEC >= nx ? 0 : x0 + VEC], inv);
#pragma unroll
            for (int k = 0; k < VEC - 1; ++k) f[i][k] = v[k + 1];
            f[i][VEC - 1] = next;
        }
    }

    // ---- IB force of this tile (Eq. ForcingTerm's f_ib): the fixed-point field
    // the spreading filled, plus the body force; the previous step's field is
    // zeroed here so that it is clean when the next step spreads into it
    C Gx[VEC], Gy[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        Gx[k] = LbConst<C>::gx(a);
        Gy[k] = LbConst<C>::gy(a);
    }
    bool flagged = false;
    if (HAS_IB) {
        flagged = flag != 0;
        const bool fo = flag_o != 0;
        // every thread has read flags_other[t] before it is cleared
        if (a.tile_h == 1 && a.tile_w <= 32 * VEC && 32 % a.tile_w == 0) __syncwarp();
        else __syncthreads();
        const size_t node = (size_t)y * nx + x0;
        if (flagged && ok) {
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
                const longlong2 g = pre_g ? gpre[k] : a.gsum[node + k];
                Gx[k] += from_fix<C>(g.x);
                Gy[k] += from_fix<C>(g.y);
            }
        }
        if (fo) {
            if (ok) {
#pragma unroll
                for (int k = 0; k < VEC; ++k) a.gclear[node + k] = make_longlong2(0, 0);
            }
            // one thread per flag: the one at the tile's first node
            if (ok && x0 % a.tile_w == 0 && y % a.tile_h == 0) a.flags_other[t] = 0;
        }
    }

    // ---- moments, Guo-corrected velocity, BGK collision with Guo source
    const C om = LbConst<C>::om(a);
    const C pre = C(1) - C(0.5) * om;
    const C om3 = LbConst<C>::om3(a);
    // Zou-He wall rows: the populations from outside rebuilt (warp-uniform: one row per warp)
    const bool zh = WALLS && a.zou_he && (y == 0 || y == ny - 1);
    C out[9][VEC];
    C rho_v[VEC], ux_v[VEC], uy_v[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        C fk[9], ok9[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) fk[i] = f[i][k];
        if (zh) zou_he<C>(fk, Gx[k], Gy[k], zh_wall_u<C>(a, y == 0), y == 0);
        collide<S>(fk, Gx[k], Gy[k], om, pre, om3, ok9, rho_v[k], ux_v[k], uy_v[k]);
#pragma unroll
        for (int i = 0; i < 9; ++i) out[i][k] = ok9[i];
    }

    if (!ok) return;
    const size_t node = (size_t)y * nx + x0;
    if (a.fields_only) {
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            if (a.rho_out) a.rho_out[node + k] = (double)rho_v[k];
            if (a.ux_out) a.ux_out[node + k] = (double)ux_v[k];
            if (a.uy_out) a.uy_out[node + k] = (double)uy_v[k];
        }
        return;
    }
    S* __restrict__ dst = static_cast<S*>(a.dst);
    const float scl = 1.0f / inv;  // 2^k, exact
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        Pack<S, VEC> p;
#pragma unroll
        for (int k = 0; k < VEC; ++k) p.v[k] = Storage<S>::store(out[i][k], scl);
        *reinterpret_cast<Pack<S, VEC>*>(dst + (size_t)i * N + node) = p;
    }
    if (HAS_IB && flagged) {
        // velocity for the interpolation to the markers (Sec. 2.3)
        Pack<C, VEC> pu, pv;
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            pu.v[k] = ux_v[k];
            pv.v[k] = uy_v[k];
        }
        *reinterpret_cast<Pack<C, VEC>*>(static_cast<C*>(a.ux) + node) = pu;
        *reinterpret_cast<Pack<C, VEC>*>(static_cast<C*>(a.uy) + node) = pv;
    }
}

template <typename S, int VEC, bool WALLS, int IB>
__global__ void __launch_bounds__(512) k_lb_step(const LbArgs a) {
    lb_tile<S, VEC, WALLS, IB>(a, blockIdx.x, blockIdx.y);
}

// Batched form: the tiles of up to kBatchMax lattices (ensemble members, each
// with its own arguments and the same tile shape) in one launch, one block per
// (lattice, tile), the tiles of a member row by row.  The member's arguments
// come from the launch parameters into shared memory; the tile then computes
// exactly what the single-lattice kernel computes.
template <typename S, int VEC, bool WALLS>
__global__ void __launch_bounds__(512) k_lb_step_batch(const __grid_constant__ LbBatch b) {
    __shared__ LbArgs s_a;
    const int m = batch_member(b.off, b.n, blockIdx.x);
    const int local = blockIdx.x - b.off[m], tx = b.tiles_x[m];
    stage_args(&s_a, &b.a[m]);
    lb_tile<S, VEC, WALLS, 1>(s_a, local % tx, local / tx);
}

template <typename S, int VEC>
static cudaError_t launch_lb_t(int ty, bool walls, bool has_ib, const LbArgs& a, cudaStream_t s) {
    dim3 block(32, ty);
    dim3 grid((a.nx + 32 * VEC - 1) / (32 * VEC), (a.ny + ty - 1) / ty);
    // the up-front force read is its own instantiation: its registers would
    // lower the occupancy of the plain form, which DRAM-bound runs need
    const int ib = has_ib ? (a.g_prefetch ? 2 : 1) : 0;
    if (walls) {
        if (ib == 2) k_lb_step<S, VEC, true, 2><<<grid, block, 0, s>>>(a);
        else if (ib == 1) k_lb_step<S, VEC, true, 1><<<grid, block, 0, s>>>(a);
        else k_lb_step<S, VEC, true, 0><<<grid, block, 0, s>>>(a);
    } else {
        if (ib == 2) k_lb_step<S, VEC, false, 2><<<grid, block, 0, s>>>(a);
        else if (ib == 1) k_lb_step<S, VEC, false, 1><<<grid, block, 0, s>>>(a);
        else k_lb_step<S, VEC, false, 0><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <typename S, int VEC>
static cudaError_t launch_lb_batch_t(int ty, bool walls, const LbBatch& b, cudaStream_t s) {
    const int nblocks = b.off[b.n];
    if (nblocks <= 0) return cudaSuccess;
    dim3 block(32, ty);
    if (walls) k_lb_step_batch<S, VEC, true><<<nblocks, block, 0, s>>>(b);
    else k_lb_step_batch<S, VEC, false><<<nblocks, block, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_lb_batch(lbib_precision prec, int vec, int ty, bool walls, const LbBatch& b, cudaStream_t s) {
    if (b.n < 1 || b.n > kBatchMax) return cudaErrorInvalidValue;
    switch (prec) {
        case LBIB_F64:
            if (vec == 1) return launch_lb_batch_t<double, 1>(ty, walls, b, s);
            if (vec == 2) return launch_lb_batch_t<double, 2>(ty, walls, b, s);
            break;
        case LBIB_F32:
            if (vec == 1) return launch_lb_batch_t<float, 1>(ty, walls, b, s);
            if (vec == 2) return launch_lb_batch_t<float, 2>(ty, walls, b, s);
            if (vec == 4) return launch_lb_batch_t<float, 4>(ty, walls, b, s);
            break;
        case LBIB_F32_STORE_F16:
            if (vec == 2) return launch_lb_batch_t<__half, 2>(ty, walls, b, s);
            if (vec == 4) return launch_lb_batch_t<__half, 4>(ty, walls, b, s);
            if (vec == 8) return launch_lb_batch_t<__half, 8>(ty, walls, b, s);
            break;
        case LBIB_F32_STORE_BF16:
            if (vec == 2) return launch_lb_batch_t<__nv_bfloat16, 2>(ty, walls, b, s);
            if (vec == 4) return launch_lb_batch_t<__nv_bfloat16, 4>(ty, walls, b, s);
            if (vec == 8) return launch_lb_batch_t<__nv_bfloat16, 8>(ty, walls, b, s);
            break;
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_lb_step(lbib_precision prec, int vec, int ty, bool walls, bool has_ib,
                           const LbArgs& a, cudaStream_t s) {
    switch (prec) {
        case LBIB_F64:
            if (vec == 1) return launch_lb_t<double, 1>(ty, walls, has_ib, a, s);
            if (vec == 2) return launch_lb_t<double, 2>(ty, walls, has_ib, a, s);
            break;
        case LBIB_F32:
            if (vec == 1) return launch_lb_t<float, 1>(ty, walls, has_ib, a, s);
            if (vec == 2) return launch_lb_t<float, 2>(ty, walls, has_ib, a, s);
            if (vec == 4) return launch_lb_t<float, 4>(ty, walls, has_ib, a, s);
            break;
        case LBIB_F32_STORE_F16:
            if (vec == 2) return launch_lb_t<__half, 2>(ty, walls, has_ib, a, s);
            if (vec == 4) return launch_lb_t<__half, 4>(ty, walls, has_ib, a, s);
            if (vec == 8) return launch_lb_t<__half, 8>(ty, walls, has_ib, a, s);
            break;
        case LBIB_F32_STORE_BF16:
            if (vec == 2) return launch_lb_t<__nv_bfloat16, 2>(ty, walls, has_ib, a, s);
            if (vec == 4) return launch_lb_t<__nv_bfloat16, 4>(ty, walls, has_ib, a, s);
            if (vec == 8) return launch_lb_t<__nv_bfloat16, 8>(ty, walls, has_ib, a, s);
            break;
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- helpers

// f^n_i(x) = w_i + d*_i(x - e_i) (or the reversed population at a wall): the
// pre-collision populations the next step starts from, as doubles.
template <typename S>
__global__ void k_stream_out(const S* __restrict__ src, double* __restrict__ out, int nx, int ny,
                             int walls, float inv, double bb_bot, double bb_top, double uw_bot, double uw_top) {
    const size_t N = (size_t)nx * ny;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(n / nx), x = (int)(n % nx);
        double d[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            int sy = y - cy(i), sx = x - cx(i);
            sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
            if (walls && (sy < 0 || sy >= ny)) {
                d[i] = (double)Storage<S>::load(src[(size_t)opp(i) * N + n], inv) +
                       (double)cx(i) * (sy < 0 ? bb_bot : bb_top);
            } else {
                sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
                d[i] = (double)Storage<S>::load(src[(size_t)i * N + (size_t)sy * nx + sx], inv);
            }
        }
        if (walls == 2 && (y == 0 || y == ny - 1)) zou_he<double>(d, 0.0, 0.0, y == 0 ? uw_bot : uw_top, y == 0);
#pragma unroll
        for (int i = 0; i < 9; ++i) out[(size_t)i * N + n] = wgt<double>(i) + d[i];
    }
}

// inverse of k_stream_out: scatter f^n back to the post-collision slots it came from
template <typename S>
__global__ void k_stream_in(const double* __restrict__ in, S* __restrict__ dst, int nx, int ny,
                            int walls, float inv, double bb_bot, double bb_top) {
    const size_t N = (size_t)nx * ny;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(n / nx), x = (int)(n % nx);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double d = in[(size_t)i * N + n] - wgt<double>(i);
            const auto sv = Storage<S>::store((typename Storage<S>::C)d, 1.0f / inv);
            int sy = y - cy(i), sx = x - cx(i);
            sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
            if (walls && (sy < 0 || sy >= ny)) {
                // a moving wall's momentum is not stored
                const double dw = d - (double)cx(i) * (sy < 0 ? bb_bot : bb_top);
                dst[(size_t)opp(i) * N + n] = Storage<S>::store((typename Storage<S>::C)dw, 1.0f / inv);
            } else {
                sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
                dst[(size_t)i * N + (size_t)sy * nx + sx] = sv;
            }
        }
    }
}

// tau = 1 discrete Poiseuille fixed point (Sec. 3 drive): the post-collision
// state is feq(1, u(y)) + Guo source with u(y) = G/(2 nu) (y+1/2)(NY-1/2-y) + G/4.
template <typename S>
__global__ void k_init_poiseuille(S* __restrict__ dst, int nx, int ny, double tau, double G, float inv) {
    const size_t N = (size_t)nx * ny;
    const double nu = (tau - 0.5) / 3.0;
    const double pre = 1.0 - 0.5 / tau;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        const double y = (double)(n / nx);
        const double u = G / (2.0 * nu) * (y + 0.5) * ((double)ny - 0.5 - y) + 0.25 * G;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double eu = cx(i) * u;
            const double deq = wgt<double>(i) * (3.0 * eu + 4.5 * eu * eu - 1.5 * u * u);
            const double src = pre * wgt<double>(i) * (3.0 * (cx(i) - u) + 9.0 * eu * cx(i)) * G;
            dst[(size_t)i * N + n] = Storage<S>::store((typename Storage<S>::C)(deq + src), 1.0f / inv);
        }
    }
}

// tau = 1 planar Couette state (Sec. 4, cell-free layer): post-collision
// deviations feq(1, u(y)) - w with u(y) = u_bot + (u_top - u_bot)(y + 1/2)/NY
template <typename S>
__global__ void k_init_couette(S* __restrict__ dst, int nx, int ny, double u_bot, double u_top, float inv) {
    const size_t N = (size_t)nx * ny;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        const double y = (double)(n / nx);
        const double u = u_bot + (u_top - u_bot) * (y + 0.5) / (double)ny;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double eu = cx(i) * u;
            const double deq = wgt<double>(i) * (3.0 * eu + 4.5 * eu * eu - 1.5 * u * u);
            dst[(size_t)i * N + n] = Storage<S>::store((typename Storage<S>::C)deq, 1.0f / inv);
        }
    }
}

// rest state f_i = w_i beside moving walls: the stored deviations are zero
// except in the slots that the wall rows pull back from the walls, which hold
// minus the wall's momentum term (so that the pulled populations are w_i)
template <typename S>
__global__ void k_init_rest_walls(S* __restrict__ dst, int nx, int ny, double bb_bot, double bb_top, float inv) {
    const size_t N = (size_t)nx * ny;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 5; i < 9; ++i) {
            const bool from_bottom = cy(i) > 0;  // 5, 6 leave the lower wall; 7, 8 the upper
            const size_t node = from_bottom ? (size_t)x : (size_t)(ny - 1) * nx + x;
            const double t = (double)cx(i) * (from_bottom ? bb_bot : bb_top);
            dst[(size_t)opp(i) * N + node] = Storage<S>::store((typename Storage<S>::C)(-t), 1.0f / inv);
        }
    }
}

// FP64 sum of all stored deviations: per-block partials, then one block adds
// them in a fixed order (run-to-run deterministic).
template <typename S>
__global__ void k_sum_dev(const S* __restrict__ src, long long n, double* partials, float inv) {
    double acc = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        acc += (double)Storage<S>::load(src[k], inv);
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(FULL, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(FULL, acc, o);
        if (threadIdx.x == 0) partials[blockIdx.x] = acc;
    }
}

__global__ void k_sum_partials(const double* partials, int n, double base, double* out) {
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) acc += partials[k];
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(FULL, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(FULL, acc, o);
        if (threadIdx.x == 0) *out = base + acc;
    }
}

static int grid_for(size_t n, int block) {
    size_t g = (n + block - 1) / block;
    return (int)(g > 4096 ? 4096 : (g == 0 ? 1 : g));
}

#define LBIB_DISPATCH_S(prec, CALL)                                          \
    switch (prec) {                                                          \
        case LBIB_F64: { using S = double; CALL; } break;                    \
        case LBIB_F32: { using S = float; CALL; } break;                     \
        case LBIB_F32_STORE_F16: { using S = __half; CALL; } break;          \
        case LBIB_F32_STORE_BF16: { using S = __nv_bfloat16; CALL; } break;  \
        default: return cudaErrorInvalidValue;                               \
    }

cudaError_t launch_stream_out(lbib_precision prec, const void* src, double* out, int nx, int ny,
                              int walls, float inv_scale, double bb_bot, double bb_top, double uw_bot,
                              double uw_top, cudaStream_t s) {
    const int g = grid_for((size_t)nx * ny, 256);
    LBIB_DISPATCH_S(prec, (k_stream_out<S><<<g, 256, 0, s>>>(static_cast<const S*>(src), out, nx, ny, walls,
                                                              inv_scale, bb_bot, bb_top, uw_bot, uw_top)));
    return cudaGetLastError();
}

cudaError_t launch_stream_in(lbib_precision prec, const double* in, void* dst, int nx, int ny,
                             bool walls, float inv_scale, double bb_bot, double bb_top, cudaStream_t s) {
    const int g = grid_for((size_t)nx * ny, 256);
    LBIB_DISPATCH_S(prec, (k_stream_in<S><<<g, 256, 0, s>>>(in, static_cast<S*>(dst), nx, ny,
                                                             walls ? 1 : 0, inv_scale, bb_bot, bb_top)));
    return cudaGetLastError();
}

cudaError_t launch_init_rest_walls(lbib_precision prec, void* dst, int nx, int ny, double bb_bot, double bb_top,
                                   float inv_scale, cudaStream_t s) {
    const int g = grid_for((size_t)nx, 256);
    LBIB_DISPATCH_S(prec, (k_init_rest_walls<S><<<g, 256, 0, s>>>(static_cast<S*>(dst), nx, ny, bb_bot, bb_top,
                                                                   inv_scale)));
    return cudaGetLastError();
}

cudaError_t launch_init_couette(lbib_precision prec, void* dst, int nx, int ny, double u_bot, double u_top,
                                float inv_scale, cudaStream_t s) {
    const int g = grid_for((size_t)nx * ny, 256);
    LBIB_DISPATCH_S(prec, (k_init_couette<S><<<g, 256, 0, s>>>(static_cast<S*>(dst), nx, ny, u_bot, u_top,
                                                                inv_scale)));
    return cudaGetLastError();
}

cudaError_t launch_init_poiseuille(lbib_precision prec, void* dst, int nx, int ny, double tau,
                                   double gx, float inv_scale, cudaStream_t s) {
    const int g = grid_for((size_t)nx * ny, 256);
    LBIB_DISPATCH_S(prec, (k_init_poiseuille<S><<<g, 256, 0, s>>>(static_cast<S*>(dst), nx, ny,
                                                                   tau, gx, inv_scale)));
    return cudaGetLastError();
}

cudaError_t launch_mass(lbib_precision prec, const void* src, long long n_elems, double* partials,
                        int n_partials, double* out, float inv_scale, cudaStream_t s) {
    LBIB_DISPATCH_S(prec, (k_sum_dev<S><<<n_partials, 256, 0, s>>>(static_cast<const S*>(src),
                                                                    n_elems, partials, inv_scale)));
    // sum_i w_i = 1 per node, so the mass is N + sum of deviations
    k_sum_partials<<<1, 1024, 0, s>>>(partials, n_partials, (double)(n_elems / 9), out);
    return cudaGetLastError();
}

}  // namespace lbib
