// Persistent bulk-copy form of the fused collide-stream kernel.
//
// The row-tile kernel (lb_kernels.cu) keeps its nine pulled populations in
// registers, so the bytes it has in flight per SM are bounded by how many
// warps fit: on large lattices it waits on DRAM latency.  This form decouples
// the two: each CTA (one to three per SM, for the whole lattice) walks a strided
// list of row segments of W = 256 * NPT nodes and streams, for every segment,
// the nine source rows it pulls from into a 4-stage shared-memory ring with
// cp.async.bulk copies that complete on an mbarrier.  While the threads
// collide segment k, the copies of segments k+1 .. k+3 are in flight.  Each
// thread takes NPT consecutive nodes: one vector shared-memory load per
// direction (plus one element for the x-shifted directions) and one vector
// global store per direction.  The spread IB force is read straight from
// global memory in the few segments whose tile holds markers.
//
// Staged row of direction i (HALO = one 16-byte chunk on each side):
//   [x0 - HALO, x0 + W + HALO) of plane i, row y - e_iy   (interior rows)
//   [x0 - HALO, x0 + W + HALO) of plane opp(i), row y      (half-way bounce-back)
// The periodic x neighbours at the ends of a row come from separate 16-byte
// copies of the other end of the row.  The arithmetic per node is
// collide_node(), the same as the row-tile kernel's, so both forms give the
// same bits.  The force-tile geometry is one tile per segment (W x 1).
//
// Paper: Coclite, arXiv 1907.00080, Sec. 2.1 (Eqs. BGK, feq, GaussHermite),
// Sec. 2.2 (Eqs. forcedBGK, ForcingTerm), Sec. 3 (periodic x, walls in y).
#include <cstdint>

#include "lb_node.cuh"

namespace lbib {
namespace {

constexpr int kThreads = 256;                   // consumer threads (8 warps) per CTA
constexpr int kConsumerWarps = kThreads / 32;
constexpr int kBlock = kThreads + 32;           // plus one producer warp
constexpr int kStages = 4;
// try_wait polls before a CTA gives up on a copy (each poll may suspend for a
// while in hardware; the bound is far beyond any healthy copy, about a second)
constexpr int kSpinLimit = 1 << 22;

template <typename S, int NPT>
struct Geom {
    static constexpr int H = 16 / (int)sizeof(S);          // halo elements (16 bytes)
    static constexpr int W = kThreads * NPT;               // nodes per segment
    static constexpr int ROW = W + 2 * H;                  // staged elements per row
    static constexpr int ROW_BYTES = ROW * (int)sizeof(S);
    static constexpr int STAGE_BYTES = 9 * ROW_BYTES;
    static constexpr int SMEM = kStages * STAGE_BYTES;
    static_assert(ROW_BYTES % 16 == 0, "16-byte aligned stage rows");
    static_assert(NPT <= H, "a thread's nodes never straddle the end of a row");
};

template <typename T, int V>
struct alignas(sizeof(T) * V) Vec {
    T v[V];
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// bounded wait for the phase with the given parity; false if it never completed
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
// the same wait with a short sleep between polls, for the consumer warps: their
// polling would otherwise take issue slots from the producer on the same SM
__device__ __forceinline__ bool mbar_wait_sleep(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        __nanosleep(64);
    }
    return false;
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, unsigned bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Producer-warp schedule (16-bit storage): 288 threads.  Warps 0-7 consume
// (collide the staged segment; they leave each segment together through named
// barrier 1), warp 8 produces: lane 0 waits for the stage's "empty" barrier
// (one arrival once the consumers have passed the segment), then lanes 0-8
// each issue the copies of one direction.  Stage s also has a "full" barrier
// (the producer's expect-tx plus the copies' bytes).  Issuing from nine lanes
// instead of one thread keeps the producer ahead of the short 16-bit segments.
template <typename S, int NPT, bool WALLS>
__global__ void __launch_bounds__(kBlock) k_lb_stream_ws(const LbArgs a) {
    using C = typename Storage<S>::C;
    using Gm = Geom<S, NPT>;
    constexpr int H = Gm::H, W = Gm::W;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bars[kStages];
    __shared__ __align__(8) unsigned long long empty[kStages];
    __shared__ int s_meta[kStages];
    __shared__ int s_last_issued[kStages];
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const int nseg = (nx + W - 1) / W;
    const long long n_items = (long long)ny * nseg;
    const size_t N = (size_t)nx * ny;
    const S* __restrict__ src = static_cast<const S*>(a.src);
    S* __restrict__ dst = static_cast<S*>(a.dst);
    const bool has_ib = a.flags != nullptr;
    const long long first = blockIdx.x, stride = gridDim.x;
    const int my_n = first < n_items ? (int)((n_items - 1 - first) / stride + 1) : 0;
    const uint32_t smem0 = smem_addr(smem);

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_addr(&bars[s]), 1);
            mbar_init(smem_addr(&empty[s]), 1);
            s_last_issued[s] = -1;
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // producer warp: stage the rows of the k-th item of this CTA into stage
    // k % kStages; lane 0 sets the expected bytes, then lane i < 9 copies the
    // source row of direction i
    auto issue = [&](int k, int flagged, int fo, int ln) {
        const long long item = first + (long long)k * stride;
        const int stage = k % kStages;
        const int y = (int)(item / nseg);
        const int x0 = (int)(item % nseg) * W;
        const int wlen = min(W, nx - x0);
        const uint32_t bar = smem_addr(&bars[stage]);
        const uint32_t base = smem0 + stage * Gm::STAGE_BYTES;
        const unsigned row_bytes = (unsigned)((wlen + 2 * H) * sizeof(S));
        if (ln == 0) {
            s_meta[stage] = flagged | (fo << 1);
            mbar_expect_tx(bar, 9u * row_bytes);
        }
        __syncwarp();
        if (ln < 9) {
            const int i = ln;
            int sy = y - cy(i), plane = i;
            if (WALLS) {
                if (sy < 0 || sy >= ny) {
                    plane = opp(i);
                    sy = y;
                }
            } else {
                sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
            }
            const S* row = src + (size_t)plane * N + (size_t)sy * nx;
            const uint32_t d = base + i * Gm::ROW_BYTES;
            if (x0 >= H && x0 + wlen + H <= nx) {
                bulk_g2s(d, row + (x0 - H), row_bytes, bar);
            } else {
                bulk_g2s(d, row + (x0 == 0 ? nx - H : x0 - H), 16u, bar);
                bulk_g2s(d + 16u, row + x0, (unsigned)(wlen * sizeof(S)), bar);
                bulk_g2s(d + 16u + (unsigned)(wlen * sizeof(S)), row + (x0 + wlen == nx ? 0 : x0 + wlen), 16u, bar);
            }
        }
    };
    auto item_flags = [&](int k, int& flagged, int& fo) {
        const long long item = first + (long long)k * stride;
        flagged = has_ib && a.flags[item] != 0;
        fo = (has_ib && a.clear_other && a.flags_other[item] != 0) ? 1 : 0;
    };

    const int warp = tid >> 5, lane = tid & 31;
    if (warp == kConsumerWarps) {
        // ---- producer: stage segment k once the consumers have left the
        // segment k - kStages that used the same stage; tile flags fetched three
        // segments ahead by lane 0 (their latency stays off the producer's path)
        int fl = 0, fo = 0, f1 = 0, o1 = 0, f2 = 0, o2 = 0;
        if (lane == 0) {
            if (my_n > 0) item_flags(0, fl, fo);
            if (my_n > 1) item_flags(1, f1, o1);
            if (my_n > 2) item_flags(2, f2, o2);
        }
        for (int k = 0; k < my_n; ++k) {
            const int stage = k % kStages;
            int stop = 0;
            if (lane == 0) {
                if (k >= kStages &&
                    !mbar_wait(smem_addr(&empty[stage]), (uint32_t)(((k / kStages) - 1) & 1)))
                    s_abort = 1;
                stop = s_abort;
                // the previous parity's flag of this tile is read here and only here
                if (!stop && fo) a.flags_other[first + (long long)k * stride] = 0;
            }
            stop = __shfl_sync(0xffffffffu, stop, 0);
            if (stop) break;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const int flb = __shfl_sync(0xffffffffu, fl, 0), fob = __shfl_sync(0xffffffffu, fo, 0);
            issue(k, flb, fob, lane);
            if (lane == 0) {
                s_last_issued[stage] = k;
                fl = f1;
                fo = o1;
                f1 = f2;
                o1 = o2;
                if (k + 3 < my_n) item_flags(k + 3, f2, o2);
            }
        }
    } else {
        // ---- consumers
        const C om = C(a.omega);
        const C pre = C(1) - C(0.5) * om;
        const C om3 = C(3.0 * a.omega);
        const float inv = a.inv_scale;
        const float scl = 1.0f / inv;  // 2^k, exact
        C* __restrict__ uxf = static_cast<C*>(a.ux);
        C* __restrict__ uyf = static_cast<C*>(a.uy);
        for (int k = 0; k < my_n; ++k) {
            const int stage = k % kStages;
            const bool ok = mbar_wait_sleep(smem_addr(&bars[stage]), (uint32_t)((k / kStages) & 1));
            const long long item = first + (long long)k * stride;
            const int y = (int)(item / nseg);
            const int x0 = (int)(item % nseg) * W;
            const int wlen = min(W, nx - x0);
            const int meta = s_meta[stage];
            const S* sp = reinterpret_cast<const S*>(smem + stage * Gm::STAGE_BYTES);
            const int j0 = tid * NPT;
            if (ok && j0 < wlen) {
                // pull: f_i(x) = d*_i(x - e_i), or d*_opp(i)(x) where x - e_i is outside the walls
                C f[9][NPT];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const bool bb = WALLS && (y - cy(i) < 0 || y - cy(i) >= ny);
                    const S* rp = sp + i * Gm::ROW + H + j0;
                    const Vec<S, NPT> v = *reinterpret_cast<const Vec<S, NPT>*>(rp);
                    if (bb || cx(i) == 0) {
#pragma unroll
                        for (int q = 0; q < NPT; ++q) f[i][q] = Storage<S>::load(v.v[q], inv);
                        if (bb && cx(i) != 0) {
                            // the momentum of a moving wall (diagonals only)
                            const C t = C(cx(i)) * wall_term<C>(a, cy(i) > 0);
#pragma unroll
                            for (int q = 0; q < NPT; ++q) f[i][q] += t;
                        }
                    } else if (cx(i) == 1) {
                        f[i][0] = Storage<S>::load(rp[-1], inv);
#pragma unroll
                        for (int q = 1; q < NPT; ++q) f[i][q] = Storage<S>::load(v.v[q - 1], inv);
                    } else {
#pragma unroll
                        for (int q = 0; q < NPT - 1; ++q) f[i][q] = Storage<S>::load(v.v[q + 1], inv);
                        f[i][NPT - 1] = Storage<S>::load(rp[NPT], inv);
                    }
                }
                const size_t node0 = (size_t)y * nx + x0 + j0;
                Vec<S, NPT> o[9];
                Vec<C, NPT> pu, pv;
#pragma unroll
                for (int q = 0; q < NPT; ++q) {
                    C Gx = C(a.gx), Gy = C(a.gy);
                    if (meta & 1) {
                        const longlong2 g = a.gsum[node0 + q];
                        Gx += from_fix<C>(g.x);
                        Gy += from_fix<C>(g.y);
                    }
                    C fq[9], out[9], rho;
#pragma unroll
                    for (int i = 0; i < 9; ++i) fq[i] = f[i][q];
                    collide<S>(fq, Gx, Gy, om, pre, om3, out, rho, pu.v[q], pv.v[q]);
#pragma unroll
                    for (int i = 0; i < 9; ++i) o[i].v[q] = Storage<S>::store(out[i], scl);
                }
#pragma unroll
                for (int i = 0; i < 9; ++i) *reinterpret_cast<Vec<S, NPT>*>(dst + (size_t)i * N + node0) = o[i];
                if (meta & 1) {
                    // velocity for the interpolation to the markers (Sec. 2.3)
                    *reinterpret_cast<Vec<C, NPT>*>(uxf + node0) = pu;
                    *reinterpret_cast<Vec<C, NPT>*>(uyf + node0) = pv;
                }
                if (meta & 2) {
#pragma unroll
                    for (int q = 0; q < NPT; ++q) a.gclear[node0 + q] = make_longlong2(0, 0);
                }
            }
            // the consumer warps leave the segment together (named barrier 1):
            // their stores go out as one burst per segment; one arrival frees the stage
            uint32_t any_bad;
            asm volatile(
                "{\n .reg .pred p, q;\n setp.eq.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n"
                " selp.u32 %0, 1, 0, q;\n}"
                : "=r"(any_bad)
                : "r"((uint32_t)ok), "r"(kThreads)
                : "memory");
            if (any_bad) {
                if (tid == 0) s_abort = 1;
                break;
            }
            if (tid == 0) mbar_arrive(smem_addr(&empty[stage]));
        }
    }
    __syncthreads();
    if (s_abort && tid == 0) {
        // a wait gave up: report it, then wait (bounded) for the copies still in
        // flight (the last segment staged into each stage) before the shared
        // memory is released
        atomicOr(a.status, ST_TIMEOUT);
        for (int st = 0; st < kStages; ++st) {
            const int m = s_last_issued[st];
            if (m >= 0) mbar_wait(smem_addr(&bars[st]), (uint32_t)((m / kStages) & 1));
        }
    }
}

// Barrier schedule (FP32, FP64): 256 threads; a CTA barrier ends each segment
// and thread 0 then refills the stage that segment used with the segment
// kStages ahead (its expected bytes and the nine row copies).
template <typename S, int NPT, bool WALLS>
__global__ void __launch_bounds__(kThreads) k_lb_stream_bar(const LbArgs a) {
    using C = typename Storage<S>::C;
    using Gm = Geom<S, NPT>;
    constexpr int H = Gm::H, W = Gm::W;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bars[kStages];
    __shared__ int s_meta[kStages];

    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const int nseg = (nx + W - 1) / W;
    const long long n_items = (long long)ny * nseg;
    const size_t N = (size_t)nx * ny;
    const S* __restrict__ src = static_cast<const S*>(a.src);
    S* __restrict__ dst = static_cast<S*>(a.dst);
    const bool has_ib = a.flags != nullptr;
    const long long first = blockIdx.x, stride = gridDim.x;
    const int my_n = first < n_items ? (int)((n_items - 1 - first) / stride + 1) : 0;
    const uint32_t smem0 = smem_addr(smem);

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(smem_addr(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // thread 0: stage the rows of the k-th item of this CTA into stage k % kStages
    auto issue = [&](int k, int flagged, int fo) {
        const long long item = first + (long long)k * stride;
        const int stage = k % kStages;
        const int y = (int)(item / nseg);
        const int x0 = (int)(item % nseg) * W;
        const int wlen = min(W, nx - x0);
        const uint32_t bar = smem_addr(&bars[stage]);
        const uint32_t base = smem0 + stage * Gm::STAGE_BYTES;
        s_meta[stage] = flagged | (fo << 1);
        const unsigned row_bytes = (unsigned)((wlen + 2 * H) * sizeof(S));
        mbar_expect_tx(bar, 9u * row_bytes);
        const bool interior = x0 >= H && x0 + wlen + H <= nx;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            int sy = y - cy(i), plane = i;
            if (WALLS) {
                if (sy < 0 || sy >= ny) {
                    plane = opp(i);
                    sy = y;
                }
            } else {
                sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
            }
            const S* row = src + (size_t)plane * N + (size_t)sy * nx;
            const uint32_t d = base + i * Gm::ROW_BYTES;
            if (interior) {
                bulk_g2s(d, row + (x0 - H), row_bytes, bar);
            } else {
                bulk_g2s(d, row + (x0 == 0 ? nx - H : x0 - H), 16u, bar);
                bulk_g2s(d + 16u, row + x0, (unsigned)(wlen * sizeof(S)), bar);
                bulk_g2s(d + 16u + (unsigned)(wlen * sizeof(S)), row + (x0 + wlen == nx ? 0 : x0 + wlen), 16u, bar);
            }
        }
    };
    auto item_flags = [&](int k, int& flagged, int& fo) {
        const long long item = first + (long long)k * stride;
        flagged = has_ib && a.flags[item] != 0;
        fo = (has_ib && a.clear_other && a.flags_other[item] != 0) ? 1 : 0;
    };

    if (tid == 0) {
        for (int k = 0; k < kStages && k < my_n; ++k) {
            int fl, fo;
            item_flags(k, fl, fo);
            issue(k, fl, fo);
        }
    }

    const C om = C(a.omega);
    const C pre = C(1) - C(0.5) * om;
    const C om3 = C(3.0 * a.omega);
    const float inv = a.inv_scale;
    const float scl = 1.0f / inv;  // 2^k, exact
    C* __restrict__ uxf = static_cast<C*>(a.ux);
    C* __restrict__ uyf = static_cast<C*>(a.uy);
    bool bad = false;
    int k = 0;
    for (; k < my_n; ++k) {
        const int stage = k % kStages;
        // thread 0 fetches the flags of the item it stages at the end of this one
        int nfl = 0, nfo = 0;
        if (tid == 0 && k + kStages < my_n) item_flags(k + kStages, nfl, nfo);

        const bool ok = mbar_wait(smem_addr(&bars[stage]), (uint32_t)((k / kStages) & 1));
        const long long item = first + (long long)k * stride;
        const int y = (int)(item / nseg);
        const int x0 = (int)(item % nseg) * W;
        const int wlen = min(W, nx - x0);
        const int meta = s_meta[stage];
        const S* sp = reinterpret_cast<const S*>(smem + stage * Gm::STAGE_BYTES);
        const int j0 = tid * NPT;
        if (j0 < wlen) {
            // pull: f_i(x) = d*_i(x - e_i), or d*_opp(i)(x) where x - e_i is outside the walls
            C f[9][NPT];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const bool bb = WALLS && (y - cy(i) < 0 || y - cy(i) >= ny);
                const S* rp = sp + i * Gm::ROW + H + j0;
                const Vec<S, NPT> v = *reinterpret_cast<const Vec<S, NPT>*>(rp);
                if (bb || cx(i) == 0) {
#pragma unroll
                    for (int q = 0; q < NPT; ++q) f[i][q] = Storage<S>::load(v.v[q], inv);
                    if (bb && cx(i) != 0) {
                        // the momentum of a moving wall (diagonals only)
                        const C t = C(cx(i)) * wall_term<C>(a, cy(i) > 0);
#pragma unroll
                        for (int q = 0; q < NPT; ++q) f[i][q] += t;
                    }
                } else if (cx(i) == 1) {
                    f[i][0] = Storage<S>::load(rp[-1], inv);
#pragma unroll
                    for (int q = 1; q < NPT; ++q) f[i][q] = Storage<S>::load(v.v[q - 1], inv);
                } else {
#pragma unroll
                    for (int q = 0; q < NPT - 1; ++q) f[i][q] = Storage<S>::load(v.v[q + 1], inv);
                    f[i][NPT - 1] = Storage<S>::load(rp[NPT], inv);
                }
            }
            const size_t node0 = (size_t)y * nx + x0 + j0;
            Vec<S, NPT> o[9];
            Vec<C, NPT> pu, pv;
#pragma unroll
            for (int q = 0; q < NPT; ++q) {
                C Gx = C(a.gx), Gy = C(a.gy);
                if (meta & 1) {
                    const longlong2 g = a.gsum[node0 + q];
                    Gx += from_fix<C>(g.x);
                    Gy += from_fix<C>(g.y);
                }
                C fq[9], out[9], rho;
#pragma unroll
                for (int i = 0; i < 9; ++i) fq[i] = f[i][q];
                collide<S>(fq, Gx, Gy, om, pre, om3, out, rho, pu.v[q], pv.v[q]);
#pragma unroll
                for (int i = 0; i < 9; ++i) o[i].v[q] = Storage<S>::store(out[i], scl);
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) *reinterpret_cast<Vec<S, NPT>*>(dst + (size_t)i * N + node0) = o[i];
            if (meta & 1) {
                // velocity for the interpolation to the markers (Sec. 2.3)
                *reinterpret_cast<Vec<C, NPT>*>(uxf + node0) = pu;
                *reinterpret_cast<Vec<C, NPT>*>(uyf + node0) = pv;
            }
            if (meta & 2) {
#pragma unroll
                for (int q = 0; q < NPT; ++q) a.gclear[node0 + q] = make_longlong2(0, 0);
            }
        }
        // every thread is done with this stage (and every wait ended) before it is refilled
        bad = __syncthreads_or(!ok) != 0;
        if (bad) break;
        if (tid == 0) {
            if (meta & 2) a.flags_other[item] = 0;
            if (k + kStages < my_n) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(k + kStages, nfl, nfo);
            }
        }
    }
    if (bad && tid == 0) {
        // a copy never completed: report it, then wait (bounded) for the copies
        // this CTA still has in flight before its shared memory is released
        atomicOr(a.status, ST_TIMEOUT);
        for (int m = k; m < my_n && m < k + kStages; ++m)
            mbar_wait(smem_addr(&bars[m % kStages]), (uint32_t)((m / kStages) & 1));
    }
}

// the producer-warp schedule for 16-bit storage, the barrier schedule otherwise
// (measured on the 8192 x 2048 probe: FP32 npt 2 199 us vs 223 us; FP16 npt 4
// 158 us vs 138 us)
template <typename S>
constexpr bool kWarpSpecialised = sizeof(S) == 2;

template <typename S, int NPT, bool WALLS>
constexpr auto stream_kernel() {
    if constexpr (kWarpSpecialised<S>) return k_lb_stream_ws<S, NPT, WALLS>;
    else return k_lb_stream_bar<S, NPT, WALLS>;
}

template <typename S, int NPT, bool WALLS>
cudaError_t prepare_t(int* grid) {
    auto kern = stream_kernel<S, NPT, WALLS>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Geom<S, NPT>::SMEM);
    if (e != cudaSuccess) return e;
    const int threads = kWarpSpecialised<S> ? kBlock : kThreads;
    int occ = 0, dev = 0, nsm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, Geom<S, NPT>::SMEM)) != cudaSuccess)
        return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    *grid = occ * nsm;
    return cudaSuccess;
}

template <typename S, int NPT>
cudaError_t dispatch(bool prepare, bool walls, int grid, int* grid_out, const LbArgs* a, cudaStream_t s) {
    if (prepare) return walls ? prepare_t<S, NPT, true>(grid_out) : prepare_t<S, NPT, false>(grid_out);
    const int threads = kWarpSpecialised<S> ? kBlock : kThreads;
    const int nseg = (a->nx + Geom<S, NPT>::W - 1) / Geom<S, NPT>::W;
    const long long items = (long long)a->ny * nseg;
    const int g = (int)(items < grid ? items : grid);
    if (walls)
        stream_kernel<S, NPT, true>()<<<g, threads, Geom<S, NPT>::SMEM, s>>>(*a);
    else
        stream_kernel<S, NPT, false>()<<<g, threads, Geom<S, NPT>::SMEM, s>>>(*a);
    return cudaGetLastError();
}

cudaError_t dispatch_all(lbib_precision prec, int npt, bool prepare, bool walls, int grid, int* grid_out,
                         const LbArgs* a, cudaStream_t s) {
    switch (prec) {
        case LBIB_F64:
            if (npt == 1) return dispatch<double, 1>(prepare, walls, grid, grid_out, a, s);
            if (npt == 2) return dispatch<double, 2>(prepare, walls, grid, grid_out, a, s);
            break;
        case LBIB_F32:
            if (npt == 1) return dispatch<float, 1>(prepare, walls, grid, grid_out, a, s);
            if (npt == 2) return dispatch<float, 2>(prepare, walls, grid, grid_out, a, s);
            if (npt == 4) return dispatch<float, 4>(prepare, walls, grid, grid_out, a, s);
            break;
        case LBIB_F32_STORE_F16:
            if (npt == 2) return dispatch<__half, 2>(prepare, walls, grid, grid_out, a, s);
            if (npt == 4) return dispatch<__half, 4>(prepare, walls, grid, grid_out, a, s);
            if (npt == 8) return dispatch<__half, 8>(prepare, walls, grid, grid_out, a, s);
            break;
        case LBIB_F32_STORE_BF16:
            if (npt == 2) return dispatch<__nv_bfloat16, 2>(prepare, walls, grid, grid_out, a, s);
            if (npt == 4) return dispatch<__nv_bfloat16, 4>(prepare, walls, grid, grid_out, a, s);
            if (npt == 8) return dispatch<__nv_bfloat16, 8>(prepare, walls, grid, grid_out, a, s);
            break;
    }
    return cudaErrorInvalidValue;
}

}  // namespace

int lb_stream_halo(lbib_precision prec) {
    return prec == LBIB_F64 ? 2 : (prec == LBIB_F32 ? 4 : 8);
}

cudaError_t prepare_lb_stream(lbib_precision prec, int npt, bool walls, bool, int* grid) {
    return dispatch_all(prec, npt, true, walls, 0, grid, nullptr, nullptr);
}

cudaError_t launch_lb_stream(lbib_precision prec, int npt, bool walls, bool, int grid, const LbArgs& a,
                             cudaStream_t s) {
    return dispatch_all(prec, npt, false, walls, grid, nullptr, &a, s);
}

}  // namespace lbib
