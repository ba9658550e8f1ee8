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
// global memory where the segment's 32-node force tiles hold markers (their
// flags are fetched kStages segments ahead by one warp and kept in shared
// memory with the stage).
//
// Staged row of direction i (HALO = one 16-byte chunk on each side):
//   [x0 - HALO, x0 + W + HALO) of plane i, row y - e_iy   (interior rows)
//   [x0 - HALO, x0 + W + HALO) of plane opp(i), row y      (half-way bounce-back)
// The periodic x neighbours at the ends of a row come from a separate 16-byte
// copy of the other end of the row, for the three directions that pull
// across that end (e_ix = 1 at x = 0, e_ix = -1 at x = NX - 1).  The arithmetic per node is
// collide_node(), the same as the row-tile kernel's, so both forms give the
// same bits.  The force tiles are 32 nodes of one row, as in the row-tile
// form.  The same bodies serve one lattice (arguments in the kernel's
// parameters) and a batch of lattices (ensemble members: the work list runs
// over all members' segments, and the member's arguments are copied into the
// stage's slot of shared memory when its segment is staged).
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
    static_assert(W / 32 <= 64, "the tile flags of a segment fit two 32-bit masks");
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
// a population store marked streaming (st.global.cs: evict first in the
// caches).  The 16-bit kernels store this way: FP16 probe 59.5 -> 55.7 us per
// 8192 x 1024 launch (a buffer of 151 MB, about the L2), unchanged at 8192 x
// 2048; the same stores slowed FP32 (97.7 -> 104.3 us), and an evict-first
// policy on the bulk loads helped neither.
template <typename V>
__device__ __forceinline__ void st_stream(V* p, const V& v) {
    static_assert(sizeof(V) == 4 || sizeof(V) == 8 || sizeof(V) == 16, "vector stores of 4, 8 or 16 bytes");
    if constexpr (sizeof(V) == 4) __stcs(reinterpret_cast<unsigned*>(p), *reinterpret_cast<const unsigned*>(&v));
    else if constexpr (sizeof(V) == 8) __stcs(reinterpret_cast<uint2*>(p), *reinterpret_cast<const uint2*>(&v));
    else __stcs(reinterpret_cast<uint4*>(p), *reinterpret_cast<const uint4*>(&v));
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, unsigned bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}


// ---------------------------------------------------------------- work lists
// Where the items (row segments) of the work list lie, and the arguments of
// the lattice each belongs to.  locate() is valid at any time; staged(st)
// is the copy the staging thread made into stage st (for one lattice, the
// kernel's own parameters), and staged_pos(st) the position of the item it
// staged there.
struct ItemRef {
    int y, x0;
};

template <typename S, int NPT>
struct OneLattice {
    static constexpr int W = Geom<S, NPT>::W;
    const LbArgs& a;
    int nseg;
    ItemRef* s_pos;  // [kStages] in shared memory
    __device__ OneLattice(const LbArgs& a_, ItemRef* sp) : a(a_), nseg((a_.nx + W - 1) / W), s_pos(sp) {}
    __device__ long long count() const { return (long long)a.ny * nseg; }
    // (32-bit: the launch refuses work lists of 2^31 items or more)
    __device__ ItemRef pos(long long item) const {
        const int it = (int)item, y = it / nseg;
        return {y, (it - y * nseg) * W};
    }
    __device__ const LbArgs& locate(long long item, ItemRef& p, int& m) const {
        p = pos(item);
        m = 0;
        return a;
    }
    __device__ const LbArgs& locate(long long item, ItemRef& p) const {
        int m = 0;
        return locate(item, p, m);
    }
    // the staging warp (all lanes) prepares a stage for the item located as
    // (p, m): lane 0 keeps its position in the stage's slot, so that the
    // consumer threads need no division per segment
    __device__ void stage_args(ItemRef p, int, int st, int lane) const {
        if (lane == 0) s_pos[st] = p;
    }
    __device__ const LbArgs& staged(int) const { return a; }
    __device__ ItemRef staged_pos(long long, int st) const { return s_pos[st]; }
};

// b.off: first item of each member; b.tiles_x: segments per row of each member
template <typename S, int NPT>
struct ManyLattices {
    static constexpr int W = Geom<S, NPT>::W;
    const LbBatch& b;
    LbArgs* s_args;  // [kStages] in shared memory
    ItemRef* s_pos;  // [kStages]
    __device__ long long count() const { return b.off[b.n]; }
    // m: on entry a member at or before the item's (a CTA's items ascend:
    // its previous item's member), on return the item's member
    __device__ const LbArgs& locate(long long item, ItemRef& p, int& m) const {
        while (m + 1 < b.n && b.off[m + 1] <= (int)item) ++m;
        const int l = (int)item - b.off[m], ns = b.tiles_x[m];
        p = {l / ns, (l % ns) * W};
        return b.a[m];
    }
    __device__ const LbArgs& locate(long long item, ItemRef& p) const {
        int m = batch_member(b.off, b.n, (int)item);
        return locate(item, p, m);
    }
    // the staging warp (all lanes) copies the arguments of member m, 8-byte
    // words, and lane 0 the item's position p, into stage st's slots (the
    // item was located when its flags were fetched)
    __device__ void stage_args(ItemRef p, int m, int st, int lane) const {
        const LbArgs& A = b.a[m];
        constexpr int NW = (int)(sizeof(LbArgs) / 8);
        for (int w = lane; w < NW; w += 32)
            reinterpret_cast<long long*>(&s_args[st])[w] = reinterpret_cast<const long long*>(&A)[w];
        if (lane == 0) s_pos[st] = p;
    }
    __device__ const LbArgs& staged(int st) const { return s_args[st]; }
    __device__ ItemRef staged_pos(long long, int st) const { return s_pos[st]; }
};

// Force-tile flags of one item (segment): W / 32 tiles of 32 nodes, lane q of
// the fetching warp taking tiles q and q + 32.  Fetched kStages items ahead into
// registers, stored into the stage's shared slot once that stage is free.
// The fetch also keeps where the item lies (p, and m, its member in a batch)
// for its staging.
struct FlagRegs {
    int f[2], o[2];
    ItemRef p;
    int m;
};
// (hint: a member at or before the item's, e.g. the CTA's previous item's)
template <int W, typename Items>
__device__ __forceinline__ void fetch_flags(const Items& it, long long item, int lane, FlagRegs& r, int hint) {
    constexpr int NF = W / 32;
    r.f[0] = r.f[1] = r.o[0] = r.o[1] = 0;
    r.m = hint;
    const LbArgs& A = it.locate(item, r.p, r.m);
    const ItemRef p = r.p;
    if (A.flags == nullptr) return;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = lane + 32 * h;
        if (q < NF && p.x0 + 32 * q < A.nx) {
            const long long t = (long long)p.y * A.tiles_x + (p.x0 >> 5) + q;
            r.f[h] = A.flags[t];
            r.o[h] = A.clear_other ? A.flags_other[t] : 0;
        }
    }
}
// the whole warp: the item's flags as bit masks (tile q: bit q % 32 of word
// q / 32), written by lane 0 into the stage's slot {flags 0-31, 32-63,
// other parity's 0-31, 32-63}
__device__ __forceinline__ void keep_flags(const FlagRegs& r, int lane, uint4* slot) {
    const unsigned f0 = __ballot_sync(0xffffffffu, r.f[0] != 0), f1 = __ballot_sync(0xffffffffu, r.f[1] != 0);
    const unsigned o0 = __ballot_sync(0xffffffffu, r.o[0] != 0), o1 = __ballot_sync(0xffffffffu, r.o[1] != 0);
    if (lane == 0) *slot = make_uint4(f0, f1, o0, o1);
}
// tile q's flag and other-parity flag from a stage's masks
__device__ __forceinline__ int flag_of(const uint4& m, int q) { return ((q < 32 ? m.x : m.y) >> (q & 31)) & 1; }
__device__ __forceinline__ int flag_other_of(const uint4& m, int q) { return ((q < 32 ? m.z : m.w) >> (q & 31)) & 1; }

// Stage the nine source rows of `item` (plane i row y - e_iy, or plane opp(i)
// row y at a wall; W nodes and a 16-byte halo each side, the periodic ends by
// separate copies) into stage `st`: lane ln of the issuing group copies the
// rows i = ln, ln + nl, ...; the caller has set the stage's expected bytes
template <typename S, int NPT, bool WALLS>
__device__ __forceinline__ void stage_rows(const LbArgs& A, ItemRef p, uint32_t base, uint32_t bar, int ln, int nl) {
    using Gm = Geom<S, NPT>;
    constexpr int H = Gm::H, W = Gm::W;
    const int nx = A.nx, ny = A.ny;
    const size_t N = (size_t)nx * ny;
    const S* __restrict__ src = static_cast<const S*>(A.src);
    const int wlen = min(W, nx - p.x0);
    const unsigned row_bytes = (unsigned)((wlen + 2 * H) * sizeof(S));
    const bool interior = p.x0 >= H && p.x0 + wlen + H <= nx;
    for (int i = ln; i < 9; i += nl) {
        int sy = p.y - cy(i), plane = i;
        if (WALLS) {
            if (sy < 0 || sy >= ny) {
                plane = opp(i);
                sy = p.y;
            }
        } else {
            sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
        }
        const S* row = src + (size_t)plane * N + (size_t)sy * nx;
        const uint32_t d = base + i * Gm::ROW_BYTES;
        if (interior) {
            bulk_g2s(d, row + (p.x0 - H), row_bytes, bar);
        } else if (p.x0 >= H) {
            // the row's last segment: its left halo and nodes in one copy; the
            // periodic right halo (the row's first 16 bytes) only for the
            // directions that pull from it (e_ix = -1)
            bulk_g2s(d, row + (p.x0 - H), (unsigned)((wlen + H) * sizeof(S)), bar);
            if (cx(i) == -1) bulk_g2s(d + (unsigned)((wlen + H) * sizeof(S)), row, 16u, bar);
        } else if (p.x0 + wlen + H <= nx) {
            // the row's first segment: the periodic left halo (the row's last
            // 16 bytes) only for e_ix = 1, then its nodes and right halo
            if (cx(i) == 1) bulk_g2s(d, row + (nx - H), 16u, bar);
            bulk_g2s(d + 16u, row, (unsigned)((wlen + H) * sizeof(S)), bar);
        } else {
            // the whole row in one segment
            if (cx(i) == 1) bulk_g2s(d, row + (nx - H), 16u, bar);
            bulk_g2s(d + 16u, row, (unsigned)(wlen * sizeof(S)), bar);
            if (cx(i) == -1) bulk_g2s(d + 16u + (unsigned)(wlen * sizeof(S)), row, 16u, bar);
        }
    }
}
// the bytes stage_rows copies: nine rows of the segment's nodes, with both
// halos inside the row, one halo at an end of the row plus the periodic halo
// of the three directions that pull across that end
template <typename S, int NPT>
__device__ __forceinline__ unsigned stage_bytes(const LbArgs& A, ItemRef p) {
    using Gm = Geom<S, NPT>;
    constexpr int H = Gm::H;
    const int wlen = min(Gm::W, A.nx - p.x0);
    const bool interior = p.x0 >= H && p.x0 + wlen + H <= A.nx;
    const bool whole = p.x0 < H && p.x0 + wlen + H > A.nx;
    const int halos = interior ? 18 : (whole ? 6 : 12);
    return (unsigned)((9 * wlen + halos * H) * (int)sizeof(S));
}

// a staged value in the collision's units: the deviation for FP64 and FP32,
// the stored (scaled) value for 16-bit storage; and back to storage
template <typename S>
__device__ __forceinline__ typename Storage<S>::C pulled(S v, float inv) {
    if constexpr (sizeof(S) == 2) return Storage<S>::raw(v);
    else return Storage<S>::load(v, inv);
}
template <typename S>
__device__ __forceinline__ S stored(typename Storage<S>::C c, float scl) {
    if constexpr (sizeof(S) == 2) return Storage<S>::store_raw(c);
    else return Storage<S>::store(c, scl);
}

// One thread's NPT nodes of a staged segment: pull from the stage, add the
// spread force where its tile is flagged, collide, store; write u where
// flagged; clear the other parity's force where its tile was flagged (and the
// flag, by the thread at the tile's first node).  Three forms, chosen per warp
// (see consume_warp), with the same arithmetic per node: EDGE, a row next to a
// wall (bounce-back pulls and the Zou-He rebuild checked per direction);
// otherwise FORCED, a warp with a flagged force tile among its own, or neither,
// where the body force is the only force and the collision's force terms are
// the same for every node.
template <typename S, int NPT, bool WALLS, bool FORCED, bool EDGE>
__device__ __forceinline__ void consume(const LbArgs& A, ItemRef p, const S* sp, int j0, int flag, int flag_o) {
    using C = typename Storage<S>::C;
    using Gm = Geom<S, NPT>;
    constexpr int H = Gm::H;
    const int nx = A.nx, ny = A.ny, y = p.y;
    const size_t N = (size_t)nx * ny;
    S* __restrict__ dst = static_cast<S*>(A.dst);
    const C om = LbConst<C>::om(A);
    const C pre = C(1) - C(0.5) * om;
    const C om3 = LbConst<C>::om3(A);
    const float inv = A.inv_scale;
    const float scl = 1.0f / inv;  // 2^k, exact
    // 16-bit storage collides on the stored (scaled) values and, with an even
    // node count per thread, converts value pairs
    constexpr bool kHalf = sizeof(S) == 2;
    constexpr bool kPair = kHalf && NPT % 2 == 0;
    // pull: f_i(x) = d*_i(x - e_i), or d*_opp(i)(x) where x - e_i is outside the walls
    C f[9][NPT];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const bool bb = WALLS && EDGE && (y - cy(i) < 0 || y - cy(i) >= ny);
        const S* rp = sp + i * Gm::ROW + H + j0;
        const Vec<S, NPT> v = *reinterpret_cast<const Vec<S, NPT>*>(rp);
        // the thread's NPT staged values of this direction in the compute type
        // (16-bit storage: the stored values, d 2^k)
        C t[NPT];
        if constexpr (kPair) {
#pragma unroll
            for (int q = 0; q < NPT; q += 2) {
                const float2 u = Storage<S>::load2(*reinterpret_cast<const typename Storage<S>::S2*>(&v.v[q]));
                t[q] = u.x;
                t[q + 1] = u.y;
            }
        } else {
#pragma unroll
            for (int q = 0; q < NPT; ++q) t[q] = pulled<S>(v.v[q], inv);
        }
        if (bb || cx(i) == 0) {
#pragma unroll
            for (int q = 0; q < NPT; ++q) f[i][q] = t[q];
            if (bb && cx(i) != 0) {
                // the momentum of a moving wall (diagonals only; scaled by 2^k
                // with the stored values: exact)
                C w = C(cx(i)) * wall_term<C>(A, cy(i) > 0);
                if constexpr (kHalf) w *= scl;
#pragma unroll
                for (int q = 0; q < NPT; ++q) f[i][q] += w;
            }
        } else if (cx(i) == 1) {
            f[i][0] = pulled<S>(rp[-1], inv);
#pragma unroll
            for (int q = 1; q < NPT; ++q) f[i][q] = t[q - 1];
        } else {
#pragma unroll
            for (int q = 0; q < NPT - 1; ++q) f[i][q] = t[q + 1];
            f[i][NPT - 1] = pulled<S>(rp[NPT], inv);
        }
    }
    const size_t node0 = (size_t)y * nx + p.x0 + j0;
    Vec<S, NPT> o[9];
    Vec<C, NPT> pu, pv;
    C prev[9];  // paired stores: the even node's results wait for the odd one's
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
        C Gx = LbConst<C>::gx(A), Gy = LbConst<C>::gy(A);
        if (FORCED && flag) {
            const longlong2 g = A.gsum[node0 + q];
            Gx += from_fix<C>(g.x);
            Gy += from_fix<C>(g.y);
        }
        C fq[9], out[9], rho;
#pragma unroll
        for (int i = 0; i < 9; ++i) fq[i] = f[i][q];
        // Zou-He wall rows: the populations from outside rebuilt
        const bool zh = WALLS && EDGE && A.zou_he && (y == 0 || y == ny - 1);
        if constexpr (kHalf) {
            if (zh) {
                // on the unscaled deviations, then back to the stored scale (exact)
#pragma unroll
                for (int i = 0; i < 9; ++i) fq[i] *= inv;
                zou_he<C>(fq, Gx, Gy, zh_wall_u<C>(A, y == 0), y == 0);
                collide_node<C>(fq, Gx, Gy, om, pre, out, rho, pu.v[q], pv.v[q]);
#pragma unroll
                for (int i = 0; i < 9; ++i) out[i] *= scl;
            } else {
                collide_node_scaled(fq, Gx, Gy, om, pre, inv, scl, out, rho, pu.v[q], pv.v[q]);
            }
        } else {
            if (zh) zou_he<C>(fq, Gx, Gy, zh_wall_u<C>(A, y == 0), y == 0);
            collide<S>(fq, Gx, Gy, om, pre, om3, out, rho, pu.v[q], pv.v[q]);
        }
        if constexpr (kPair) {
            if (q & 1) {
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    *reinterpret_cast<typename Storage<S>::S2*>(&o[i].v[q - 1]) = Storage<S>::store2(prev[i], out[i]);
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i) prev[i] = out[i];
            }
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) o[i].v[q] = stored<S>(out[i], scl);
        }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        Vec<S, NPT>* d = reinterpret_cast<Vec<S, NPT>*>(dst + (size_t)i * N + node0);
        if constexpr (kHalf) st_stream(d, o[i]);
        else *d = o[i];
    }
    if (FORCED && flag) {
        // velocity for the interpolation to the markers (Sec. 2.3)
        *reinterpret_cast<Vec<C, NPT>*>(static_cast<C*>(A.ux) + node0) = pu;
        *reinterpret_cast<Vec<C, NPT>*>(static_cast<C*>(A.uy) + node0) = pv;
    }
    if (flag_o) {
#pragma unroll
        for (int q = 0; q < NPT; ++q) A.gclear[node0 + q] = make_longlong2(0, 0);
        // the tile's flag was fetched kStages segments ago; nothing reads it again
        if (((p.x0 + j0) & 31) == 0) A.flags_other[(long long)y * A.tiles_x + ((p.x0 + j0) >> 5)] = 0;
    }
}

// A consumer warp's part of a staged segment (the threads with nodes in it):
// with SPLIT, the form of consume for the warp, from the segment's row and the
// flags of the NPT force tiles the warp covers (tiles warp * NPT .. + NPT - 1,
// all in one word of the stage's masks), a choice uniform over the warp;
// without, the general form for every warp (the barrier schedule: on the
// FP32 probe the three forms took 7% longer there, for 13% fewer
// instructions, while the producer-warp kernels gained).
template <typename S, int NPT, bool WALLS, bool SPLIT>
__device__ __forceinline__ void consume_warp(const LbArgs& A, ItemRef p, const S* sp, int tid, const uint4& fm) {
    static_assert(32 % NPT == 0, "a warp's tiles lie in one mask word");
    const int j0 = tid * NPT, q0 = (tid >> 5) * NPT;
    const int flag = flag_of(fm, j0 >> 5), flag_o = flag_other_of(fm, j0 >> 5);
    const unsigned warp_tiles = ((q0 < 32 ? fm.x : fm.y) >> (q0 & 31)) & ((1u << NPT) - 1u);
    if (!SPLIT || (WALLS && (p.y == 0 || p.y == A.ny - 1)))
        consume<S, NPT, WALLS, true, true>(A, p, sp, j0, flag, flag_o);
    else if (warp_tiles != 0u)
        consume<S, NPT, WALLS, true, false>(A, p, sp, j0, flag, flag_o);
    else
        consume<S, NPT, WALLS, false, false>(A, p, sp, j0, flag, flag_o);
}

// Producer-warp schedule (16-bit storage, batches): 288 threads.  Warps 0-7
// consume (collide the staged segment; each frees the stage for its part with
// its own arrival on the stage's "empty" barrier), warp 8 produces: lane 0
// waits for that barrier (eight arrivals once the consumers have passed the
// segment), the lanes store
// the segment's tile flags, lane 0 sets the expected bytes, then lanes 0-8
// each issue the copies of one direction.  Stage s also has a "full" barrier
// (the producer's expect-tx plus the copies' bytes).  Issuing from nine lanes
// instead of one thread keeps the producer ahead of the short 16-bit segments.
template <typename S, int NPT, bool WALLS, typename Items>
__device__ __forceinline__ void stream_ws(const Items& it) {
    using Gm = Geom<S, NPT>;
    constexpr int W = Gm::W;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bars[kStages];
    __shared__ __align__(8) unsigned long long empty[kStages];
    __shared__ uint4 s_fm[kStages];  // tile-flag masks of each stage's item (see keep_flags)
    __shared__ int s_last_issued[kStages];
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x;
    const long long n_items = it.count();
    const long long first = blockIdx.x, stride = gridDim.x;
    const int my_n = first < n_items ? (int)((n_items - 1 - first) / stride + 1) : 0;
    const uint32_t smem0 = smem_addr(smem);

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_addr(&bars[s]), 1);
            mbar_init(smem_addr(&empty[s]), kConsumerWarps);
            s_last_issued[s] = -1;
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int warp = tid >> 5, lane = tid & 31;
    if (warp == kConsumerWarps) {
        // ---- producer: stage segment k once the consumers have left the
        // segment k - kStages that used the same stage; its tile flags were
        // fetched three segments ahead (their latency stays off the producer's path)
        FlagRegs r0, r1, r2;
        r0 = r1 = r2 = FlagRegs{{0, 0}, {0, 0}, {0, 0}, 0};
        if (my_n > 0) fetch_flags<W>(it, first, lane, r0, 0);
        if (my_n > 1) fetch_flags<W>(it, first + stride, lane, r1, r0.m);
        if (my_n > 2) fetch_flags<W>(it, first + 2 * stride, lane, r2, r1.m);
        for (int k = 0; k < my_n; ++k) {
            const int stage = k % kStages;
            const long long item = first + (long long)k * stride;
            int stop = 0;
            if (lane == 0) {
                if (k >= kStages && !mbar_wait(smem_addr(&empty[stage]), (uint32_t)(((k / kStages) - 1) & 1)))
                    s_abort = 1;
                stop = s_abort;
            }
            stop = __shfl_sync(0xffffffffu, stop, 0);
            if (stop) break;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            keep_flags(r0, lane, &s_fm[stage]);
            it.stage_args(r0.p, r0.m, stage, lane);
            __syncwarp();
            const LbArgs& A = it.staged(stage);
            const ItemRef p = it.staged_pos(item, stage);
            const uint32_t bar = smem_addr(&bars[stage]);
            if (lane == 0) mbar_expect_tx(bar, stage_bytes<S, NPT>(A, p));
            __syncwarp();
            if (lane < 9) stage_rows<S, NPT, WALLS>(A, p, smem0 + stage * Gm::STAGE_BYTES, bar, lane, 9);
            if (lane == 0) s_last_issued[stage] = k;
            r0 = r1;
            r1 = r2;
            if (k + 3 < my_n) fetch_flags<W>(it, first + (long long)(k + 3) * stride, lane, r2, r1.m);
        }
    } else {
        // ---- consumers
        for (int k = 0; k < my_n; ++k) {
            const int stage = k % kStages;
            const bool ok = mbar_wait_sleep(smem_addr(&bars[stage]), (uint32_t)((k / kStages) & 1));
            const long long item = first + (long long)k * stride;
            const LbArgs& A = it.staged(stage);
            const ItemRef p = it.staged_pos(item, stage);
            const int wlen = min(W, A.nx - p.x0);
            const int j0 = tid * NPT;
            if (ok && j0 < wlen) {
                const S* sp = reinterpret_cast<const S*>(smem + stage * Gm::STAGE_BYTES);
                consume_warp<S, NPT, WALLS, true>(A, p, sp, tid, s_fm[stage]);
            }
            // each consumer warp frees its share of the stage as soon as it is
            // done with it (the stage's empty barrier counts the eight warps)
            if (!ok) {
                if ((tid & 31) == 0) s_abort = 1;
                break;
            }
            __syncwarp();
            if ((tid & 31) == 0) mbar_arrive(smem_addr(&empty[stage]));
        }
    }
    __syncthreads();
    if (s_abort && tid == 0) {
        // a wait gave up: report it, then wait (bounded) for the copies still in
        // flight (the last segment staged into each stage) before the shared
        // memory is released
        ItemRef p0;
        atomicOr(it.locate(first, p0).status, ST_TIMEOUT);
        for (int st = 0; st < kStages; ++st) {
            const int m = s_last_issued[st];
            if (m >= 0) mbar_wait(smem_addr(&bars[st]), (uint32_t)((m / kStages) & 1));
        }
    }
}

// Barrier schedule (FP32, FP64): 256 threads; a CTA barrier ends each segment;
// then warp 0 refills the stage with the segment kStages ahead: the tile flags
// it fetched at the start of this one, the arguments (batches), the expected
// bytes and the nine row copies (lanes 0-8, one direction each).
template <typename S, int NPT, bool WALLS, typename Items>
__device__ __forceinline__ void stream_bar(const Items& it) {
    using Gm = Geom<S, NPT>;
    constexpr int W = Gm::W;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bars[kStages];
    __shared__ uint4 s_fm[kStages];  // tile-flag masks of each stage's item (see keep_flags)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long n_items = it.count();
    const long long first = blockIdx.x, stride = gridDim.x;
    const int my_n = first < n_items ? (int)((n_items - 1 - first) / stride + 1) : 0;
    const uint32_t smem0 = smem_addr(smem);

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(smem_addr(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // warp 0 (all lanes): stage the k-th item of this CTA into stage k % kStages
    // (its arguments and position, then lane 0 the expected bytes, then lanes
    // 0-8 the copies of one direction each)
    auto issue = [&](int k, const FlagRegs& r) {
        const long long item = first + (long long)k * stride;
        const int stage = k % kStages;
        it.stage_args(r.p, r.m, stage, lane);
        __syncwarp();
        const LbArgs& A = it.staged(stage);
        const ItemRef p = it.staged_pos(item, stage);
        const uint32_t bar = smem_addr(&bars[stage]);
        if (lane == 0) mbar_expect_tx(bar, stage_bytes<S, NPT>(A, p));
        __syncwarp();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (lane < 9) stage_rows<S, NPT, WALLS>(A, p, smem0 + stage * Gm::STAGE_BYTES, bar, lane, 9);
    };

    // (the member hint stays 0: this schedule serves single lattices, whose
    // items have no member to search)
    if (warp == 0) {
        for (int k = 0; k < kStages && k < my_n; ++k) {
            FlagRegs r;
            fetch_flags<W>(it, first + (long long)k * stride, lane, r, 0);
            keep_flags(r, lane, &s_fm[k]);
            issue(k, r);
        }
    }
    __syncthreads();

    bool bad = false;
    int k = 0;
    for (; k < my_n; ++k) {
        const int stage = k % kStages;
        // warp 0 fetches the flags of the item it stages at the end of this one
        FlagRegs nf{{0, 0}, {0, 0}, {0, 0}, 0};
        if (warp == 0 && k + kStages < my_n) fetch_flags<W>(it, first + (long long)(k + kStages) * stride, lane, nf, 0);

        const bool ok = mbar_wait(smem_addr(&bars[stage]), (uint32_t)((k / kStages) & 1));
        const long long item = first + (long long)k * stride;
        const LbArgs& A = it.staged(stage);
        const ItemRef p = it.staged_pos(item, stage);
        const int wlen = min(W, A.nx - p.x0);
        const int j0 = tid * NPT;
        if (j0 < wlen) {
            const S* sp = reinterpret_cast<const S*>(smem + stage * Gm::STAGE_BYTES);
            consume_warp<S, NPT, WALLS, false>(A, p, sp, tid, s_fm[stage]);
        }
        // every thread is done with this stage (and every wait ended) before it is refilled
        bad = __syncthreads_or(!ok) != 0;
        if (bad) break;
        if (warp == 0 && k + kStages < my_n) {
            keep_flags(nf, lane, &s_fm[stage]);
            issue(k + kStages, nf);
        }
    }
    if (bad && tid == 0) {
        // a copy never completed: report it, then wait (bounded) for the copies
        // this CTA still has in flight before its shared memory is released
        ItemRef p0;
        atomicOr(it.locate(first + (long long)k * stride, p0).status, ST_TIMEOUT);
        for (int m = k; m < my_n && m < k + kStages; ++m)
            mbar_wait(smem_addr(&bars[m % kStages]), (uint32_t)((m / kStages) & 1));
    }
}

// ---------------------------------------------------------------- kernels
// (the producer-warp kernels are bounded to the registers of as many CTAs per
// SM as their stages fit in shared memory, at most four)
constexpr int ctas_per_sm(int smem) {
    const int c = (220 * 1024) / smem;
    return c > 4 ? 4 : (c < 1 ? 1 : c);
}
template <typename S, int NPT, bool WALLS>
__global__ void __launch_bounds__(kBlock, ctas_per_sm(Geom<S, NPT>::SMEM)) k_lb_stream_ws(const LbArgs a) {
    __shared__ ItemRef s_pos[kStages];
    stream_ws<S, NPT, WALLS>(OneLattice<S, NPT>(a, s_pos));
}
template <typename S, int NPT, bool WALLS>
__global__ void __launch_bounds__(kThreads) k_lb_stream_bar(const LbArgs a) {
    __shared__ ItemRef s_pos[kStages];
    stream_bar<S, NPT, WALLS>(OneLattice<S, NPT>(a, s_pos));
}
// batched: the segments of up to kBatchMax lattices (b.off: first item of each
// member, b.tiles_x: its segments per row)
template <typename S, int NPT, bool WALLS>
__global__ void __launch_bounds__(kBlock, ctas_per_sm(Geom<S, NPT>::SMEM))
    k_lb_stream_ws_batch(const __grid_constant__ LbBatch b) {
    __shared__ LbArgs s_args[kStages];
    __shared__ ItemRef s_pos[kStages];
    stream_ws<S, NPT, WALLS>(ManyLattices<S, NPT>{b, s_args, s_pos});
}
template <typename S, int NPT, bool WALLS>
__global__ void __launch_bounds__(kThreads) k_lb_stream_bar_batch(const __grid_constant__ LbBatch b) {
    __shared__ LbArgs s_args[kStages];
    __shared__ ItemRef s_pos[kStages];
    stream_bar<S, NPT, WALLS>(ManyLattices<S, NPT>{b, s_args, s_pos});
}

// the producer-warp schedule for 16-bit storage, the barrier schedule otherwise
// (measured on the 8192 x 2048 probe: FP32 npt 2 199 us vs 223 us; FP16 npt 4
// 158 us vs 138 us)
template <typename S>
constexpr bool kWarpSpecialised = sizeof(S) == 2;
// batches: the staging of a segment also copies its member's arguments, which
// keeps the producer warp off the consumers' path in every storage type
template <typename S>
constexpr bool kBatchWarpSpecialised = true;

template <typename S, int NPT, bool WALLS, bool BATCH>
constexpr auto stream_kernel() {
    if constexpr (BATCH) {
        if constexpr (kBatchWarpSpecialised<S>) return k_lb_stream_ws_batch<S, NPT, WALLS>;
        else return k_lb_stream_bar_batch<S, NPT, WALLS>;
    } else {
        if constexpr (kWarpSpecialised<S>) return k_lb_stream_ws<S, NPT, WALLS>;
        else return k_lb_stream_bar<S, NPT, WALLS>;
    }
}

template <typename S, int NPT, bool WALLS, bool BATCH>
cudaError_t prepare_t(int* grid) {
    auto kern = stream_kernel<S, NPT, WALLS, BATCH>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Geom<S, NPT>::SMEM);
    if (e != cudaSuccess) return e;
    const bool ws = BATCH ? kBatchWarpSpecialised<S> : kWarpSpecialised<S>;
    const int threads = ws ? kBlock : kThreads;
    int occ = 0, dev = 0, nsm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, Geom<S, NPT>::SMEM)) != cudaSuccess)
        return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    *grid = occ * nsm;
    return cudaSuccess;
}

// one entry for the four uses: prepare (grid_out) or launch, one lattice (a)
// or a batch (b)
template <typename S, int NPT>
cudaError_t dispatch(bool prepare, bool walls, int grid, int* grid_out, const LbArgs* a, const LbBatch* b,
                     cudaStream_t s) {
    const bool batch = b != nullptr;
    if (prepare) {
        if (batch) return walls ? prepare_t<S, NPT, true, true>(grid_out) : prepare_t<S, NPT, false, true>(grid_out);
        return walls ? prepare_t<S, NPT, true, false>(grid_out) : prepare_t<S, NPT, false, false>(grid_out);
    }
    const int threads = (batch ? kBatchWarpSpecialised<S> : kWarpSpecialised<S>) ? kBlock : kThreads;
    long long items;
    if (batch) {
        if (b->n < 1 || b->n > kBatchMax) return cudaErrorInvalidValue;
        items = b->off[b->n];
    } else {
        items = (long long)a->ny * ((a->nx + Geom<S, NPT>::W - 1) / Geom<S, NPT>::W);
    }
    if (items >= (1LL << 31)) return cudaErrorInvalidValue;  // item indices are 32-bit in the kernel
    const int g = (int)(items < grid ? items : grid);
    if (g <= 0) return cudaSuccess;
    constexpr int SM = Geom<S, NPT>::SMEM;
    if (batch) {
        if (walls) stream_kernel<S, NPT, true, true>()<<<g, threads, SM, s>>>(*b);
        else stream_kernel<S, NPT, false, true>()<<<g, threads, SM, s>>>(*b);
    } else {
        if (walls) stream_kernel<S, NPT, true, false>()<<<g, threads, SM, s>>>(*a);
        else stream_kernel<S, NPT, false, false>()<<<g, threads, SM, s>>>(*a);
    }
    return cudaGetLastError();
}

cudaError_t dispatch_all(lbib_precision prec, int npt, bool prepare, bool walls, int grid, int* grid_out,
                         const LbArgs* a, const LbBatch* b, cudaStream_t s) {
    switch (prec) {
        case LBIB_F64:
            if (npt == 1) return dispatch<double, 1>(prepare, walls, grid, grid_out, a, b, s);
            if (npt == 2) return dispatch<double, 2>(prepare, walls, grid, grid_out, a, b, s);
            break;
        case LBIB_F32:
            if (npt == 1) return dispatch<float, 1>(prepare, walls, grid, grid_out, a, b, s);
            if (npt == 2) return dispatch<float, 2>(prepare, walls, grid, grid_out, a, b, s);
            if (npt == 4) return dispatch<float, 4>(prepare, walls, grid, grid_out, a, b, s);
            break;
        case LBIB_F32_STORE_F16:
            if (npt == 2) return dispatch<__half, 2>(prepare, walls, grid, grid_out, a, b, s);
            if (npt == 4) return dispatch<__half, 4>(prepare, walls, grid, grid_out, a, b, s);
            if (npt == 8) return dispatch<__half, 8>(prepare, walls, grid, grid_out, a, b, s);
            break;
        case LBIB_F32_STORE_BF16:
            if (npt == 2) return dispatch<__nv_bfloat16, 2>(prepare, walls, grid, grid_out, a, b, s);
            if (npt == 4) return dispatch<__nv_bfloat16, 4>(prepare, walls, grid, grid_out, a, b, s);
            if (npt == 8) return dispatch<__nv_bfloat16, 8>(prepare, walls, grid, grid_out, a, b, s);
            break;
    }
    return cudaErrorInvalidValue;
}

}  // namespace

int lb_stream_halo(lbib_precision prec) {
    return prec == LBIB_F64 ? 2 : (prec == LBIB_F32 ? 4 : 8);
}

cudaError_t prepare_lb_stream(lbib_precision prec, int npt, bool walls, bool, int* grid) {
    return dispatch_all(prec, npt, true, walls, 0, grid, nullptr, nullptr, nullptr);
}

cudaError_t launch_lb_stream(lbib_precision prec, int npt, bool walls, bool, int grid, const LbArgs& a,
                             cudaStream_t s) {
    return dispatch_all(prec, npt, false, walls, grid, nullptr, &a, nullptr, s);
}

cudaError_t prepare_lb_stream_batch(lbib_precision prec, int npt, bool walls, int* grid) {
    LbBatch dummy;
    dummy.n = 0;
    return dispatch_all(prec, npt, true, walls, 0, grid, nullptr, &dummy, nullptr);
}

cudaError_t launch_lb_stream_batch(lbib_precision prec, int npt, bool walls, int grid, const LbBatch& b,
                                   cudaStream_t s) {
    return dispatch_all(prec, npt, false, walls, grid, nullptr, nullptr, &b, s);
}

}  // namespace lbib
