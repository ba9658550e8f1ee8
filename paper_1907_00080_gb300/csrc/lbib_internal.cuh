// Internal declarations of the lbib CUDA library (not part of the public ABI).
//
// Layout in HBM (one context):
//   populations  two buffers A/B, [9][NY][NX] of the storage type, x fastest;
//                each holds the post-collision deviations d*_i = f*_i - w_i of
//                one step (pull scheme: the fused kernel streams while reading)
//   u field      ux, uy [NY][NX] of the compute type, written by the fused
//                kernel only in tiles that IB stencils touch
//   markers      X^n, X^{n-1} as interleaved (x, y) doubles; F^n, U^n, the nine
//                shape-function weights and the stencil origin per vertex
//   IB force     two fixed-point (int64 x 2) per-node fields alternating with the
//                step parity, plus a flag per fused-kernel tile that spreading touched
//   adhesion     per ligand: element vertices, bond, candidate; per receptor:
//                position, owner, claim; receptors bucketed in a uniform grid
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lbib.h"

namespace lbib {

// ---------------------------------------------------------------- D2Q9
// Velocity set of Eq. GaussHermite: 0 rest; 1..4 axis (E, N, W, S);
// 5..8 diagonals (NE, NW, SW, SE).  Weights 4/9, 1/9, 1/36.
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5);
}
template <typename C>
__host__ __device__ constexpr C wgt(int i) {
    return i == 0 ? C(4.0 / 9.0) : (i <= 4 ? C(1.0 / 9.0) : C(1.0 / 36.0));
}
static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "axis opposites");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "diagonal opposites");

// ---------------------------------------------------------------- storage
// Conversion between stored values and the compute type; 16-bit forms carry a
// power-of-two scale: stored = d_i * 2^k, so load multiplies by inv = 2^-k and
// store by scale = 2^k (both exact).
template <typename S> struct Storage;
template <> struct Storage<double> {
    using C = double;
    __device__ static double load(double s, float) { return s; }
    __device__ static double store(double d, float) { return d; }
};
template <> struct Storage<float> {
    using C = float;
    __device__ static float load(float s, float) { return s; }
    __device__ static float store(float d, float) { return d; }
};
// 16-bit storage also converts the stored values as they are (raw, store_raw:
// for the collision on the scaled values) and in pairs (two neighbouring
// nodes' values of one direction in one step; the pair conversions round each
// value exactly as the single ones do)
template <> struct Storage<__half> {
    using C = float;
    using S2 = __half2;
    __device__ static float load(__half s, float inv) { return __half2float(s) * inv; }
    __device__ static __half store(float d, float scale) { return __float2half_rn(d * scale); }
    __device__ static float raw(__half s) { return __half2float(s); }
    __device__ static __half store_raw(float s) { return __float2half_rn(s); }
    __device__ static float2 load2(__half2 s) { return __half22float2(s); }
    __device__ static __half2 store2(float a, float b) { return __floats2half2_rn(a, b); }
};
template <> struct Storage<__nv_bfloat16> {
    using C = float;
    using S2 = __nv_bfloat162;
    __device__ static float load(__nv_bfloat16 s, float inv) { return __bfloat162float(s) * inv; }
    __device__ static __nv_bfloat16 store(float d, float scale) { return __float2bfloat16_rn(d * scale); }
    __device__ static float raw(__nv_bfloat16 s) { return __bfloat162float(s); }
    __device__ static __nv_bfloat16 store_raw(float s) { return __float2bfloat16_rn(s); }
    __device__ static float2 load2(__nv_bfloat162 s) { return __bfloat1622float2(s); }
    __device__ static __nv_bfloat162 store2(float a, float b) { return __floats2bfloat162_rn(a, b); }
};

// ---------------------------------------------------------------- kernel args
// The IB force is spread into a per-node fixed-point field (int64 pairs scaled
// by 2^52): integer addition is associative, so the atomics of the spreading
// give the same bits in any order.  Two fields alternate with the step parity;
// tiles that a step's spreading touched are flagged, and the fused kernel of
// the following step zeroes them again.
constexpr double kFixScale = 4503599627370496.0;          // 2^52
constexpr double kFixInv = 1.0 / 4503599627370496.0;      // 2^-52

struct LbArgs {
    const void* src;       // post-collision deviations of step n-1
    void* dst;             // post-collision deviations of step n
    void* ux;              // u field (compute type), written in flagged tiles
    void* uy;
    double* rho_out;       // fields mode: rho, ux, uy as doubles (may be null)
    double* ux_out;
    double* uy_out;
    const longlong2* gsum; // [N] fixed-point IB force of this step (flagged tiles)
    longlong2* gclear;     // [N] the other parity's field, zeroed in its flagged tiles
    const int* flags;      // [ntiles] force tiles (32 nodes of a row) this step's spreading touched
    int* flags_other;      // [ntiles] tiles the previous step's spreading touched
    int clear_other;       // 1 during a step, 0 for read-backs and profiling
    int nx, ny;
    double omega;          // 1/tau
    double gx, gy;         // body force
    float omf, om3f;       // omega and 3 omega rounded to FP32 (no FP64 conversion in the FP32 kernels)
    float gxf, gyf;        // the body force rounded to FP32
    float inv_scale;       // 2^-k for 16-bit storage, 1 otherwise
    double bb_bot, bb_top; // moving walls: 6 w_d u_w (w_d = 1/36) of the lower / upper wall; a
                           // diagonal population bounced back there gains cx(i) times it
    float bbf_bot, bbf_top;  // the same rounded to FP32 (no FP64 conversion in the FP32 kernels)
    int zou_he;            // 1: the walls are Zou-He wall rows y = 0, NY - 1 (bb_* are 0)
    double uw_bot, uw_top; // Zou-He: x velocities of the lower and upper wall rows
    float uwf_bot, uwf_top;
    int fields_only;       // 1: write rho/ux/uy doubles, skip populations
    int g_prefetch;        // row tiles: read the spread force of every node up front (L2-resident lattices)
    int tile_w, tile_h, tiles_x;  // force-tile geometry of the flags (32 x 1 nodes; tiles_x = ceil(nx / 32))
    int* status;           // device status word (StatusBits)
};

struct MarkerArgs {
    int nx, ny, walls;
    double inv_nx, inv_ny;    // 1/nx, 1/ny (periodic wrapping without a division)
    int nmem, nv;
    const int* mem_off;
    const int* mem_n;
    const int* mem_kind;
    const double* mem_ks;
    const double* mem_kb;
    const double* mem_ka;
    const double* mem_A0;
    const double* mem_qa;     // [nmem] k_a p_ref / A_0: the area coefficient is mem_qa (A - A_0)
    const int* mem_lig_off;   // ligands of membrane m: [lig_off[m], lig_off[m+1])
    void* X;                  // [nv] current positions (unwrapped): double (x, y) in
                              // FP64 mode, float-float {x.hi, y.hi, x.lo, y.lo} otherwise
    void* Xp;                 // [nv] previous positions, same layout
    void* F;                  // [nv][2] compute type
    void* U;                  // [nv][2] compute type
    void* W;                  // [nv][9] compute type
    int* stencil;             // [nv][2]
    const void* rest;         // [nv] rest records (32 bytes): |x_{v+1}-x_v|^2, the cross and
                              // dot products of the two edges at v, |x_{v+1}-x_v|
    const int* elem_lig;      // [nv] ligand on element (v, v+1) or -1
    // repulsion
    double d_rep;
    int nseg;
    const int* seg_mem;       // [nseg]
    const int* seg_v0;        // [nseg] first global vertex
    const int* seg_n;         // [nseg]
    float4* seg_box;          // [nseg] centre x wrapped to [0,nx), centre y, half extents
    const int* mem_seg_off;   // segments of membrane m: [mem_seg_off[m], mem_seg_off[m+1])
    // work units: (membrane, first local vertex, vertex count); the force kernel
    // cuts every membrane into chunks of kChunkV vertices, the advance kernel
    // cuts kinematic membranes the same way and keeps rigid-projected ones whole
    int nfu, nau;
    int adv_threads;          // threads per advance block: 64, or the longest rigid ring rounded up to a warp
    const int4* fu;           // [nfu][2]: {m, k0, kn, off} {n, kind, lig0, nlig} (see kUnitInts)
    const int4* au;           // [nau][2], same records
    // bonds
    int nlig, nrec;
    const int* lig_a;         // [nlig] first vertex of the ligand element
    const int* lig_b;         // [nlig] second vertex
    int* bond_of_lig;         // [nlig]
    int* cand;                // [nlig]
    int* rupt;                // [nlig]
    const double* rec_xy;     // [nrec][2] receptor positions (FP64 decisions)
    const void* rec_e;        // [nrec] the same in the marker position layout
    int* owner;               // [nrec]
    int* owner_cell;          // [nrec] the same in cell order (owner_cell[p] = owner[rcell_ids[p]])
    const int* rcell_of_rec;  // [nrec] cell-order position of receptor r
    int* claim;               // [nrec]
    const int* rcell_start;   // [ncell + 1]
    const int* rcell_ids;     // [nrec] receptor ids in cell order
    const void* rcell_pos;    // [nrec] their positions, same order, marker position layout
    int rc_nx, rc_ny;         // receptor grid
    double rc_w, rc_h, rc_y0; // cell size, y origin
    double inv_rc_w, inv_rc_h, inv_y_eq;
    double d_cut2;            // (d_cut (1 + 1e-12))^2, a conservative pre-check
    double sigma, y_eq, d_cut, d_break, kf_dt, kr0_dt, beta_f, beta_r;
    uint64_t seed, instance;
    // tiles of the fused kernel, spreading target of this step
    int tile_w, tile_h, tiles_x, tiles_y;
    longlong2* gsum;
    int* flags;
    // step counter, status and the arrival counters of the last-block epilogues
    long long* d_step;
    int* status;
    unsigned int* tickets;    // arrival counter of the advance kernel's last-block epilogue
    // u field (compute type)
    const void* ux;
    const void* uy;
    // FP32 copies of the scalar parameters (no double->float conversion in the kernels)
    struct {
        float nx, ny, inv_nx, inv_ny, sigma, y_eq, inv_y_eq, d_rep, d_cut, d_break;
        float kf_dt, kr0_dt, beta_f, beta_r, inv_rc_w, inv_rc_h, rc_y0;
    } f;
    // ligands decided by each advance unit (element inside the unit, CSR), and
    // the ligands whose element straddles two units (decided by the last block)
    const int4* au_ligs;      // {ligand, local vertex a, local vertex b, 0} per unit ligand
    int nstrad;
    const int* strad_ligs;
    // dynamic particles (Sec. 2.4): compute-type [nv][2] arrays, meaningful on
    // the vertices of dynamic membranes only
    void* V;                  // particle velocity u_p^n
    void* Hf;                 // hydrodynamic force of this step (k_hydro)
    void* Dib;                // forcing term spread into the fluid (k_hydro)
    double* rb;               // [nmem][6] rigid state: u, v, u_prev, v_prev, omega, omega_prev
    const double* mem_dyn;    // [nmem][3] mass rho_P A_0, inertia rho_P J_0, vertex mass m / n
    int has_dyn;              // 1 if any membrane is dynamic
};

// Arguments of the hydrodynamic-stress kernel: the populations the step
// starts from and what turns them into p and u
struct HydroArgs {
    const void* src;          // post-collision deviations d* of step n-1 (f^n = w + pulled d*)
    float inv_scale;
    double bb_bot, bb_top;    // moving-wall terms of the bounce-back (as in LbArgs)
    float bbf_bot, bbf_top;
    double gx, gy;            // body force (u = (sum f e + G_body / 2) / rho)
    double nu;                // (tau - 1/2) / 3
    int nunits;               // blocks: chunks of hydro_chunk() vertices of the dynamic membranes
    const int4* units;        // [nunits] {first local vertex, vertex count, membrane offset, membrane size}
};

// ST_FIXRANGE: a spread force or a repulsion magnitude left the range of its
// fixed-point accumulator (see clamp_fix)
enum StatusBits { ST_NONFINITE = 1, ST_TILE_OVERFLOW = 2, ST_TIMEOUT = 4, ST_FIXRANGE = 8 };

constexpr int kChunkV = 64;   // vertices per marker-kernel block (a multiple of 32)
constexpr int kUnitInts = 8;  // ints per work-unit record (two int4)
constexpr int kSegV = 8;      // vertices per repulsion-screening segment (divides kChunkV)

// Copy kernel arguments (a struct of the library's argument types) into
// shared memory, all threads of the block taking 8-byte words; ends with a
// block barrier.  Batched kernels stage the arguments of the member a block
// works for this way, from global memory or (generic pointer) from the
// launch's own parameters.
template <typename T>
__device__ __forceinline__ void stage_args(T* dst, const T* src) {
    static_assert(sizeof(T) % 8 == 0 && alignof(T) >= 8, "argument structs are 8-byte words");
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    for (int k = tid; k < (int)(sizeof(T) / 8); k += nt)
        reinterpret_cast<long long*>(dst)[k] = reinterpret_cast<const long long*>(src)[k];
    __syncthreads();
}

// Batched launches (ensembles): up to kBatchMax members per launch.  The block
// of a launch that a member's work starts at is off[member]; a block finds its
// member by a binary search over these offsets, which travel in the launch's
// parameters (no memory round trip before the first data load).
constexpr int kBatchMax = 64;
__device__ __forceinline__ int batch_member(const int* off, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
// fused kernel: the members' arguments themselves are parameters (192 B each)
struct LbBatch {
    int n;
    int off[kBatchMax + 1];     // row tiles: first block of each member; persistent form: first segment
    int tiles_x[kBatchMax];     // row tiles: tiles per row; persistent form: segments per row
    LbArgs a[kBatchMax];
};
// marker kernels: the members' arguments (744 B each) stay in global memory
// block -> member for the first kBlockTable blocks of a launch (one parameter
// load where a search over off[] would take several dependent ones)
constexpr int kBlockTable = 8192;
static_assert(kBatchMax <= 255, "members fit the byte table");
struct MarkerBatch {
    int n;
    int off[kBatchMax + 1];     // first block of each member's units
    const MarkerArgs* args;     // [n]
    unsigned char member[kBlockTable];  // member of block b < min(off[n], kBlockTable)
};
__device__ __forceinline__ int marker_member(const MarkerBatch& b, int blk) {
    return blk < kBlockTable ? (int)b.member[blk] : batch_member(b.off, b.n, blk);
}

// ---------------------------------------------------------------- launchers
// lb_kernels.cu
cudaError_t launch_lb_step(lbib_precision prec, int vec, int ty, bool walls, bool has_ib,
                           const LbArgs& a, cudaStream_t s);
// batched row tiles of up to kBatchMax lattices with markers, all with the
// tile shape (vec, ty); b.off[b.n] blocks
cudaError_t launch_lb_batch(lbib_precision prec, int vec, int ty, bool walls, const LbBatch& b, cudaStream_t s);
// lb_stream_kernel.cu: the persistent bulk-copy form of the fused kernel (one
// CTA per SM slot streams row segments of 256 * npt nodes through a 4-stage
// shared-memory pipeline); prepare_ sets its shared-memory limit and returns
// the grid size, outside any stream capture
int lb_stream_halo(lbib_precision prec);  // elements per 16-byte halo chunk
cudaError_t prepare_lb_stream(lbib_precision prec, int npt, bool walls, bool has_ib, int* grid);
cudaError_t launch_lb_stream(lbib_precision prec, int npt, bool walls, bool has_ib, int grid,
                             const LbArgs& a, cudaStream_t s);
// the persistent form over the segments of up to kBatchMax lattices (b.off:
// first segment of each member, b.tiles_x: its segments per row)
cudaError_t prepare_lb_stream_batch(lbib_precision prec, int npt, bool walls, int* grid);
cudaError_t launch_lb_stream_batch(lbib_precision prec, int npt, bool walls, int grid, const LbBatch& b,
                                   cudaStream_t s);
// walls: 0 periodic, 1 bounce-back (bb_* the moving-wall terms), 2 Zou-He (uw_* the wall
// velocities; the unknown populations of the wall rows rebuilt without a force)
cudaError_t launch_stream_out(lbib_precision prec, const void* src, double* out, int nx, int ny,
                              int walls, float inv_scale, double bb_bot, double bb_top, double uw_bot,
                              double uw_top, cudaStream_t s);
cudaError_t launch_stream_in(lbib_precision prec, const double* in, void* dst, int nx, int ny,
                             bool walls, float inv_scale, double bb_bot, double bb_top, cudaStream_t s);
cudaError_t launch_init_rest_walls(lbib_precision prec, void* dst, int nx, int ny, double bb_bot, double bb_top,
                                   float inv_scale, cudaStream_t s);
cudaError_t launch_init_couette(lbib_precision prec, void* dst, int nx, int ny, double u_bot, double u_top,
                                float inv_scale, cudaStream_t s);
cudaError_t launch_init_poiseuille(lbib_precision prec, void* dst, int nx, int ny, double tau,
                                   double gx, float inv_scale, cudaStream_t s);
cudaError_t launch_mass(lbib_precision prec, const void* src, long long n_elems, double* partials,
                        int n_partials, double* out, float inv_scale, cudaStream_t s);
// ib_kernels.cu
cudaError_t launch_rest(lbib_precision prec, const MarkerArgs& a, void* rest, double* A0, double* qa,
                        cudaStream_t s);
cudaError_t launch_forces(lbib_precision prec, const MarkerArgs& a, int max_n, cudaStream_t s);
cudaError_t launch_advance(lbib_precision prec, const MarkerArgs& a, cudaStream_t s);
// batched marker kernels of up to kBatchMax contexts (b.off[b.n] blocks); the
// advance blocks have `threads` threads (the widest member's)
cudaError_t launch_forces_batch(lbib_precision prec, const MarkerBatch& b, cudaStream_t s);
cudaError_t launch_advance_batch(lbib_precision prec, bool dyn, const MarkerBatch& b, int threads, cudaStream_t s);
cudaError_t launch_seg_boxes(lbib_precision prec, const MarkerArgs& a, cudaStream_t s);
cudaError_t launch_areas(lbib_precision prec, const MarkerArgs& a, double* areas, cudaStream_t s);
// dynamic_kernels.cu: hydrodynamic stresses and forcing terms of the dynamic
// particles at the start of a step (before launch_forces)
cudaError_t launch_hydro(lbib_precision prec, const MarkerArgs& a, const HydroArgs& h, cudaStream_t s);
int hydro_chunk(lbib_precision prec);  // vertices per block of the hydrodynamic kernel
// observables.cu: 8 doubles per membrane (see lbib_membrane_observables)
cudaError_t launch_observables(lbib_precision prec, const MarkerArgs& a, double* out, cudaStream_t s);
cudaError_t launch_pos_in(lbib_precision prec, const double* xy, void* X, int nv, cudaStream_t s);
cudaError_t launch_pos_out(lbib_precision prec, const void* X, double* xy, int nv, cudaStream_t s);

}  // namespace lbib

// ---------------------------------------------------------------- context
struct lbib_ctx {
    int nx = 0, ny = 0;
    lbib_precision prec = LBIB_F32;
    lbib_init init = LBIB_INIT_REST;
    double tau = 1.0, gx = 0.0, gy = 0.0;
    lbib_walls walls = LBIB_WALLS_Y_BOUNCEBACK;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t pop_elem = 4;      // bytes per stored population
    size_t cmp_elem = 4;      // bytes per compute-type value
    int scale_exp = 0;        // 16-bit storage scale 2^k
    float inv_scale = 1.0f;
    double uw_bot = 0.0, uw_top = 0.0;  // x velocities of the lower and upper walls

    void* f[2] = {nullptr, nullptr};
    int cur = 0;              // buffer holding d*^{n-1}
    void* ux = nullptr;
    void* uy = nullptr;
    double* stage = nullptr;  // 9*N doubles, lazily allocated for read/write
    double* partials = nullptr;
    double* dscalar = nullptr; // small device scratch for results
    int n_partials = 0;

    int vec = 0, ty = 0;      // tiling of the fused kernel (ty = 0: persistent bulk-copy form, vec = npt)
    int stream_grid = 0;      // CTAs of the persistent form (SMs x resident CTAs)
    int tile_w = 0, tile_h = 0, tiles_x = 0, tiles_y = 0, ntiles = 0;

    // host-side membrane staging
    std::vector<double> h_xy;
    std::vector<int> h_mem_off, h_mem_n, h_mem_kind, h_lig_elem_local, h_mem_lig_off;
    std::vector<double> h_ks, h_kb, h_ka;
    std::vector<double> h_rhop;   // rho_P / rho of each membrane (dynamic ones)
    int nmem = 0, nv = 0, nlig = 0;
    int ndyn = 0;                 // dynamic membranes
    int4* d_hydro_units = nullptr; // chunks of their vertices (in the arena)
    int n_hydro_units = 0;
    // receptors
    std::vector<double> h_rec;
    lbib_bond_params bp{};
    bool have_receptors = false;
    double d_rep = 2.0;

    // device marker state (allocated at finalize)
    bool finalized = false;
    int max_mem_n = 0;
    int nseg = 0;
    void* dmem = nullptr;     // one arena for all marker / tile / bond arrays
    size_t dmem_bytes = 0;
    lbib::MarkerArgs ma{};
    longlong2* G[2] = {nullptr, nullptr};   // fixed-point IB force fields (by parity)
    int* flags[2] = {nullptr, nullptr};      // spread-touched tiles (by parity)
    double* d_areas = nullptr;
    double* xy_stage = nullptr;             // 2*nv doubles for marker read/write
    double* d_obs = nullptr;                // 8*nmem doubles of membrane observables (lazy)
    unsigned int* tickets = nullptr;

    long long* d_step = nullptr;
    int* d_status = nullptr;
    long long steps = 0;
    bool fields_valid = false;
    bool poisoned = false;

    // captured step graphs: [start buffer][0: one step, 1: chunk of kChunk steps]
    cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    cudaGraph_t graph_tmpl[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // kept for ensembles
    bool graphs_ready = false;
    bool no_g_prefetch = false;  // set for ensemble members (see lb_args)

    std::string err;
};
