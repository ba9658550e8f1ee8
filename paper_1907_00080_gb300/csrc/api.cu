// C ABI of the lbib library: context set-up, device arena, captured step
// graphs, ensembles and read-backs.  Every step of the time integration runs
// in the CUDA kernels of lb_kernels.cu / lb_stream_kernel.cu, ib_kernels.cu
// and advance_kernel.cu; this file only arranges memory, validates arguments
// and enqueues work.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "lbib_internal.cuh"
#include "adjoint.cuh"
#include "slabs.cuh"
#include "tangent.cuh"

using namespace lbib;

namespace {

constexpr int kChunk = 16;  // steps per captured chunk graph (even)
constexpr int kMaxGridY = 65535;  // largest y extent of a launch grid

lbib_status fail(lbib_ctx* c, lbib_status st, const std::string& msg) {
    if (c) c->err = msg;
    return st;
}

lbib_status cuda_fail(lbib_ctx* c, cudaError_t e, const char* where) {
    if (c) c->err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? LBIB_E_OOM : LBIB_E_CUDA;
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);     \
    } while (0)

size_t elem_size(lbib_precision p) {
    switch (p) {
        case LBIB_F64: return 8;
        case LBIB_F32: return 4;
        default: return 2;
    }
}

bool is_dynamic(int kind) { return kind == LBIB_MEMBRANE_DYNAMIC || kind == LBIB_MEMBRANE_DYNAMIC_RIGID; }
// membranes advanced by one block over the whole ring (their sums span it)
bool whole_ring(int kind) { return kind == LBIB_MEMBRANE_RIGID_PROJECTED || kind == LBIB_MEMBRANE_DYNAMIC_RIGID; }

// Area A_0 and polar second moment J_0 about the area centroid of a rest
// polygon (CCW, xy interleaved), summed over the triangles (vertex 0, v, v+1):
// with a, b their corners relative to vertex 0 and c = a x b, the triangle has
// area c/2, centroid (a + b)/3 and polar moment c (|a|^2 + a.b + |b|^2)/12
// about vertex 0; the parallel-axis theorem moves the sum to the centroid.
// A_0 is the shoelace sum about vertex 0 the rest of the library uses.
void rest_mass_properties(int n, const double* xy, double* A0, double* J0) {
    double sa = 0.0, s2 = 0.0, sx = 0.0, sy = 0.0, sj = 0.0;
    const double xr = xy[0], yr = xy[1];
    for (int v = 0; v < n; ++v) {
        const int w = (v + 1) % n;
        const double ax = xy[2 * v] - xr, ay = xy[2 * v + 1] - yr;
        const double bx = xy[2 * w] - xr, by = xy[2 * w + 1] - yr;
        sa += ax * by - bx * ay;
        const double c = ax * by - ay * bx;
        s2 += c;
        sx += c * (ax + bx);
        sy += c * (ay + by);
        sj += c * ((ax * ax + ay * ay) + (ax * bx + ay * by) + (bx * bx + by * by));
    }
    const double area = 0.5 * s2;
    const double gx = sx / (3.0 * s2), gy = sy / (3.0 * s2);
    *A0 = 0.5 * sa;
    *J0 = sj / 12.0 - area * (gx * gx + gy * gy);
}

struct Arena {
    char* base = nullptr;
    size_t used = 0;
    template <typename T>
    T* take(size_t n) {
        used = (used + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base + used);
        used += sizeof(T) * (n ? n : 1);
        return p;
    }
};

bool valid_vec(lbib_precision p, int vec, int nx) {
    if (vec <= 0 || nx % vec) return false;
    switch (p) {
        case LBIB_F64: return vec == 1 || vec == 2;
        case LBIB_F32: return vec == 1 || vec == 2 || vec == 4;
        default: return vec == 2 || vec == 4 || vec == 8;
    }
}

// persistent bulk-copy form: npt nodes per thread (segments of 256 npt nodes);
// rows must split into whole 16-byte chunks
bool valid_stream(lbib_precision p, int npt, int nx) {
    if (nx % lb_stream_halo(p)) return false;
    switch (p) {
        case LBIB_F64: return npt == 1 || npt == 2;
        case LBIB_F32: return npt == 1 || npt == 2 || npt == 4;
        default: return npt == 2 || npt == 4 || npt == 8;
    }
}

void default_tiling(const lbib_ctx* c, int* vec, int* ty) {
    // lattices whose two population buffers exceed L2 (129 MB) stream through
    // the persistent bulk-copy form, which keeps enough bytes in flight for DRAM
    // (FP64 stays on row tiles: it is bound by the FP64 pipe, not by DRAM)
    const double two_buffers = 2.0 * 9.0 * (double)c->pop_elem * c->nx * c->ny;
    const int npt = c->prec == LBIB_F32 ? 2 : 4;
    if (c->prec != LBIB_F64 && two_buffers > 128e6 && valid_stream(c->prec, npt, c->nx)) {
        *vec = npt;
        *ty = 0;
        return;
    }
    const long long nodes = (long long)c->nx * c->ny;
    // 16-bit storage from a million nodes on: the row tiles' occupancy is capped
    // by registers and they wait on their loads, while the persistent form's
    // bulk copies keep the bytes in flight (512-node segments for L2-sized lattices)
    const bool half = c->prec == LBIB_F32_STORE_F16 || c->prec == LBIB_F32_STORE_BF16;
    if (half && nodes >= (1LL << 20) && valid_stream(c->prec, 2, c->nx)) {
        *vec = 2;
        *ty = 0;
        return;
    }
    int v = c->prec == LBIB_F64 ? 2 : 4;
    while (v > 1 && !valid_vec(c->prec, v, c->nx)) v /= 2;
    const long long N = (long long)c->nx * c->ny;
    // small lattices: fewer nodes per thread so that every SM has warps to switch between
    while (v > 1 && N / v < 152LL * 1024 && valid_vec(c->prec, v / 2, c->nx)) v /= 2;
    const long long tiles_x = (c->nx + 32LL * v - 1) / (32LL * v);
    // large lattices: two rows per block (one-warp blocks would hit the limit of
    // 32 resident blocks per SM); small ones: up to 4 rows while the grid still
    // has four blocks per SM (the 640 x 160 capillary measured fastest at 4 rows)
    int t = N >= (1LL << 20) ? 2 : 4;
    while (t > 1 && tiles_x * ((c->ny + t - 1) / t) < 152LL * 4) t /= 2;
    // the grid's y extent (rows / t) is limited to 65535 blocks
    while (t < 16 && (c->ny + t - 1) / t > kMaxGridY) t *= 2;
    *vec = v;
    *ty = t;
}

}  // namespace

// ------------------------------------------------------------------ create
// FP16 storage: scale the deviations so that the expected peak (a few times
// the Poiseuille peak deviation w_1 * 3 u_max, or the largest wall velocity's)
// sits near 2^12
void choose_scale(lbib_ctx* c) {
    if (c->prec != LBIB_F32_STORE_F16) return;
    const double nu = (c->tau - 0.5) / 3.0;
    const double umax = std::max(1e-12, std::fabs(c->gx) * (double)c->ny * c->ny / (8.0 * nu) +
                                             std::fabs(c->gy) * (double)c->nx * c->nx / (8.0 * nu) +
                                             std::max(std::fabs(c->uw_bot), std::fabs(c->uw_top)));
    const double dmax = std::max(umax / 3.0, 1e-9);
    int k = (int)std::floor(std::log2(4096.0 / dmax));
    k = std::max(0, std::min(k, 40));
    c->scale_exp = k;
    c->inv_scale = std::ldexp(1.0f, -k);
}

double bb_term(double u_wall);

// the initial state in f[0]: rest (pre-collision f_i = w_i), or the
// post-collision state of the Poiseuille or Couette fixed point
cudaError_t init_populations(lbib_ctx* c) {
    const size_t N = (size_t)c->nx * c->ny;
    cudaError_t e = cudaMemsetAsync(c->f[0], 0, 9 * N * c->pop_elem, c->stream);
    if (e == cudaSuccess && c->init == LBIB_INIT_REST && c->walls == LBIB_WALLS_Y_BOUNCEBACK &&
        (c->uw_bot != 0.0 || c->uw_top != 0.0))
        e = launch_init_rest_walls(c->prec, c->f[0], c->nx, c->ny, bb_term(c->uw_bot), bb_term(c->uw_top),
                                   c->inv_scale, c->stream);
    if (e == cudaSuccess && c->init == LBIB_INIT_POISEUILLE)
        e = launch_init_poiseuille(c->prec, c->f[0], c->nx, c->ny, c->tau, c->gx, c->inv_scale, c->stream);
    if (e == cudaSuccess && c->init == LBIB_INIT_COUETTE)
        e = launch_init_couette(c->prec, c->f[0], c->nx, c->ny, c->uw_bot, c->uw_top, c->inv_scale, c->stream);
    return e;
}

// momentum a moving wall gives a bounced-back diagonal population: 6 w_d u_w
double bb_term(double u_wall) { return 6.0 * (1.0 / 36.0) * u_wall; }

extern "C" lbib_status lbib_create(const lbib_lattice* lat, double tau, const double body_force[2],
                                   lbib_walls walls, void* cuda_stream, lbib_ctx** out) {
    if (!lat || !out) return LBIB_E_INVALID;
    *out = nullptr;
    if (lat->nx < 4 || lat->ny < 4) return LBIB_E_INVALID;
    if (!(tau > 0.5)) return LBIB_E_INVALID;
    if (lat->prec < LBIB_F64 || lat->prec > LBIB_F32_STORE_BF16) return LBIB_E_INVALID;
    if (walls != LBIB_WALLS_NONE && walls != LBIB_WALLS_Y_BOUNCEBACK && walls != LBIB_WALLS_ZOU_HE)
        return LBIB_E_INVALID;
    if (lat->init == LBIB_INIT_POISEUILLE && (walls != LBIB_WALLS_Y_BOUNCEBACK || tau != 1.0))
        return LBIB_E_INVALID;
    if (lat->init == LBIB_INIT_COUETTE && walls != LBIB_WALLS_Y_BOUNCEBACK) return LBIB_E_INVALID;
    if (lat->init < LBIB_INIT_REST || lat->init > LBIB_INIT_COUETTE) return LBIB_E_INVALID;
    if (lat->prec != LBIB_F64 && lat->prec != LBIB_F32 && (lat->nx % 2)) return LBIB_E_INVALID;
    lbib_ctx* c = new lbib_ctx();
    c->nx = lat->nx;
    c->ny = lat->ny;
    c->prec = lat->prec;
    c->init = lat->init;
    c->tau = tau;
    c->gx = body_force ? body_force[0] : 0.0;
    c->gy = body_force ? body_force[1] : 0.0;
    c->walls = walls;
    c->pop_elem = elem_size(c->prec);
    c->cmp_elem = c->prec == LBIB_F64 ? 8 : 4;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return LBIB_E_CUDA;
    }
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return LBIB_E_CUDA;
        }
        c->own_stream = true;
    }
    choose_scale(c);
    const size_t N = (size_t)c->nx * c->ny;
    cudaError_t e;
    for (int b = 0; b < 2; ++b) {
        e = cudaMalloc(&c->f[b], 9 * N * c->pop_elem);
        if (e != cudaSuccess) {
            lbib_destroy(c);
            return LBIB_E_OOM;
        }
    }
    e = cudaMalloc(&c->ux, N * c->cmp_elem);
    if (e == cudaSuccess) e = cudaMalloc(&c->uy, N * c->cmp_elem);
    c->n_partials = 1024;
    if (e == cudaSuccess) e = cudaMalloc(&c->partials, sizeof(double) * c->n_partials);
    if (e == cudaSuccess) e = cudaMalloc(&c->dscalar, sizeof(double) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_step, sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(int));
    if (e != cudaSuccess) {
        lbib_destroy(c);
        return LBIB_E_OOM;
    }
    e = cudaMemsetAsync(c->ux, 0, N * c->cmp_elem, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->uy, 0, N * c->cmp_elem, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_step, 0, sizeof(long long), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = init_populations(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        lbib_destroy(c);
        return LBIB_E_CUDA;
    }
    c->cur = 0;
    *out = c;
    return LBIB_OK;
}

extern "C" lbib_status lbib_add_membrane(lbib_ctx* c, const double* xy, int32_t n, double k_s,
                                         double k_b, double k_area, lbib_kind kind,
                                         const int32_t* ligand_elems, int32_t n_ligands,
                                         int32_t* membrane_id_out) {
    if (!c) return LBIB_E_INVALID;
    if (c->finalized) return fail(c, LBIB_E_STATE, "membranes must be added before the first step");
    if (!xy || n < 3) return fail(c, LBIB_E_INVALID, "a membrane needs >= 3 vertices");
    if (kind != LBIB_MEMBRANE_KINEMATIC && kind != LBIB_MEMBRANE_RIGID_PROJECTED &&
        kind != LBIB_MEMBRANE_DYNAMIC && kind != LBIB_MEMBRANE_DYNAMIC_RIGID)
        return fail(c, LBIB_E_INVALID, "unknown membrane kind");
    if (whole_ring(kind) && n > 4 * kChunkV)
        return fail(c, LBIB_E_INVALID, "rigid-projected and rigid dynamic membranes are limited to 256 vertices");
    if (is_dynamic(kind) && c->walls == LBIB_WALLS_ZOU_HE)
        return fail(c, LBIB_E_INVALID, "dynamic particles need half-way or no walls");
    if (n_ligands < 0 || (n_ligands > 0 && !ligand_elems))
        return fail(c, LBIB_E_INVALID, "ligand list");
    for (int k = 0; k < 2 * n; ++k)
        if (!std::isfinite(xy[k])) return fail(c, LBIB_E_INVALID, "non-finite vertex");
    std::vector<char> used(n, 0);
    for (int k = 0; k < n_ligands; ++k) {
        if (ligand_elems[k] < 0 || ligand_elems[k] >= n) return fail(c, LBIB_E_INVALID, "ligand element out of range");
        if (used[ligand_elems[k]]) return fail(c, LBIB_E_INVALID, "at most one ligand per element");
        used[ligand_elems[k]] = 1;
    }
    const int m = c->nmem;
    c->h_mem_off.push_back(c->nv);
    c->h_mem_n.push_back(n);
    c->h_mem_kind.push_back((int)kind);
    c->h_ks.push_back(k_s);
    c->h_kb.push_back(k_b);
    c->h_ka.push_back(k_area);
    c->h_rhop.push_back(1.1);  // rho_P / rho of the particles (Sec. 3)
    if (kind == LBIB_MEMBRANE_DYNAMIC || kind == LBIB_MEMBRANE_DYNAMIC_RIGID) c->ndyn += 1;
    c->h_xy.insert(c->h_xy.end(), xy, xy + 2 * n);
    if (c->h_mem_lig_off.empty()) c->h_mem_lig_off.push_back(0);
    for (int k = 0; k < n_ligands; ++k) c->h_lig_elem_local.push_back(c->nv + ligand_elems[k]);
    c->nlig += n_ligands;
    c->h_mem_lig_off.push_back(c->nlig);
    c->nv += n;
    c->nmem += 1;
    c->max_mem_n = std::max(c->max_mem_n, n);
    if (membrane_id_out) *membrane_id_out = m;
    return LBIB_OK;
}

extern "C" lbib_status lbib_set_receptors(lbib_ctx* c, const double* xy, int32_t n,
                                          const lbib_bond_params* p) {
    if (!c) return LBIB_E_INVALID;
    if (c->finalized) return fail(c, LBIB_E_STATE, "receptors must be set before the first step");
    if (n < 0 || (n > 0 && !xy) || !p) return fail(c, LBIB_E_INVALID, "receptor arguments");
    if (n > 0 && c->walls == LBIB_WALLS_NONE) return fail(c, LBIB_E_INVALID, "receptors need walls");
    if (!(p->d_cut > 0.0) || !(p->y_eq > 0.0) || !(p->d_break > 0.0))
        return fail(c, LBIB_E_INVALID, "bond lengths must be positive");
    for (int k = 0; k < 2 * n; ++k)
        if (!std::isfinite(xy[k])) return fail(c, LBIB_E_INVALID, "non-finite receptor");
    c->h_rec.assign(xy, xy + 2 * n);
    c->bp = *p;
    c->have_receptors = true;
    return LBIB_OK;
}

extern "C" lbib_status lbib_set_repulsion(lbib_ctx* c, double d_rep) {
    if (!c || !(d_rep >= 0.0)) return LBIB_E_INVALID;
    c->d_rep = d_rep;
    return LBIB_OK;
}

extern "C" lbib_status lbib_set_wall_velocity(lbib_ctx* c, double u_bottom, double u_top) {
    if (!c) return LBIB_E_INVALID;
    if (c->walls == LBIB_WALLS_NONE) return fail(c, LBIB_E_INVALID, "moving walls need walls");
    if (!std::isfinite(u_bottom) || !std::isfinite(u_top)) return fail(c, LBIB_E_INVALID, "non-finite wall velocity");
    if (c->graphs_ready || c->steps > 0) return fail(c, LBIB_E_STATE, "wall velocities are fixed at the first step");
    c->uw_bot = u_bottom;
    c->uw_top = u_top;
    choose_scale(c);
    c->cur = 0;
    CK(init_populations(c));
    CK(cudaStreamSynchronize(c->stream));
    c->fields_valid = false;
    return LBIB_OK;
}

extern "C" lbib_status lbib_set_tiling(lbib_ctx* c, int32_t vec, int32_t ty) {
    if (!c) return LBIB_E_INVALID;
    if (c->finalized) return fail(c, LBIB_E_STATE, "tiling is fixed at the first step");
    if (vec == 0 && ty == 0) {
        c->vec = c->ty = 0;
        return LBIB_OK;
    }
    const bool ok = ty == 0 ? valid_stream(c->prec, vec, c->nx)
                            : (valid_vec(c->prec, vec, c->nx) && ty >= 1 && ty <= 16 && (c->ny + ty - 1) / ty <= kMaxGridY);
    if (!ok) return fail(c, LBIB_E_INVALID, "unsupported tiling");
    c->vec = vec;
    c->ty = ty;
    return LBIB_OK;
}

extern "C" lbib_status lbib_get_tiling(const lbib_ctx* c, int32_t* vec, int32_t* ty) {
    if (!c || !vec || !ty) return LBIB_E_INVALID;
    if (c->vec) {
        *vec = c->vec;
        *ty = c->ty;
    } else {
        default_tiling(c, vec, ty);
    }
    return LBIB_OK;
}

// ------------------------------------------------------------------ finalize
static lbib_status finalize(lbib_ctx* c) {
    if (c->finalized) return LBIB_OK;
    if (!c->vec) default_tiling(c, &c->vec, &c->ty);
    if (c->ty == 0) {
        CK(prepare_lb_stream(c->prec, c->vec, c->walls != LBIB_WALLS_NONE, c->nv > 0, &c->stream_grid));
    } else {
        if ((c->ny + c->ty - 1) / c->ty > kMaxGridY)
            return fail(c, LBIB_E_INVALID, "lattice too tall for the row-tile form: more than 65535 x 16 rows");
    }
    // force flags per 32 nodes of a row, in both kernel forms: a flagged tile
    // reads and later clears the spread force and writes u only there (with
    // tiles of a whole block or segment, red cells that cross most of them
    // made nearly every node pay those 40 bytes)
    c->tile_w = 32;
    c->tile_h = 1;
    c->tiles_x = (c->nx + c->tile_w - 1) / c->tile_w;
    c->tiles_y = (c->ny + c->tile_h - 1) / c->tile_h;
    c->ntiles = c->tiles_x * c->tiles_y;

    const int nv = c->nv, nm = c->nmem, nl = c->nlig;
    const int nr = c->have_receptors ? (int)(c->h_rec.size() / 2) : 0;
    // repulsion-screening segments of kSegV consecutive vertices per membrane
    std::vector<int> seg_mem, seg_v0, seg_n, mem_seg_off(nm + 1, 0);
    for (int m = 0; m < nm; ++m) {
        mem_seg_off[m] = (int)seg_mem.size();
        for (int s = 0; s < c->h_mem_n[m]; s += kSegV) {
            seg_mem.push_back(m);
            seg_v0.push_back(c->h_mem_off[m] + s);
            seg_n.push_back(std::min(kSegV, c->h_mem_n[m] - s));
        }
    }
    mem_seg_off[nm] = (int)seg_mem.size();
    c->nseg = (int)seg_mem.size();
    // ligand element vertices and element -> ligand map
    std::vector<int> lig_a(nl), lig_b(nl), elem_lig(std::max(nv, 1), -1), vmem(std::max(nv, 1));
    for (int m = 0; m < nm; ++m)
        for (int k = 0; k < c->h_mem_n[m]; ++k) vmem[c->h_mem_off[m] + k] = m;
    for (int l = 0; l < nl; ++l) {
        const int a = c->h_lig_elem_local[l];
        const int m = vmem[a];
        lig_a[l] = a;
        lig_b[l] = c->h_mem_off[m] + (a - c->h_mem_off[m] + 1) % c->h_mem_n[m];
        elem_lig[a] = l;
    }
    std::vector<int> mem_lig_off = c->h_mem_lig_off;
    if (mem_lig_off.empty()) mem_lig_off.assign(nm + 1, 0);
    // receptor grid: cells at least d_cut wide so a 3x3 block covers the cut-off disc
    int rc_nx = 1, rc_ny = 1;
    double rc_w = c->nx, rc_h = 1.0, rc_y0 = 0.0;
    std::vector<int> rcell_start(2, 0), rcell_ids;
    if (nr > 0) {
        const double dc = c->bp.d_cut;
        rc_nx = std::max(1, (int)std::floor(c->nx / dc));
        rc_w = (double)c->nx / rc_nx;
        double ymin = 1e300, ymax = -1e300;
        for (int r = 0; r < nr; ++r) {
            ymin = std::min(ymin, c->h_rec[2 * r + 1]);
            ymax = std::max(ymax, c->h_rec[2 * r + 1]);
        }
        const double span = ymax - ymin;
        rc_ny = std::max(1, (int)std::floor(span / dc));
        rc_h = span > 0 ? std::max(span / rc_ny, dc) : dc;
        rc_y0 = ymin;
        std::vector<int> cell(nr);
        std::vector<int> cnt((size_t)rc_nx * rc_ny + 1, 0);
        for (int r = 0; r < nr; ++r) {
            const double x = c->h_rec[2 * r] - c->nx * std::floor(c->h_rec[2 * r] / c->nx);
            int gx = std::min(rc_nx - 1, (int)std::floor(x / rc_w));
            int gy = std::min(rc_ny - 1, std::max(0, (int)std::floor((c->h_rec[2 * r + 1] - rc_y0) / rc_h)));
            cell[r] = gy * rc_nx + gx;
            cnt[cell[r] + 1]++;
        }
        for (size_t k = 1; k < cnt.size(); ++k) cnt[k] += cnt[k - 1];
        rcell_start = cnt;
        rcell_ids.assign(nr, 0);
        std::vector<int> cur(cnt.begin(), cnt.end() - 1);
        for (int r = 0; r < nr; ++r) rcell_ids[cur[cell[r]]++] = r;  // ascending id within a cell
    }
    // work units, kUnitInts ints each (one 32-byte read per block):
    // {membrane, first local vertex, vertex count, membrane offset, membrane size,
    //  kind, then for force units the membrane's first segment, for advance
    //  units the first ligand record and the number of ligand records}
    std::vector<int> fu, au;
    for (int m = 0; m < nm; ++m) {
        const int n = c->h_mem_n[m], off = c->h_mem_off[m], kind = c->h_mem_kind[m];
        for (int k0 = 0; k0 < n; k0 += kChunkV) {
            fu.insert(fu.end(), {m, k0, std::min(kChunkV, n - k0), off, n, kind, mem_seg_off[m], 0});
            if (!whole_ring(kind)) au.insert(au.end(), {m, k0, std::min(kChunkV, n - k0), off, n, kind, 0, 0});
        }
        if (whole_ring(kind)) au.insert(au.end(), {m, 0, n, off, n, kind, 0, 0});
    }
    // ligands decided inside each advance unit (both element vertices in it),
    // as records {ligand, local index of its element's two vertices, 0}, and
    // the straddling rest, decided by the kernel's last block
    const int nau = (int)(au.size() / kUnitInts);
    std::vector<int> au_ligs, strad;
    {
        std::vector<std::vector<int>> per(nau);
        std::vector<int> unit_of(std::max(nv, 1), -1);
        for (int q = 0; q < nau; ++q) {
            const int* u = &au[kUnitInts * q];
            for (int k = 0; k < u[2]; ++k) unit_of[u[3] + u[1] + k] = q;
        }
        for (int l = 0; l < nl; ++l) {
            const int ua = unit_of[lig_a[l]], ub = unit_of[lig_b[l]];
            if (ua == ub) per[ua].push_back(l);
            else strad.push_back(l);
        }
        for (int q = 0; q < nau; ++q) {
            int* u = &au[kUnitInts * q];
            u[6] = (int)(au_ligs.size() / 4);
            u[7] = (int)per[q].size();  // <= vertices of the unit <= 4 kChunkV (one per advance thread)
            for (int l : per[q]) au_ligs.insert(au_ligs.end(), {l, lig_a[l] - u[3] - u[1], lig_b[l] - u[3] - u[1], 0});
        }
    }

    // dynamic particles: mass rho_P A_0, inertia rho_P J_0 (J_0 the polar moment
    // of the rest polygon about its area centroid) and vertex mass per membrane
    // and the blocks of the hydrodynamic kernel, {k0, count, membrane offset, membrane size}
    std::vector<double> dyn_consts(3 * (size_t)std::max(nm, 1), 0.0);
    std::vector<int> hydro_units;
    for (int m = 0; m < nm; ++m) {
        if (!is_dynamic(c->h_mem_kind[m])) continue;
        const int n = c->h_mem_n[m];
        const int hc = hydro_chunk(c->prec);
        for (int k0 = 0; k0 < n; k0 += hc)
            hydro_units.insert(hydro_units.end(), {k0, std::min(hc, n - k0), c->h_mem_off[m], n});
        const double* p = c->h_xy.data() + 2 * (size_t)c->h_mem_off[m];
        double A0, J0;
        rest_mass_properties(n, p, &A0, &J0);
        dyn_consts[3 * m] = c->h_rhop[m] * A0;
        dyn_consts[3 * m + 1] = c->h_rhop[m] * J0;
        dyn_consts[3 * m + 2] = c->h_rhop[m] * A0 / n;
    }

    // ---- one arena for every marker / tile / bond array
    const size_t cs = c->cmp_elem;
    size_t bytes = 0;
    {
        Arena probe;
        probe.base = nullptr;
        auto add = [&](size_t b) { probe.used = ((probe.used + 255) & ~size_t(255)) + (b ? b : 1); };
        add(4 * (nm + 1)); add(4 * (nm + 1)); add(4 * (nm + 1)); add(8 * (nm + 1)); add(8 * (nm + 1));
        add(8 * (nm + 1)); add(8 * (nm + 1)); add(8 * (nm + 1)); add(4 * (nm + 2));
        add(16 * nv); add(16 * nv); add(2 * cs * nv); add(2 * cs * nv); add(9 * cs * nv); add(8 * nv);
        add(32 * nv); add(4 * nv); add(16 * nv + 16 * nr);
        add(4 * c->nseg); add(4 * c->nseg); add(4 * c->nseg); add(16 * c->nseg); add(4 * (nm + 1));
        add(4 * nl); add(4 * nl); add(4 * nl); add(4 * nl); add(4 * nl);
        add(16 * nr); add(16 * nr); add(4 * nr); add(4 * nr); add(4 * rcell_start.size()); add(4 * rcell_ids.size()); add(16 * nr);
        add(4 * nr); add(4 * nr);
        add(4 * c->ntiles); add(4 * c->ntiles); add(8 * (nm + 1)); add(16);
        add(4 * fu.size()); add(4 * au.size());
        add(4 * au_ligs.size()); add(4 * strad.size());
        add(2 * cs * nv); add(2 * cs * nv); add(2 * cs * nv); add(48 * (nm + 1)); add(24 * (nm + 1));
        add(4 * hydro_units.size());
        bytes = probe.used + 256;
    }
    lbib_status st = LBIB_OK;
    cudaError_t e = cudaMalloc(&c->dmem, bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, "arena");
    c->dmem_bytes = bytes;
    Arena ar;
    ar.base = static_cast<char*>(c->dmem);
    MarkerArgs& a = c->ma;
    a = MarkerArgs{};
    a.nx = c->nx; a.ny = c->ny; a.walls = c->walls != LBIB_WALLS_NONE ? 1 : 0;
    a.inv_nx = 1.0 / c->nx; a.inv_ny = 1.0 / c->ny;
    a.nmem = nm; a.nv = nv;
    int* mem_off = ar.take<int>(nm + 1);
    int* mem_n = ar.take<int>(nm + 1);
    int* mem_kind = ar.take<int>(nm + 1);
    double* ks = ar.take<double>(nm + 1);
    double* kb = ar.take<double>(nm + 1);
    double* ka = ar.take<double>(nm + 1);
    double* A0 = ar.take<double>(nm + 1);
    double* qa = ar.take<double>(nm + 1);
    int* lig_off = ar.take<int>(nm + 2);
    a.X = ar.take<double>(2 * (size_t)nv);   // 16 bytes per vertex in either layout
    a.Xp = ar.take<double>(2 * (size_t)nv);
    c->xy_stage = ar.take<double>(2 * (size_t)nv + 2 * (size_t)nr);
    a.F = ar.take<char>(2 * cs * nv);
    a.U = ar.take<char>(2 * cs * nv);
    a.W = ar.take<char>(9 * cs * nv);
    a.stencil = ar.take<int>(2 * (size_t)nv);
    double* rest = ar.take<double>(4 * (size_t)nv);
    int* elig = ar.take<int>(nv);
    int* d_seg_mem = ar.take<int>(c->nseg);
    int* d_seg_v0 = ar.take<int>(c->nseg);
    int* d_seg_n = ar.take<int>(c->nseg);
    a.seg_box = ar.take<float4>(c->nseg);
    int* d_mem_seg_off = ar.take<int>(nm + 1);
    int* d_lig_a = ar.take<int>(nl);
    int* d_lig_b = ar.take<int>(nl);
    a.bond_of_lig = ar.take<int>(nl);
    a.cand = ar.take<int>(nl);
    a.rupt = ar.take<int>(nl);
    double* rec_xy = ar.take<double>(2 * (size_t)nr);
    void* rec_e = ar.take<double>(2 * (size_t)nr);
    a.owner = ar.take<int>(nr);
    a.owner_cell = ar.take<int>(nr);
    int* d_rcell_of_rec = ar.take<int>(nr);
    a.claim = ar.take<int>(nr);
    int* d_rcs = ar.take<int>(rcell_start.size());
    int* d_rci = ar.take<int>(rcell_ids.size());
    void* d_rcpos = ar.take<double>(2 * (size_t)nr);
    c->flags[0] = ar.take<int>(c->ntiles);
    c->flags[1] = ar.take<int>(c->ntiles);
    c->d_areas = ar.take<double>(nm + 1);
    c->tickets = ar.take<unsigned int>(4);
    int* d_fu = ar.take<int>(fu.size());
    int* d_au = ar.take<int>(au.size());
    int* d_au_ligs = ar.take<int>(au_ligs.size());
    int* d_strad = ar.take<int>(strad.size());
    void* V = ar.take<char>(2 * cs * nv);
    void* Hf = ar.take<char>(2 * cs * nv);
    void* Dib = ar.take<char>(2 * cs * nv);
    double* rb = ar.take<double>(6 * (size_t)(nm + 1));
    double* mem_dyn = ar.take<double>(3 * (size_t)(nm + 1));
    int* d_hydro_units = ar.take<int>(hydro_units.size());
    if (ar.used > bytes) return fail(c, LBIB_E_STATE, "internal arena sizing error");

    auto H2D = [&](void* d, const void* h, size_t b) -> cudaError_t {
        if (b == 0) return cudaSuccess;
        return cudaMemcpyAsync(d, h, b, cudaMemcpyHostToDevice, c->stream);
    };
    std::vector<double> zeros;
    if (nm > 0) {
        CK(H2D(mem_off, c->h_mem_off.data(), 4 * nm));
        CK(H2D(mem_n, c->h_mem_n.data(), 4 * nm));
        CK(H2D(mem_kind, c->h_mem_kind.data(), 4 * nm));
        CK(H2D(ks, c->h_ks.data(), 8 * nm));
        CK(H2D(kb, c->h_kb.data(), 8 * nm));
        CK(H2D(ka, c->h_ka.data(), 8 * nm));
        CK(H2D(lig_off, mem_lig_off.data(), 4 * (nm + 1)));
        CK(H2D(c->xy_stage, c->h_xy.data(), 16 * (size_t)nv));
        CK(launch_pos_in(c->prec, c->xy_stage, a.X, nv, c->stream));
        CK(launch_pos_in(c->prec, c->xy_stage, a.Xp, nv, c->stream));
        CK(cudaMemsetAsync(a.F, 0, 2 * cs * nv, c->stream));
        CK(cudaMemsetAsync(a.U, 0, 2 * cs * nv, c->stream));
        CK(H2D(elig, elem_lig.data(), 4 * (size_t)nv));
        CK(H2D(d_seg_mem, seg_mem.data(), 4 * seg_mem.size()));
        CK(H2D(d_seg_v0, seg_v0.data(), 4 * seg_v0.size()));
        CK(H2D(d_seg_n, seg_n.data(), 4 * seg_n.size()));
        CK(H2D(d_mem_seg_off, mem_seg_off.data(), 4 * (nm + 1)));
        CK(H2D(d_fu, fu.data(), 4 * fu.size()));
        CK(H2D(d_au, au.data(), 4 * au.size()));
        if (!au_ligs.empty()) CK(H2D(d_au_ligs, au_ligs.data(), 4 * au_ligs.size()));
        if (!strad.empty()) CK(H2D(d_strad, strad.data(), 4 * strad.size()));
        CK(cudaMemsetAsync(V, 0, 2 * cs * nv, c->stream));
        CK(cudaMemsetAsync(Hf, 0, 2 * cs * nv, c->stream));
        CK(cudaMemsetAsync(Dib, 0, 2 * cs * nv, c->stream));
        CK(cudaMemsetAsync(rb, 0, 48 * (size_t)nm, c->stream));
        CK(H2D(mem_dyn, dyn_consts.data(), 24 * (size_t)nm));
        if (!hydro_units.empty()) CK(H2D(d_hydro_units, hydro_units.data(), 4 * hydro_units.size()));
        CK(cudaStreamSynchronize(c->stream));  // dyn_consts, hydro_units leave scope
    }
    if (nl > 0) {
        CK(H2D(d_lig_a, lig_a.data(), 4 * nl));
        CK(H2D(d_lig_b, lig_b.data(), 4 * nl));
        CK(cudaMemsetAsync(a.bond_of_lig, 0xFF, 4 * nl, c->stream));
        CK(cudaMemsetAsync(a.cand, 0xFF, 4 * nl, c->stream));
        CK(cudaMemsetAsync(a.rupt, 0xFF, 4 * nl, c->stream));
    }
    if (nr > 0) {
        CK(H2D(rec_xy, c->h_rec.data(), 16 * (size_t)nr));
        CK(launch_pos_in(c->prec, rec_xy, rec_e, nr, c->stream));
        CK(cudaMemsetAsync(a.owner, 0xFF, 4 * nr, c->stream));
        CK(cudaMemsetAsync(a.owner_cell, 0xFF, 4 * nr, c->stream));
        CK(cudaMemsetAsync(a.claim, 0x7F, 4 * nr, c->stream));  // 0x7F7F7F7F: no claim
    }
    CK(H2D(d_rcs, rcell_start.data(), 4 * rcell_start.size()));
    if (!rcell_ids.empty()) {
        CK(H2D(d_rci, rcell_ids.data(), 4 * rcell_ids.size()));
        std::vector<int> rcell_of_rec(nr);
        for (int p = 0; p < nr; ++p) rcell_of_rec[rcell_ids[p]] = p;
        CK(H2D(d_rcell_of_rec, rcell_of_rec.data(), 4 * nr));
        // receptor positions permuted into cell order (staged through xy_stage)
        std::vector<double> rp(2 * (size_t)nr);
        for (int p = 0; p < nr; ++p) {
            rp[2 * p] = c->h_rec[2 * rcell_ids[p]];
            rp[2 * p + 1] = c->h_rec[2 * rcell_ids[p] + 1];
        }
        CK(H2D(c->xy_stage, rp.data(), 16 * (size_t)nr));
        CK(launch_pos_in(c->prec, c->xy_stage, d_rcpos, nr, c->stream));
        CK(cudaStreamSynchronize(c->stream));  // rp leaves scope
    }
    CK(cudaMemsetAsync(c->flags[0], 0, 4 * c->ntiles, c->stream));
    CK(cudaMemsetAsync(c->flags[1], 0, 4 * c->ntiles, c->stream));
    CK(cudaMemsetAsync(c->tickets, 0, 16, c->stream));
    if (nv > 0) {
        const size_t gb = sizeof(longlong2) * (size_t)c->nx * c->ny;
        for (int p = 0; p < 2; ++p) {
            CK(cudaMalloc(&c->G[p], gb));
            CK(cudaMemsetAsync(c->G[p], 0, gb, c->stream));
        }
    }

    a.mem_off = mem_off; a.mem_n = mem_n; a.mem_kind = mem_kind;
    a.mem_ks = ks; a.mem_kb = kb; a.mem_ka = ka; a.mem_A0 = A0; a.mem_qa = qa; a.mem_lig_off = lig_off;
    a.rest = rest; a.elem_lig = elig;
    a.d_rep = c->d_rep; a.nseg = c->nseg;
    a.seg_mem = d_seg_mem; a.seg_v0 = d_seg_v0; a.seg_n = d_seg_n; a.mem_seg_off = d_mem_seg_off;
    a.nfu = (int)(fu.size() / kUnitInts); a.nau = nau;
    // advance blocks: one thread per vertex of the longest rigid ring, at least
    // a chunk; small blocks leave room for other work (ensembles) on the SMs
    {
        int longest = kChunkV;
        for (int m = 0; m < nm; ++m)
            if (whole_ring(c->h_mem_kind[m])) longest = std::max(longest, c->h_mem_n[m]);
        a.adv_threads = (longest + 31) / 32 * 32;
    }
    // dynamic particles: states at rest, the ids for the hydrodynamic kernel
    a.V = V; a.Hf = Hf; a.Dib = Dib; a.rb = rb; a.mem_dyn = mem_dyn; a.has_dyn = c->ndyn > 0 ? 1 : 0;
    c->d_hydro_units = reinterpret_cast<int4*>(d_hydro_units);
    c->n_hydro_units = (int)(hydro_units.size() / 4);
    a.fu = reinterpret_cast<const int4*>(d_fu);
    a.au = reinterpret_cast<const int4*>(d_au);
    a.au_ligs = reinterpret_cast<const int4*>(d_au_ligs);
    a.nstrad = (int)strad.size(); a.strad_ligs = d_strad;
    a.nlig = nl; a.nrec = nr; a.lig_a = d_lig_a; a.lig_b = d_lig_b;
    a.rec_xy = rec_xy; a.rec_e = rec_e; a.rcell_start = d_rcs; a.rcell_ids = d_rci; a.rcell_pos = d_rcpos;
    a.rcell_of_rec = d_rcell_of_rec;
    a.rc_nx = rc_nx; a.rc_ny = rc_ny; a.rc_w = rc_w; a.rc_h = rc_h; a.rc_y0 = rc_y0;
    a.inv_rc_w = 1.0 / rc_w; a.inv_rc_h = 1.0 / rc_h;
    a.inv_y_eq = c->bp.y_eq > 0 ? 1.0 / c->bp.y_eq : 0.0;
    a.d_cut2 = (c->bp.d_cut * (1.0 + 1e-12)) * (c->bp.d_cut * (1.0 + 1e-12));
    a.sigma = c->bp.sigma; a.y_eq = c->bp.y_eq; a.d_cut = c->bp.d_cut; a.d_break = c->bp.d_break;
    a.kf_dt = c->bp.kf_dt; a.kr0_dt = c->bp.kr0_dt; a.beta_f = c->bp.beta_f; a.beta_r = c->bp.beta_r;
    a.seed = c->bp.seed; a.instance = c->bp.instance;
    a.tile_w = c->tile_w; a.tile_h = c->tile_h; a.tiles_x = c->tiles_x; a.tiles_y = c->tiles_y;
    a.d_step = c->d_step; a.status = c->d_status; a.tickets = c->tickets;
    a.f.nx = (float)c->nx; a.f.ny = (float)c->ny; a.f.inv_nx = (float)a.inv_nx; a.f.inv_ny = (float)a.inv_ny;
    a.f.sigma = (float)a.sigma; a.f.y_eq = (float)a.y_eq; a.f.inv_y_eq = (float)a.inv_y_eq;
    a.f.d_rep = (float)a.d_rep; a.f.d_cut = (float)a.d_cut; a.f.d_break = (float)a.d_break;
    a.f.kf_dt = (float)a.kf_dt; a.f.kr0_dt = (float)a.kr0_dt; a.f.beta_f = (float)a.beta_f;
    a.f.beta_r = (float)a.beta_r; a.f.inv_rc_w = (float)a.inv_rc_w; a.f.inv_rc_h = (float)a.inv_rc_h;
    a.f.rc_y0 = (float)a.rc_y0;
    a.ux = c->ux; a.uy = c->uy;

    if (nm > 0) {
        CK(launch_rest(c->prec, a, rest, A0, qa, c->stream));
        CK(launch_seg_boxes(c->prec, a, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    c->finalized = true;
    return st;
}

// ------------------------------------------------------------------ one step
static LbArgs lb_args(const lbib_ctx* c, int src, int gpar, int clear_other) {
    LbArgs l{};
    l.src = c->f[src];
    l.dst = c->f[1 - src];
    l.ux = c->ux;
    l.uy = c->uy;
    l.gsum = c->G[gpar];
    l.gclear = c->G[1 - gpar];
    l.flags = c->flags[gpar];
    l.flags_other = c->flags[1 - gpar];
    l.clear_other = clear_other;
    l.nx = c->nx;
    l.ny = c->ny;
    l.omega = 1.0 / c->tau;
    l.gx = c->gx;
    l.gy = c->gy;
    l.omf = (float)l.omega;
    l.om3f = (float)(3.0 * l.omega);
    l.gxf = (float)l.gx;
    l.gyf = (float)l.gy;
    l.inv_scale = c->inv_scale;
    // half-way walls: the moving-wall term of the bounced-back diagonals;
    // Zou-He wall rows: the wall velocities themselves
    const bool zh = c->walls == LBIB_WALLS_ZOU_HE;
    l.bb_bot = zh ? 0.0 : bb_term(c->uw_bot);
    l.bb_top = zh ? 0.0 : bb_term(c->uw_top);
    l.bbf_bot = (float)l.bb_bot;
    l.bbf_top = (float)l.bb_top;
    l.zou_he = zh ? 1 : 0;
    l.uw_bot = zh ? c->uw_bot : 0.0;
    l.uw_top = zh ? c->uw_top : 0.0;
    l.uwf_bot = (float)l.uw_bot;
    l.uwf_top = (float)l.uw_top;
    l.fields_only = 0;
    // the two population buffers and the force field well inside the 129 MB L2
    // (not for ensemble members: together they leave L2, and the extra reads
    // cost DRAM bandwidth)
    l.g_prefetch = !c->no_g_prefetch &&
                   (size_t)c->nx * c->ny * (2 * 9 * c->pop_elem + sizeof(longlong2)) <= (size_t)64 << 20;
    l.tile_w = c->tile_w;
    l.tile_h = c->tile_h;
    l.tiles_x = c->tiles_x;
    l.status = c->d_status;
    if (c->nv == 0) {
        l.flags = nullptr;
        l.flags_other = nullptr;
    }
    return l;
}

// the hydrodynamic-stress kernel's view of the populations in buffer `src`
static HydroArgs hydro_args(const lbib_ctx* c, int src) {
    HydroArgs h{};
    h.src = c->f[src];
    h.inv_scale = c->inv_scale;
    h.bb_bot = bb_term(c->uw_bot);
    h.bb_top = bb_term(c->uw_top);
    h.bbf_bot = (float)h.bb_bot;
    h.bbf_top = (float)h.bb_top;
    h.gx = c->gx;
    h.gy = c->gy;
    h.nu = (c->tau - 0.5) / 3.0;
    h.nunits = c->n_hydro_units;
    h.units = c->d_hydro_units;
    return h;
}

// the fused collide-stream kernel in the context's form
static cudaError_t launch_fused(const lbib_ctx* c, const LbArgs& l, cudaStream_t s) {
    const bool walls = c->walls != LBIB_WALLS_NONE;
    if (c->ty == 0) return launch_lb_stream(c->prec, c->vec, walls, c->nv > 0, c->stream_grid, l, s);
    return launch_lb_step(c->prec, c->vec, c->ty, walls, c->nv > 0, l, s);
}

// one time step from population buffer `src`: forces + weights + spreading,
// fused collide-stream, interpolation + advance, bond kinetics
static cudaError_t enqueue_step(lbib_ctx* c, int src, cudaStream_t s) {
    MarkerArgs a = c->ma;
    a.gsum = c->G[src];
    a.flags = c->flags[src];
    cudaError_t e;
    const bool has_ib = c->nv > 0;
    if (c->ndyn > 0 && (e = launch_hydro(c->prec, a, hydro_args(c, src), s)) != cudaSuccess) return e;
    if (has_ib && (e = launch_forces(c->prec, a, c->max_mem_n, s)) != cudaSuccess) return e;
    const LbArgs l = lb_args(c, src, src, 1);
    if ((e = launch_fused(c, l, s)) != cudaSuccess) return e;
    if (has_ib && (e = launch_advance(c->prec, a, s)) != cudaSuccess) return e;
    return cudaSuccess;
}

// discard the captured step graphs (they are captured again on next use)
static void drop_graphs(lbib_ctx* c) {
    for (int s = 0; s < 2; ++s)
        for (int k = 0; k < 2; ++k) {
            if (c->graph[s][k]) cudaGraphExecDestroy(c->graph[s][k]);
            if (c->graph_tmpl[s][k]) cudaGraphDestroy(c->graph_tmpl[s][k]);
            c->graph[s][k] = nullptr;
            c->graph_tmpl[s][k] = nullptr;
        }
    c->graphs_ready = false;
}

static lbib_status build_graphs(lbib_ctx* c) {
    if (c->graphs_ready) return LBIB_OK;
    cudaStream_t cap;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    for (int start = 0; start < 2; ++start) {
        for (int kind = 0; kind < 2; ++kind) {
            cudaGraph_t g;
            cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) {
                cudaStreamDestroy(cap);
                return cuda_fail(c, e, "begin capture");
            }
            const int nsteps = kind == 0 ? 1 : kChunk;
            int src = start;
            cudaError_t le = cudaSuccess;
            for (int k = 0; k < nsteps && le == cudaSuccess; ++k) {
                le = enqueue_step(c, src, cap);
                src = 1 - src;
            }
            e = cudaStreamEndCapture(cap, &g);
            if (le != cudaSuccess || e != cudaSuccess) {
                cudaStreamDestroy(cap);
                return cuda_fail(c, le != cudaSuccess ? le : e, "capture step");
            }
            e = cudaGraphInstantiate(&c->graph[start][kind], g, 0);
            c->graph_tmpl[start][kind] = g;  // an ensemble embeds it as a child graph
            if (e != cudaSuccess) {
                cudaStreamDestroy(cap);
                return cuda_fail(c, e, "instantiate step graph");
            }
        }
    }
    cudaStreamDestroy(cap);
    c->graphs_ready = true;
    return LBIB_OK;
}

extern "C" lbib_status lbib_step(lbib_ctx* c, int64_t n) {
    if (!c || n < 0) return LBIB_E_INVALID;
    if (c->poisoned) return fail(c, LBIB_E_STATE, "context poisoned by an earlier device-side failure");
    lbib_status st = finalize(c);
    if (st != LBIB_OK) return st;
    st = build_graphs(c);
    if (st != LBIB_OK) return st;
    int64_t left = n;
    while (left >= kChunk) {
        CK(cudaGraphLaunch(c->graph[c->cur][1], c->stream));
        left -= kChunk;  // even number of steps: the buffer roles are unchanged
    }
    while (left > 0) {
        CK(cudaGraphLaunch(c->graph[c->cur][0], c->stream));
        c->cur = 1 - c->cur;
        --left;
    }
    c->steps += n;
    if (n > 0) c->fields_valid = true;
    return LBIB_OK;
}

extern "C" lbib_status lbib_sync(lbib_ctx* c) {
    if (!c) return LBIB_E_INVALID;
    CK(cudaStreamSynchronize(c->stream));
    int st = 0;
    CK(cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & ST_NONFINITE) {
        c->poisoned = true;
        return fail(c, LBIB_E_NONFINITE, "a marker position became non-finite");
    }
    if (st & ST_FIXRANGE) {
        c->poisoned = true;
        return fail(c, LBIB_E_NONFINITE,
                    "a spread marker force (|w F| >= 64 lu per node) or a repulsion magnitude (>= 1, membranes "
                    "overlapping) left its fixed-point range or was not finite");
    }
    if (st & ST_TIMEOUT) {
        c->poisoned = true;
        return fail(c, LBIB_E_TIMEOUT, "a bulk copy of the fused kernel never completed");
    }
    return LBIB_OK;
}

extern "C" int64_t lbib_step_count(const lbib_ctx* c) { return c ? c->steps : -1; }

extern "C" int32_t lbib_kernels_per_step(const lbib_ctx* c) {
    if (!c) return -1;
    // forces with spreading, fused LB, interpolation + advance + bond kinetics,
    // and the hydrodynamic stresses when there are dynamic particles
    return c->nv > 0 ? (c->ndyn > 0 ? 4 : 3) : 1;
}

extern "C" int32_t lbib_storage_scale_exponent(const lbib_ctx* c) { return c ? c->scale_exp : 0; }

// ------------------------------------------------------------------ read / write
static lbib_status ensure_stage(lbib_ctx* c) {
    if (c->stage) return LBIB_OK;
    CK(cudaMalloc(&c->stage, 9 * sizeof(double) * (size_t)c->nx * c->ny));
    return LBIB_OK;
}

extern "C" lbib_status lbib_read_fields(lbib_ctx* c, double* rho, double* ux, double* uy, int on_device) {
    if (!c) return LBIB_E_INVALID;
    if (!c->fields_valid) return fail(c, LBIB_E_STATE, "no completed step since the populations were set");
    lbib_status st = finalize(c);
    if (st != LBIB_OK) return st;
    const size_t N = (size_t)c->nx * c->ny;
    double *dr = rho, *du = ux, *dv = uy;
    if (!on_device) {
        if ((st = ensure_stage(c)) != LBIB_OK) return st;
        dr = rho ? c->stage : nullptr;
        du = ux ? c->stage + N : nullptr;
        dv = uy ? c->stage + 2 * N : nullptr;
    }
    // recompute rho^n, u^n from the buffer the last step read, with its force field
    LbArgs l = lb_args(c, 1 - c->cur, 1 - c->cur, 0);
    l.dst = nullptr;
    l.rho_out = dr;
    l.ux_out = du;
    l.uy_out = dv;
    l.fields_only = 1;
    // the row-tile kernel serves the read-back in either form (it looks the
    // force flags up by the context's tile geometry)
    const int rv = c->ty != 0 ? c->vec : (c->prec == LBIB_F32_STORE_F16 || c->prec == LBIB_F32_STORE_BF16 ? 2 : 1);
    int rt = c->ty != 0 ? c->ty : 4;
    while (rt < 16 && (c->ny + rt - 1) / rt > kMaxGridY) rt *= 2;
    CK(launch_lb_step(c->prec, rv, rt, c->walls != LBIB_WALLS_NONE, c->nv > 0, l, c->stream));
    if (!on_device) {
        if (rho) CK(cudaMemcpyAsync(rho, dr, N * 8, cudaMemcpyDeviceToHost, c->stream));
        if (ux) CK(cudaMemcpyAsync(ux, du, N * 8, cudaMemcpyDeviceToHost, c->stream));
        if (uy) CK(cudaMemcpyAsync(uy, dv, N * 8, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return LBIB_OK;
}

extern "C" lbib_status lbib_read_populations(lbib_ctx* c, double* f, int on_device) {
    if (!c || !f) return LBIB_E_INVALID;
    const size_t N = (size_t)c->nx * c->ny;
    lbib_status st;
    double* out = f;
    if (!on_device) {
        if ((st = ensure_stage(c)) != LBIB_OK) return st;
        out = c->stage;
    }
    const bool zh = c->walls == LBIB_WALLS_ZOU_HE;
    CK(launch_stream_out(c->prec, c->f[c->cur], out, c->nx, c->ny, (int)c->walls, c->inv_scale,
                         zh ? 0.0 : bb_term(c->uw_bot), zh ? 0.0 : bb_term(c->uw_top), c->uw_bot, c->uw_top,
                         c->stream));
    if (!on_device) CK(cudaMemcpyAsync(f, out, 9 * N * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LBIB_OK;
}

// the upload of a context's populations, enqueued on stream s (no wait)
static lbib_status write_populations_on(lbib_ctx* c, const double* f, int on_device, cudaStream_t s) {
    const size_t N = (size_t)c->nx * c->ny;
    lbib_status st;
    const double* in = f;
    if (!on_device) {
        if ((st = ensure_stage(c)) != LBIB_OK) return st;
        CK(cudaMemcpyAsync(c->stage, f, 9 * N * 8, cudaMemcpyHostToDevice, s));
        in = c->stage;
    }
    // Zou-He walls: the slots the wall rows would stream out through are
    // never pulled; the bounce-back inverse fills them harmlessly
    const bool zh = c->walls == LBIB_WALLS_ZOU_HE;
    CK(launch_stream_in(c->prec, in, c->f[c->cur], c->nx, c->ny, c->walls != LBIB_WALLS_NONE, c->inv_scale,
                        zh ? 0.0 : bb_term(c->uw_bot), zh ? 0.0 : bb_term(c->uw_top), s));
    c->fields_valid = false;
    return LBIB_OK;
}

extern "C" lbib_status lbib_write_populations(lbib_ctx* c, const double* f, int on_device) {
    if (!c || !f) return LBIB_E_INVALID;
    const lbib_status st = write_populations_on(c, f, on_device, c->stream);
    if (st != LBIB_OK) return st;
    CK(cudaStreamSynchronize(c->stream));
    return LBIB_OK;
}

// the read-back of marker positions, enqueued on stream s (no wait)
static lbib_status read_markers_on(lbib_ctx* c, int32_t m, double* xy, cudaStream_t s) {
    lbib_status st = finalize(c);
    if (st != LBIB_OK) return st;
    if (c->nv == 0) return LBIB_OK;
    const int off = m < 0 ? 0 : c->h_mem_off[m];
    const int n = m < 0 ? c->nv : c->h_mem_n[m];
    CK(launch_pos_out(c->prec, c->ma.X, c->xy_stage, c->nv, s));
    CK(cudaMemcpyAsync(xy, c->xy_stage + 2 * (size_t)off, 16 * (size_t)n, cudaMemcpyDeviceToHost, s));
    return LBIB_OK;
}

extern "C" lbib_status lbib_read_markers(lbib_ctx* c, int32_t m, double* xy) {
    if (!c || !xy || m < -1 || m >= c->nmem) return LBIB_E_INVALID;
    const lbib_status st = read_markers_on(c, m, xy, c->stream);
    if (st != LBIB_OK) return st;
    CK(cudaStreamSynchronize(c->stream));
    return LBIB_OK;
}

// the upload of marker positions X^n and X^{n-1}, enqueued on stream s (no wait)
static lbib_status write_markers_on(lbib_ctx* c, const double* xy, const double* xy_prev, cudaStream_t s) {
    lbib_status st = finalize(c);
    if (st != LBIB_OK) return st;
    if (c->nv == 0) return LBIB_OK;
    const size_t b = 16 * (size_t)c->nv;
    CK(cudaMemcpyAsync(c->xy_stage, xy, b, cudaMemcpyHostToDevice, s));
    CK(launch_pos_in(c->prec, c->xy_stage, c->ma.X, c->nv, s));
    // X^{n-1} = X^n: the staged copy serves both
    if (xy_prev && xy_prev != xy) CK(cudaMemcpyAsync(c->xy_stage, xy_prev, b, cudaMemcpyHostToDevice, s));
    CK(launch_pos_in(c->prec, c->xy_stage, c->ma.Xp, c->nv, s));
    CK(launch_seg_boxes(c->prec, c->ma, s));
    return LBIB_OK;
}

extern "C" lbib_status lbib_write_markers(lbib_ctx* c, const double* xy, const double* xy_prev) {
    if (!c || !xy) return LBIB_E_INVALID;
    const lbib_status st = write_markers_on(c, xy, xy_prev, c->stream);
    if (st != LBIB_OK) return st;
    CK(cudaStreamSynchronize(c->stream));
    return LBIB_OK;
}

template <typename C>
static void widen(const std::vector<char>& raw, double* out, size_t n) {
    const C* p = reinterpret_cast<const C*>(raw.data());
    for (size_t k = 0; k < n; ++k) out[k] = (double)p[k];
}

static lbib_status read_cvec(lbib_ctx* c, const void* dptr, double* out) {
    if (!out) return LBIB_E_INVALID;
    lbib_status st = finalize(c);
    if (st != LBIB_OK) return st;
    if (c->nv == 0) return LBIB_OK;
    const size_t n = 2 * (size_t)c->nv;
    std::vector<char> raw(n * c->cmp_elem);
    CK(cudaMemcpyAsync(raw.data(), dptr, raw.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (c->cmp_elem == 8) widen<double>(raw, out, n);
    else widen<float>(raw, out, n);
    return LBIB_OK;
}

extern "C" lbib_status lbib_read_marker_forces(lbib_ctx* c, double* fxy) {
    if (!c) return LBIB_E_INVALID;
    lbib_status st = finalize(c);
    if (st != LBIB_OK) return st;
    return read_cvec(c, c->ma.F, fxy);
}

extern "C" lbib_status lbib_set_particle_density(lbib_ctx* c, int32_t m, double rho_ratio) {
    if (!c) return LBIB_E_INVALID;
    if (c->finalized) return fail(c, LBIB_E_STATE, "particle densities must be set before the first step");
    if (m < 0 || m >= c->nmem || !is_dynamic(c->h_mem_kind[m]))
        return fail(c, LBIB_E_INVALID, "not a dynamic membrane");
    if (!(rho_ratio > 0.0) || !std::isfinite(rho_ratio)) return fail(c, LBIB_E_INVALID, "density ratio");
    c->h_rhop[m] = rho_ratio;
    return LBIB_OK;
}

extern "C" lbib_status lbib_read_particle_velocity(lbib_ctx* c, int32_t m, double* uv) {
    if (!c || !uv) return LBIB_E_INVALID;
    if (m < 0 || m >= c->nmem || !is_dynamic(c->h_mem_kind[m]))
        return fail(c, LBIB_E_INVALID, "not a dynamic membrane");
    std::vector<double> all(2 * (size_t)c->nv);
    lbib_status st = read_cvec(c, c->ma.V, all.data());
    if (st != LBIB_OK) return st;
    std::copy(all.begin() + 2 * (size_t)c->h_mem_off[m],
              all.begin() + 2 * (size_t)(c->h_mem_off[m] + c->h_mem_n[m]), uv);
    return LBIB_OK;
}

extern "C" lbib_status lbib_read_marker_velocity(lbib_ctx* c, double* uxy) {
    if (!c) return LBIB_E_INVALID;
    lbib_status st = finalize(c);
    if (st != LBIB_OK) return st;
    return read_cvec(c, c->ma.U, uxy);
}

extern "C" lbib_status lbib_read_bonds(lbib_ctx* c, int32_t* lig, int32_t* rec, int32_t cap, int32_t* n_out) {
    if (!c || cap < 0 || (cap > 0 && (!lig || !rec))) return LBIB_E_INVALID;
    lbib_status st = finalize(c);
    if (st != LBIB_OK) return st;
    std::vector<int> b(c->nlig);
    if (c->nlig > 0) {
        CK(cudaMemcpyAsync(b.data(), c->ma.bond_of_lig, 4 * (size_t)c->nlig, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    int cnt = 0;
    for (int l = 0; l < c->nlig; ++l) {
        if (b[l] < 0) continue;
        if (cnt < cap) {
            lig[cnt] = l;
            rec[cnt] = b[l];
        }
        ++cnt;
    }
    if (n_out) *n_out = cnt;
    return LBIB_OK;
}

extern "C" lbib_status lbib_diagnostics(lbib_ctx* c, double* mass, double* areas) {
    if (!c) return LBIB_E_INVALID;
    lbib_status st = finalize(c);
    if (st != LBIB_OK) return st;
    if (mass) {
        const long long n = 9LL * c->nx * c->ny;
        CK(launch_mass(c->prec, c->f[c->cur], n, c->partials, c->n_partials, c->dscalar, c->inv_scale,
                       c->stream));
        CK(cudaMemcpyAsync(mass, c->dscalar, 8, cudaMemcpyDeviceToHost, c->stream));
    }
    if (areas && c->nmem > 0) {
        CK(launch_areas(c->prec, c->ma, c->d_areas, c->stream));
        CK(cudaMemcpyAsync(areas, c->d_areas, 8 * (size_t)c->nmem, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return LBIB_OK;
}

extern "C" lbib_status lbib_membrane_observables(lbib_ctx* c, double* out) {
    if (!c || !out) return LBIB_E_INVALID;
    lbib_status st = finalize(c);
    if (st != LBIB_OK) return st;
    if (c->nmem == 0) return LBIB_OK;
    if (!c->d_obs) CK(cudaMalloc(&c->d_obs, 8 * sizeof(double) * (size_t)c->nmem));
    CK(launch_observables(c->prec, c->ma, c->d_obs, c->stream));
    CK(cudaMemcpyAsync(out, c->d_obs, 8 * sizeof(double) * (size_t)c->nmem, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LBIB_OK;
}

extern "C" lbib_status lbib_profile_fused(lbib_ctx* c, int32_t reps, double* ms_per_launch) {
    if (!c || reps < 1 || !ms_per_launch) return LBIB_E_INVALID;
    if (!c->finalized || c->steps == 0) return fail(c, LBIB_E_STATE, "profile after at least one step");
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // the force field of the last completed step stays fixed for every launch
    const int gpar = 1 - c->cur;
    LbArgs l = lb_args(c, c->cur, gpar, 0);
    CK(cudaEventRecord(e0, c->stream));
    for (int r = 0; r < reps; ++r) {
        l.src = c->f[c->cur];
        l.dst = c->f[1 - c->cur];
        l.gsum = c->G[gpar];
        l.flags = c->nv > 0 ? c->flags[gpar] : nullptr;
        CK(launch_fused(c, l, c->stream));
        c->cur = 1 - c->cur;
    }
    CK(cudaEventRecord(e1, c->stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_per_launch = (double)ms / reps;
    c->fields_valid = false;
    return LBIB_OK;
}

extern "C" lbib_status lbib_profile_hydro(lbib_ctx* c, int32_t reps, double* ms_per_launch) {
    if (!c || reps < 1 || !ms_per_launch) return LBIB_E_INVALID;
    if (!c->finalized || c->steps == 0) return fail(c, LBIB_E_STATE, "profile after at least one step");
    *ms_per_launch = 0.0;
    if (c->ndyn == 0) return LBIB_OK;
    cudaEvent_t ev[2];
    for (int k = 0; k < 2; ++k) CK(cudaEventCreate(&ev[k]));
    CK(cudaEventRecord(ev[0], c->stream));
    for (int r = 0; r < reps; ++r) CK(launch_hydro(c->prec, c->ma, hydro_args(c, c->cur), c->stream));
    CK(cudaEventRecord(ev[1], c->stream));
    CK(cudaEventSynchronize(ev[1]));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ev[0], ev[1]));
    *ms_per_launch = (double)ms / reps;
    for (int k = 0; k < 2; ++k) cudaEventDestroy(ev[k]);
    return LBIB_OK;
}

extern "C" lbib_status lbib_profile_kernels(lbib_ctx* c, int32_t reps, double* ms_per_launch) {
    if (!c || reps < 1 || !ms_per_launch) return LBIB_E_INVALID;
    if (!c->finalized || c->steps == 0) return fail(c, LBIB_E_STATE, "profile after at least one step");
    cudaEvent_t ev[6];
    for (int k = 0; k < 6; ++k) CK(cudaEventCreate(&ev[k]));
    const bool has_ib = c->nv > 0;
    MarkerArgs a = c->ma;
    a.gsum = c->G[c->cur];
    a.flags = c->flags[c->cur];
    // forces + spreading (accumulates into the field of the current parity)
    CK(cudaEventRecord(ev[0], c->stream));
    for (int r = 0; r < reps && has_ib; ++r) CK(launch_forces(c->prec, a, c->max_mem_n, c->stream));
    CK(cudaEventRecord(ev[1], c->stream));
    // fused collide-stream, ping-pong between the buffers
    const int gpar = 1 - c->cur;
    LbArgs l = lb_args(c, c->cur, gpar, 0);
    CK(cudaEventRecord(ev[2], c->stream));
    for (int r = 0; r < reps; ++r) {
        l.src = c->f[c->cur];
        l.dst = c->f[1 - c->cur];
        CK(launch_fused(c, l, c->stream));
        c->cur = 1 - c->cur;
    }
    CK(cudaEventRecord(ev[3], c->stream));
    // interpolation + advance + bond kinetics
    CK(cudaEventRecord(ev[4], c->stream));
    for (int r = 0; r < reps && has_ib; ++r) CK(launch_advance(c->prec, a, c->stream));
    CK(cudaEventRecord(ev[5], c->stream));
    CK(cudaEventSynchronize(ev[5]));
    for (int k = 0; k < 3; ++k) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]));
        ms_per_launch[k] = (k != 1 && !has_ib) ? 0.0 : (double)ms / reps;
    }
    for (int k = 0; k < 6; ++k) cudaEventDestroy(ev[k]);
    c->fields_valid = false;
    return LBIB_OK;
}

extern "C" const char* lbib_last_error(const lbib_ctx* c) { return c ? c->err.c_str() : "null context"; }

extern "C" void lbib_destroy(lbib_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (int s = 0; s < 2; ++s)
        for (int k = 0; k < 2; ++k) {
            if (c->graph[s][k]) cudaGraphExecDestroy(c->graph[s][k]);
            if (c->graph_tmpl[s][k]) cudaGraphDestroy(c->graph_tmpl[s][k]);
        }
    for (int b = 0; b < 2; ++b)
        if (c->f[b]) cudaFree(c->f[b]);
    if (c->ux) cudaFree(c->ux);
    if (c->uy) cudaFree(c->uy);
    if (c->stage) cudaFree(c->stage);
    if (c->partials) cudaFree(c->partials);
    if (c->dscalar) cudaFree(c->dscalar);
    if (c->d_step) cudaFree(c->d_step);
    if (c->d_status) cudaFree(c->d_status);
    if (c->dmem) cudaFree(c->dmem);
    if (c->d_obs) cudaFree(c->d_obs);
    for (int p = 0; p < 2; ++p)
        if (c->G[p]) cudaFree(c->G[p]);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

// ------------------------------------------------------------------ ensembles
// Independent contexts advanced together: one graph per chunk of steps holds
// every member's captured step graph as a child node with no edges between
// them, so the members' kernels run side by side on the GPU.
//
// Members that share a precision, walls and the form and shape of the fused
// kernel (row tiles (vec, ty), or the persistent form with npt = vec) and have
// markers but no dynamic particles are advanced in the batched form: per time
// step one launch of each kernel covers every member of a group (one block per
// (member, force unit) and per (member, advance unit); the fused kernel one
// block per (member, tile), or persistent CTAs walking all members'
// segments), with the members' arguments in the launch parameters or in
// device memory.  Groups (at most kBatchMax members each,
// contiguous, balanced by nodes) are independent branches of the captured
// chunk graph, so one group's latency-bound marker kernels can run beside
// another group's bandwidth-bound fused kernel.  Any other set of members
// runs as a graph of the members' own step graphs.
struct lbib_ensemble {
    std::vector<lbib_ctx*> m;
    cudaStream_t stream = nullptr;
    // [flip][kind]: members at their parity at creation (flip 0) or the other
    // one (flip 1); kind 0 one step, kind 1 a chunk of kChunk steps
    cudaGraphExec_t g[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int flip = 0;
    std::vector<int> cur0;
    bool own_stream = false;
    std::string err;
    // batched form
    bool batched = false;
    lbib::MarkerArgs* margs = nullptr;             // [2][n] in device memory: [phase][member]
    std::vector<int> gstart;                       // group g: members [gstart[g], gstart[g + 1])
    std::vector<lbib::LbBatch> lbb[2];             // [phase][group]
    std::vector<lbib::MarkerBatch> fbb[2], abb[2];  // [phase][group]
    int adv_threads = 0;
    int stream_grid = 0;                           // CTAs of the batched persistent form
};

namespace {
lbib_status ens_fail(lbib_ensemble* e, lbib_status st, const std::string& msg) {
    if (e) e->err = msg;
    return st;
}
}  // namespace

#define ECK(call)                                                                     \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) return ens_fail(e, LBIB_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// whether the members can run in the batched form (see lbib_ensemble)
static bool batchable(const std::vector<lbib_ctx*>& m) {
    const lbib_ctx* c0 = m[0];
    for (const lbib_ctx* c : m) {
        if (c->prec != c0->prec || c->walls != c0->walls || c->vec != c0->vec || c->ty != c0->ty || c->nv == 0 ||
            c->ndyn > 0 || c->ma.nfu == 0 || c->ma.nau == 0)
            return false;
    }
    return true;
}

static void drop_ensemble_graphs(lbib_ensemble* e) {
    for (int f = 0; f < 2; ++f)
        for (int k = 0; k < 2; ++k) {
            if (e->g[f][k]) cudaGraphExecDestroy(e->g[f][k]);
            e->g[f][k] = nullptr;
        }
}

// group boundaries: ngroups contiguous ranges with about equal nodes, none
// above kBatchMax members (ceil(n / kBatchMax) <= ngroups <= n)
static std::vector<int> ensemble_groups(const lbib_ensemble* e, int ngroups) {
    const int n = (int)e->m.size();
    std::vector<double> cum(n + 1, 0.0);  // nodes of members [0, i)
    for (int i = 0; i < n; ++i) cum[i + 1] = cum[i] + (double)e->m[i]->nx * e->m[i]->ny;
    std::vector<int> start{0};
    for (int g = 1; g < ngroups; ++g) {
        const int lo = std::max(start.back() + 1, n - (ngroups - g) * kBatchMax);
        const int hi = std::min(n - (ngroups - g), start.back() + kBatchMax);
        int b = hi;
        for (int i = lo; i <= hi; ++i)
            if (cum[i] >= cum[n] * g / ngroups) {
                b = i;
                break;
            }
        start.push_back(b);
    }
    start.push_back(n);
    return start;
}

// the parameter blocks of the batched launches and the device table of the
// members' marker arguments, for `ngroups` groups
static lbib_status ensemble_batch_tables(lbib_ensemble* e, int ngroups) {
    const size_t n = e->m.size();
    if (!e->margs) {
        std::vector<MarkerArgs> ma(2 * n);
        for (size_t i = 0; i < n; ++i) {
            lbib_ctx* c = e->m[i];
            for (int p = 0; p < 2; ++p) {
                const int src = e->cur0[i] ^ p;
                MarkerArgs a = c->ma;
                a.gsum = c->G[src];
                a.flags = c->flags[src];
                ma[p * n + i] = a;
            }
        }
        ECK(cudaMalloc(&e->margs, sizeof(MarkerArgs) * 2 * n));
        ECK(cudaMemcpy(e->margs, ma.data(), sizeof(MarkerArgs) * 2 * n, cudaMemcpyHostToDevice));
    }
    e->gstart = ensemble_groups(e, ngroups);
    const int G = (int)e->gstart.size() - 1;
    e->adv_threads = 0;
    for (int p = 0; p < 2; ++p) {
        e->lbb[p].assign(G, LbBatch{});
        e->fbb[p].assign(G, MarkerBatch{});
        e->abb[p].assign(G, MarkerBatch{});
        for (int g = 0; g < G; ++g) {
            LbBatch& lb = e->lbb[p][g];
            MarkerBatch& fb = e->fbb[p][g];
            MarkerBatch& ab = e->abb[p][g];
            const int i0 = e->gstart[g], i1 = e->gstart[g + 1];
            lb.n = fb.n = ab.n = i1 - i0;
            fb.args = ab.args = e->margs + p * n + i0;
            int kb = 0, fu = 0, au = 0;
            for (int i = i0; i < i1; ++i) {
                lbib_ctx* c = e->m[i];
                const int k = i - i0, src = e->cur0[i] ^ p;
                // row tiles: blocks of (32 vec) x ty nodes; persistent form: segments of 256 vec nodes
                const int gx = c->ty > 0 ? (c->nx + 32 * c->vec - 1) / (32 * c->vec)
                                         : (c->nx + 256 * c->vec - 1) / (256 * c->vec);
                const int gy = c->ty > 0 ? (c->ny + c->ty - 1) / c->ty : c->ny;
                lb.off[k] = kb;
                lb.tiles_x[k] = gx;
                lb.a[k] = lb_args(c, src, src, 1);
                fb.off[k] = fu;
                ab.off[k] = au;
                kb += gx * gy;
                fu += c->ma.nfu;
                au += c->ma.nau;
                e->adv_threads = std::max(e->adv_threads, c->ma.adv_threads);
            }
            lb.off[lb.n] = kb;
            fb.off[fb.n] = fu;
            ab.off[ab.n] = au;
            for (MarkerBatch* mb : {&fb, &ab})
                for (int k = 0; k < mb->n; ++k)
                    for (int blk = mb->off[k]; blk < mb->off[k + 1] && blk < kBlockTable; ++blk)
                        mb->member[blk] = (unsigned char)k;
        }
    }
    const lbib_ctx* c0 = e->m[0];
    if (c0->ty == 0)
        ECK(prepare_lb_stream_batch(c0->prec, c0->vec, c0->walls != LBIB_WALLS_NONE, &e->stream_grid));
    return LBIB_OK;
}

// one time step of every member of group g in the batched form, at phase p
static cudaError_t ensemble_batch_step(const lbib_ensemble* e, int g, int p, cudaStream_t s) {
    const lbib_ctx* c0 = e->m[0];
    const bool walls = c0->walls != LBIB_WALLS_NONE;
    cudaError_t r = launch_forces_batch(c0->prec, e->fbb[p][g], s);
    if (r == cudaSuccess)
        r = c0->ty > 0 ? launch_lb_batch(c0->prec, c0->vec, c0->ty, walls, e->lbb[p][g], s)
                       : launch_lb_stream_batch(c0->prec, c0->vec, walls, e->stream_grid, e->lbb[p][g], s);
    if (r == cudaSuccess) r = launch_advance_batch(c0->prec, false, e->abb[p][g], e->adv_threads, s);
    return r;
}

// capture the batched chunk graphs: each group's steps on a stream of its own,
// forked from and joined to the capturing stream
static lbib_status ensemble_build_batched(lbib_ensemble* e, int ngroups) {
    lbib_status st = ensemble_batch_tables(e, ngroups);
    if (st != LBIB_OK) return st;
    const int G = (int)e->gstart.size() - 1;
    std::vector<cudaStream_t> gs(G, nullptr);
    std::vector<cudaEvent_t> ev(G + 1, nullptr);
    cudaStream_t cap = nullptr;
    cudaError_t r = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    for (int g = 0; g < G && r == cudaSuccess; ++g) r = cudaStreamCreateWithFlags(&gs[g], cudaStreamNonBlocking);
    for (int k = 0; k <= G && r == cudaSuccess; ++k) r = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
    for (int flip = 0; flip < 2 && r == cudaSuccess; ++flip) {
        for (int kind = 0; kind < 2 && r == cudaSuccess; ++kind) {
            const int nsteps = kind == 0 ? 1 : kChunk;
            cudaGraph_t gr = nullptr;
            r = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (r != cudaSuccess) break;
            cudaError_t le = cudaEventRecord(ev[G], cap);
            for (int g = 0; g < G && le == cudaSuccess; ++g) {
                cudaStream_t s = G == 1 ? cap : gs[g];
                if (G > 1) le = cudaStreamWaitEvent(s, ev[G], 0);
                for (int k = 0; k < nsteps && le == cudaSuccess; ++k) le = ensemble_batch_step(e, g, flip ^ (k & 1), s);
                if (G > 1 && le == cudaSuccess) le = cudaEventRecord(ev[g], s);
                if (G > 1 && le == cudaSuccess) le = cudaStreamWaitEvent(cap, ev[g], 0);
            }
            r = cudaStreamEndCapture(cap, &gr);
            if (r == cudaSuccess) r = le;
            if (r == cudaSuccess) r = cudaGraphInstantiate(&e->g[flip][kind], gr, 0);
            if (gr) cudaGraphDestroy(gr);
        }
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    for (cudaStream_t x : gs)
        if (x) cudaStreamDestroy(x);
    if (cap) cudaStreamDestroy(cap);
    if (r != cudaSuccess) {
        drop_ensemble_graphs(e);
        return ens_fail(e, LBIB_E_CUDA, std::string("capture batched step: ") + cudaGetErrorString(r));
    }
    e->batched = true;
    return LBIB_OK;
}

static lbib_status ensemble_build(lbib_ensemble* e) {
    if (batchable(e->m))
        return ensemble_build_batched(e, ((int)e->m.size() + kBatchMax - 1) / kBatchMax);
    for (int flip = 0; flip < 2; ++flip) {
        for (int kind = 0; kind < 2; ++kind) {
            cudaGraph_t g;
            ECK(cudaGraphCreate(&g, 0));
            for (size_t i = 0; i < e->m.size(); ++i) {
                lbib_ctx* c = e->m[i];
                cudaGraphNode_t node;
                const cudaError_t r = cudaGraphAddChildGraphNode(&node, g, nullptr, 0,
                                                                 c->graph_tmpl[e->cur0[i] ^ flip][kind]);
                if (r != cudaSuccess) {
                    cudaGraphDestroy(g);
                    return ens_fail(e, LBIB_E_CUDA, std::string("add member graph: ") + cudaGetErrorString(r));
                }
            }
            const cudaError_t r = cudaGraphInstantiate(&e->g[flip][kind], g, 0);
            cudaGraphDestroy(g);
            if (r != cudaSuccess) return ens_fail(e, LBIB_E_CUDA, std::string("instantiate: ") + cudaGetErrorString(r));
        }
    }
    return LBIB_OK;
}

extern "C" lbib_status lbib_ensemble_create(lbib_ctx* const* members, int32_t n, void* cuda_stream,
                                            lbib_ensemble** out) {
    if (!members || n < 1 || !out) return LBIB_E_INVALID;
    for (int i = 0; i < n; ++i) {
        if (!members[i]) return LBIB_E_INVALID;
        for (int j = 0; j < i; ++j)
            if (members[j] == members[i]) return LBIB_E_INVALID;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBIB_E_CUDA;
    for (int i = 0; i < n; ++i) {
        lbib_ctx* c = members[i];
        if (c->device != dev || c->poisoned) return LBIB_E_INVALID;
        lbib_status st = finalize(c);
        if (st == LBIB_OK && !c->no_g_prefetch) {
            // the members' row tiles read the force field only in flagged tiles
            if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LBIB_E_CUDA;
            c->no_g_prefetch = true;
            drop_graphs(c);
        }
        if (st == LBIB_OK) st = build_graphs(c);
        if (st != LBIB_OK) return st;
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LBIB_E_CUDA;
    }
    lbib_ensemble* e = new lbib_ensemble();
    e->m.assign(members, members + n);
    for (int i = 0; i < n; ++i) e->cur0.push_back(members[i]->cur);
    if (cuda_stream) {
        e->stream = static_cast<cudaStream_t>(cuda_stream);
    } else if (cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete e;
        return LBIB_E_CUDA;
    } else {
        e->own_stream = true;
    }
    e->err.clear();
    const lbib_status st = ensemble_build(e);
    if (st != LBIB_OK) {
        for (int f = 0; f < 2; ++f)
            for (int k = 0; k < 2; ++k)
                if (e->g[f][k]) cudaGraphExecDestroy(e->g[f][k]);
        if (e->margs) cudaFree(e->margs);
        if (e->own_stream) cudaStreamDestroy(e->stream);
        delete e;
        return st;
    }
    *out = e;
    return LBIB_OK;
}

extern "C" lbib_status lbib_ensemble_step(lbib_ensemble* e, int64_t n) {
    if (!e || n < 0) return LBIB_E_INVALID;
    for (lbib_ctx* c : e->m)
        if (c->poisoned) return ens_fail(e, LBIB_E_STATE, "a member is poisoned by an earlier device-side failure");
    int64_t left = n;
    while (left >= kChunk) {
        ECK(cudaGraphLaunch(e->g[e->flip][1], e->stream));
        left -= kChunk;  // even: every member keeps its buffer roles
    }
    while (left > 0) {
        ECK(cudaGraphLaunch(e->g[e->flip][0], e->stream));
        e->flip ^= 1;
        --left;
    }
    for (size_t i = 0; i < e->m.size(); ++i) {
        lbib_ctx* c = e->m[i];
        c->cur = e->cur0[i] ^ e->flip;
        c->steps += n;
        if (n > 0) c->fields_valid = true;
    }
    return LBIB_OK;
}

extern "C" lbib_status lbib_ensemble_sync(lbib_ensemble* e) {
    if (!e) return LBIB_E_INVALID;
    ECK(cudaStreamSynchronize(e->stream));
    for (lbib_ctx* c : e->m) {
        const lbib_status st = lbib_sync(c);
        if (st != LBIB_OK) return ens_fail(e, st, c->err);
    }
    return LBIB_OK;
}

extern "C" int32_t lbib_ensemble_size(const lbib_ensemble* e) { return e ? (int32_t)e->m.size() : -1; }

// Every member's state from host (or device) buffers in one call: the copies
// and conversions of all members are enqueued on the ensemble's stream, after
// its pending steps, with one wait at the end.
extern "C" lbib_status lbib_ensemble_write_state(lbib_ensemble* e, const double* const* f,
                                                 const double* const* xy, const double* const* xy_prev,
                                                 int32_t on_device) {
    if (!e || (on_device && xy)) return LBIB_E_INVALID;
    // the members' own streams may hold work of their own
    for (lbib_ctx* c : e->m) ECK(cudaStreamSynchronize(c->stream));
    for (lbib_ctx* c : e->m)
        if (c->poisoned) return ens_fail(e, LBIB_E_STATE, "a member is poisoned by an earlier device-side failure");
    // host populations: every member's copy first (back to back on the copy
    // engine), then the conversions
    const size_t n = e->m.size();
    if (f && !on_device) {
        for (size_t i = 0; i < n; ++i) {
            lbib_ctx* c = e->m[i];
            if (!f[i]) continue;
            const lbib_status st = ensure_stage(c);
            if (st != LBIB_OK) return ens_fail(e, st, c->err);
            ECK(cudaMemcpyAsync(c->stage, f[i], 9 * sizeof(double) * (size_t)c->nx * c->ny, cudaMemcpyHostToDevice,
                                e->stream));
        }
    }
    for (size_t i = 0; i < n; ++i) {
        lbib_ctx* c = e->m[i];
        lbib_status st;
        if (f && f[i] && (st = write_populations_on(c, on_device ? f[i] : c->stage, 1, e->stream)) != LBIB_OK)
            return ens_fail(e, st, c->err);
        if (xy && xy[i] && (st = write_markers_on(c, xy[i], xy_prev ? xy_prev[i] : nullptr, e->stream)) != LBIB_OK)
            return ens_fail(e, st, c->err);
    }
    ECK(cudaStreamSynchronize(e->stream));
    return LBIB_OK;
}

extern "C" lbib_status lbib_ensemble_read_markers(lbib_ensemble* e, double* const* xy) {
    if (!e || !xy) return LBIB_E_INVALID;
    for (size_t i = 0; i < e->m.size(); ++i) {
        if (!xy[i]) continue;
        const lbib_status st = read_markers_on(e->m[i], -1, xy[i], e->stream);
        if (st != LBIB_OK) return ens_fail(e, st, e->m[i]->err);
    }
    ECK(cudaStreamSynchronize(e->stream));
    return LBIB_OK;
}

extern "C" int32_t lbib_ensemble_form(const lbib_ensemble* e) { return e ? (e->batched ? 1 : 0) : -1; }

extern "C" lbib_status lbib_ensemble_set_groups(lbib_ensemble* e, int32_t groups) {
    if (!e) return LBIB_E_INVALID;
    if (!e->batched) return ens_fail(e, LBIB_E_STATE, "groups apply to the batched form only");
    const int n = (int)e->m.size();
    if (groups < (n + kBatchMax - 1) / kBatchMax || groups > n)
        return ens_fail(e, LBIB_E_INVALID, "groups must lie in [ceil(n / 64), n]");
    ECK(cudaStreamSynchronize(e->stream));
    drop_ensemble_graphs(e);
    return ensemble_build_batched(e, groups);
}

extern "C" lbib_status lbib_ensemble_profile_kernels(lbib_ensemble* e, int32_t reps, double* ms_per_launch) {
    if (!e || reps < 1 || !ms_per_launch) return LBIB_E_INVALID;
    if (!e->batched) return ens_fail(e, LBIB_E_STATE, "kernel times apply to the batched form only");
    const lbib_ctx* c0 = e->m[0];
    const bool walls = c0->walls != LBIB_WALLS_NONE;
    const int G = (int)e->gstart.size() - 1;
    cudaEvent_t ev[4];
    for (int k = 0; k < 4; ++k) ECK(cudaEventCreate(&ev[k]));
    ECK(cudaEventRecord(ev[0], e->stream));
    for (int r = 0; r < reps; ++r)
        for (int g = 0; g < G; ++g) ECK(launch_forces_batch(c0->prec, e->fbb[e->flip][g], e->stream));
    ECK(cudaEventRecord(ev[1], e->stream));
    for (int r = 0; r < reps; ++r)
        for (int g = 0; g < G; ++g) {
            const int p = e->flip ^ (r & 1);
            ECK(c0->ty > 0 ? launch_lb_batch(c0->prec, c0->vec, c0->ty, walls, e->lbb[p][g], e->stream)
                           : launch_lb_stream_batch(c0->prec, c0->vec, walls, e->stream_grid, e->lbb[p][g], e->stream));
        }
    ECK(cudaEventRecord(ev[2], e->stream));
    for (int r = 0; r < reps; ++r)
        for (int g = 0; g < G; ++g)
            ECK(launch_advance_batch(c0->prec, false, e->abb[e->flip][g], e->adv_threads, e->stream));
    ECK(cudaEventRecord(ev[3], e->stream));
    ECK(cudaEventSynchronize(ev[3]));
    for (int k = 0; k < 3; ++k) {
        float ms = 0.f;
        ECK(cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
        ms_per_launch[k] = ms / reps;
    }
    for (int k = 0; k < 4; ++k) cudaEventDestroy(ev[k]);
    // the members' state is no longer a time step's: the ensemble is spent
    for (lbib_ctx* c : e->m) c->poisoned = true;
    return LBIB_OK;
}

extern "C" int32_t lbib_ensemble_groups(const lbib_ensemble* e) {
    return e ? (e->batched ? (int32_t)e->gstart.size() - 1 : 0) : -1;
}

extern "C" int32_t lbib_ensemble_launches_per_step(const lbib_ensemble* e) {
    if (!e) return -1;
    if (e->batched) return 3 * ((int32_t)e->gstart.size() - 1);
    int k = 0;
    for (const lbib_ctx* c : e->m) k += lbib_kernels_per_step(c);
    return k;
}

extern "C" lbib_ctx* lbib_ensemble_member(lbib_ensemble* e, int32_t i) {
    if (!e || i < 0 || i >= (int32_t)e->m.size()) return nullptr;
    return e->m[i];
}

extern "C" const char* lbib_ensemble_last_error(const lbib_ensemble* e) { return e ? e->err.c_str() : "null ensemble"; }

extern "C" void lbib_ensemble_destroy(lbib_ensemble* e) {
    if (!e) return;
    cudaStreamSynchronize(e->stream);
    for (int f = 0; f < 2; ++f)
        for (int k = 0; k < 2; ++k)
            if (e->g[f][k]) cudaGraphExecDestroy(e->g[f][k]);
    if (e->margs) cudaFree(e->margs);
    for (lbib_ctx* c : e->m) lbib_destroy(c);
    if (e->own_stream) cudaStreamDestroy(e->stream);
    delete e;
}

// ------------------------------------------------------------------ tangent
// Forward-mode derivative of an FP64 context's trajectory along one direction
// of (k_s, k_b per membrane, sigma, initial marker positions); the bond events
// of the primal run are taken as given.
struct lbib_tangent {
    lbib_ctx* c = nullptr;  // primal (not owned)
    double* fd[2] = {nullptr, nullptr};
    double* dX[3] = {nullptr, nullptr, nullptr};  // roles rotate: X^{n-1}, X^n, X^{n+1}
    int ip = 0, ix = 1, in = 2, cf = 0;
    double *Gv = nullptr, *Gd = nullptr, *u = nullptr, *ud = nullptr, *Wv = nullptr, *Wd = nullptr;
    double *Fv = nullptr, *Fd = nullptr, *A = nullptr, *Ad = nullptr, *dks = nullptr, *dkb = nullptr;
    double* box = nullptr;
    double* th0 = nullptr;
    double* l0 = nullptr;
    int* st = nullptr;
    double dsigma = 0.0;
    std::vector<void*> allocs;
};

extern "C" void lbib_tangent_destroy(lbib_tangent* t) {
    if (!t) return;
    if (t->c && t->c->stream) cudaStreamSynchronize(t->c->stream);
    for (void* p : t->allocs) cudaFree(p);
    delete t;
}

extern "C" lbib_status lbib_tangent_create(lbib_ctx* c, lbib_tangent** out) {
    if (!c || !out) return LBIB_E_INVALID;
    if (c->prec != LBIB_F64) return fail(c, LBIB_E_INVALID, "the tangent needs an FP64 context");
    if (c->uw_bot != 0.0 || c->uw_top != 0.0) return fail(c, LBIB_E_INVALID, "the tangent needs resting walls");
    if (c->walls == LBIB_WALLS_ZOU_HE) return fail(c, LBIB_E_INVALID, "the tangent needs half-way or no walls");
    for (int k : c->h_mem_kind)
        if (k != LBIB_MEMBRANE_KINEMATIC)
            return fail(c, LBIB_E_INVALID, "the tangent supports kinematic membranes only");
    lbib_status st = finalize(c);
    if (st == LBIB_OK) st = build_graphs(c);
    if (st != LBIB_OK) return st;
    lbib_tangent* t = new lbib_tangent();
    t->c = c;
    const size_t N = (size_t)c->nx * c->ny, nv = std::max(c->nv, 1), nm = std::max(c->nmem, 1);
    auto get = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
        t->allocs.push_back(p);
        return p;
    };
    bool ok = true;
    for (int b = 0; b < 2; ++b) ok = ok && (t->fd[b] = (double*)get(9 * N * 8));
    for (int b = 0; b < 3; ++b) ok = ok && (t->dX[b] = (double*)get(2 * nv * 8));
    ok = ok && (t->Gv = (double*)get(2 * N * 8)) && (t->Gd = (double*)get(2 * N * 8));
    ok = ok && (t->u = (double*)get(2 * N * 8)) && (t->ud = (double*)get(2 * N * 8));
    ok = ok && (t->Wv = (double*)get(9 * nv * 8)) && (t->Wd = (double*)get(9 * nv * 8));
    ok = ok && (t->Fv = (double*)get(2 * nv * 8)) && (t->Fd = (double*)get(2 * nv * 8));
    ok = ok && (t->A = (double*)get(nm * 8)) && (t->Ad = (double*)get(nm * 8)) && (t->box = (double*)get(4 * nm * 8));
    ok = ok && (t->dks = (double*)get(nm * 8)) && (t->dkb = (double*)get(nm * 8));
    ok = ok && (t->st = (int*)get(2 * nv * 4)) && (t->th0 = (double*)get(nv * 8)) && (t->l0 = (double*)get(nv * 8));
    if (!ok) {
        lbib_tangent_destroy(t);
        return fail(c, LBIB_E_OOM, "tangent buffers");
    }
    launch_rest_fp64(c->prec, c->ma, t->l0, t->th0, c->stream);
    cudaMemsetAsync(t->fd[0], 0, 9 * N * 8, c->stream);
    cudaMemsetAsync(t->fd[1], 0, 9 * N * 8, c->stream);
    for (int b = 0; b < 3; ++b) cudaMemsetAsync(t->dX[b], 0, 2 * nv * 8, c->stream);
    cudaMemsetAsync(t->dks, 0, nm * 8, c->stream);
    cudaMemsetAsync(t->dkb, 0, nm * 8, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        lbib_tangent_destroy(t);
        return fail(c, LBIB_E_CUDA, "tangent set-up");
    }
    *out = t;
    return LBIB_OK;
}

extern "C" lbib_status lbib_tangent_seed(lbib_tangent* t, const double* dks, const double* dkb, double dsigma,
                                         const double* dxy, const double* dxy_prev) {
    if (!t) return LBIB_E_INVALID;
    lbib_ctx* c = t->c;
    const size_t N = (size_t)c->nx * c->ny;
    const size_t nv = (size_t)c->nv, nm = (size_t)c->nmem;
    CK(cudaMemsetAsync(t->fd[t->cf], 0, 9 * N * 8, c->stream));
    if (nm) {
        if (dks) CK(cudaMemcpyAsync(t->dks, dks, nm * 8, cudaMemcpyHostToDevice, c->stream));
        else CK(cudaMemsetAsync(t->dks, 0, nm * 8, c->stream));
        if (dkb) CK(cudaMemcpyAsync(t->dkb, dkb, nm * 8, cudaMemcpyHostToDevice, c->stream));
        else CK(cudaMemsetAsync(t->dkb, 0, nm * 8, c->stream));
    }
    if (nv) {
        if (dxy) CK(cudaMemcpyAsync(t->dX[t->ix], dxy, nv * 16, cudaMemcpyHostToDevice, c->stream));
        else CK(cudaMemsetAsync(t->dX[t->ix], 0, nv * 16, c->stream));
        const double* pv = dxy_prev ? dxy_prev : dxy;
        if (pv) CK(cudaMemcpyAsync(t->dX[t->ip], pv, nv * 16, cudaMemcpyHostToDevice, c->stream));
        else CK(cudaMemsetAsync(t->dX[t->ip], 0, nv * 16, c->stream));
    }
    t->dsigma = dsigma;
    CK(cudaStreamSynchronize(c->stream));
    return LBIB_OK;
}

extern "C" lbib_status lbib_tangent_step(lbib_tangent* t, int64_t n) {
    if (!t || n < 0) return LBIB_E_INVALID;
    lbib_ctx* c = t->c;
    if (c->poisoned) return fail(c, LBIB_E_STATE, "context poisoned by an earlier device-side failure");
    for (int64_t k = 0; k < n; ++k) {
        TangentArgs a{};
        a.m = c->ma;
        a.f = static_cast<const double*>(c->f[c->cur]);
        a.fd_src = t->fd[t->cf];
        a.fd_dst = t->fd[1 - t->cf];
        a.dX = t->dX[t->ix];
        a.dXp = t->dX[t->ip];
        a.dXn = t->dX[t->in];
        a.Gv = t->Gv; a.Gd = t->Gd; a.u = t->u; a.ud = t->ud; a.Wv = t->Wv; a.Wd = t->Wd;
        a.st = t->st; a.Fv = t->Fv; a.Fd = t->Fd; a.A = t->A; a.Ad = t->Ad; a.box = t->box;
        a.dks = t->dks; a.dkb = t->dkb; a.dsigma = t->dsigma; a.th0 = t->th0; a.l0 = t->l0;
        a.omega = 1.0 / c->tau; a.gx = c->gx; a.gy = c->gy;
        a.step = c->steps;
        CK(launch_tangent_step(a, c->stream));
        // the primal step (its captured one-step graph) follows on the same stream
        CK(cudaGraphLaunch(c->graph[c->cur][0], c->stream));
        c->cur = 1 - c->cur;
        c->steps += 1;
        c->fields_valid = true;
        t->cf = 1 - t->cf;
        const int op = t->ip;
        t->ip = t->ix;
        t->ix = t->in;
        t->in = op;
    }
    return LBIB_OK;
}

extern "C" lbib_status lbib_tangent_read(lbib_tangent* t, double* dxy, double* dxy_prev) {
    if (!t) return LBIB_E_INVALID;
    lbib_ctx* c = t->c;
    const size_t nv = (size_t)c->nv;
    if (dxy && nv) CK(cudaMemcpyAsync(dxy, t->dX[t->ix], nv * 16, cudaMemcpyDeviceToHost, c->stream));
    if (dxy_prev && nv) CK(cudaMemcpyAsync(dxy_prev, t->dX[t->ip], nv * 16, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return lbib_sync(c);
}

// ------------------------------------------------------------------ adjoint
// Reverse-mode derivative of an FP64 context's trajectory (the transpose of
// the tangent above).  lbib_adjoint_record runs the primal and keeps the full
// step state every K steps; lbib_adjoint_reverse walks the segments backwards:
// it restores a segment's first state, re-runs the segment with the context's
// own step graph (bit-identical to the recorded run: fixed-point spreading and
// counter-based bond draws) while copying each step's state to a tape, then
// applies the adjoint step to the tape in reverse order.
namespace {

// the context's full step state at a step boundary (in the context's own
// storage and position layouts)
struct Snap {
    void* mem = nullptr;
    void* f = nullptr;
    double *X = nullptr, *Xp = nullptr;
    int *bond = nullptr, *owner = nullptr, *owner_cell = nullptr;
    float4* seg_box = nullptr;
    long long* d_step = nullptr;
    long long step = 0;
};

size_t snap_bytes(const lbib_ctx* c) {
    Arena a;
    const size_t N = (size_t)c->nx * c->ny, nv = c->nv, nlig = c->nlig, nrec = c->ma.nrec;
    a.take<char>(9 * N * c->pop_elem);
    a.take<double>(2 * nv);
    a.take<double>(2 * nv);
    a.take<int>(nlig);
    a.take<int>(nrec);
    a.take<int>(nrec);
    a.take<float4>(c->nseg);
    a.take<long long>(1);
    return a.used + 256;
}

void snap_layout(const lbib_ctx* c, Snap& s) {
    Arena a;
    a.base = static_cast<char*>(s.mem);
    const size_t N = (size_t)c->nx * c->ny, nv = c->nv, nlig = c->nlig, nrec = c->ma.nrec;
    s.f = a.take<char>(9 * N * c->pop_elem);
    s.X = a.take<double>(2 * nv);
    s.Xp = a.take<double>(2 * nv);
    s.bond = a.take<int>(nlig);
    s.owner = a.take<int>(nrec);
    s.owner_cell = a.take<int>(nrec);
    s.seg_box = a.take<float4>(c->nseg);
    s.d_step = a.take<long long>(1);
}

// copy the state between the context and a snapshot (to_snap: context -> snapshot)
cudaError_t snap_copy(lbib_ctx* c, Snap& s, bool to_snap) {
    const size_t N = (size_t)c->nx * c->ny, nv = c->nv, nlig = c->nlig, nrec = c->ma.nrec;
    auto cp = [&](void* snap, void* ctx, size_t bytes) -> cudaError_t {
        if (bytes == 0) return cudaSuccess;
        return cudaMemcpyAsync(to_snap ? snap : ctx, to_snap ? ctx : snap, bytes, cudaMemcpyDeviceToDevice,
                               c->stream);
    };
    cudaError_t e;
    if ((e = cp(s.f, c->f[c->cur], 9 * N * c->pop_elem)) != cudaSuccess) return e;
    if ((e = cp(s.X, c->ma.X, 16 * nv)) != cudaSuccess) return e;
    if ((e = cp(s.Xp, c->ma.Xp, 16 * nv)) != cudaSuccess) return e;
    if ((e = cp(s.bond, c->ma.bond_of_lig, 4 * nlig)) != cudaSuccess) return e;
    if ((e = cp(s.owner, c->ma.owner, 4 * nrec)) != cudaSuccess) return e;
    if ((e = cp(s.owner_cell, c->ma.owner_cell, 4 * nrec)) != cudaSuccess) return e;
    if ((e = cp(s.seg_box, c->ma.seg_box, sizeof(float4) * c->nseg)) != cudaSuccess) return e;
    if ((e = cp(s.d_step, c->d_step, 8)) != cudaSuccess) return e;
    if (to_snap) s.step = c->steps;
    else c->steps = s.step;
    return cudaSuccess;
}

}  // namespace

struct lbib_adjoint {
    lbib_ctx* c = nullptr;  // primal (not owned)
    int K = 0;              // checkpoint interval (steps per segment)
    std::vector<Snap> snaps;  // state at the first step of each recorded segment
    Snap end;                 // state after the recorded run
    int64_t n_rec = 0;
    bool seeded = false, reversed = false;
    // tape of one segment, per step: the state it starts from (deviations,
    // positions, bonds) and what the context's step computed from it (marker
    // forces, shape functions, stencil origins, fixed-point spread force)
    double* tape_f = nullptr;
    double* tape_X = nullptr;
    int* tape_bond = nullptr;
    double* tape_F = nullptr;
    double* tape_W = nullptr;
    int* tape_st = nullptr;
    longlong2* tape_G = nullptr;
    // adjoint state and per-step work arrays
    double* fbar[2] = {nullptr, nullptr};
    int cb = 0;
    double* XB[2] = {nullptr, nullptr};  // adjoint of the current positions (roles alternate per step)
    int xb = 0;
    double *XPB = nullptr, *ubar = nullptr, *Gbar = nullptr, *Wbar = nullptr;
    double *Abar = nullptr, *ksb = nullptr, *kbb = nullptr, *sgb = nullptr, *fio = nullptr;
    // areas and boxes re-evaluated per step (tangent area kernel, zero tangent)
    double *A = nullptr, *Ad = nullptr, *box = nullptr, *zero = nullptr, *th0 = nullptr, *l0 = nullptr;
    std::vector<void*> allocs;
};

namespace {

void adjoint_free_snaps(lbib_adjoint* a) {
    for (Snap& s : a->snaps) cudaFree(s.mem);
    a->snaps.clear();
    if (a->end.mem) cudaFree(a->end.mem);
    a->end = Snap{};
}

}  // namespace

extern "C" void lbib_adjoint_destroy(lbib_adjoint* a) {
    if (!a) return;
    if (a->c && a->c->stream) cudaStreamSynchronize(a->c->stream);
    adjoint_free_snaps(a);
    for (void* p : a->allocs) cudaFree(p);
    delete a;
}

extern "C" lbib_status lbib_adjoint_create(lbib_ctx* c, int32_t checkpoint_every, lbib_adjoint** out) {
    if (!c || !out) return LBIB_E_INVALID;
    *out = nullptr;
    if (checkpoint_every < 1) return fail(c, LBIB_E_INVALID, "checkpoint interval must be at least 1");
    if (c->uw_bot != 0.0 || c->uw_top != 0.0) return fail(c, LBIB_E_INVALID, "the adjoint needs resting walls");
    if (c->walls == LBIB_WALLS_ZOU_HE) return fail(c, LBIB_E_INVALID, "the adjoint needs half-way or no walls");
    for (size_t m = 0; m < c->h_mem_kind.size(); ++m) {
        if (c->h_mem_kind[m] != LBIB_MEMBRANE_KINEMATIC)
            return fail(c, LBIB_E_INVALID, "the adjoint supports kinematic membranes only");
        if (c->h_mem_n[m] < 5) return fail(c, LBIB_E_INVALID, "the adjoint needs membranes of at least 5 vertices");
    }
    lbib_status st = finalize(c);
    if (st == LBIB_OK) st = build_graphs(c);
    if (st != LBIB_OK) return st;
    lbib_adjoint* a = new lbib_adjoint();
    a->c = c;
    a->K = checkpoint_every;
    const size_t N = (size_t)c->nx * c->ny, nv = std::max(c->nv, 1), nm = std::max(c->nmem, 1);
    const size_t nl = std::max(c->nlig, 1), K = (size_t)checkpoint_every;
    auto get = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        a->allocs.push_back(p);
        return p;
    };
    bool ok = (a->tape_f = (double*)get(K * 9 * N * 8)) && (a->tape_X = (double*)get(K * 2 * nv * 8)) &&
              (a->tape_bond = (int*)get(K * nl * 4));
    ok = ok && (a->tape_F = (double*)get(K * 2 * nv * 8)) && (a->tape_W = (double*)get(K * 9 * nv * 8)) &&
         (a->tape_st = (int*)get(K * 2 * nv * 4)) && (a->tape_G = (longlong2*)get(K * N * sizeof(longlong2)));
    ok = ok && (a->fbar[0] = (double*)get(9 * N * 8)) && (a->fbar[1] = (double*)get(9 * N * 8)) &&
         (a->fio = (double*)get(9 * N * 8));
    ok = ok && (a->XB[0] = (double*)get(2 * nv * 8)) && (a->XB[1] = (double*)get(2 * nv * 8)) &&
         (a->XPB = (double*)get(2 * nv * 8)) && (a->Wbar = (double*)get(9 * nv * 8));
    ok = ok && (a->ubar = (double*)get(2 * N * 8)) && (a->Gbar = (double*)get(2 * N * 8));
    ok = ok && (a->Abar = (double*)get(nm * 8)) && (a->ksb = (double*)get(nm * 8)) && (a->kbb = (double*)get(nm * 8)) &&
         (a->sgb = (double*)get(8));
    // areas and boxes of every taped step (one launch per segment)
    ok = ok && (a->A = (double*)get(K * nm * 8)) && (a->Ad = (double*)get(nm * 8)) &&
         (a->box = (double*)get(K * 4 * nm * 8));
    ok = ok && (a->zero = (double*)get(std::max(2 * nv, nm) * 8)) && (a->th0 = (double*)get(nv * 8)) &&
         (a->l0 = (double*)get(nv * 8));
    if (!ok) {
        lbib_adjoint_destroy(a);
        return fail(c, LBIB_E_OOM, "adjoint buffers (tape of the checkpoint interval)");
    }
    cudaError_t e = cudaMemsetAsync(a->ubar, 0, 2 * N * 8, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(a->zero, 0, std::max(2 * nv, nm) * 8, c->stream);
    // without markers there is no spread force: the tape's field stays zero
    if (e == cudaSuccess && c->nv == 0) e = cudaMemsetAsync(a->tape_G, 0, K * N * sizeof(longlong2), c->stream);
    if (e == cudaSuccess) e = launch_rest_fp64(c->prec, c->ma, a->l0, a->th0, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        lbib_adjoint_destroy(a);
        return cuda_fail(c, e, "adjoint set-up");
    }
    *out = a;
    return LBIB_OK;
}

extern "C" lbib_status lbib_adjoint_record(lbib_adjoint* a, int64_t n) {
    if (!a || n < 1) return LBIB_E_INVALID;
    lbib_ctx* c = a->c;
    if (c->poisoned) return fail(c, LBIB_E_STATE, "context poisoned by an earlier device-side failure");
    CK(cudaStreamSynchronize(c->stream));
    adjoint_free_snaps(a);
    a->n_rec = 0;
    a->seeded = a->reversed = false;
    const size_t bytes = snap_bytes(c);
    const int64_t nseg = (n + a->K - 1) / a->K;
    auto alloc_snap = [&](Snap& s) -> bool {
        if (cudaMalloc(&s.mem, bytes) != cudaSuccess) {
            cudaGetLastError();
            s.mem = nullptr;
            return false;
        }
        snap_layout(c, s);
        return true;
    };
    for (int64_t j = 0; j < nseg; ++j) {
        Snap s;
        if (!alloc_snap(s)) {
            adjoint_free_snaps(a);
            return fail(c, LBIB_E_OOM, "adjoint checkpoint");
        }
        a->snaps.push_back(s);
        CK(snap_copy(c, a->snaps.back(), true));
        const lbib_status st = lbib_step(c, std::min<int64_t>(a->K, n - j * a->K));
        if (st != LBIB_OK) return st;
    }
    if (!alloc_snap(a->end)) {
        adjoint_free_snaps(a);
        return fail(c, LBIB_E_OOM, "adjoint checkpoint");
    }
    CK(snap_copy(c, a->end, true));
    const lbib_status st = lbib_sync(c);
    if (st != LBIB_OK) return st;
    a->n_rec = n;
    return LBIB_OK;
}

extern "C" lbib_status lbib_adjoint_seed(lbib_adjoint* a, const double* xy_bar, const double* xy_prev_bar,
                                         const double* f_bar) {
    if (!a) return LBIB_E_INVALID;
    lbib_ctx* c = a->c;
    if (a->n_rec == 0) return fail(c, LBIB_E_STATE, "nothing recorded: call lbib_adjoint_record first");
    const size_t N = (size_t)c->nx * c->ny, nv = (size_t)c->nv, nm = std::max(c->nmem, 1);
    if (nv) {
        if (xy_bar) CK(cudaMemcpyAsync(a->XB[a->xb], xy_bar, 16 * nv, cudaMemcpyHostToDevice, c->stream));
        else CK(cudaMemsetAsync(a->XB[a->xb], 0, 16 * nv, c->stream));
        if (xy_prev_bar) CK(cudaMemcpyAsync(a->XPB, xy_prev_bar, 16 * nv, cudaMemcpyHostToDevice, c->stream));
        else CK(cudaMemsetAsync(a->XPB, 0, 16 * nv, c->stream));
    }
    if (f_bar) {
        CK(cudaMemcpyAsync(a->fio, f_bar, 9 * N * 8, cudaMemcpyHostToDevice, c->stream));
        CK(launch_adjoint_perm(a->fio, a->fbar[a->cb], c->nx, c->ny, c->walls != LBIB_WALLS_NONE, 1,
                               c->stream));
    } else {
        CK(cudaMemsetAsync(a->fbar[a->cb], 0, 9 * N * 8, c->stream));
    }
    CK(cudaMemsetAsync(a->ksb, 0, nm * 8, c->stream));
    CK(cudaMemsetAsync(a->kbb, 0, nm * 8, c->stream));
    CK(cudaMemsetAsync(a->sgb, 0, 8, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    a->seeded = true;
    a->reversed = false;
    return LBIB_OK;
}

extern "C" lbib_status lbib_adjoint_reverse(lbib_adjoint* a) {
    if (!a) return LBIB_E_INVALID;
    lbib_ctx* c = a->c;
    if (!a->seeded || a->reversed) return fail(c, LBIB_E_STATE, "the adjoint needs a fresh lbib_adjoint_seed");
    if (c->poisoned) return fail(c, LBIB_E_STATE, "context poisoned by an earlier device-side failure");
    const size_t N = (size_t)c->nx * c->ny, nv = std::max(c->nv, 1), nl = std::max(c->nlig, 1);
    for (int64_t j = (int64_t)a->snaps.size() - 1; j >= 0; --j) {
        Snap& s = a->snaps[j];
        const int len = (int)std::min<int64_t>(a->K, a->n_rec - j * a->K);
        // re-run the segment, keeping each step's state and what the step
        // computed from it (the spread field before the next step clears it)
        CK(snap_copy(c, s, false));
        auto d2d = [&](void* dst, const void* src, size_t bytes) {
            return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream);
        };
        const size_t nvr = (size_t)c->nv;
        const bool f64 = c->prec == LBIB_F64;  // other precisions: FP64 copies on the tape
        for (int k = 0; k < len; ++k) {
            if (f64) {
                // the state the step starts from, in one launch
                CopyList l{};
                l.src[0] = c->f[c->cur]; l.dst[0] = a->tape_f + (size_t)k * 9 * N; l.words[0] = 18 * N;
                l.src[1] = c->ma.X; l.dst[1] = a->tape_X + (size_t)k * 2 * nv; l.words[1] = 4 * nvr;
                l.src[2] = c->ma.bond_of_lig; l.dst[2] = a->tape_bond + (size_t)k * nl; l.words[2] = (size_t)c->nlig;
                l.n = 3;
                CK(launch_copy_words(l, c->stream));
            } else {
                CK(launch_widen_storage(c->prec, c->f[c->cur], a->tape_f + (size_t)k * 9 * N, 9 * N, c->inv_scale,
                                        c->stream));
                if (nvr) CK(launch_pos_out(c->prec, c->ma.X, a->tape_X + (size_t)k * 2 * nv, c->nv, c->stream));
                if (c->nlig) CK(d2d(a->tape_bond + (size_t)k * nl, c->ma.bond_of_lig, 4 * (size_t)c->nlig));
            }
            const int src = c->cur;
            CK(cudaGraphLaunch(c->graph[c->cur][0], c->stream));
            c->cur = 1 - c->cur;
            c->steps += 1;
            if (nvr && f64) {
                // what the step computed, in one launch
                CopyList l{};
                l.src[0] = c->ma.F; l.dst[0] = a->tape_F + (size_t)k * 2 * nv; l.words[0] = 4 * nvr;
                l.src[1] = c->ma.W; l.dst[1] = a->tape_W + (size_t)k * 9 * nv; l.words[1] = 18 * nvr;
                l.src[2] = c->ma.stencil; l.dst[2] = a->tape_st + (size_t)k * 2 * nv; l.words[2] = 2 * nvr;
                l.src[3] = c->G[src]; l.dst[3] = a->tape_G + (size_t)k * N; l.words[3] = 4 * N;
                l.n = 4;
                CK(launch_copy_words(l, c->stream));
            } else if (nvr) {
                CK(launch_widen_compute(c->prec, c->ma.F, a->tape_F + (size_t)k * 2 * nv, 2 * nvr, c->stream));
                CK(launch_widen_compute(c->prec, c->ma.W, a->tape_W + (size_t)k * 9 * nv, 9 * nvr, c->stream));
                CK(d2d(a->tape_st + (size_t)k * 2 * nv, c->ma.stencil, 8 * nvr));
                CK(d2d(a->tape_G + (size_t)k * N, c->G[src], N * sizeof(longlong2)));
            }
        }
        // areas and bounding boxes of the segment's taped positions
        CK(launch_tape_areas(c->ma, a->tape_X, len, a->A, a->box, c->stream));
        // adjoint steps, last to first
        const size_t nm = std::max(c->nmem, 1);
        for (int k = len - 1; k >= 0; --k) {
            AdjointArgs g{};
            TangentArgs& t = g.t;
            t.m = c->ma;
            t.m.X = a->tape_X + (size_t)k * 2 * nv;
            t.m.bond_of_lig = a->tape_bond + (size_t)k * nl;
            t.f = a->tape_f + (size_t)k * 9 * N;
            t.dX = a->zero;
            t.dXp = a->zero;
            t.Fv = a->tape_F + (size_t)k * 2 * nv;
            t.Wv = a->tape_W + (size_t)k * 9 * nv;
            t.st = a->tape_st + (size_t)k * 2 * nv;
            t.A = a->A + (size_t)k * nm; t.Ad = a->zero; t.box = a->box + (size_t)k * 4 * nm;
            t.dks = a->zero; t.dkb = a->zero; t.dsigma = 0.0; t.th0 = a->th0; t.l0 = a->l0;
            g.gfix = a->tape_G + (size_t)k * N;
            t.omega = 1.0 / c->tau; t.gx = c->gx; t.gy = c->gy;
            t.step = s.step + k;
            g.fbar = a->fbar[a->cb];
            g.fbar_out = a->fbar[1 - a->cb];
            g.XB = a->XB[a->xb]; g.XB_out = a->XB[1 - a->xb];
            g.XPB = a->XPB; g.ubar = a->ubar; g.Gbar = a->Gbar; g.Wbar = a->Wbar;
            g.Abar = a->Abar; g.ks_bar = a->ksb; g.kb_bar = a->kbb; g.sigma_bar = a->sgb;
            CK(launch_adjoint_step(g, c->stream));
            a->cb = 1 - a->cb;
            a->xb = 1 - a->xb;
        }
    }
    // leave the context as the recorded run left it
    CK(snap_copy(c, a->end, false));
    c->fields_valid = false;
    a->reversed = true;
    return lbib_sync(c);
}

extern "C" lbib_status lbib_adjoint_read(lbib_adjoint* a, double* xy_bar, double* xy_prev_bar, double* ks_bar,
                                         double* kb_bar, double* sigma_bar, double* f_bar) {
    if (!a) return LBIB_E_INVALID;
    lbib_ctx* c = a->c;
    if (!a->seeded) return fail(c, LBIB_E_STATE, "the adjoint has not been seeded");
    const size_t N = (size_t)c->nx * c->ny, nv = (size_t)c->nv, nm = (size_t)c->nmem;
    if (xy_bar && nv) CK(cudaMemcpyAsync(xy_bar, a->XB[a->xb], 16 * nv, cudaMemcpyDeviceToHost, c->stream));
    if (xy_prev_bar && nv) CK(cudaMemcpyAsync(xy_prev_bar, a->XPB, 16 * nv, cudaMemcpyDeviceToHost, c->stream));
    if (ks_bar && nm) CK(cudaMemcpyAsync(ks_bar, a->ksb, 8 * nm, cudaMemcpyDeviceToHost, c->stream));
    if (kb_bar && nm) CK(cudaMemcpyAsync(kb_bar, a->kbb, 8 * nm, cudaMemcpyDeviceToHost, c->stream));
    if (sigma_bar) CK(cudaMemcpyAsync(sigma_bar, a->sgb, 8, cudaMemcpyDeviceToHost, c->stream));
    if (f_bar) {
        CK(launch_adjoint_perm(a->fbar[a->cb], a->fio, c->nx, c->ny, c->walls != LBIB_WALLS_NONE, 0,
                               c->stream));
        CK(cudaMemcpyAsync(f_bar, a->fio, 9 * N * 8, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return LBIB_OK;
}

extern "C" int64_t lbib_adjoint_recorded_steps(const lbib_adjoint* a) { return a ? a->n_rec : -1; }

// ------------------------------------------------------------------ save / load
// The full step state of a context in a binary file: a header that identifies
// the set-up, then the stored populations of the current buffer (storage
// format), X^n, X^{n-1}, the bonds, the receptor occupancy (both orders), the
// repulsion segment boxes and the step counter.  Host byte order.
namespace {

constexpr char kSaveMagic[8] = {'L', 'B', 'I', 'B', 'S', 'A', 'V', '1'};

struct SaveHeader {
    char magic[8];
    int32_t version, nx, ny, prec, walls, nmem, nv, nlig, nrec, nseg, scale_exp, ndyn;
    double tau, gx, gy, uw_bot, uw_top, d_rep;
    int64_t steps;
    uint64_t setup_hash;  // of the membranes, ligands, receptors and bond parameters
};
constexpr int32_t kSaveVersion = 2;

// FNV-1a over the bytes of the set-up that the header's sizes do not pin:
// rest shapes, stiffnesses, kinds, densities, ligand elements, receptor
// positions and bond parameters
struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void bytes(const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        for (size_t k = 0; k < n; ++k) h = (h ^ b[k]) * 1099511628211ull;
    }
    template <typename T>
    void vec(const std::vector<T>& v) {
        const uint64_t n = v.size();
        bytes(&n, sizeof(n));
        if (n) bytes(v.data(), n * sizeof(T));
    }
    template <typename T>
    void val(T x) { bytes(&x, sizeof(x)); }
};

uint64_t setup_hash(const lbib_ctx* c) {
    Fnv f;
    f.vec(c->h_xy);
    f.vec(c->h_mem_off);
    f.vec(c->h_mem_n);
    f.vec(c->h_mem_kind);
    f.vec(c->h_lig_elem_local);
    f.vec(c->h_mem_lig_off);
    f.vec(c->h_ks);
    f.vec(c->h_kb);
    f.vec(c->h_ka);
    f.vec(c->h_rhop);
    f.val<int>(c->have_receptors ? 1 : 0);
    if (c->have_receptors) {
        f.vec(c->h_rec);
        const lbib_bond_params& b = c->bp;
        for (double v : {b.d_cut, b.y_eq, b.sigma, b.kf_dt, b.kr0_dt, b.beta_f, b.beta_r, b.d_break}) f.val(v);
        f.val(b.seed);
        f.val(b.instance);
    }
    return f.h;
}

SaveHeader header_of(const lbib_ctx* c) {
    SaveHeader h{};
    std::memcpy(h.magic, kSaveMagic, 8);
    h.version = kSaveVersion;
    h.nx = c->nx; h.ny = c->ny; h.prec = (int32_t)c->prec; h.walls = (int32_t)c->walls;
    h.nmem = c->nmem; h.nv = c->nv; h.nlig = c->nlig; h.nrec = c->ma.nrec; h.nseg = c->nseg;
    h.scale_exp = c->scale_exp;
    h.ndyn = c->ndyn;
    h.tau = c->tau; h.gx = c->gx; h.gy = c->gy; h.uw_bot = c->uw_bot; h.uw_top = c->uw_top; h.d_rep = c->d_rep;
    h.steps = c->steps;
    h.setup_hash = setup_hash(c);
    return h;
}

// the device arrays of the state, with their sizes in bytes
struct StatePart {
    void* dev;
    size_t bytes;
};

std::vector<StatePart> state_parts(lbib_ctx* c) {
    const size_t N = (size_t)c->nx * c->ny, nv = c->nv, nlig = c->nlig, nrec = c->ma.nrec;
    return {{c->f[c->cur], 9 * N * c->pop_elem}, {c->ma.X, 16 * nv},          {c->ma.Xp, 16 * nv},
            {c->ma.bond_of_lig, 4 * nlig},       {c->ma.owner, 4 * nrec},     {c->ma.owner_cell, 4 * nrec},
            {c->ma.seg_box, sizeof(float4) * (size_t)c->nseg},              {c->d_step, 8},
            // dynamic particles: vertex velocities and rigid states
            {c->ma.V, c->ndyn > 0 ? 2 * c->cmp_elem * nv : 0},
            {c->ma.rb, c->ndyn > 0 ? 6 * sizeof(double) * (size_t)c->nmem : 0}};
}

}  // namespace

extern "C" lbib_status lbib_save(lbib_ctx* c, const char* path) {
    if (!c || !path) return LBIB_E_INVALID;
    if (c->poisoned) return fail(c, LBIB_E_STATE, "context poisoned by an earlier device-side failure");
    lbib_status st = finalize(c);
    if (st != LBIB_OK) return st;
    CK(cudaStreamSynchronize(c->stream));
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(c, LBIB_E_INVALID, std::string("cannot open for writing: ") + path);
    const SaveHeader h = header_of(c);
    bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1;
    std::vector<char> buf;
    for (const StatePart& p : state_parts(c)) {
        if (!ok || p.bytes == 0) continue;
        buf.resize(p.bytes);
        const cudaError_t e = cudaMemcpy(buf.data(), p.dev, p.bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            std::fclose(fp);
            return cuda_fail(c, e, "save: read-back");
        }
        ok = std::fwrite(buf.data(), 1, p.bytes, fp) == p.bytes;
    }
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok) return fail(c, LBIB_E_INVALID, std::string("cannot write: ") + path);
    return LBIB_OK;
}

extern "C" lbib_status lbib_load(lbib_ctx* c, const char* path) {
    if (!c || !path) return LBIB_E_INVALID;
    lbib_status st = finalize(c);
    if (st == LBIB_OK) st = build_graphs(c);
    if (st != LBIB_OK) return st;
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(c, LBIB_E_INVALID, std::string("cannot open for reading: ") + path);
    SaveHeader h{};
    if (std::fread(&h, sizeof(h), 1, fp) != 1 || std::memcmp(h.magic, kSaveMagic, 8) != 0 || h.version != kSaveVersion) {
        std::fclose(fp);
        return fail(c, LBIB_E_INVALID, "not a saved lbib state");
    }
    const SaveHeader mine = header_of(c);
    const bool same = h.nx == mine.nx && h.ny == mine.ny && h.prec == mine.prec && h.walls == mine.walls &&
                      h.nmem == mine.nmem && h.nv == mine.nv && h.nlig == mine.nlig && h.nrec == mine.nrec &&
                      h.nseg == mine.nseg && h.scale_exp == mine.scale_exp && h.tau == mine.tau &&
                      h.gx == mine.gx && h.gy == mine.gy && h.uw_bot == mine.uw_bot && h.uw_top == mine.uw_top &&
                      h.d_rep == mine.d_rep && h.ndyn == mine.ndyn && h.setup_hash == mine.setup_hash;
    if (!same) {
        std::fclose(fp);
        return fail(c, LBIB_E_INVALID, "the saved state belongs to another set-up (lattice, precision, membranes, "
                                       "receptors or parameters differ)");
    }
    // read everything before touching the context, so that a short file leaves it as it was
    std::vector<StatePart> parts = state_parts(c);
    std::vector<std::vector<char>> data(parts.size());
    for (size_t k = 0; k < parts.size(); ++k) {
        data[k].resize(parts[k].bytes);
        if (parts[k].bytes && std::fread(data[k].data(), 1, parts[k].bytes, fp) != parts[k].bytes) {
            std::fclose(fp);
            return fail(c, LBIB_E_INVALID, "the saved state is truncated");
        }
    }
    const bool at_end = std::fgetc(fp) == EOF;
    std::fclose(fp);
    if (!at_end) return fail(c, LBIB_E_INVALID, "the saved state has bytes beyond its last part");
    CK(cudaStreamSynchronize(c->stream));
    for (size_t k = 0; k < parts.size(); ++k)
        if (parts[k].bytes)
            CK(cudaMemcpyAsync(parts[k].dev, data[k].data(), parts[k].bytes, cudaMemcpyHostToDevice, c->stream));
    // the per-step scratch back to its idle values: no spread force, no flagged
    // tiles, no bond candidates, ruptures or claims, no status
    const size_t N = (size_t)c->nx * c->ny;
    for (int p = 0; p < 2; ++p) {
        if (c->G[p]) CK(cudaMemsetAsync(c->G[p], 0, sizeof(longlong2) * N, c->stream));
        if (c->flags[p]) CK(cudaMemsetAsync(c->flags[p], 0, 4 * (size_t)c->ntiles, c->stream));
    }
    CK(cudaMemsetAsync(c->tickets, 0, 16, c->stream));
    CK(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    if (c->nlig > 0) {
        CK(cudaMemsetAsync(c->ma.cand, 0xFF, 4 * (size_t)c->nlig, c->stream));
        CK(cudaMemsetAsync(c->ma.rupt, 0xFF, 4 * (size_t)c->nlig, c->stream));
    }
    if (c->ma.nrec > 0) CK(cudaMemsetAsync(c->ma.claim, 0x7F, 4 * (size_t)c->ma.nrec, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->steps = h.steps;
    c->poisoned = false;
    c->fields_valid = false;
    return LBIB_OK;
}

// ------------------------------------------------------------------ x-slabs
// One lattice decomposed into x-slabs, each a context with two ghost columns
// (slabs.cu); one step of the group steps every slab and exchanges the ghost
// columns.
struct lbib_slabs {
    std::vector<lbib_ctx*> s;  // not owned
    cudaStream_t stream = nullptr;
    std::string err;
};

namespace {

lbib_status slabs_fail(lbib_slabs* g, lbib_status st, const std::string& msg) {
    if (g) g->err = msg;
    return st;
}

cudaError_t slabs_exchange(lbib_slabs* g) {
    SlabTable t{};
    t.n = (int)g->s.size();
    t.ny = g->s[0]->ny;
    for (int k = 0; k < t.n; ++k) {
        t.f[k] = g->s[k]->f[g->s[k]->cur];
        t.width[k] = g->s[k]->nx;
    }
    return launch_halo_exchange(t, g->s[0]->pop_elem, g->stream);
}

}  // namespace

extern "C" lbib_status lbib_slabs_create(lbib_ctx* const* slabs, int32_t n, lbib_slabs** out) {
    if (!slabs || !out || n < 2 || n > kMaxSlabs) return LBIB_E_INVALID;
    *out = nullptr;
    lbib_ctx* c0 = slabs[0];
    for (int k = 0; k < n; ++k) {
        lbib_ctx* c = slabs[k];
        if (!c) return LBIB_E_INVALID;
        for (int j = 0; j < k; ++j)
            if (slabs[j] == c) return fail(c, LBIB_E_INVALID, "a context appears twice among the slabs");
        const bool same = c->ny == c0->ny && c->prec == c0->prec && c->walls == c0->walls && c->tau == c0->tau &&
                          c->gx == c0->gx && c->gy == c0->gy && c->uw_bot == c0->uw_bot && c->uw_top == c0->uw_top &&
                          c->scale_exp == c0->scale_exp && c->stream == c0->stream;
        if (!same) return fail(c, LBIB_E_INVALID, "slabs need the same rows, precision, walls, tau, forcing and stream");
        if (c->nmem > 0) return fail(c, LBIB_E_INVALID, "slabs carry the lattice only (no membranes)");
        if (c->poisoned) return fail(c, LBIB_E_STATE, "a slab is poisoned by an earlier device-side failure");
        if (c->cur != c0->cur || c->steps != c0->steps)
            return fail(c, LBIB_E_STATE, "the slabs must be at the same step");
        lbib_status st = finalize(c);
        if (st == LBIB_OK) st = build_graphs(c);
        if (st != LBIB_OK) return st;
    }
    lbib_slabs* g = new lbib_slabs();
    g->s.assign(slabs, slabs + n);
    g->stream = c0->stream;
    cudaError_t e = slabs_exchange(g);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) {
        delete g;
        return cuda_fail(c0, e, "slab halo exchange");
    }
    *out = g;
    return LBIB_OK;
}

extern "C" lbib_status lbib_slabs_step(lbib_slabs* g, int64_t n) {
    if (!g || n < 0) return LBIB_E_INVALID;
    for (lbib_ctx* c : g->s)
        if (c->poisoned) return slabs_fail(g, LBIB_E_STATE, "a slab is poisoned by an earlier device-side failure");
    for (int64_t k = 0; k < n; ++k) {
        for (lbib_ctx* c : g->s) {
            const cudaError_t e = cudaGraphLaunch(c->graph[c->cur][0], c->stream);
            if (e != cudaSuccess) return slabs_fail(g, LBIB_E_CUDA, std::string("slab step: ") + cudaGetErrorString(e));
            c->cur = 1 - c->cur;
            c->steps += 1;
            c->fields_valid = true;
        }
        const cudaError_t e = slabs_exchange(g);
        if (e != cudaSuccess) return slabs_fail(g, LBIB_E_CUDA, std::string("halo exchange: ") + cudaGetErrorString(e));
    }
    return LBIB_OK;
}

extern "C" lbib_status lbib_slabs_sync(lbib_slabs* g) {
    if (!g) return LBIB_E_INVALID;
    for (lbib_ctx* c : g->s) {
        const lbib_status st = lbib_sync(c);
        if (st != LBIB_OK) return slabs_fail(g, st, c->err);
    }
    return LBIB_OK;
}

extern "C" const char* lbib_slabs_last_error(const lbib_slabs* g) { return g ? g->err.c_str() : "null slabs"; }

extern "C" void lbib_slabs_destroy(lbib_slabs* g) {
    if (!g) return;
    if (g->stream) cudaStreamSynchronize(g->stream);
    delete g;
}

// ------------------------------------------------------------------ slab faces
// The faces one x-slab exchanges with its neighbours when the neighbours live
// in other processes (one slab per rank): the caller moves the 3 x NY stored
// values of each face between ranks after every step.
extern "C" int32_t lbib_storage_bytes(const lbib_ctx* c) { return c ? (int32_t)c->pop_elem : -1; }

extern "C" lbib_status lbib_slab_face(lbib_ctx* c, int32_t side, int32_t out, void* buf, int32_t on_device) {
    if (!c || !buf || (side != 0 && side != 1) || (out != 0 && out != 1)) return LBIB_E_INVALID;
    if (c->nmem > 0) return fail(c, LBIB_E_INVALID, "slabs carry the lattice only (no membranes)");
    if (c->nx < 3) return fail(c, LBIB_E_INVALID, "a slab needs at least one interior column");
    lbib_status st = finalize(c);
    if (st != LBIB_OK) return st;
    // leaving: first interior column (3, 6, 7) or last interior column (1, 5, 8);
    // entering: ghost column 0 (1, 5, 8) or ghost column nx - 1 (3, 6, 7)
    static const int kPlus[3] = {1, 5, 8}, kMinus[3] = {3, 6, 7};
    const int* dirs = (side == 0) == (out == 1) ? kMinus : kPlus;
    const int col = out ? (side == 0 ? 1 : c->nx - 2) : (side == 0 ? 0 : c->nx - 1);
    const size_t e = c->pop_elem, N = (size_t)c->nx * c->ny;
    char* base = static_cast<char*>(c->f[c->cur]);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice
                                          : (out ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice);
    for (int q = 0; q < 3; ++q) {
        char* colp = base + ((size_t)dirs[q] * N + (size_t)col) * e;
        char* bufp = static_cast<char*>(buf) + (size_t)q * c->ny * e;
        if (out)
            CK(cudaMemcpy2DAsync(bufp, e, colp, (size_t)c->nx * e, e, c->ny, kind, c->stream));
        else
            CK(cudaMemcpy2DAsync(colp, (size_t)c->nx * e, bufp, e, e, c->ny, kind, c->stream));
    }
    if (!on_device) CK(cudaStreamSynchronize(c->stream));
    return LBIB_OK;
}
