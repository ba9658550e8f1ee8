// Per-membrane observables of the margination and adhesion studies (Sec. 4):
// centroid, centroid velocity, region of the channel, bonds, lowest and
// highest vertex; FP64 reductions in a fixed order (one block per membrane).
#include "ext_real.cuh"
#include "lbib_internal.cuh"

namespace lbib {
namespace {

constexpr int kObsThreads = 256;

template <typename C>
__global__ void __launch_bounds__(kObsThreads) k_observables(const MarkerArgs a, double* out) {
    const int m = blockIdx.x;
    const int off = a.mem_off[m], n = a.mem_n[m];
    double sx = 0.0, sy = 0.0, su = 0.0, sv = 0.0, ylo = 1e300, yhi = -1e300, nb = 0.0;
    for (int k = threadIdx.x; k < n; k += kObsThreads) {
        typename Ext<C>::E x, y, xp, yp;
        PosIO<C>::load(a.X, off + k, x, y);
        PosIO<C>::load(a.Xp, off + k, xp, yp);
        const double xd = etod(x), yd = etod(y);
        sx += xd;
        sy += yd;
        su += xd - etod(xp);
        sv += yd - etod(yp);
        ylo = fmin(ylo, yd);
        yhi = fmax(yhi, yd);
    }
    for (int l = a.mem_lig_off[m] + threadIdx.x; l < a.mem_lig_off[m + 1]; l += kObsThreads)
        nb += a.bond_of_lig[l] >= 0 ? 1.0 : 0.0;
    __shared__ double r[7][kObsThreads];
    r[0][threadIdx.x] = sx;
    r[1][threadIdx.x] = sy;
    r[2][threadIdx.x] = su;
    r[3][threadIdx.x] = sv;
    r[4][threadIdx.x] = nb;
    r[5][threadIdx.x] = ylo;
    r[6][threadIdx.x] = yhi;
    __syncthreads();
    for (int o = kObsThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            for (int q = 0; q < 5; ++q) r[q][threadIdx.x] += r[q][threadIdx.x + o];
            r[5][threadIdx.x] = fmin(r[5][threadIdx.x], r[5][threadIdx.x + o]);
            r[6][threadIdx.x] = fmax(r[6][threadIdx.x], r[6][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double inv = 1.0 / (double)n;
        const double yc = r[1][0] * inv;
        // the three regions of the channel by the centroid's height over H = NY
        // above the lower wall: bulk 0.3..0.7, intermediate 0.2..0.3 and 0.7..0.8,
        // cell-free layer below 0.2 and above 0.8
        const double h = (yc + 0.5) / (double)a.ny;
        const double region = (h >= 0.3 && h <= 0.7) ? 0.0 : ((h >= 0.2 && h <= 0.8) ? 1.0 : 2.0);
        double* o = out + 8 * (size_t)m;
        o[0] = r[0][0] * inv;
        o[1] = yc;
        o[2] = r[2][0] * inv;
        o[3] = r[3][0] * inv;
        o[4] = region;
        o[5] = r[4][0];
        o[6] = r[5][0] + 0.5;
        o[7] = r[6][0] + 0.5;
    }
}

}  // namespace

cudaError_t launch_observables(lbib_precision prec, const MarkerArgs& a, double* out, cudaStream_t s) {
    if (a.nmem == 0) return cudaSuccess;
    if (prec == LBIB_F64) k_observables<double><<<a.nmem, kObsThreads, 0, s>>>(a, out);
    else k_observables<float><<<a.nmem, kObsThreads, 0, s>>>(a, out);
    return cudaGetLastError();
}

}  // namespace lbib
