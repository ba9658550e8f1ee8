// Halo exchange of an x-slab decomposition of one lattice: sub-domain k is a
// context of width W_k + 2 whose columns 0 and W_k + 1 are ghost columns.
// After each step the ghost column 0 of slab k receives, for the three
// populations that stream in +x (e_x = +1: 1, 5, 8), the post-collision values
// of the last interior column of slab k - 1; the ghost column W_k + 1 receives,
// for the three that stream in -x (3, 6, 7), those of the first interior
// column of slab k + 1 (the slabs close into a ring: periodic x).  The pull of
// the next step then reads, at every interior node, exactly what it would read
// in the undivided lattice (Sec. 3: periodic x), so the interiors evolve as
// the whole lattice does.
#include "lbib_internal.cuh"
#include "slabs.cuh"

namespace lbib {
namespace {

// one thread per (slab, row, direction slot); E is the stored element
template <typename E>
__global__ void k_halo_exchange(const SlabTable t) {
    const int k = blockIdx.y;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;  // row * 6 + slot
    if (q >= 6 * t.ny) return;
    const int y = q / 6, slot = q % 6;
    const int left = (k + t.n - 1) % t.n, right = (k + 1) % t.n;
    constexpr int in_plus[3] = {1, 5, 8};   // e_x = +1: enter across the left edge
    constexpr int in_minus[3] = {3, 6, 7};  // e_x = -1: enter across the right edge
    E* mine = static_cast<E*>(t.f[k]);
    const size_t Nk = (size_t)t.width[k] * t.ny;
    if (slot < 3) {
        const int i = in_plus[slot];
        const E* src = static_cast<const E*>(t.f[left]);
        const size_t Nl = (size_t)t.width[left] * t.ny;
        mine[(size_t)i * Nk + (size_t)y * t.width[k]] = src[(size_t)i * Nl + (size_t)y * t.width[left] + t.width[left] - 2];
    } else {
        const int i = in_minus[slot - 3];
        const E* src = static_cast<const E*>(t.f[right]);
        const size_t Nr = (size_t)t.width[right] * t.ny;
        mine[(size_t)i * Nk + (size_t)y * t.width[k] + t.width[k] - 1] = src[(size_t)i * Nr + (size_t)y * t.width[right] + 1];
    }
}

}  // namespace

cudaError_t launch_halo_exchange(const SlabTable& t, size_t elem, cudaStream_t s) {
    const dim3 grid((6 * t.ny + 127) / 128, t.n);
    switch (elem) {
        case 8: k_halo_exchange<unsigned long long><<<grid, 128, 0, s>>>(t); break;
        case 4: k_halo_exchange<unsigned int><<<grid, 128, 0, s>>>(t); break;
        case 2: k_halo_exchange<unsigned short><<<grid, 128, 0, s>>>(t); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace lbib
