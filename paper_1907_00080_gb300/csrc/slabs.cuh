// Halo exchange between the x-slabs of one lattice (slabs.cu).
#pragma once

#include <cuda_runtime.h>

namespace lbib {

constexpr int kMaxSlabs = 16;

struct SlabTable {
    void* f[kMaxSlabs];      // each slab's current stored populations [9][ny][width]
    int width[kMaxSlabs];    // W_k + 2 (two ghost columns)
    int n, ny;
};

cudaError_t launch_halo_exchange(const SlabTable& t, size_t elem, cudaStream_t s);

}  // namespace lbib
