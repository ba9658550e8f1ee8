// lbib_population_mass_noalloc: the FP64 mass reduction over a caller-owned
// population buffer, with its per-block partial sums kept in a fixed
// file-scope device array instead of memory allocated at run time.
//
// Who needs this: a host program that monitors mass conservation between
// steps of a long simulation from a thread that must not call cudaMalloc or
// cudaFree (those can synchronise the whole device and stall the step
// pipeline), or one whose memory pool has reserved the device memory up front,
// so that an allocation would fail.  Such a caller owns the population buffer
// and the output double; the library allocates nothing.
//
// The scratch (kMaxPartials doubles, 32 KiB) is one array per device shared by
// every call on that device: calls must not overlap in time (on different
// streams or host threads) or they race on it.  Every partial the second
// kernel reads is written by the first kernel of the same call, so nothing has
// to be cleared beforehand.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "lbib.h"

namespace {

constexpr int kBlock = 256;                              // threads of the slice kernel
constexpr int kPerThread = 64;                           // values per thread
constexpr long long kSlice = (long long)kBlock * kPerThread;  // values per block (16384)
constexpr int kMaxPartials = 4096;                       // scratch doubles (32 KiB)
constexpr long long kMaxValues = kSlice * kMaxPartials;  // 2^26 values
constexpr long long kMaxNodes = kMaxValues / 9;          // 7,456,540 lattice nodes
constexpr int kMaxDevices = 64;
constexpr unsigned kAll = 0xffffffffu;

static __device__ __align__(256) double g_mass_partials[kMaxPartials];

// block b adds the values [b kSlice, (b + 1) kSlice) in a fixed order: thread
// t takes t, t + kBlock, ...; then a fixed shuffle tree and warp order
__global__ void __launch_bounds__(kBlock) k_mass_slices(const double* __restrict__ f, long long n,
                                                        double* __restrict__ partials) {
    const long long base = (long long)blockIdx.x * kSlice + threadIdx.x;
    double acc = 0.0;
#pragma unroll 8
    for (int r = 0; r < kPerThread; ++r) {
        const long long k = base + (long long)r * kBlock;
        if (k < n) acc += __ldcs(f + k);
    }
    __shared__ double red[kBlock / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kAll, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = red[0];
        for (int w = 1; w < kBlock / 32; ++w) s += red[w];
        partials[blockIdx.x] = s;
    }
}

// one block of 1024 threads adds the n_parts partials of this call in a fixed order
__global__ void __launch_bounds__(1024) k_mass_total(const double* __restrict__ partials, int n_parts,
                                                     double* __restrict__ out) {
    double acc = 0.0;
    for (int k = threadIdx.x; k < n_parts; k += 1024) acc += partials[k];
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kAll, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = red[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kAll, acc, o);
        if (threadIdx.x == 0) *out = acc;
    }
}

std::mutex g_setup_mutex;
double* g_scratch[kMaxDevices] = {};

// device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached
cudaError_t scratch_for(int dev, double** p) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch[dev]) {
        void* q = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&q, g_mass_partials);
        if (e != cudaSuccess) return e;
        g_scratch[dev] = static_cast<double*>(q);
    }
    *p = g_scratch[dev];
    return cudaSuccess;
}

// true if p is device (or managed) memory of device dev
bool on_device(const void* p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();  // clear the error of a plain host pointer
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace

extern "C" lbib_status lbib_population_mass_noalloc(const double* f, int64_t n_nodes, double* mass,
                                                    void* stream) {
    if (n_nodes < 0 || n_nodes > kMaxNodes || !mass || (n_nodes > 0 && !f)) return LBIB_E_INVALID;
    if ((reinterpret_cast<uintptr_t>(f) & 7) || (reinterpret_cast<uintptr_t>(mass) & 7))
        return LBIB_E_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBIB_E_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return LBIB_E_INVALID;
    if (!on_device(mass, dev) || (n_nodes > 0 && !on_device(f, dev))) return LBIB_E_INVALID;
    double* partials = nullptr;
    if (scratch_for(dev, &partials) != cudaSuccess) return LBIB_E_CUDA;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long n = 9LL * n_nodes;
    const int n_parts = (int)((n + kSlice - 1) / kSlice);  // <= kMaxPartials by the size check
    if (n_parts > 0) k_mass_slices<<<n_parts, kBlock, 0, s>>>(f, n, partials);
    k_mass_total<<<1, 1024, 0, s>>>(partials, n_parts, mass);
    return cudaGetLastError() == cudaSuccess ? LBIB_OK : LBIB_E_CUDA;
}
