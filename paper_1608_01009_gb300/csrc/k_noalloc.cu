// Field energy with no allocation at all: a variant of the library's
// field-energy reduction for callers that cannot allocate device memory.
//
// The regular diagnostic (pic_energy) keeps its per-block partial sums in
// memory the context allocated with cudaMalloc.  Some callers cannot allow
// that: a host framework that owns all device memory through its own pool and
// forbids allocations behind its back, a process that has already reserved
// the whole device for its own buffers, and latency-critical loops in which
// cudaMalloc's implicit device-wide synchronisation is not acceptable.  This
// variant takes the caller's field arrays and output pointer and keeps its
// partial sums in one file-scope device array of fixed size, which every GPU
// that loads this library holds until the process exits.
#include <cstdio>
#include <mutex>

#include "../../include/pic.h"
#include "pic_internal.cuh"

namespace picgb {

constexpr int NOALLOC_NT = 256;                  // cells per block, one partial sum per block
constexpr int NOALLOC_MAX_PARTIALS = 65536;      // 512 KiB of FP64 partial sums
constexpr long long NOALLOC_MAX_CELLS = (long long)NOALLOC_MAX_PARTIALS * NOALLOC_NT;  // 16,777,216 = 256^3
constexpr int NOALLOC_MAX_DEVICES = 64;

// Scratch of the partial sums.  In host code this name is only a stand-in for
// the symbol; kernels receive the device address cudaGetSymbolAddress returns.
static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_PARTIALS];

// Per block: sum over its NOALLOC_NT cells (in linear cell order) of
// Ex^2 + Ey^2 + Ez^2 + Bx^2 + By^2 + Bz^2, written to partials[block].
__global__ void __launch_bounds__(NOALLOC_NT) k_field_energy_flat(const double* __restrict__ Ex,
                                                                   const double* __restrict__ Ey,
                                                                   const double* __restrict__ Ez,
                                                                   const double* __restrict__ Bx,
                                                                   const double* __restrict__ By,
                                                                   const double* __restrict__ Bz, long long ncell,
                                                                   double* __restrict__ partials) {
    __shared__ double red[NOALLOC_NT / 32];
    const long long t = (long long)blockIdx.x * NOALLOC_NT + threadIdx.x;
    double e2 = 0.0;
    if (t < ncell) {
        const double v[6] = {Ex[t], Ey[t], Ez[t], Bx[t], By[t], Bz[t]};
        for (int c = 0; c < 6; ++c) e2 += v[c] * v[c];
    }
    const double s = block_sum<NOALLOC_NT>(e2, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// out = half_dV * sum of partials[0..n), fixed order.
__global__ void __launch_bounds__(1024) k_field_energy_flat_sum(const double* __restrict__ partials, int n,
                                                               double half_dV, double* __restrict__ out) {
    __shared__ double red[32];
    double a = 0.0;
    for (int i = threadIdx.x; i < n; i += 1024) a += partials[i];
    const double s = block_sum<1024>(a, red);
    if (threadIdx.x == 0) *out = half_dV * s;
}

namespace {
std::mutex g_noalloc_mutex;
double* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};
}  // namespace

}  // namespace picgb

using namespace picgb;

extern "C" PIC_API int pic_field_energy_noalloc(const double* const E[3], const double* const B[3],
                                                const int32_t n[3], const double d[3], double* wf, void* stream) {
    if (!E || !B || !n || !d || !wf) {
        fprintf(stderr, "pic_field_energy_noalloc: null argument\n");
        return PIC_ERR_ARG;
    }
    for (int c = 0; c < 3; ++c) {
        if (!E[c] || !B[c]) {
            fprintf(stderr, "pic_field_energy_noalloc: null field component\n");
            return PIC_ERR_ARG;
        }
        if (n[c] <= 0 || !(d[c] > 0)) {
            fprintf(stderr, "pic_field_energy_noalloc: n and d must be positive\n");
            return PIC_ERR_ARG;
        }
    }
    const long long ncell = (long long)n[0] * n[1] * n[2];
    if (ncell > NOALLOC_MAX_CELLS) {
        fprintf(stderr,
                "pic_field_energy_noalloc: %lld cells exceed the fixed scratch of %d partial sums "
                "(at most %lld cells); use pic_energy on a context instead\n",
                ncell, NOALLOC_MAX_PARTIALS, NOALLOC_MAX_CELLS);
        return PIC_ERR_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        cudaGetLastError();
        return PIC_ERR_CUDA;
    }
    double* partials = nullptr;
    {
        // first call on this device: look up the scratch's device address (the
        // current device is the one the address belongs to)
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                fprintf(stderr, "pic_field_energy_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
                return PIC_ERR_CUDA;
            }
            g_noalloc_addr[dev] = static_cast<double*>(p);
        }
        partials = g_noalloc_addr[dev];
    }
    const int nblocks = (int)((ncell + NOALLOC_NT - 1) / NOALLOC_NT);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // every block overwrites its own partial, so nothing needs clearing first
    k_field_energy_flat<<<nblocks, NOALLOC_NT, 0, st>>>(E[0], E[1], E[2], B[0], B[1], B[2], ncell, partials);
    k_field_energy_flat_sum<<<1, 1024, 0, st>>>(partials, nblocks, 0.5 * d[0] * d[1] * d[2], wf);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "pic_field_energy_noalloc: launch failed: %s\n", cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    return PIC_OK;
}
