// Measured FP64 fused multiply-add throughput of the device: the denominator
// of the FP64 particle kernel's roofline, taken in the same process and run
// as the kernel it judges (a library facility; the paper has no counterpart).
//
// Every thread runs PROBE_CHAINS independent chains a <- a * b + c, so each
// warp always has a DFMA ready to issue and the FP64 pipe, not latency,
// bounds the kernel.  b < 1 keeps every chain finite (a tends to c / (1 - b)).
// The grid fills every SM with PROBE_BLOCKS_PER_SM CTAs.  Nothing is
// allocated: the result of the chains goes to a file-scope sink, written only
// if it equals a value it never takes, which keeps the compiler from dropping
// the work.
#include <cstdio>

#include "../../include/pic.h"
#include "pic_internal.cuh"

namespace picgb {

constexpr int PROBE_NT = 256;
constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_BLOCKS_PER_SM = 4;

static __device__ double g_probe_sink;

__global__ void __launch_bounds__(PROBE_NT) k_dfma_rate(long long iters, double b, double c) {
    double a[PROBE_CHAINS];
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = 1e-3 * threadIdx.x + i;
#pragma unroll 4
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = fma(a[i], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) s += a[i];
    if (s == -1.25e300) g_probe_sink = s;
}

// One index outside an array of one element, checked; nothing is addressed.
__global__ void k_index_probe(int* ok) {
    const bool inside = in_range(0, 1), outside = in_range(1, 1);
    if (!inside && outside) *ok = 0;  // never: in_range(0, 1) holds in every build
}

PICGB_INDEX_FLAG_READER(probe_index_flags)

}  // namespace picgb

using namespace picgb;

extern "C" PIC_API int pic_selftest_index_check(int device) {
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return PIC_ERR_CUDA;
    }
    probe_index_flags();  // clear
    k_index_probe<<<1, 1>>>(nullptr);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        fprintf(stderr, "pic_selftest_index_check: %s\n", cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    return (probe_index_flags() & ERRBIT_INDEX) ? PIC_ERR_INDEX : PIC_OK;
}

extern "C" PIC_API int pic_probe_fp64_fma(int device, int64_t iters, double* tflops, double* ms) {
    if (!tflops || !ms || iters < 1 || iters > (1LL << 30)) {
        fprintf(stderr, "pic_probe_fp64_fma: null output or iters outside 1..2^30\n");
        return PIC_ERR_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return PIC_ERR_CUDA;
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    if (nsm < 1) return PIC_ERR_CUDA;
    const int grid = nsm * PROBE_BLOCKS_PER_SM;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.0f;
    // one untimed launch, then the best of three timed ones
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            k_dfma_rate<<<grid, PROBE_NT, 0, st>>>(rep == 0 ? iters / 8 + 1 : iters, 0.999999, 1e-6);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.0f || t < best)) best = t;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess || !(best > 0.0f)) {
        fprintf(stderr, "pic_probe_fp64_fma: %s\n", cudaGetErrorString(e));
        cudaGetLastError();
        return PIC_ERR_CUDA;
    }
    const double fma_count = (double)grid * PROBE_NT * PROBE_CHAINS * (double)iters;
    *ms = best;
    *tflops = 2.0 * fma_count / (best * 1e-3) / 1e12;
    return PIC_OK;
}
