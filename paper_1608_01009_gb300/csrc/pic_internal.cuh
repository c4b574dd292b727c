// Internal layouts and device helpers of libpicgb (not part of the C ABI).
//
// HBM layout
//   fields  FP64, one ghost-padded array per component, PAD = 2 ghost cells on
//           each side: padded extent np[a] = n[a] + 4, element (i,j,k) of the
//           domain at (i+2) + np0*((j+2) + np1*(k+2)).  E and B live in one
//           buffer EB of 6 consecutive components (Ex Ey Ez Bx By Bz), so one
//           4-D TMA box (x, y, z, component) stages a supercell's whole field
//           tile.  J (3 components) is a separate padded buffer that the
//           particle kernels add into; its ghost cells are folded onto their
//           periodic owners by the E update.  Mixed mode keeps an FP32 copy of
//           EB with the same geometry.
//   particles  structure of arrays, binned by supercell: per particle a
//           packed global cell index (10 bits per axis, sign bit = inactive),
//           the offset inside the cell (3 x R, in [0,1)), momentum u (3 x R),
//           weight (R) and an id (int32), R = double (FP64) or float (mixed).
//           bin_start[b] .. bin_start[b+1] are the particles of supercell b.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace picgb {

constexpr int PAD = 2;
constexpr int MAX_SPECIES = 8;

// Sticky device error bits (the host maps them to pic_status codes).
enum : int { ERRBIT_DRIFT = 1, ERRBIT_TIMEOUT = 2, ERRBIT_NAN = 4, ERRBIT_INDEX = 8 };

// Index checks of the debug build (PICGB_DEBUG=1, libpicgb_debug.so; a stand-in
// for a memory checker).  The particle kernels, the second-order form factor's
// kernel, the differentiable path's kernels and the sort's scatter pass every
// index they read or write through in_range(i, n) against the size of the array
// it addresses; an index outside sets ERRBIT_INDEX in the flag of its
// translation unit (each unit has its own copy of g_index_err, read and cleared
// by the host function PICGB_INDEX_FLAG_READER defines there) and the access is
// skipped.  Release builds compile every check to `true`.
#ifndef PICGB_DEBUG
#define PICGB_DEBUG 0
#endif
#if PICGB_DEBUG
static __device__ int g_index_err;
#endif
__device__ __forceinline__ bool in_range(long long i, long long n) {
#if PICGB_DEBUG
    if (i >= 0 && i < n) return true;
    atomicOr(&g_index_err, ERRBIT_INDEX);
    return false;
#else
    (void)i;
    (void)n;
    return true;
#endif
}
#if PICGB_DEBUG
#define PICGB_INDEX_FLAG_READER(fn)                                  \
    int fn() {                                                       \
        int v = 0, zero = 0;                                         \
        if (cudaMemcpyFromSymbol(&v, g_index_err, sizeof v) != cudaSuccess) return ERRBIT_INDEX; \
        cudaMemcpyToSymbol(g_index_err, &zero, sizeof zero);         \
        return v;                                                    \
    }
#else
#define PICGB_INDEX_FLAG_READER(fn) \
    int fn() { return 0; }
#endif
// readers of the units that check (the host ORs them into the sticky status)
int push_index_flags();
int push32_index_flags();
int tsc_index_flags();
int tape_index_flags();
int sort_index_flags();

constexpr int INACTIVE = (int)0x80000000;

struct GridDev {
    int n[3];      // cells
    int np[3];     // padded extent n + 2 PAD
    long long P;   // padded volume
    double d[3];
    double rd[3];  // 1 / d
    double dt;
    int bc[3];
    int S;         // supercell edge in cells
    int Sshift;    // log2(S)
    int nsc[3];    // supercells per axis
    int nbins;
    int absorb_cells;
    double absorb_sigma;
    double absorb_rL;  // 1 / absorb_cells (0 without a layer)
    // absorbing layer factors per axis, lattice index and staggering (device,
    // 2 n[a] doubles from damp_off[a]: whole then half-shifted points); null:
    // formed in the field kernels from the formula
    const double* damp;
    int damp_off[3];
};

template <class R>
struct PStore {
    int* cell;     // packed global cell, INACTIVE bit
    R* off[3];     // offset in cell, [0,1)
    R* u[3];       // momentum u = gamma v / c
    R* w;          // weight
    int* id;
};

struct Chunk {
    int sc;        // supercell (bin) index
    int start;     // first particle
    int count;     // particles in this chunk
    int pad;
};

struct PushParams {
    GridDev g;
    double qdt2m;   // q dt / (2 m)
    double dtd[3];  // dt / d[a]: velocity (in c) -> displacement in cells
    double cq[3];   // q / (dt d[p] d[r]): current density per unit weight and cell displacement
    double mass;
    // FP32 copies for the mixed kernel (a double -> float conversion runs on
    // the FP64 pipe, so none is left inside the particle loop)
    float qdt2m_f, dtd_f[3], cq_f[3];
    // mixed kernel: the species' largest |w| (device, written by the load), which
    // fixes the scale of the fixed-point current tile
    const float* wmax;
    // mixed kernel under the displacement-bounded sort schedule: the largest
    // gamma^2 = 1 + u^2 of this push as float bits (atomicMax; a particle's
    // displacement is |d_a| = sqrt(1 - 1/gamma^2) dt/d_a); null: not tracked
    unsigned* drift;
};

// Per-CTA queue of the moves that leave their start cell (structure of arrays,
// CHUNK entries per CTA starting at blockIdx.x * CHUNK): the particle kernel
// defers their Villasenor-Buneman split to one dense pass per chunk.
template <class R>
struct XQueue {
    int* key;   // J-tile corner index of the start cell
    R* a[3];    // start offset in the cell
    R* d[3];    // displacement (cells)
    R* w;       // weight
};

// Differentiable path: id-ordered FP64 particle state, its cotangents, and the
// per-species step constants.
struct TapeDev {
    double* xi[3];  // position in cells
    double* u[3];
    const double* w;
    int* act;       // 1 active; 0 deactivated at an absorbing boundary, or absent
};

struct LamDev {
    double* xi[3];  // cotangent of the position (in cells)
    double* u[3];   // cotangent of the momentum
};

struct StepParams {
    GridDev g;
    double qdt2m, dtd[3], cq[3], mass;
};

#ifndef PICGB_CHUNK
#define PICGB_CHUNK 4096
#endif
constexpr int CHUNK = PICGB_CHUNK;  // most particles of one supercell handled by one CTA pass

__host__ __device__ inline int pack_cell(int ix, int iy, int iz) { return ix | (iy << 10) | (iz << 20); }
__host__ __device__ inline int cell_x(int c) { return c & 1023; }
__host__ __device__ inline int cell_y(int c) { return (c >> 10) & 1023; }
__host__ __device__ inline int cell_z(int c) { return (c >> 20) & 1023; }

__host__ __device__ inline long long pidx(const GridDev& g, int i, int j, int k) {
    // padded linear index of domain cell (i,j,k) (ghosts: i in [-PAD, n+PAD))
    return (long long)(i + PAD) + (long long)g.np[0] * ((long long)(j + PAD) + (long long)g.np[1] * (k + PAD));
}

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase: returns false once `limit` polls or
// `limit_ns` nanoseconds (whichever comes first) pass without completion; the
// caller records a timeout and leaves.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase, uint32_t limit,
                                                  uint64_t limit_ns) {
    const uint32_t addr = smem_u32(bar);
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(phase)
            : "memory");
        if (done) return true;
        if ((it & 63u) == 63u && global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// 4-D tiled TMA load global -> shared, completion signalled on `bar`.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// Bulk (non-tensor) copy global -> shared of `bytes` bytes, completion signalled
// on `bar`: both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Budget of a TMA wait: far beyond any legitimate latency (microseconds), short
// enough that a kernel whose copy never lands returns within about a second.
constexpr uint32_t WAIT_LIMIT = 1u << 22;         // polls (each try_wait may suspend a while)
constexpr uint64_t WAIT_LIMIT_NS = 1000000000ull;  // 1 s of device time

// FP64 reciprocal square root and reciprocal for arguments >= 1 (the Lorentz
// factors and Boris denominators of the particle kernels): the PTX approximations as seeds
// and one correction from the binomial series, with e = 1 - x y0^2,
//   1/sqrt(x) = y0 (1 - e)^(-1/2) ~ y0 (1 + e/2 + 3 e^2/8),
// and with e = 1 - x r0,  1/x = r0 / (1 - e) ~ r0 (1 + e + e^2):
// third-order convergence, so the seeds (measured within 1e-6 relative) give a
// full FP64 result in 4 (rsqrt) and 3 (reciprocal) FP64 operations; both stay within
// 2.3e-16 relative of CUDA's rsqrt and of IEEE division over [1, 1e8] (c2
// particle kernel 5.32 -> 5.28 ms).
#ifndef PICGB_F64_NR
#define PICGB_F64_NR 1  // 0: CUDA's rsqrt and IEEE division
#endif
__device__ __forceinline__ double rsqrt_ge1(double x) {
#if PICGB_F64_NR
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x * y, y, 1.0);
    return fma(y * e, fma(e, 0.375, 0.5), y);
#else
    return rsqrt(x);
#endif
}
__device__ __forceinline__ double rcp_ge1(double x) {
#if PICGB_F64_NR
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    const double e = fma(-x, r, 1.0);
    return fma(fma(e, e, e), r, r);
#else
    return 1.0 / x;
#endif
}

// ------------------------------------------------------------------ warp helpers
// Warp-aggregated atomic add of 1 per lane on counters[key] (lanes with the
// same key are served by one atomic); returns each lane's slot.  All 32 lanes
// must call it; lanes with key < 0 take no slot and get -1.
__device__ __forceinline__ int warp_agg_slot(int* counters, int key) {
    unsigned peers = __match_any_sync(0xffffffffu, key);
    int lane = threadIdx.x & 31;
    int leader = __ffs(peers) - 1;
    int rank = __popc(peers & ((1u << lane) - 1u));
    int base = 0;
    if (lane == leader && key >= 0) base = atomicAdd(&counters[key], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    return key >= 0 ? base + rank : -1;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Fixed-order block sum (deterministic for a fixed block shape); result valid
// in the block's first thread.  Blocks may be 1-, 2- or 3-D (NT threads).
template <int NT>
__device__ double block_sum(double v, double* scratch) {
    v = warp_sum(v);
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int w = tid >> 5, l = tid & 31;
    __syncthreads();
    if (l == 0) scratch[w] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
        for (int i = 0; i < NT / 32; ++i) s += scratch[i];
    return s;
}

// ------------------------------------------------------------------ launchers (host)
cudaError_t wmax_launch(cudaStream_t st, int nsm, const float* w, const long long* n, float* wmax);

// FP64 particle kernel (k_push.cu, R = double, S = 2, 4, 8)
template <class R, int S>
cudaError_t push_setup(int* blocks_per_sm);
template <class R, int S>
cudaError_t push_launch(int grid, cudaStream_t st, const CUtensorMap& tm, const PushParams& pp, const PStore<R>& ps,
                        const PStore<R>& pin, const int* perm, const XQueue<R>& xq, const Chunk* chunks,
                        const int* nchunks, double* J, double* ek_part, int* err);
// mixed-precision particle kernel (k_push32.cu, S = 4, 8)
template <int S>
cudaError_t push32_setup(int* blocks_per_sm);
template <int S>
cudaError_t push32_launch(int grid, cudaStream_t st, const CUtensorMap& tm, const PushParams& pp,
                          const PStore<float>& ps, const PStore<float>& pin, const int* perm,
                          const XQueue<float>& xq, const Chunk* chunks, const int* nchunks, double* J,
                          double* ek_part, int* err);

}  // namespace picgb
