// Particle load/unload between the ABI's FP64 physical arrays and the binned
// store, and the energy diagnostics reductions.
#include "pic_internal.cuh"

namespace picgb {

constexpr int IO_NT = 256;

template <class R>
__device__ __forceinline__ R clamp_below_one(R v);
template <>
__device__ __forceinline__ double clamp_below_one<double>(double v) {
    return v < 0x1.fffffffffffffp-1 ? v : 0x1.fffffffffffffp-1;
}
template <>
__device__ __forceinline__ float clamp_below_one<float>(float v) {
    return v < 0x1.fffffep-1f ? v : 0x1.fffffep-1f;
}

// Physical position -> (cell, offset): xi = x / d, cell = floor(xi), offset =
// xi - cell, cells wrapped on periodic axes; a particle outside the domain on
// an absorbing axis is stored deactivated.  The division is a multiply by the
// host-computed 1/d (at most an ulp from the quotient; FP64 division costs
// many FP64-pipe instructions on this part), the cell a round-down conversion.
template <class R>
__device__ __forceinline__ void load_one(long long p, const double (&pos)[3], double ux, double uy, double uz,
                                         double w, const PStore<R>& dst, const GridDev& g) {
    int c[3];
    bool gone = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double xi = pos[a] * g.rd[a];
        long long ci = __double2ll_rd(xi);
        const double off = xi - (double)ci;
        if (ci < 0 || ci >= g.n[a]) {
            if (g.bc[a] == 0) {
                ci %= g.n[a];
                if (ci < 0) ci += g.n[a];
            } else {
                gone = true;
                ci = 0;
            }
        }
        c[a] = (int)ci;
        dst.off[a][p] = clamp_below_one<R>((R)off);
    }
    dst.cell[p] = gone ? (INACTIVE | pack_cell(c[0], c[1], c[2])) : pack_cell(c[0], c[1], c[2]);
    dst.u[0][p] = (R)ux;
    dst.u[1][p] = (R)uy;
    dst.u[2][p] = (R)uz;
    dst.w[p] = (R)w;
    dst.id[p] = (int)p;
}

// One particle per thread (any alignment).
template <class R>
__global__ void __launch_bounds__(IO_NT) k_load(long long n, const double* __restrict__ x, const double* __restrict__ y,
                                               const double* __restrict__ z, const double* __restrict__ ux,
                                               const double* __restrict__ uy, const double* __restrict__ uz,
                                               const double* __restrict__ w, PStore<R> dst, GridDev g) {
    const long long p = (long long)blockIdx.x * IO_NT + threadIdx.x;
    if (p >= n) return;
    const double pos[3] = {x[p], y[p], z[p]};
    load_one<R>(p, pos, ux[p], uy[p], uz[p], w[p], dst, g);
}

// Two particles per thread from 16-byte loads (all seven arrays 16-byte
// aligned): half the load instructions, which matters when the arrays are
// page-locked host memory read over the CPU-GPU link.
template <class R>
__global__ void __launch_bounds__(IO_NT) k_load2(long long n, const double2* __restrict__ x,
                                                const double2* __restrict__ y, const double2* __restrict__ z,
                                                const double2* __restrict__ ux, const double2* __restrict__ uy,
                                                const double2* __restrict__ uz, const double2* __restrict__ w,
                                                PStore<R> dst, GridDev g) {
    const long long q = (long long)blockIdx.x * IO_NT + threadIdx.x;  // pair index
    if (2 * q >= n) return;
    if (2 * q + 1 < n) {
        const double2 X = x[q], Y = y[q], Z = z[q], U = ux[q], V = uy[q], S = uz[q], Wt = w[q];
        const double p0[3] = {X.x, Y.x, Z.x}, p1[3] = {X.y, Y.y, Z.y};
        load_one<R>(2 * q, p0, U.x, V.x, S.x, Wt.x, dst, g);
        load_one<R>(2 * q + 1, p1, U.y, V.y, S.y, Wt.y, dst, g);
    } else {  // odd tail: scalar loads of the last particle
        const double* xs = reinterpret_cast<const double*>(x);
        const long long p = 2 * q;
        const double pos[3] = {xs[p], reinterpret_cast<const double*>(y)[p], reinterpret_cast<const double*>(z)[p]};
        load_one<R>(p, pos, reinterpret_cast<const double*>(ux)[p], reinterpret_cast<const double*>(uy)[p],
                    reinterpret_cast<const double*>(uz)[p], reinterpret_cast<const double*>(w)[p], dst, g);
    }
}

// Active particles -> FP64 physical arrays, compacted through one counter.
template <class R>
__global__ void __launch_bounds__(IO_NT) k_unload(PStore<R> src, const long long* __restrict__ n_cur, GridDev g,
                                                 int* __restrict__ counter, long long cap, long long* __restrict__ id,
                                                 double* __restrict__ x, double* __restrict__ y,
                                                 double* __restrict__ z, double* __restrict__ ux,
                                                 double* __restrict__ uy, double* __restrict__ uz,
                                                 double* __restrict__ w) {
    const long long N = *n_cur;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * IO_NT;
    for (long long base = (long long)blockIdx.x * IO_NT + (threadIdx.x & ~31); base < N; base += stride) {
        const long long p = base + lane;
        const int cp = p < N ? src.cell[p] : INACTIVE;
        const int q = warp_agg_slot(counter, cp < 0 ? -1 : 0);
        if (q >= 0 && q < cap) {
            id[q] = src.id[p];
            x[q] = ((double)cell_x(cp) + (double)src.off[0][p]) * g.d[0];
            y[q] = ((double)cell_y(cp) + (double)src.off[1][p]) * g.d[1];
            z[q] = ((double)cell_z(cp) + (double)src.off[2][p]) * g.d[2];
            ux[q] = (double)src.u[0][p];
            uy[q] = (double)src.u[1][p];
            uz[q] = (double)src.u[2][p];
            w[q] = (double)src.w[p];
        }
    }
}

template <class R>
__global__ void __launch_bounds__(IO_NT) k_count_active(PStore<R> src, const long long* __restrict__ n_cur,
                                                       int* __restrict__ counter) {
    const long long N = *n_cur;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * IO_NT;
    for (long long base = (long long)blockIdx.x * IO_NT + (threadIdx.x & ~31); base < N; base += stride) {
        const long long p = base + lane;
        const int cp = p < N ? src.cell[p] : INACTIVE;
        warp_agg_slot(counter, cp < 0 ? -1 : 0);
    }
}

// Kinetic energy partial sums m * sum w (gamma - 1), FP64, one per block.
template <class R>
__global__ void __launch_bounds__(IO_NT) k_kinetic(PStore<R> src, const long long* __restrict__ n_cur, double mass,
                                                  double* __restrict__ part) {
    __shared__ double red[IO_NT / 32];
    const long long N = *n_cur;
    double s = 0.0;
    for (long long p = (long long)blockIdx.x * IO_NT + threadIdx.x; p < N; p += (long long)gridDim.x * IO_NT) {
        if (src.cell[p] < 0) continue;
        const double ux = src.u[0][p], uy = src.u[1][p], uz = src.u[2][p];
        const double u2p1 = fma(ux, ux, fma(uy, uy, fma(uz, uz, 1.0)));
        s += (double)src.w[p] * fma(u2p1, rsqrt(u2p1), -1.0);
    }
    const double t = block_sum<IO_NT>(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t * mass;
}

// out[0] = 0.5 dV sum(wf_part[0..nwf)), out[1] = sum(ek_part[0..nek)); fixed order.
__global__ void k_energy_finalize(const double* __restrict__ wf_part, int nwf, const double* __restrict__ ek_part,
                                  int nek, double half_dV, double* __restrict__ out) {
    __shared__ double red[32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nwf; i += 1024) a += wf_part[i];
    for (int i = threadIdx.x; i < nek; i += 1024) b += ek_part[i];
    const double sa = block_sum<1024>(a, red);
    const double sb = block_sum<1024>(b, red);
    if (threadIdx.x == 0) {
        out[0] = half_dV * sa;
        out[1] = sb;
    }
}

// Largest |w| of an FP32 store (non-negative floats order like their bit
// patterns, so an unsigned atomicMax on the bits is a float max).
__global__ void __launch_bounds__(IO_NT) k_wmax(const float* __restrict__ w, const long long* __restrict__ n_cur,
                                               float* __restrict__ wmax) {
    const long long N = *n_cur;
    unsigned m = 0;
    for (long long p = (long long)blockIdx.x * IO_NT + threadIdx.x; p < N; p += (long long)gridDim.x * IO_NT)
        m = max(m, __float_as_uint(fabsf(w[p])));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(reinterpret_cast<unsigned*>(wmax), m);
}

cudaError_t wmax_launch(cudaStream_t st, int nsm, const float* w, const long long* n, float* wmax) {
    cudaError_t e = cudaMemsetAsync(wmax, 0, sizeof(float), st);
    if (e != cudaSuccess) return e;
    k_wmax<<<nsm * 4, IO_NT, 0, st>>>(w, n, wmax);
    return cudaGetLastError();
}

template <class R>
cudaError_t load_launch(cudaStream_t st, long long n, const double* const* src7, const PStore<R>& dst,
                        const GridDev& g) {
    if (n <= 0) return cudaSuccess;
    bool aligned = true;
    for (int k = 0; k < 7; ++k) aligned = aligned && (reinterpret_cast<uintptr_t>(src7[k]) & 15) == 0;
    if (aligned) {
        const long long pairs = (n + 1) / 2;
        const int grid = (int)((pairs + IO_NT - 1) / IO_NT);
        const double2* v[7];
        for (int k = 0; k < 7; ++k) v[k] = reinterpret_cast<const double2*>(src7[k]);
        k_load2<R><<<grid, IO_NT, 0, st>>>(n, v[0], v[1], v[2], v[3], v[4], v[5], v[6], dst, g);
    } else {
        const int grid = (int)((n + IO_NT - 1) / IO_NT);
        k_load<R><<<grid, IO_NT, 0, st>>>(n, src7[0], src7[1], src7[2], src7[3], src7[4], src7[5], src7[6], dst, g);
    }
    return cudaGetLastError();
}

template <class R>
cudaError_t unload_launch(cudaStream_t st, int nsm, const PStore<R>& src, const long long* n_cur, const GridDev& g,
                          int* counter, long long cap, long long* id, double* const* dst7) {
    k_unload<R><<<nsm * 8, IO_NT, 0, st>>>(src, n_cur, g, counter, cap, id, dst7[0], dst7[1], dst7[2], dst7[3],
                                          dst7[4], dst7[5], dst7[6]);
    return cudaGetLastError();
}

template <class R>
cudaError_t count_launch(cudaStream_t st, int nsm, const PStore<R>& src, const long long* n_cur, int* counter) {
    k_count_active<R><<<nsm * 8, IO_NT, 0, st>>>(src, n_cur, counter);
    return cudaGetLastError();
}

template <class R>
cudaError_t kinetic_launch(cudaStream_t st, int grid, const PStore<R>& src, const long long* n_cur, double mass,
                           double* part) {
    k_kinetic<R><<<grid, IO_NT, 0, st>>>(src, n_cur, mass, part);
    return cudaGetLastError();
}

cudaError_t energy_finalize_launch(cudaStream_t st, const double* wf_part, int nwf, const double* ek_part, int nek,
                                   double half_dV, double* out) {
    k_energy_finalize<<<1, 1024, 0, st>>>(wf_part, nwf, ek_part, nek, half_dV, out);
    return cudaGetLastError();
}

#define PICGB_IO_INST(R)                                                                                             \
    template cudaError_t load_launch<R>(cudaStream_t, long long, const double* const*, const PStore<R>&,            \
                                        const GridDev&);                                                            \
    template cudaError_t unload_launch<R>(cudaStream_t, int, const PStore<R>&, const long long*, const GridDev&,    \
                                          int*, long long, long long*, double* const*);                             \
    template cudaError_t count_launch<R>(cudaStream_t, int, const PStore<R>&, const long long*, int*);              \
    template cudaError_t kinetic_launch<R>(cudaStream_t, int, const PStore<R>&, const long long*, double, double*);
PICGB_IO_INST(double)
PICGB_IO_INST(float)

}  // namespace picgb
