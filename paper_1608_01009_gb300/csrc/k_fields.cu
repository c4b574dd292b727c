// Yee FDTD field update (the Maxwell stage of arXiv:1608.01009 Sec. 2, which
// the paper times as "Other"), one thread per cell, x fastest (coalesced).
//
//   k_fdtd_b : B <- B - (dt/2) curl E   (forward differences of E)
//   k_fdtd_e : E <- E + dt (curl B - J) (backward differences of B); folds the
//              ghost images of J onto their owner, records the folded J and
//              zeroes every J entry it read, ready for the next deposit
// Each kernel writes its result into the cell's periodic ghost images too, so
// the next stencil and the next TMA field tile read valid ghosts with no
// separate exchange pass.  The second B half step also refreshes the FP32
// field copy (mixed mode) and writes per-block field-energy partial sums.
// Along an absorbing axis the ghosts stay zero (no field outside the domain)
// and each updated component is damped inside the layer.
#include "pic_internal.cuh"

namespace picgb {

// Image list of domain index i along an axis: the cell itself plus, on a
// periodic axis, the ghost copy at i+n (i < PAD) or i-n (i >= n-PAD).  On an
// absorbing axis the ghosts i-PAD (i < PAD) / i+PAD (i >= n-PAD) are listed
// with fold = false, so the J fold zeroes them without adding them.
struct Img {
    int idx[2];
    bool fold[2];
    int cnt;
};

__device__ __forceinline__ Img images(int i, int n, int bc) {
    Img m;
    m.idx[0] = i;
    m.fold[0] = true;
    m.cnt = 1;
    if (i < PAD) {
        m.idx[1] = bc == 0 ? i + n : i - PAD;
        m.fold[1] = bc == 0;
        m.cnt = 2;
    } else if (i >= n - PAD) {
        m.idx[1] = bc == 0 ? i - n : i + PAD;
        m.fold[1] = bc == 0;
        m.cnt = 2;
    }
    return m;
}

// Damping of the absorbing layer at lattice coordinate p (cells) along an axis of n cells.
__device__ __forceinline__ double damp1(const GridDev& g, double p, int n) {
    double dist = fmin(p, (double)n - p);
    double L = (double)g.absorb_cells;
    if (g.absorb_cells <= 0 || dist >= L) return 1.0;
    double r = (L - dist) * g.absorb_rL;
    return 1.0 - g.absorb_sigma * r * r;
}

// Product of the layer factors for component `comp` at cell (i,j,k);
// `magnetic` selects the B staggering.  The factors come from the context's
// table (g.damp, filled once by k_damp_table with damp1), which spares the
// field kernels about 8 FP64 operations per component and absorbing axis.
__device__ __forceinline__ double damping(const GridDev& g, int comp, bool magnetic, int i, int j, int k) {
    double f = 1.0;
    int ijk[3] = {i, j, k};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (g.bc[a] == 0) continue;
        const bool half = magnetic ? comp != a : comp == a;
        if (g.damp)
            f *= g.damp[g.damp_off[a] + (half ? g.n[a] : 0) + ijk[a]];
        else
            f *= damp1(g, ijk[a] + (half ? 0.5 : 0.0), g.n[a]);
    }
    return f;
}

// The layer factors of every absorbing axis at its whole and half-shifted
// lattice points (1 on periodic axes); one thread per entry.
__global__ void k_damp_table(GridDev g, double* __restrict__ tab) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    int a = 0, r = t;
    while (a < 3 && r >= 2 * g.n[a]) r -= 2 * g.n[a++];
    if (a >= 3) return;
    const int half = r >= g.n[a], i = half ? r - g.n[a] : r;
    tab[g.damp_off[a] + r] = g.bc[a] != 0 ? damp1(g, i + (half ? 0.5 : 0.0), g.n[a]) : 1.0;
}

__device__ __forceinline__ bool any_absorbing(const GridDev& g) { return (g.bc[0] | g.bc[1] | g.bc[2]) != 0; }

// Store v at the cell and at its periodic ghost images (absorbing ghosts stay 0).
// (Loops run to the fixed bound of two images, so the image lists stay in
// registers.)
template <class R>
__device__ __forceinline__ void store_images(R* A, const GridDev& g, const Img& ix, const Img& iy, const Img& iz,
                                             R v) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (c >= iz.cnt || !iz.fold[c]) continue;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            if (b >= iy.cnt || !iy.fold[b]) continue;
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                if (a >= ix.cnt || !ix.fold[a]) continue;
                A[pidx(g, ix.idx[a], iy.idx[b], iz.idx[c])] = v;
            }
        }
    }
}

// Launch geometry: blocks of 32 x 4 cells in x,y, one z plane per grid z, so
// (i,j,k) come from the block and thread indices without integer division;
// the update kernels are held to 64 registers, 8 blocks per SM (measured:
// field stage 0.340 -> 0.323 ms per step at 128^3, 0.730 -> 0.685 ms on the
// 256 x 128 x 128 laser ramp, against 32 x 8 blocks at 70 registers).
#ifndef PICGB_FDTD_BX
#define PICGB_FDTD_BX 32
#endif
#ifndef PICGB_FDTD_BY
#define PICGB_FDTD_BY 4
#endif
#ifndef PICGB_FDTD_MINB
#define PICGB_FDTD_MINB 8
#endif
constexpr int FDTD_BX = PICGB_FDTD_BX, FDTD_BY = PICGB_FDTD_BY, FDTD_NT = FDTD_BX * FDTD_BY;

__device__ __forceinline__ bool cell_of_thread(const GridDev& g, int& i, int& j, int& k) {
    i = blockIdx.x * FDTD_BX + threadIdx.x;
    j = blockIdx.y * FDTD_BY + threadIdx.y;
    k = blockIdx.z;
    return i < g.n[0] && j < g.n[1];
}

__device__ __forceinline__ int flat_block() { return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z); }

// hr[a] = h / d_a and dtr[a] = dt / d_a come from the host: each component's
// update is then two differences and two (B) or three (E) fused multiply-adds,
// FP64-pipe issue being what these kernels spend most.
struct Fac3 {
    double v[3];
};

__global__ void __launch_bounds__(FDTD_NT, PICGB_FDTD_MINB) k_fdtd_b(double* __restrict__ EB, GridDev g, Fac3 hr, int last,
                                                    float* __restrict__ EB32, double* __restrict__ wf_part) {
    __shared__ double red[FDTD_NT / 32];
    double e2 = 0.0;
    int i, j, k;
    if (cell_of_thread(g, i, j, k)) {
        const long long o = pidx(g, i, j, k);
        const long long sy = g.np[0], sz = (long long)g.np[0] * g.np[1];
        const double* Ex = EB;
        const double* Ey = EB + g.P;
        const double* Ez = EB + 2 * g.P;
        double* B = EB + 3 * g.P;
        const double hx = hr.v[0], hy = hr.v[1], hz = hr.v[2];
        const double ex = Ex[o], ey = Ey[o], ez = Ez[o];
        // B - h curl E, curl E = (dy Ez - dz Ey, dz Ex - dx Ez, dx Ey - dy Ex) by forward differences
        double b[3] = {fma(-hy, Ez[o + sy] - ez, fma(hz, Ey[o + sz] - ey, B[o])),
                       fma(-hz, Ex[o + sz] - ex, fma(hx, Ez[o + 1] - ez, B[g.P + o])),
                       fma(-hx, Ey[o + 1] - ey, fma(hy, Ex[o + sy] - ex, B[2 * g.P + o]))};
        if (any_absorbing(g))
            for (int c = 0; c < 3; ++c) b[c] *= damping(g, c, true, i, j, k);
        const Img ix = images(i, g.n[0], g.bc[0]), iy = images(j, g.n[1], g.bc[1]), iz = images(k, g.n[2], g.bc[2]);
        for (int c = 0; c < 3; ++c) store_images(B + c * g.P, g, ix, iy, iz, b[c]);
        if (last) {
            if (EB32) {
                const double e[3] = {ex, ey, ez};
                for (int c = 0; c < 3; ++c) {
                    store_images(EB32 + c * g.P, g, ix, iy, iz, (float)e[c]);
                    store_images(EB32 + (3 + c) * g.P, g, ix, iy, iz, (float)b[c]);
                }
            }
            e2 = ex * ex + ey * ey + ez * ez + b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
        }
    }
    if (last) {
        const double s = block_sum<FDTD_NT>(e2, red);
        if (threadIdx.x == 0 && threadIdx.y == 0) wf_part[flat_block()] = s;
    }
}

__global__ void __launch_bounds__(FDTD_NT, PICGB_FDTD_MINB) k_fdtd_e(double* __restrict__ EB, double* __restrict__ J,
                                                    double* __restrict__ Jlast, GridDev g, Fac3 dtr) {
    const long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
    int i, j, k;
    if (!cell_of_thread(g, i, j, k)) return;
    const long long t = i + (long long)g.n[0] * (j + (long long)g.n[1] * k);
    const long long o = pidx(g, i, j, k);
    const long long sy = g.np[0], sz = (long long)g.np[0] * g.np[1];
    const double* Bx = EB + 3 * g.P;
    const double* By = EB + 4 * g.P;
    const double* Bz = EB + 5 * g.P;
    // every load of the cell first (they are independent), then the ghost fold
    const double bx = Bx[o], by = By[o], bz = Bz[o];
    const double bz_y = Bz[o - sy], by_z = By[o - sz], bx_z = Bx[o - sz], bz_x = Bz[o - 1], by_x = By[o - 1],
                 bx_y = Bx[o - sy];
    const double e0 = EB[o], e1 = EB[g.P + o], e2 = EB[2 * g.P + o];
    double jc[3] = {J[o], J[g.P + o], J[2 * g.P + o]};
    const Img ix = images(i, g.n[0], g.bc[0]), iy = images(j, g.n[1], g.bc[1]), iz = images(k, g.n[2], g.bc[2]);
    if (ix.cnt * iy.cnt * iz.cnt > 1) {
        // boundary cell: add the periodic ghost images of J, zero every image read
#pragma unroll
        for (int c3 = 0; c3 < 2; ++c3)
#pragma unroll
            for (int b3 = 0; b3 < 2; ++b3)
#pragma unroll
                for (int a3 = 0; a3 < 2; ++a3) {
                    if (c3 >= iz.cnt || b3 >= iy.cnt || a3 >= ix.cnt || (a3 | b3 | c3) == 0) continue;
                    const long long q = pidx(g, ix.idx[a3], iy.idx[b3], iz.idx[c3]);
                    const bool fold = ix.fold[a3] && iy.fold[b3] && iz.fold[c3];
                    for (int c = 0; c < 3; ++c) {
                        if (fold) jc[c] += J[c * g.P + q];
                        J[c * g.P + q] = 0.0;
                    }
                }
    }
    for (int c = 0; c < 3; ++c) {
        J[c * g.P + o] = 0.0;
        Jlast[c * ncell + t] = jc[c];
    }
    // E + dt (curl B - J), curl B by backward differences
    const double tx = dtr.v[0], ty = dtr.v[1], tz = dtr.v[2], dt = g.dt;
    double e[3] = {fma(ty, bz - bz_y, fma(-tz, by - by_z, fma(-dt, jc[0], e0))),
                   fma(tz, bx - bx_z, fma(-tx, bz - bz_x, fma(-dt, jc[1], e1))),
                   fma(tx, by - by_x, fma(-ty, bx - bx_y, fma(-dt, jc[2], e2)))};
    if (any_absorbing(g))
        for (int c = 0; c < 3; ++c) e[c] *= damping(g, c, false, i, j, k);
    for (int c = 0; c < 3; ++c) store_images(EB + c * g.P, g, ix, iy, iz, e[c]);
}

// Refresh ghosts (and the FP32 copy) from the domain values after E/B are set.
__global__ void __launch_bounds__(FDTD_NT) k_refresh(double* __restrict__ EB, GridDev g, float* __restrict__ EB32) {
    int i, j, k;
    if (!cell_of_thread(g, i, j, k)) return;
    const long long o = pidx(g, i, j, k);
    const Img ix = images(i, g.n[0], g.bc[0]), iy = images(j, g.n[1], g.bc[1]), iz = images(k, g.n[2], g.bc[2]);
    for (int c = 0; c < 6; ++c) {
        const double v = EB[c * g.P + o];
        store_images(EB + c * g.P, g, ix, iy, iz, v);
        if (EB32) store_images(EB32 + c * g.P, g, ix, iy, iz, (float)v);
    }
}

// Field-energy partial sums of the current state (sum of E^2 + B^2 per block).
__global__ void __launch_bounds__(FDTD_NT) k_field_energy(const double* __restrict__ EB, GridDev g,
                                                          double* __restrict__ wf_part) {
    __shared__ double red[FDTD_NT / 32];
    double e2 = 0.0;
    int i, j, k;
    if (cell_of_thread(g, i, j, k)) {
        const long long o = pidx(g, i, j, k);
        for (int c = 0; c < 6; ++c) {
            const double v = EB[c * g.P + o];
            e2 += v * v;
        }
    }
    const double s = block_sum<FDTD_NT>(e2, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) wf_part[flat_block()] = s;
}

static dim3 fdtd_grid(const GridDev& g) {
    return dim3((g.n[0] + FDTD_BX - 1) / FDTD_BX, (g.n[1] + FDTD_BY - 1) / FDTD_BY, g.n[2]);
}

int fdtd_blocks(const GridDev& g) {
    const dim3 b = fdtd_grid(g);
    return (int)(b.x * b.y * b.z);
}

cudaError_t fdtd_b_launch(cudaStream_t st, double* EB, const GridDev& g, double h, int last, float* EB32,
                          double* wf_part) {
    const Fac3 hr{{h * g.rd[0], h * g.rd[1], h * g.rd[2]}};
    k_fdtd_b<<<fdtd_grid(g), dim3(FDTD_BX, FDTD_BY), 0, st>>>(EB, g, hr, last, EB32, wf_part);
    return cudaGetLastError();
}

cudaError_t fdtd_e_launch(cudaStream_t st, double* EB, double* J, double* Jlast, const GridDev& g) {
    const Fac3 dtr{{g.dt * g.rd[0], g.dt * g.rd[1], g.dt * g.rd[2]}};
    k_fdtd_e<<<fdtd_grid(g), dim3(FDTD_BX, FDTD_BY), 0, st>>>(EB, J, Jlast, g, dtr);
    return cudaGetLastError();
}

// Fill the layer-factor table (2 (n0 + n1 + n2) doubles at damp_off[]) of g.
cudaError_t damp_table_launch(cudaStream_t st, const GridDev& g, double* tab) {
    const int n = 2 * (g.n[0] + g.n[1] + g.n[2]);
    k_damp_table<<<(n + 255) / 256, 256, 0, st>>>(g, tab);
    return cudaGetLastError();
}

cudaError_t refresh_launch(cudaStream_t st, double* EB, const GridDev& g, float* EB32) {
    k_refresh<<<fdtd_grid(g), dim3(FDTD_BX, FDTD_BY), 0, st>>>(EB, g, EB32);
    return cudaGetLastError();
}

cudaError_t field_energy_launch(cudaStream_t st, const double* EB, const GridDev& g, double* wf_part) {
    k_field_energy<<<fdtd_grid(g), dim3(FDTD_BX, FDTD_BY), 0, st>>>(EB, g, wf_part);
    return cudaGetLastError();
}

}  // namespace picgb
