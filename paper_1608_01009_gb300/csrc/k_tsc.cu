// Second-order (TSC) form factor path, FP64: field gather with quadratic
// B-spline weights, Boris push, move, and Esirkepov's charge-conserving
// current, for one species.
//
// The paper fixes the cloud-in-cell form factor (Sec. 3); this is the usual
// next order of PIC codes.  The form factor is the quadratic B-spline: on the
// three lattice points nearest the particle, with delta its offset from the
// nearest one (in [-1/2, 1/2)), the weights are (1/2 - delta)^2 / 2,
// 3/4 - delta^2 and (1/2 + delta)^2 / 2, per axis, multiplied over the axes.
// Esirkepov (Comput. Phys. Commun. 135, 144 (2001)) splits the density change
// of a move, S1x S1y S1z - S0x S0y S0z, into three directional parts,
//   W_x = dSx (S0y S0z + dSy S0z / 2 + S0y dSz / 2 + dSy dSz / 3),  dS = S1 - S0,
// (y, z cyclic); the x current on the edge (i+1/2, j, k) is -Q times the
// running sum of W_x along x, Q = q w / (dt dy dz).
//
// As in the VB path the displacement enters as given: the new offset is
// taken from the old nearest node, and when that node stays the nearest the
// weight changes are the exact factored differences of the spline pieces,
// -d (1 - delta0 - delta1)/2, -d (delta0 + delta1), d (1 + delta0 + delta1)/2,
// free of the cancellation of two rounded weights for small moves.
//
// GB300 design: one thread per particle over the binned store (lanes next to
// each other share cells, so the 27-point gathers mostly hit L1), the fields
// read from the ghost-padded global grid, each non-zero current value one FP64
// RED into J with the periodic image folded in the kernel (absorbing axes drop
// what falls outside the domain).  It needs no supercell slack, so any sort
// interval works.  Spreading a warp's lanes over different cells (to keep
// their REDs off common addresses) measured 13% slower: same-cell lanes share
// the gather's cache lines, and the REDs are not the limit.
#include "pic_internal.cuh"

namespace picgb {

constexpr int TSC_NT = 256;
#ifndef PICGB_TSC_MINB
#define PICGB_TSC_MINB 2  // resident CTAs per SM the register budget is cut for
#endif
constexpr int TSC_MINB = PICGB_TSC_MINB;

// Quadratic B-spline weights of an offset delta in [-1/2, 1/2) from the
// nearest lattice point, on the points -1, 0, +1.
__device__ __forceinline__ void tsc_weights(double delta, double w[3]) {
    const double a = 0.5 - delta, b = 0.5 + delta;
    w[0] = 0.5 * a * a;
    w[1] = fma(-delta, delta, 0.75);
    w[2] = 0.5 * b * b;
}

// Offsets lie in [0, 1): compare on the bit pattern (integer ALU).
__device__ __forceinline__ bool at_least_half(double f) { return __double2hiint(f) >= 0x3FE00000; }

// End point b = offset + displacement in (-1, 2): -1, 0 or +1 cells.
__device__ __forceinline__ int tsc_cell_shift(double b) {
    const int h = __double2hiint(b);
    return h < 0 ? -1 : (h >= 0x3FF00000 ? 1 : 0);
}

// 27-point interpolation of one ghost-padded component around lattice point
// (ix, iy, iz), separable: z of y of x.
__device__ __forceinline__ double interp27(const double* __restrict__ F, const GridDev& g, int ix, int iy, int iz,
                                           const double (&wx)[3], const double (&wy)[3], const double (&wz)[3]) {
    double sum = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double sy = 0.0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const long long r0 =
                (ix - 1 + PAD) + (long long)g.np[0] * ((iy - 1 + b + PAD) + (long long)g.np[1] * (iz - 1 + c + PAD));
            if (!in_range(r0, g.P - 2)) continue;  // debug build only: the row's 3 points in the component
            const double* row = F + r0;
            const double sx = fma(wx[2], row[2], fma(wx[1], row[1], wx[0] * row[0]));
            sy = fma(wy[b], sx, sy);
        }
        sum = fma(wz[c], sy, sum);
    }
    return sum;
}

// Add v to one padded J component at domain lattice index (i, j, k), each in
// [-2, n+2]: periodic axes wrap to the owner, absorbing axes drop outside.
__device__ __forceinline__ void add_current(double* __restrict__ Jc, const GridDev& g, int i, int j, int k, double v) {
    int ijk[3] = {i, j, k};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (ijk[a] < 0 || ijk[a] >= g.n[a]) {
            if (g.bc[a] != 0) return;
            ijk[a] += ijk[a] < 0 ? g.n[a] : -g.n[a];
        }
    }
    const long long o = (ijk[0] + PAD) + (long long)g.np[0] * ((ijk[1] + PAD) + (long long)g.np[1] * (ijk[2] + PAD));
    if (in_range(o, g.P)) atomicAdd(Jc + o, v);
}

// Esirkepov current of component C.  Window index k of every axis a is the
// lattice node base[a] - 2 + k; S0, dS are zero outside [lo[a], hi[a]], so
// only those transverse rows and the edges between those nodes are visited.
// The loops stay rolled: unrolled, the three components' guarded 5 x 5 x 4
// bodies overflow the instruction cache.
template <int C>
__device__ __forceinline__ void esirkepov_component(double* __restrict__ Jc, const GridDev& g, const int (&base)[3],
                                                    const double (&S0)[3][5], const double (&dS)[3][5],
                                                    const int (&lo)[3], const int (&hi)[3], double Q) {
    constexpr int P = (C + 1) % 3, R = (C + 2) % 3;
#pragma unroll 1
    for (int jp = lo[P]; jp <= hi[P]; ++jp) {
#pragma unroll 1
        for (int jr = lo[R]; jr <= hi[R]; ++jr) {
            const double t = fma(S0[P][jp], S0[R][jr],
                                 fma(0.5 * dS[P][jp], S0[R][jr],
                                     fma(0.5 * S0[P][jp], dS[R][jr], dS[P][jp] * dS[R][jr] * (1.0 / 3.0))));
            double run = 0.0;
#pragma unroll 1
            for (int i = lo[C]; i < hi[C]; ++i) {
                run = fma(dS[C][i], t, run);
                int idx[3];
                idx[C] = base[C] - 2 + i;
                idx[P] = base[P] - 2 + jp;
                idx[R] = base[R] - 2 + jr;
                add_current(Jc, g, idx[0], idx[1], idx[2], -Q * run);
            }
        }
    }
}

__global__ void __launch_bounds__(TSC_NT, TSC_MINB) k_push_tsc(PStore<double> ps, const long long* __restrict__ n_cur,
                                                     PushParams pp, const double* __restrict__ EB,
                                                     double* __restrict__ J, double* __restrict__ ek_part) {
    __shared__ double red[TSC_NT / 32];
    const GridDev& g = pp.g;
    const long long N = *n_cur;
    const long long P = g.P;
    double ek = 0.0;
    for (long long p = (long long)blockIdx.x * TSC_NT + threadIdx.x; p < N; p += (long long)gridDim.x * TSC_NT) {
        const int cp = ps.cell[p];
        if (cp < 0) continue;
        const int gc[3] = {cell_x(cp), cell_y(cp), cell_z(cp)};
        const double f[3] = {ps.off[0][p], ps.off[1][p], ps.off[2][p]};
        double ux = ps.u[0][p], uy = ps.u[1][p], uz = ps.u[2][p];
        const double w = ps.w[p];

        // ---- gather: node lattice (centre = nearest node) and half-shifted
        // lattice (centre = the cell itself) weights per axis
        int cN[3], cH[3];
        double s0[3], wN[3][3], wH[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const bool up = at_least_half(f[a]);
            cN[a] = gc[a] + (up ? 1 : 0);
            s0[a] = up ? f[a] - 1.0 : f[a];
            cH[a] = gc[a];
            tsc_weights(s0[a], wN[a]);
            tsc_weights(f[a] - 0.5, wH[a]);
        }
        const double Ex = interp27(EB + 0 * P, g, cH[0], cN[1], cN[2], wH[0], wN[1], wN[2]);
        const double Ey = interp27(EB + 1 * P, g, cN[0], cH[1], cN[2], wN[0], wH[1], wN[2]);
        const double Ez = interp27(EB + 2 * P, g, cN[0], cN[1], cH[2], wN[0], wN[1], wH[2]);
        const double Bx = interp27(EB + 3 * P, g, cN[0], cH[1], cH[2], wN[0], wH[1], wH[2]);
        const double By = interp27(EB + 4 * P, g, cH[0], cN[1], cH[2], wH[0], wN[1], wH[2]);
        const double Bz = interp27(EB + 5 * P, g, cH[0], cH[1], cN[2], wH[0], wH[1], wN[2]);

        // ---- Boris: half electric kick, rotation t = (q dt / 2 m gamma^-) B, half kick
        const double h = pp.qdt2m;
        const double umx = fma(h, Ex, ux), umy = fma(h, Ey, uy), umz = fma(h, Ez, uz);
        const double hg = h * rsqrt(fma(umx, umx, fma(umy, umy, fma(umz, umz, 1.0))));
        const double tbx = hg * Bx, tby = hg * By, tbz = hg * Bz;
        const double sf = 2.0 / fma(tbx, tbx, fma(tby, tby, fma(tbz, tbz, 1.0)));
        const double upx = fma(umy, tbz, fma(-umz, tby, umx));
        const double upy = fma(umz, tbx, fma(-umx, tbz, umy));
        const double upz = fma(umx, tby, fma(-umy, tbx, umz));
        ux = fma(h, Ex, fma(upy, sf * tbz, fma(-upz, sf * tby, umx)));
        uy = fma(h, Ey, fma(upz, sf * tbx, fma(-upx, sf * tbz, umy)));
        uz = fma(h, Ez, fma(upx, sf * tby, fma(-upy, sf * tbx, umz)));

        // ---- move: displacement in cells
        const double u2p1 = fma(ux, ux, fma(uy, uy, fma(uz, uz, 1.0)));
        const double gi = rsqrt(u2p1);
        const double d[3] = {ux * (gi * pp.dtd[0]), uy * (gi * pp.dtd[1]), uz * (gi * pp.dtd[2])};

        // ---- Esirkepov current on the 5-node windows around the old nearest node
        if (w != 0.0) {
            double S0[3][5], dS[3][5];
            int lo[3], hi[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double s1 = s0[a] + d[a];  // new offset from the old nearest node
                const int m1 = s1 >= 0.5 ? 1 : (s1 < -0.5 ? -1 : 0);
#pragma unroll
                for (int k = 0; k < 5; ++k) S0[a][k] = (k >= 1 && k <= 3) ? wN[a][k - 1] : 0.0;
                if (m1 == 0) {
                    // same nearest node: exact factored differences of the spline pieces
                    const double sum = s0[a] + s1;
                    dS[a][0] = 0.0;
                    dS[a][1] = -0.5 * d[a] * (1.0 - sum);
                    dS[a][2] = -d[a] * sum;
                    dS[a][3] = 0.5 * d[a] * (1.0 + sum);
                    dS[a][4] = 0.0;
                } else {
                    double w1[3];
                    tsc_weights(s1 - (double)m1, w1);
#pragma unroll
                    for (int k = 0; k < 5; ++k) {
                        const int k1 = k - 1 - m1;  // index into the new weights
                        const double nw = k1 == 0 ? w1[0] : (k1 == 1 ? w1[1] : (k1 == 2 ? w1[2] : 0.0));
                        dS[a][k] = nw - S0[a][k];
                    }
                }
                lo[a] = 1 + (m1 < 0 ? m1 : 0);
                hi[a] = 3 + (m1 > 0 ? m1 : 0);
            }
            esirkepov_component<0>(J + 0 * P, g, cN, S0, dS, lo, hi, pp.cq[0] * w);
            esirkepov_component<1>(J + 1 * P, g, cN, S0, dS, lo, hi, pp.cq[1] * w);
            esirkepov_component<2>(J + 2 * P, g, cN, S0, dS, lo, hi, pp.cq[2] * w);
        }

        // ---- new cell and offset
        int ng[3];
        double nf[3];
        bool gone = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double b = f[a] + d[a];
            const int s = tsc_cell_shift(b);
            nf[a] = s ? fmin(b - (double)s, 0x1.fffffffffffffp-1) : b;
            ng[a] = gc[a] + s;
            if (ng[a] < 0 || ng[a] >= g.n[a]) {
                if (g.bc[a] == 0) ng[a] += ng[a] < 0 ? g.n[a] : -g.n[a];
                else gone = true;
            }
        }
        ps.cell[p] = gone ? (INACTIVE | cp) : pack_cell(ng[0], ng[1], ng[2]);
        ps.off[0][p] = nf[0];
        ps.off[1][p] = nf[1];
        ps.off[2][p] = nf[2];
        ps.u[0][p] = ux;
        ps.u[1][p] = uy;
        ps.u[2][p] = uz;
        if (!gone) ek = fma(w, fma(u2p1, gi, -1.0), ek);
    }
    const double s = block_sum<TSC_NT>(ek, red);
    if (threadIdx.x == 0) ek_part[blockIdx.x] = s * pp.mass;
}

cudaError_t tsc_launch(int grid, cudaStream_t st, const PushParams& pp, const PStore<double>& ps,
                       const long long* n_cur, const double* EB, double* J, double* ek_part) {
    k_push_tsc<<<grid, TSC_NT, 0, st>>>(ps, n_cur, pp, EB, J, ek_part);
    return cudaGetLastError();
}

PICGB_INDEX_FLAG_READER(tsc_index_flags)

}  // namespace picgb
