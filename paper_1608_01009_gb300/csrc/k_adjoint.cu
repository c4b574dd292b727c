// Differentiable FP64 path: the PIC step on id-ordered particles, and its
// hand-written discrete adjoint.
//
// Forward (one thread per particle; the same step as the fused kernel --
// cloud-in-cell gather, relativistic Boris push, move and Villasenor-Buneman
// deposit, arXiv:1608.01009 Secs. 2-3 -- but with particles kept in a fixed
// order, gathering from the ghost-padded FP64 field buffer in global memory
// and depositing with global atomics).  No sort is needed, so a run can be
// replayed from a checkpoint particle for particle.
//
// Adjoint of one step, given the cotangents of the new state (lambda_x of
// x^{n+1}, lambda_u of u^{n+1/2}, lambda_E of E^{n+1}, lambda_B of B^{n+1}):
//   fields    the Yee sub-steps in reverse.  With C_E the forward-difference
//             curl (E lattice -> B lattice) and C_B the backward-difference
//             curl (B -> E), C_B = C_E^T (also with zero fields outside an
//             absorbing axis), and the damping masks M are diagonal:
//               B^{n+1} = M_B (B' - h C_E E^{n+1})     -> lB' = M_B lB1, lE1 -= h C_B lB'
//               E^{n+1} = M_E (E^n + dt C_B B' - dt J)  -> lE^n = M_E lE1, lB' += dt C_E lE^n,
//                                                          lJ = -dt lE^n
//               B'      = M_B (B^n - h C_E E^n)        -> lB^n = M_B lB', lE^n -= h C_B lB^n
//   particles reverse mode through deposit (the edge currents as functions of
//             the piece start, displacement and crossing times), move, Boris
//             and the trilinear gather (a weighted scatter of lambda_E,
//             lambda_B to the grid and a position gradient).
#include "pic_internal.cuh"

namespace picgb {

constexpr int TAPE_NT = 256;

// Thread -> particle map of the per-particle kernels: inside each block's tile
// of TAPE_NT consecutive particles, lane l of warp w takes particle
// l * (TAPE_NT / 32) + w.  Id order is usually cell order (a cell's particles
// are consecutive), so the 32 lanes of a warp fall in up to 32 different
// cells and their atomics rarely hit the same grid nodes, while each block
// still reads one contiguous tile (the other warps find it in L1).
__device__ __forceinline__ long long lane_strided(long long n, bool& ok) {
    constexpr int W = TAPE_NT / 32;
    const int t = threadIdx.x;
    const long long p = (long long)blockIdx.x * TAPE_NT + (t & 31) * W + (t >> 5);
    ok = p < n;
    return p;
}

__device__ __forceinline__ double stag(int comp, int axis, bool magnetic) {
    return magnetic ? (comp == axis ? 0.0 : 0.5) : (comp == axis ? 0.5 : 0.0);
}

// Cell of xi along each axis and the two lattices a component can sit on:
// the node lattice (base = cell, fraction = offset a in [0,1)) and the
// half-shifted one (xi - 1/2: base cell - 1 and a + 1/2 when a < 1/2, else
// cell and a - 1/2).  One floor and one conversion per axis serve all six
// components, whose lattices are these per axis (the floor and the FP64 ->
// int conversion run on the FP64 pipe, which bounds the differentiable path).
struct Lat {
    int c0[3], c1[3];      // base on the node / half-shifted lattice
    double f0[3], f1[3];   // fractions
};

__device__ __forceinline__ Lat lattices(const double xi[3]) {
    Lat L;
    for (int a = 0; a < 3; ++a) {
        const double fl = floor(xi[a]);
        const int ci = (int)fl;
        const double o = xi[a] - fl;
        const bool lo = __double2hiint(o) < 0x3FE00000;  // o < 1/2 (o >= 0: bit patterns order like integers)
        L.c0[a] = ci;
        L.f0[a] = o;
        L.c1[a] = lo ? ci - 1 : ci;
        L.f1[a] = o + (lo ? 0.5 : -0.5);
    }
    return L;
}

// Lattice base and fractions of component c (0..5: Ex..Ez, Bx..Bz).
__device__ __forceinline__ void lattice(int c, const Lat& L, int base[3], double f[3]) {
    for (int a = 0; a < 3; ++a) {
        // E_c is half-shifted along axis c, B_c along the two other axes
        const bool half = c < 3 ? c == a : c - 3 != a;
        base[a] = half ? L.c1[a] : L.c0[a];
        f[a] = half ? L.f1[a] : L.f0[a];
    }
}

__device__ __forceinline__ double tri_val(const double v[8], const double f[3]) {
    const double c00 = fma(f[0], v[1] - v[0], v[0]), c10 = fma(f[0], v[3] - v[2], v[2]);
    const double c01 = fma(f[0], v[5] - v[4], v[4]), c11 = fma(f[0], v[7] - v[6], v[6]);
    const double c0 = fma(f[1], c10 - c00, c00), c1 = fma(f[1], c11 - c01, c01);
    return fma(f[2], c1 - c0, c0);
}

// 8 corner values v[bx + 2 by + 4 bz] of component c around `base`.
__device__ __forceinline__ void corners(const double* EB, const GridDev& g, int c, const int base[3], double v[8]) {
    const double* F = EB + (long long)c * g.P;
    for (int q = 0; q < 8; ++q) {
        const long long o = pidx(g, base[0] + (q & 1), base[1] + ((q >> 1) & 1), base[2] + (q >> 2));
        v[q] = in_range(o, g.P) ? F[o] : 0.0;  // the check is compiled in the debug build only
    }
}

__device__ __forceinline__ void cross(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Boris step u -> un (half electric kick, rotation, half kick) with the
// intermediates its adjoint reuses: um = u + h E, rgm = 1/gamma^-, t = h rgm B,
// k = 2/(1 + t.t), s = k t, up = um + um x t.  The differentiable path's
// forward step and its adjoint both call it, so they see the same trajectory.
struct BorisFwd {
    double um[3], rgm, gg, t[3], k, s[3], up[3];
};

__device__ __forceinline__ void boris_fwd(const double u[3], const double E[3], const double B[3], double h,
                                          double un[3], BorisFwd& f) {
    for (int a = 0; a < 3; ++a) f.um[a] = fma(h, E[a], u[a]);
    f.rgm = rsqrt_ge1(fma(f.um[0], f.um[0], fma(f.um[1], f.um[1], fma(f.um[2], f.um[2], 1.0))));
    f.gg = h * f.rgm;
    for (int a = 0; a < 3; ++a) f.t[a] = f.gg * B[a];
    f.k = 2.0 * rcp_ge1(1.0 + fma(f.t[0], f.t[0], fma(f.t[1], f.t[1], f.t[2] * f.t[2])));
    for (int a = 0; a < 3; ++a) f.s[a] = f.k * f.t[a];
    f.up[0] = fma(f.um[1], f.t[2], fma(-f.um[2], f.t[1], f.um[0]));
    f.up[1] = fma(f.um[2], f.t[0], fma(-f.um[0], f.t[2], f.um[1]));
    f.up[2] = fma(f.um[0], f.t[1], fma(-f.um[1], f.t[0], f.um[2]));
    un[0] = fma(h, E[0], fma(f.up[1], f.s[2], fma(-f.up[2], f.s[1], f.um[0])));
    un[1] = fma(h, E[1], fma(f.up[2], f.s[0], fma(-f.up[0], f.s[2], f.um[1])));
    un[2] = fma(h, E[2], fma(f.up[0], f.s[1], fma(-f.up[1], f.s[0], f.um[2])));
}

// Reverse mode of the Boris step from its forward intermediates: given lun
// (cotangent of the new u), returns lu (old u) and adds the cotangents of the
// particle fields into lE, lB.
__device__ void boris_adjoint(const BorisFwd& f, const double B[3], double h, const double lun[3], double lu[3],
                              double lE[3], double lB[3]) {
    // un = upl + h E ; upl = um + up x s
    double lum[3], lup[3], ls[3], lt[3], tmp[3];
    for (int a = 0; a < 3; ++a) {
        lE[a] += h * lun[a];
        lum[a] = lun[a];
    }
    cross(f.s, lun, lup);  // lambda_up = s x lambda_upl
    cross(lun, f.up, ls);  // lambda_s = lambda_upl x up
    // up = um + um x t
    cross(f.t, lup, tmp);
    for (int a = 0; a < 3; ++a) lum[a] += lup[a] + tmp[a];
    cross(lup, f.um, lt);  // lambda_t = lambda_up x um
    // s = k t, k = 2 / (1 + t.t)
    const double lk = ls[0] * f.t[0] + ls[1] * f.t[1] + ls[2] * f.t[2];
    const double lt2 = -0.5 * f.k * f.k * lk;
    for (int a = 0; a < 3; ++a) lt[a] += f.k * ls[a] + 2.0 * f.t[a] * lt2;
    // t = g B, g = h / gamma^-, gamma^- = sqrt(1 + um.um)
    const double lg = lt[0] * B[0] + lt[1] * B[1] + lt[2] * B[2];
    for (int a = 0; a < 3; ++a) lB[a] += f.gg * lt[a];
    // d gamma^- / d um = um / gamma^-, d g / d gamma^- = -g / gamma^-
    const double lgm = -lg * f.gg * f.rgm;
    for (int a = 0; a < 3; ++a) lum[a] += (lgm * f.rgm) * f.um[a];
    // um = u + h E
    for (int a = 0; a < 3; ++a) {
        lu[a] = lum[a];
        lE[a] += h * lum[a];
    }
}

// The pieces of the move a -> a + d (a relative to cell cell0, in cells): the
// crossing parameters t (1 where an axis is not crossed), sorted with the axis
// each belongs to.
struct Pieces {
    double t[3];
    int ax[3];
    bool cr[3];  // the axis is crossed
    int n;       // number of pieces
};

__device__ __forceinline__ Pieces pieces_of(const double a[3], const double d[3]) {
    Pieces P;
    P.n = 1;
    for (int c = 0; c < 3; ++c) {
        const double b = a[c] + d[c];
        P.ax[c] = c;
        P.cr[c] = b >= 1.0 || b < 0.0;
        if (P.cr[c]) {
            P.t[c] = ((b >= 1.0 ? 1.0 : 0.0) - a[c]) / d[c];
            P.n += 1;
        } else {
            P.t[c] = 1.0;
        }
    }
    // sort (t, axis) ascending; on a tie a crossed axis goes first, so the
    // first n - 1 entries are exactly the crossings
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2 - i; ++j)
            if (P.t[j + 1] < P.t[j] || (P.t[j + 1] == P.t[j] && P.cr[j + 1] && !P.cr[j])) {
                const double tt = P.t[j];
                P.t[j] = P.t[j + 1];
                P.t[j + 1] = tt;
                const int aa = P.ax[j];
                P.ax[j] = P.ax[j + 1];
                P.ax[j + 1] = aa;
                const bool cc = P.cr[j];
                P.cr[j] = P.cr[j + 1];
                P.cr[j + 1] = cc;
            }
    return P;
}

__device__ __forceinline__ int off_of(double m) { return m < 0.0 ? -1 : (m >= 1.0 ? 1 : 0); }

// Forward deposit of the move from cell0 + a with displacement d into J
// (padded, global atomics).
__device__ void deposit_global(double* J, const GridDev& g, const int cell0[3], const double a[3], const double d[3],
                               const double Q[3]) {
    const Pieces P = pieces_of(a, d);
    double ta = 0.0;
    for (int s = 0; s < P.n; ++s) {
        const double tb = s + 1 < P.n ? P.t[s] : 1.0;
        if (tb > ta) {
            double pa[3], dd[3];
            int cell[3];
            for (int c = 0; c < 3; ++c) {
                pa[c] = fma(ta, d[c], a[c]);
                dd[c] = (tb - ta) * d[c];
                const int o = off_of(fma(0.5, dd[c], pa[c]));
                cell[c] = cell0[c] + o;
                pa[c] -= o;
            }
            double m[3], om[3];
            for (int c = 0; c < 3; ++c) {
                m[c] = fma(0.5, dd[c], pa[c]);
                om[c] = 1.0 - m[c];
            }
            for (int c = 0; c < 3; ++c) {
                const int p = (c + 1) % 3, r = (c + 2) % 3;
                const double q = Q[c] * dd[c], k = dd[p] * dd[r] * (1.0 / 12.0);
                double* Jc = J + (long long)c * g.P;
                for (int s1 = 0; s1 < 2; ++s1)
                    for (int s2 = 0; s2 < 2; ++s2) {
                        const double wp = s1 ? m[p] : om[p], wr = s2 ? m[r] : om[r];
                        const double sig = s1 == s2 ? 1.0 : -1.0;
                        int idx[3] = {cell[0], cell[1], cell[2]};
                        idx[p] += s1;
                        idx[r] += s2;
                        const long long o = pidx(g, idx[0], idx[1], idx[2]);
                        if (in_range(o, g.P)) atomicAdd(&Jc[o], q * fma(sig, k, wp * wr));
                    }
            }
        }
        ta = tb;
    }
}

// Reverse mode of deposit_global: reads lJ (padded, ghosts filled) and adds
// the cotangents of the start a and displacement d.
__device__ void deposit_adjoint(const double* LJ, const GridDev& g, const int cell0[3], const double a[3],
                                const double d[3], const double Q[3], double la[3], double ld[3]) {
    const Pieces P = pieces_of(a, d);
    const double Q12[3] = {Q[0] * (1.0 / 12.0), Q[1] * (1.0 / 12.0), Q[2] * (1.0 / 12.0)};
    double lt[3] = {0.0, 0.0, 0.0};  // cotangents of the sorted crossing parameters
    double ta = 0.0;
    for (int s = 0; s < P.n; ++s) {
        const double tb = s + 1 < P.n ? P.t[s] : 1.0;
        if (tb > ta) {
            double pa[3], dd[3];
            int cell[3];
            for (int c = 0; c < 3; ++c) {
                pa[c] = fma(ta, d[c], a[c]);
                dd[c] = (tb - ta) * d[c];
                const int o = off_of(fma(0.5, dd[c], pa[c]));
                cell[c] = cell0[c] + o;
                pa[c] -= o;
            }
            double m[3];
            for (int c = 0; c < 3; ++c) m[c] = fma(0.5, dd[c], pa[c]);
            double lm[3] = {0, 0, 0}, ldd[3] = {0, 0, 0};  // cotangents of the midpoint and of dd
            for (int c = 0; c < 3; ++c) {
                const int p = (c + 1) % 3, r = (c + 2) % 3;
                const double* Lc = LJ + (long long)c * g.P;
                int i0[3] = {cell[0], cell[1], cell[2]};
                double L[2][2];
                for (int s1 = 0; s1 < 2; ++s1)
                    for (int s2 = 0; s2 < 2; ++s2) {
                        int idx[3] = {i0[0], i0[1], i0[2]};
                        idx[p] += s1;
                        idx[r] += s2;
                        const long long o = pidx(g, idx[0], idx[1], idx[2]);
                        L[s1][s2] = in_range(o, g.P) ? Lc[o] : 0.0;
                    }
                // f = Q d_c [Sum L W_p W_r + K d_p d_r / 12]: S = Sum L W_p W_r is the
                // bilinear interpolant of the four edge cotangents at (m_p, m_r),
                // Dp, Dr its slopes and K its cross slope
                const double a0 = L[1][0] - L[0][0], a1 = L[1][1] - L[0][1];
                const double K = a1 - a0;
                const double Sp0 = fma(m[p], a0, L[0][0]), Sp1 = fma(m[p], a1, L[0][1]);
                const double Dr = Sp1 - Sp0;
                const double S = fma(m[r], Dr, Sp0);
                const double Dp = fma(m[r], K, a0);
                const double qd = Q[c] * dd[c];
                const double kq = K * Q12[c];  // Q_c K / 12
                const double kk = kq * dd[c];  // Q_c d_c K / 12
                // df/dd_c = Q_c (S + K d_p d_r / 12); df/dm_p = Q_c d_c Dp, df/dm_r = Q_c d_c Dr;
                // df/dd_p = Q_c d_c K d_r / 12, df/dd_r = Q_c d_c K d_p / 12
                ldd[c] = fma(Q[c], S, fma(kq * dd[p], dd[r], ldd[c]));
                lm[p] = fma(qd, Dp, lm[p]);
                lm[r] = fma(qd, Dr, lm[r]);
                ldd[p] = fma(kk, dd[r], ldd[p]);
                ldd[r] = fma(kk, dd[p], ldd[r]);
            }
            // m = pa + dd / 2
            double lpa[3];
            for (int c = 0; c < 3; ++c) {
                lpa[c] = lm[c];
                ldd[c] = fma(0.5, lm[c], ldd[c]);
            }
            // pa = a + ta d - o, dd = (tb - ta) d
            double lta = 0.0, ltb = 0.0;
            for (int c = 0; c < 3; ++c) {
                la[c] += lpa[c];
                ld[c] += ta * lpa[c] + (tb - ta) * ldd[c];
                lta += d[c] * (lpa[c] - ldd[c]);
                ltb += d[c] * ldd[c];
            }
            if (s > 0) lt[s - 1] += lta;
            if (s + 1 < P.n) lt[s] += ltb;
        }
        ta = tb;
    }
    // t = (face - a_ax) / d_ax
    for (int s = 0; s + 1 < P.n; ++s) {
        const int c = P.ax[s];
        const double q = lt[s] / d[c];
        la[c] -= q;
        ld[c] -= q * P.t[s];
    }
}

// Displacement d = dtd u / gamma of a step (u = u^{n+1/2}) and the new position x^{n+1} = x^n + d:
// periodic axes wrap, and the return value says whether the particle left an absorbing axis.
// The tape's forward step and the rebuild of positions from a checkpoint (k_tape_move) both
// call it; the products and sums are explicitly rounded (never contracted into an FMA), so a
// rebuilt position equals the recorded one bit for bit.  The bounds are tested on the bit
// patterns with integer compares, off the FP64 pipe that bounds both kernels.  As signed
// integers the patterns of -0 .. -inf lie at or below that of -inf, and those of n .. +inf
// between the patterns of n and +inf; a NaN falls in neither range, so like a floating-point
// compare the tests leave it in place (and -0 counts as below 0, wrapping to +0).
__device__ __forceinline__ bool below0(long long bx) { return bx <= (long long)0xFFF0000000000000ULL; }
__device__ __forceinline__ bool at_or_above(long long bx, long long bn) {
    return bx >= bn && bx <= 0x7FF0000000000000LL;
}

// The grid's cells per axis as doubles (the position bounds), formed on the host.
struct Ext3 {
    double n[3];
};
static Ext3 ext_of(const StepParams& sp) { return Ext3{{(double)sp.g.n[0], (double)sp.g.n[1], (double)sp.g.n[2]}}; }

__device__ __forceinline__ bool move_of(const double xi[3], const double u[3], const StepParams& sp, const Ext3& ext,
                                        double d[3], double x1[3]) {
    const double gi = rsqrt_ge1(fma(u[0], u[0], fma(u[1], u[1], fma(u[2], u[2], 1.0))));
    bool gone = false;
    for (int c = 0; c < 3; ++c) {
        d[c] = __dmul_rn(u[c], __dmul_rn(gi, sp.dtd[c]));
        double x = __dadd_rn(xi[c], d[c]);
        const long long bn = __double_as_longlong(ext.n[c]);
        long long bx = __double_as_longlong(x);
        if (sp.g.bc[c] == 0) {
            if (below0(bx)) {
                x = __dadd_rn(x, ext.n[c]);
                bx = __double_as_longlong(x);
            }
            if (at_or_above(bx, bn)) x = __dadd_rn(x, -ext.n[c]);
        } else if (below0(bx) || at_or_above(bx, bn)) {
            gone = true;
        }
        x1[c] = x;
    }
    return gone;
}

// One forward step of every particle.
__global__ void __launch_bounds__(TAPE_NT) k_tape_step(TapeDev T, long long n, StepParams sp, Ext3 ext,
                                                      const double* __restrict__ EB, double* __restrict__ J) {
    bool ok;
    const long long p = lane_strided(n, ok);
    if (!ok || !T.act[p]) return;
    const GridDev& g = sp.g;
    double xi[3] = {T.xi[0][p], T.xi[1][p], T.xi[2][p]};
    double u[3] = {T.u[0][p], T.u[1][p], T.u[2][p]};
    const Lat lat = lattices(xi);
    double F[6];
    for (int c = 0; c < 6; ++c) {
        int base[3];
        double f[3], v[8];
        lattice(c, lat, base, f);
        corners(EB, g, c, base, v);
        F[c] = tri_val(v, f);
    }
    {
        BorisFwd bf;
        const double u0[3] = {u[0], u[1], u[2]};
        boris_fwd(u0, F, F + 3, sp.qdt2m, u, bf);
    }
    double d[3], x1[3];
    const bool gone = move_of(xi, u, sp, ext, d, x1);
    const double w = T.w[p];
    if (w != 0.0 && sp.cq[0] != 0.0) {
        const double Q[3] = {sp.cq[0] * w, sp.cq[1] * w, sp.cq[2] * w};
        deposit_global(J, g, lat.c0, lat.f0, d, Q);
    }
    for (int c = 0; c < 3; ++c) {
        T.xi[c][p] = x1[c];
        T.u[c][p] = u[c];
    }
    if (gone) T.act[p] = 0;
}

// Rebuild of the next position from a recorded state: src holds x^n and its active flag,
// with src.u = u^{n+1/2} (the momentum after the step); dst.xi and dst.act receive x^{n+1} and
// its flag, exactly as k_tape_step moves the particle (dst may alias src; dst.u is unused).
__global__ void __launch_bounds__(TAPE_NT) k_tape_move(TapeDev src, TapeDev dst, long long n, StepParams sp, Ext3 ext) {
    const long long p = (long long)blockIdx.x * TAPE_NT + threadIdx.x;
    if (p >= n) return;
    const double xi[3] = {src.xi[0][p], src.xi[1][p], src.xi[2][p]};
    const int act = src.act[p];
    if (!act) {
        if (dst.xi[0] != src.xi[0])
            for (int c = 0; c < 3; ++c) dst.xi[c][p] = xi[c];
        dst.act[p] = 0;
        return;
    }
    const double u[3] = {src.u[0][p], src.u[1][p], src.u[2][p]};
    double d[3], x1[3];
    const bool gone = move_of(xi, u, sp, ext, d, x1);
    for (int c = 0; c < 3; ++c) dst.xi[c][p] = x1[c];
    dst.act[p] = gone ? 0 : 1;
}

// Cotangent of the final kinetic energy: lambda_u = weight * m w u / gamma, lambda_x = 0.
__global__ void __launch_bounds__(TAPE_NT) k_tape_seed(TapeDev T, LamDev L, long long n, double mass, double weight) {
    const long long p = (long long)blockIdx.x * TAPE_NT + threadIdx.x;
    if (p >= n) return;
    const double u[3] = {T.u[0][p], T.u[1][p], T.u[2][p]};
    const double gi = rsqrt(fma(u[0], u[0], fma(u[1], u[1], fma(u[2], u[2], 1.0))));
    const double s = T.act[p] ? weight * mass * T.w[p] * gi : 0.0;
    for (int c = 0; c < 3; ++c) {
        L.u[c][p] = s * u[c];
        L.xi[c][p] = 0.0;
    }
}

// Reverse of one particle step.  T holds the state at step n (x^n, u^{n-1/2});
// L holds the cotangents of x^{n+1}, u^{n+1/2} on entry and of x^n, u^{n-1/2}
// on exit; EB = E^n, B^n; LJ = lambda_J (ghosts filled); scat receives the
// gather cotangents lambda_E, lambda_B (padded, atomics; ghosts folded later).
#ifndef PICGB_TAPE_MINB
#define PICGB_TAPE_MINB 2  // CTAs per SM the adjoint kernel's register budget is set for
#endif
__global__ void __launch_bounds__(TAPE_NT, PICGB_TAPE_MINB)
    k_tape_adjoint(TapeDev T, LamDev L, long long n, StepParams sp, Ext3 ext, const double* __restrict__ EB,
                   const double* __restrict__ LJ, double* __restrict__ scat) {
    bool ok;
    const long long p = lane_strided(n, ok);
    if (!ok || !T.act[p]) return;  // inactive: the step is the identity
    const GridDev& g = sp.g;
    const double xi[3] = {T.xi[0][p], T.xi[1][p], T.xi[2][p]};
    const double u0[3] = {T.u[0][p], T.u[1][p], T.u[2][p]};
    // recompute the forward gather, with the position derivatives of each
    // interpolant from the same lerp tree: v = lerp_z(lerp_y(lerp_x(corners)))
    const Lat lat = lattices(xi);
    double F[6], dF[6][3];
    int bs[6][3];
    for (int c = 0; c < 6; ++c) {
        double v[8], f[3];
        lattice(c, lat, bs[c], f);
        corners(EB, g, c, bs[c], v);
        const double a0 = v[1] - v[0], a1 = v[3] - v[2], a2 = v[5] - v[4], a3 = v[7] - v[6];
        const double c00 = fma(f[0], a0, v[0]), c10 = fma(f[0], a1, v[2]);
        const double c01 = fma(f[0], a2, v[4]), c11 = fma(f[0], a3, v[6]);
        const double e0 = c10 - c00, e1 = c11 - c01;
        const double c0 = fma(f[1], e0, c00), c1 = fma(f[1], e1, c01);
        const double b0 = fma(f[1], a1 - a0, a0), b1 = fma(f[1], a3 - a2, a2);
        dF[c][2] = c1 - c0;
        dF[c][1] = fma(f[2], e1 - e0, e0);
        dF[c][0] = fma(f[2], b1 - b0, b0);
        F[c] = fma(f[2], dF[c][2], c0);
    }
    double u1[3];
    BorisFwd bf;
    boris_fwd(u0, F, F + 3, sp.qdt2m, u1, bf);
    const double gi = rsqrt_ge1(fma(u1[0], u1[0], fma(u1[1], u1[1], fma(u1[2], u1[2], 1.0))));
    double d[3];
    {
        double x1[3];
        move_of(xi, u1, sp, ext, d, x1);  // the forward's displacement, bit for bit
    }
    // cotangents of the outputs
    double lx1[3] = {L.xi[0][p], L.xi[1][p], L.xi[2][p]};
    double lu1[3] = {L.u[0][p], L.u[1][p], L.u[2][p]};
    // deposit
    double la[3] = {0, 0, 0}, ld[3] = {0, 0, 0};
    const double w = T.w[p];
    if (w != 0.0 && sp.cq[0] != 0.0) {
        const double Q[3] = {sp.cq[0] * w, sp.cq[1] * w, sp.cq[2] * w};
        deposit_adjoint(LJ, g, lat.c0, lat.f0, d, Q, la, ld);
    }
    // move: x^{n+1} = x^n + d, d = dtd u / gamma
    double lx0[3];
    for (int c = 0; c < 3; ++c) {
        lx0[c] = lx1[c] + la[c];
        ld[c] += lx1[c];
    }
    double ldv[3], dot = 0.0;
    for (int c = 0; c < 3; ++c) {
        ldv[c] = sp.dtd[c] * ld[c];
        dot += ldv[c] * u1[c];
    }
    const double gi3 = gi * gi * gi;
    for (int c = 0; c < 3; ++c) lu1[c] += ldv[c] * gi - u1[c] * dot * gi3;
    // Boris
    double lu0[3], lF[6] = {0, 0, 0, 0, 0, 0};
    boris_adjoint(bf, F + 3, sp.qdt2m, lu1, lu0, lF, lF + 3);
    // gather: scatter lambda_F with the separable CIC weights, and the position gradient.
    // The 1-D weights (1 - f, f) come from the two lattices of each axis, and the (y, z)
    // weight products are shared by the components on the same pair of y and z lattices
    // (Ex; Ey and Bz; Ez and By; Bx).
    double gl[2][3];  // 1 - f on the node / half-shifted lattice
    for (int a = 0; a < 3; ++a) {
        gl[0][a] = 1.0 - lat.f0[a];
        gl[1][a] = 1.0 - lat.f1[a];
    }
    double yz[4][4];  // [half along y + 2 half along z][by + 2 bz]
    for (int l = 0; l < 4; ++l) {
        const double fy = (l & 1) ? lat.f1[1] : lat.f0[1], gy = gl[l & 1][1];
        const double fz = (l >> 1) ? lat.f1[2] : lat.f0[2], gz = gl[l >> 1][2];
        yz[l][0] = gy * gz;
        yz[l][1] = fy * gz;
        yz[l][2] = gy * fz;
        yz[l][3] = fy * fz;
    }
    for (int c = 0; c < 6; ++c) {
        const double sc = lF[c];
        lx0[0] = fma(sc, dF[c][0], lx0[0]);
        lx0[1] = fma(sc, dF[c][1], lx0[1]);
        lx0[2] = fma(sc, dF[c][2], lx0[2]);
        // half-shifted axes: E_c along c, B_c along the two others
        const bool hx = c == 0 || c == 4 || c == 5, hy = c == 1 || c == 3 || c == 5, hz = c == 2 || c == 3 || c == 4;
        const double s1 = sc * (hx ? lat.f1[0] : lat.f0[0]), s0 = sc * gl[hx ? 1 : 0][0];
        const double* wyz = yz[(hy ? 1 : 0) + (hz ? 2 : 0)];
        double* S = scat + (long long)c * g.P;
        for (int q = 0; q < 4; ++q) {
            const long long o = pidx(g, bs[c][0], bs[c][1] + (q & 1), bs[c][2] + (q >> 1));
            if (!in_range(o, g.P - 1)) continue;  // debug build only: o and o + 1
            atomicAdd(&S[o], wyz[q] * s0);
            atomicAdd(&S[o + 1], wyz[q] * s1);
        }
    }
    for (int c = 0; c < 3; ++c) {
        L.xi[c][p] = lx0[c];
        L.u[c][p] = lu0[c];
    }
}

// Kinetic-energy partials of the tape state.
__global__ void __launch_bounds__(TAPE_NT) k_tape_kinetic(TapeDev T, long long n, double mass, double* __restrict__ part) {
    __shared__ double red[TAPE_NT / 32];
    double s = 0.0;
    for (long long p = (long long)blockIdx.x * TAPE_NT + threadIdx.x; p < n; p += (long long)gridDim.x * TAPE_NT) {
        if (!T.act[p]) continue;
        const double u2p1 = fma(T.u[0][p], T.u[0][p], fma(T.u[1][p], T.u[1][p], fma(T.u[2][p], T.u[2][p], 1.0)));
        s += T.w[p] * fma(u2p1, rsqrt(u2p1), -1.0);
    }
    const double t = block_sum<TAPE_NT>(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t * mass;
}

// Store (binned) -> id-ordered tape arrays (positions in cells).
template <class R>
__global__ void __launch_bounds__(TAPE_NT) k_tape_from_store(PStore<R> ps, const long long* __restrict__ n_cur, TapeDev T,
                                                            double* __restrict__ w_out, long long nid) {
    const long long N = *n_cur;
    for (long long p = (long long)blockIdx.x * TAPE_NT + threadIdx.x; p < N; p += (long long)gridDim.x * TAPE_NT) {
        const int cp = ps.cell[p];
        if (cp < 0) continue;
        const long long id = ps.id[p];
        if (id < 0 || id >= nid) continue;
        T.xi[0][id] = (double)cell_x(cp) + (double)ps.off[0][p];
        T.xi[1][id] = (double)cell_y(cp) + (double)ps.off[1][p];
        T.xi[2][id] = (double)cell_z(cp) + (double)ps.off[2][p];
        for (int c = 0; c < 3; ++c) T.u[c][id] = (double)ps.u[c][p];
        w_out[id] = (double)ps.w[p];
        T.act[id] = 1;
    }
}

// Tape -> FP64 physical arrays (x,y,z,ux,uy,uz,w), for re-loading the store.
__global__ void __launch_bounds__(TAPE_NT) k_tape_to_phys(TapeDev T, long long n, GridDev g, double* const* out) {
    const long long p = (long long)blockIdx.x * TAPE_NT + threadIdx.x;
    if (p >= n) return;
    for (int c = 0; c < 3; ++c) {
        // absent or deactivated particles are placed outside the domain so that the load drops them
        out[c][p] = T.act[p] ? T.xi[c][p] * g.d[c] : (g.bc[c] ? -1.0 : T.xi[c][p] * g.d[c]);
        out[3 + c][p] = T.u[c][p];
    }
    out[6][p] = T.w[p];
}

// Particle cotangents -> gradients in physical units (lambda_x / d).
__global__ void __launch_bounds__(TAPE_NT) k_lam_to_phys(LamDev L, long long n, GridDev g, double* const* out) {
    const long long p = (long long)blockIdx.x * TAPE_NT + threadIdx.x;
    if (p >= n) return;
    for (int c = 0; c < 3; ++c) {
        if (out[c]) out[c][p] = L.xi[c][p] * g.rd[c];
        if (out[3 + c]) out[3 + c][p] = L.u[c][p];
    }
}

// ------------------------------------------------------------------ adjoint fields
// Ghost bookkeeping as in the forward FDTD: periodic images of the owner; on
// absorbing axes the ghosts stand for the fixed zero field outside.
__device__ __forceinline__ void img(int i, int n, int bc, int idx[2], bool fold[2], int& cnt) {
    idx[0] = i;
    fold[0] = true;
    cnt = 1;
    if (i < PAD) {
        idx[1] = bc == 0 ? i + n : i - PAD;
        fold[1] = bc == 0;
        cnt = 2;
    } else if (i >= n - PAD) {
        idx[1] = bc == 0 ? i - n : i + PAD;
        fold[1] = bc == 0;
        cnt = 2;
    }
}

__device__ __forceinline__ double damp_of(const GridDev& g, int comp, bool magnetic, int i, int j, int k) {
    double f = 1.0;
    const int ijk[3] = {i, j, k};
    for (int a = 0; a < 3; ++a) {
        if (g.bc[a] == 0 || g.absorb_cells <= 0) continue;
        if (g.damp) {  // the forward's table of the same factors
            f *= g.damp[g.damp_off[a] + (stag(comp, a, magnetic) != 0.0 ? g.n[a] : 0) + ijk[a]];
            continue;
        }
        const double pos = ijk[a] + stag(comp, a, magnetic);
        const double dist = fmin(pos, (double)g.n[a] - pos);
        const double L = (double)g.absorb_cells;
        if (dist >= L) continue;
        const double r = (L - dist) * g.absorb_rL;
        f *= 1.0 - g.absorb_sigma * r * r;
    }
    return f;
}

constexpr int AF_BX = 32, AF_BY = 8;

__device__ __forceinline__ bool acell(const GridDev& g, int& i, int& j, int& k) {
    i = blockIdx.x * AF_BX + threadIdx.x;
    j = blockIdx.y * AF_BY + threadIdx.y;
    k = blockIdx.z;
    return i < g.n[0] && j < g.n[1];
}

template <class F>
__device__ __forceinline__ void for_images(const GridDev& g, int i, int j, int k, bool only_fold, F fn) {
    int ix[2], iy[2], iz[2], cx, cy, cz;
    bool fx[2], fy[2], fz[2];
    img(i, g.n[0], g.bc[0], ix, fx, cx);
    img(j, g.n[1], g.bc[1], iy, fy, cy);
    img(k, g.n[2], g.bc[2], iz, fz, cz);
    for (int c = 0; c < cz; ++c)
        for (int b = 0; b < cy; ++b)
            for (int a = 0; a < cx; ++a) {
                const bool f = fx[a] && fy[b] && fz[c];
                if (only_fold && !f) continue;
                fn(pidx(g, ix[a], iy[b], iz[c]), f, (a | b | c) == 0);
            }
}

// L[comp] <- mask * L[comp] on the domain, copied to the periodic ghost images
// (comp0 = 0: E components, 3: B components).
__global__ void k_adj_mask_fill(double* __restrict__ L, GridDev g, int comp0) {
    int i, j, k;
    if (!acell(g, i, j, k)) return;
    const long long o = pidx(g, i, j, k);
    for (int c = 0; c < 3; ++c) {
        double* A = L + (long long)(comp0 + c) * g.P;
        const double v = A[o] * damp_of(g, c, comp0 == 3, i, j, k);
        for_images(g, i, j, k, true, [&](long long q, bool, bool) { A[q] = v; });
    }
}

// lE += coef * C_B lB (backward differences; reads lB ghosts).
__global__ void k_adj_curlB(double* __restrict__ L, GridDev g, double coef) {
    int i, j, k;
    if (!acell(g, i, j, k)) return;
    const long long o = pidx(g, i, j, k), sy = g.np[0], sz = (long long)g.np[0] * g.np[1];
    const double* Bx = L + 3 * g.P;
    const double* By = L + 4 * g.P;
    const double* Bz = L + 5 * g.P;
    const double rx = g.rd[0], ry = g.rd[1], rz = g.rd[2];
    const double cx = (Bz[o] - Bz[o - sy]) * ry - (By[o] - By[o - sz]) * rz;
    const double cy = (Bx[o] - Bx[o - sz]) * rz - (Bz[o] - Bz[o - 1]) * rx;
    const double cz = (By[o] - By[o - 1]) * rx - (Bx[o] - Bx[o - sy]) * ry;
    L[o] += coef * cx;
    L[g.P + o] += coef * cy;
    L[2 * g.P + o] += coef * cz;
}

// lB += coef * C_E lE (forward differences; reads lE ghosts); and
// lJ = jcoef * lE on the cell and its periodic images.
__global__ void k_adj_curlE(double* __restrict__ L, double* __restrict__ LJ, GridDev g, double coef, double jcoef) {
    int i, j, k;
    if (!acell(g, i, j, k)) return;
    const long long o = pidx(g, i, j, k), sy = g.np[0], sz = (long long)g.np[0] * g.np[1];
    const double* Ex = L;
    const double* Ey = L + g.P;
    const double* Ez = L + 2 * g.P;
    const double rx = g.rd[0], ry = g.rd[1], rz = g.rd[2];
    const double ex = Ex[o], ey = Ey[o], ez = Ez[o];
    const double cx = (Ez[o + sy] - ez) * ry - (Ey[o + sz] - ey) * rz;
    const double cy = (Ex[o + sz] - ex) * rz - (Ez[o + 1] - ez) * rx;
    const double cz = (Ey[o + 1] - ey) * rx - (Ex[o + sy] - ex) * ry;
    L[3 * g.P + o] += coef * cx;
    L[4 * g.P + o] += coef * cy;
    L[5 * g.P + o] += coef * cz;
    const double e[3] = {ex, ey, ez};
    for (int c = 0; c < 3; ++c) {
        double* A = LJ + (long long)c * g.P;
        const double v = jcoef * e[c];
        for_images(g, i, j, k, true, [&](long long q, bool, bool) { A[q] = v; });
    }
}

// L (domain cells) += scat summed over the cell and its periodic images; every
// scat entry read is zeroed (absorbing ghosts are dropped: no field lives there).
__global__ void k_adj_fold_add(double* __restrict__ L, double* __restrict__ scat, GridDev g) {
    int i, j, k;
    if (!acell(g, i, j, k)) return;
    const long long o = pidx(g, i, j, k);
    int ix[2], iy[2], iz[2], cx, cy, cz;
    bool fx[2], fy[2], fz[2];
    img(i, g.n[0], g.bc[0], ix, fx, cx);
    img(j, g.n[1], g.bc[1], iy, fy, cy);
    img(k, g.n[2], g.bc[2], iz, fz, cz);
    double s[6];
    for (int c = 0; c < 6; ++c) {
        s[c] = scat[(long long)c * g.P + o];
        scat[(long long)c * g.P + o] = 0.0;
    }
    if (cx * cy * cz > 1) {
        for (int c3 = 0; c3 < cz; ++c3)
            for (int b3 = 0; b3 < cy; ++b3)
                for (int a3 = 0; a3 < cx; ++a3) {
                    if ((a3 | b3 | c3) == 0) continue;
                    const long long q = pidx(g, ix[a3], iy[b3], iz[c3]);
                    const bool f = fx[a3] && fy[b3] && fz[c3];
                    for (int c = 0; c < 6; ++c) {
                        if (f) s[c] += scat[(long long)c * g.P + q];
                        scat[(long long)c * g.P + q] = 0.0;
                    }
                }
    }
    for (int c = 0; c < 6; ++c) L[(long long)c * g.P + o] += s[c];
}

// ------------------------------------------------------------------ launchers
static dim3 agrid(const GridDev& g) { return dim3((g.n[0] + AF_BX - 1) / AF_BX, (g.n[1] + AF_BY - 1) / AF_BY, g.n[2]); }
static int pgrid(long long n) { return (int)((n + TAPE_NT - 1) / TAPE_NT); }

cudaError_t tape_step_launch(cudaStream_t st, const TapeDev& T, long long n, const StepParams& sp, const double* EB,
                             double* J) {
    if (n > 0) k_tape_step<<<pgrid(n), TAPE_NT, 0, st>>>(T, n, sp, ext_of(sp), EB, J);
    return cudaGetLastError();
}

cudaError_t tape_move_launch(cudaStream_t st, const TapeDev& src, const TapeDev& dst, long long n, const StepParams& sp) {
    if (n > 0) k_tape_move<<<pgrid(n), TAPE_NT, 0, st>>>(src, dst, n, sp, ext_of(sp));
    return cudaGetLastError();
}

cudaError_t tape_seed_launch(cudaStream_t st, const TapeDev& T, const LamDev& L, long long n, double mass,
                             double weight) {
    if (n > 0) k_tape_seed<<<pgrid(n), TAPE_NT, 0, st>>>(T, L, n, mass, weight);
    return cudaGetLastError();
}

cudaError_t tape_adjoint_launch(cudaStream_t st, const TapeDev& T, const LamDev& L, long long n, const StepParams& sp,
                                const double* EB, const double* LJ, double* scat) {
    if (n > 0) k_tape_adjoint<<<pgrid(n), TAPE_NT, 0, st>>>(T, L, n, sp, ext_of(sp), EB, LJ, scat);
    return cudaGetLastError();
}

cudaError_t tape_kinetic_launch(cudaStream_t st, int grid, const TapeDev& T, long long n, double mass, double* part) {
    k_tape_kinetic<<<grid, TAPE_NT, 0, st>>>(T, n, mass, part);
    return cudaGetLastError();
}

template <class R>
cudaError_t tape_from_store_launch(cudaStream_t st, int nsm, const PStore<R>& ps, const long long* n_cur,
                                   const TapeDev& T, double* w_out, long long nid) {
    k_tape_from_store<R><<<nsm * 8, TAPE_NT, 0, st>>>(ps, n_cur, T, w_out, nid);
    return cudaGetLastError();
}
template cudaError_t tape_from_store_launch<double>(cudaStream_t, int, const PStore<double>&, const long long*,
                                                    const TapeDev&, double*, long long);
template cudaError_t tape_from_store_launch<float>(cudaStream_t, int, const PStore<float>&, const long long*,
                                                   const TapeDev&, double*, long long);

cudaError_t tape_to_phys_launch(cudaStream_t st, const TapeDev& T, long long n, const GridDev& g, double* const* out) {
    if (n > 0) k_tape_to_phys<<<pgrid(n), TAPE_NT, 0, st>>>(T, n, g, out);
    return cudaGetLastError();
}

cudaError_t lam_to_phys_launch(cudaStream_t st, const LamDev& L, long long n, const GridDev& g, double* const* out) {
    if (n > 0) k_lam_to_phys<<<pgrid(n), TAPE_NT, 0, st>>>(L, n, g, out);
    return cudaGetLastError();
}

// One adjoint field step on L = (lE, lB) (padded), producing LJ.
cudaError_t adj_fields_launch(cudaStream_t st, double* L, double* LJ, const GridDev& g) {
    const dim3 gr = agrid(g), bl(AF_BX, AF_BY);
    const double h = 0.5 * g.dt;
    k_adj_mask_fill<<<gr, bl, 0, st>>>(L, g, 3);           // lB' = M_B lB1
    k_adj_curlB<<<gr, bl, 0, st>>>(L, g, -h);              // lE1 -= h C_B lB'
    k_adj_mask_fill<<<gr, bl, 0, st>>>(L, g, 0);           // lE^n = M_E lE1
    k_adj_curlE<<<gr, bl, 0, st>>>(L, LJ, g, g.dt, -g.dt);  // lB' += dt C_E lE^n, lJ = -dt lE^n
    k_adj_mask_fill<<<gr, bl, 0, st>>>(L, g, 3);           // lB^n = M_B lB'
    k_adj_curlB<<<gr, bl, 0, st>>>(L, g, -h);              // lE^n -= h C_B lB^n
    return cudaGetLastError();
}

cudaError_t adj_fold_add_launch(cudaStream_t st, double* L, double* scat, const GridDev& g) {
    k_adj_fold_add<<<agrid(g), dim3(AF_BX, AF_BY), 0, st>>>(L, scat, g);
    return cudaGetLastError();
}

PICGB_INDEX_FLAG_READER(tape_index_flags)

}  // namespace picgb
