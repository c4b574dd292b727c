// Plain FP64 CPU oracle of one particle-in-cell time step.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
// calls this file; only the test suite, the smoke check and the CPU-baseline leg
// of the benchmark load it.  It shares no code, header, table or constant with
// the CUDA path.
//
// What it computes follows the method overview of arXiv:1608.01009 (Surmin et
// al., "Co-design of a particle-in-cell plasma simulation code for Intel Xeon
// Phi"):
//   * Sec. 2: the PIC cycle -- numerical integration of Maxwell's equations on a
//     grid, interpolation of the field to the particles, the relativistic
//     equations of motion of the macro-particles, and the current density
//     they create;
//   * Sec. 3: double precision, the cloud-in-cell (first-order) form factor and
//     the Villasenor-Buneman charge-conserving current deposition.
// The paper names neither the pusher nor the field solver; the readings taken
// here are the relativistic Boris pusher and the Yee FDTD scheme on the
// standard Yee staggering, with B advanced in two half steps so that E and B
// both live at integer time levels when the particles are pushed.
//
// Beyond the paper (which uses CIC only), form_factor = 2 selects the
// second-order (triangular-shaped cloud, TSC) form factor -- the quadratic
// B-spline, weights 1/2 (1/2 - delta)^2, 3/4 - delta^2, 1/2 (1/2 + delta)^2 on
// the three lattice points nearest the particle -- for both the gather and the
// charge density, with the charge-conserving current of Esirkepov (Comput.
// Phys. Commun. 135, 144 (2001)) for an arbitrary form factor.
//
// Units are normalised: time 1/w, length c/w, momentum u = p/(mc), fields
// m c w / e, so that  dE/dt = curl B - J,  dB/dt = -curl E,
// du/dt = (q/m)(E + u x B / gamma),  dx/dt = u / gamma.
//
// Everything is written in natural loop order, one particle after another,
// with no blocking or fusion, so that each stage can be read against the
// method by eye.  The scalar type is a template parameter: T = double is the
// oracle proper; T = Dual (value + one directional derivative) runs the very
// same statements in forward-mode differentiation and is the CPU reference
// gradient for the adjoint (floor() of a Dual takes its value, so the
// derivative is the almost-everywhere derivative of the piecewise-smooth step).
//
// Build: g++ -O2 -ffp-contract=off -fPIC -shared (oracle/build_oracle.py).
// -ffp-contract=off keeps every product and sum rounded separately, as written.
// A second build with -fopenmp (libpic_oracle_threads.so) runs whole steps'
// particle loop on all host cores; it exists to time the oracle on the host,
// and the tests check it against the serial build.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <cstdlib>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- dual numbers
struct Dual {
    double v, d;
    Dual() : v(0), d(0) {}
    Dual(double a) : v(a), d(0) {}
    Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
    double q = a.v / b.v;
    return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }
inline double sqrt(double a) { return std::sqrt(a); }
inline double val(double a) { return a; }
inline double val(Dual a) { return a.v; }
inline double tan_of(double) { return 0.0; }
inline double tan_of(Dual a) { return a.d; }

// ---------------------------------------------------------------- grid
enum { BC_PERIODIC = 0, BC_ABSORBING = 1 };

}  // namespace

extern "C" {

// Grid descriptor.  n = cells per axis, d = cell size, dt = time step,
// bc = boundary per axis, absorb_cells / absorb_sigma = damping layer.
typedef struct {
    int n[3];
    double d[3];
    double dt;
    int bc[3];
    int absorb_cells;
    double absorb_sigma;
    int form_factor;  // 1 (or 0): cloud-in-cell; 2: TSC with the Esirkepov current
} or_grid;

// One species.  Positions are physical (x in [0, n*d) on periodic axes),
// momenta u = gamma v / c, w = macro-particle weight (number density times
// volume), active = 0 once a particle has left through an absorbing boundary.
typedef struct {
    double q, m;
    int64_t n;
    double *x, *y, *z, *ux, *uy, *uz, *w;
    int8_t* active;
} or_species;

}  // extern "C"

namespace {

// Staggered positions of the Yee components, in cells (Yee 1966):
//   Ex (i+1/2, j, k)      Bx (i, j+1/2, k+1/2)
//   Ey (i, j+1/2, k)      By (i+1/2, j, k+1/2)
//   Ez (i, j, k+1/2)      Bz (i+1/2, j+1/2, k)
// The current J shares the positions of E.
inline double stagE(int comp, int axis) { return comp == axis ? 0.5 : 0.0; }
inline double stagB(int comp, int axis) { return comp == axis ? 0.0 : 0.5; }

inline long long lin(const or_grid& g, long long i, long long j, long long k) {
    return i + (long long)g.n[0] * (j + (long long)g.n[1] * k);
}

inline long long wrap(long long i, int n) {
    long long r = i % n;
    return r < 0 ? r + n : r;
}

// Grid value of one component at lattice index (i,j,k).  Periodic axes wrap;
// outside the domain along an absorbing axis the field is zero.
template <class T>
T at(const or_grid& g, const T* F, long long i, long long j, long long k) {
    long long ijk[3] = {i, j, k};
    for (int a = 0; a < 3; ++a) {
        if (ijk[a] < 0 || ijk[a] >= g.n[a]) {
            if (g.bc[a] == BC_PERIODIC) ijk[a] = wrap(ijk[a], g.n[a]);
            else return T(0.0);
        }
    }
    return F[lin(g, ijk[0], ijk[1], ijk[2])];
}

// ------------------------------------------------------------------ gather
// Cloud-in-cell interpolation (Sec. 3): trilinear weights of the particle
// position relative to the component's own staggered lattice, summed over the
// 8 surrounding lattice points.  xi is the position in cells.
template <class T>
T interp(const or_grid& g, const T* F, const double off[3], const T xi[3]) {
    long long i0[3];
    T f[3];
    for (int a = 0; a < 3; ++a) {
        T s = xi[a] - off[a];
        double fl = std::floor(val(s));
        i0[a] = (long long)fl;
        f[a] = s - fl;
    }
    T sum = 0.0;
    for (int c = 0; c < 8; ++c) {
        int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
        T wx = bx ? f[0] : T(1.0) - f[0];
        T wy = by ? f[1] : T(1.0) - f[1];
        T wz = bz ? f[2] : T(1.0) - f[2];
        sum += wx * wy * wz * at(g, F, i0[0] + bx, i0[1] + by, i0[2] + bz);
    }
    return sum;
}

// Second-order form factor (TSC, quadratic B-spline) weights of a position s
// (in lattice units) on the lattice points i0-1, i0, i0+1 nearest to it:
// i0 = floor(s + 1/2), delta = s - i0 in [-1/2, 1/2).
template <class T>
long long tsc_weights(T s, T w[3]) {
    double fl = std::floor(val(s) + 0.5);
    T delta = s - fl;
    T a = T(0.5) - delta, b = T(0.5) + delta;
    w[0] = T(0.5) * a * a;
    w[1] = T(0.75) - delta * delta;
    w[2] = T(0.5) * b * b;
    return (long long)fl;
}

// TSC interpolation: the 27 lattice points of the component's own staggered
// lattice around the particle, weighted by the product of the three 1-D
// quadratic-spline weights.
template <class T>
T interp_tsc(const or_grid& g, const T* F, const double off[3], const T xi[3]) {
    long long i0[3];
    T w[3][3];
    for (int a = 0; a < 3; ++a) i0[a] = tsc_weights(T(xi[a] - off[a]), w[a]);
    T sum = 0.0;
    for (int c = 0; c < 3; ++c)
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a)
                sum += w[0][a] * w[1][b] * w[2][c] * at(g, F, i0[0] - 1 + a, i0[1] - 1 + b, i0[2] - 1 + c);
    return sum;
}

template <class T>
void gather_one(const or_grid& g, T* const E[3], T* const B[3], const T xi[3], T Ep[3], T Bp[3]) {
    for (int c = 0; c < 3; ++c) {
        double oe[3] = {stagE(c, 0), stagE(c, 1), stagE(c, 2)};
        double ob[3] = {stagB(c, 0), stagB(c, 1), stagB(c, 2)};
        if (g.form_factor == 2) {
            Ep[c] = interp_tsc(g, E[c], oe, xi);
            Bp[c] = interp_tsc(g, B[c], ob, xi);
        } else {
            Ep[c] = interp(g, E[c], oe, xi);
            Bp[c] = interp(g, B[c], ob, xi);
        }
    }
}

// ------------------------------------------------------------------ Boris push
// Relativistic equations of motion (Sec. 2), advanced with the Boris scheme:
// half electric kick, magnetic rotation with t = (q dt / 2 m gamma^-) B and
// s = 2 t / (1 + t^2), second half electric kick.
template <class T>
void boris(T u[3], const T E[3], const T B[3], double q, double m, double dt) {
    double h = 0.5 * q * dt / m;
    T um[3], t[3], s[3], up[3];
    for (int a = 0; a < 3; ++a) um[a] = u[a] + h * E[a];
    T gm = sqrt(T(1.0) + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    for (int a = 0; a < 3; ++a) t[a] = h * B[a] / gm;
    T t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int a = 0; a < 3; ++a) s[a] = T(2.0) * t[a] / (T(1.0) + t2);
    up[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    up[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    up[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    T pl[3];
    pl[0] = um[0] + (up[1] * s[2] - up[2] * s[1]);
    pl[1] = um[1] + (up[2] * s[0] - up[0] * s[2]);
    pl[2] = um[2] + (up[0] * s[1] - up[1] * s[0]);
    for (int a = 0; a < 3; ++a) u[a] = pl[a] + h * E[a];
}

// ------------------------------------------------------------------ deposit
// Add a contribution to a J component at lattice index (i,j,k).  Periodic axes
// wrap; contributions outside the domain along an absorbing axis are dropped.
template <class T>
void add_at(const or_grid& g, T* F, long long i, long long j, long long k, T v) {
    long long ijk[3] = {i, j, k};
    for (int a = 0; a < 3; ++a) {
        if (ijk[a] < 0 || ijk[a] >= g.n[a]) {
            if (g.bc[a] == BC_PERIODIC) ijk[a] = wrap(ijk[a], g.n[a]);
            else return;
        }
    }
    F[lin(g, ijk[0], ijk[1], ijk[2])] += v;
}

// Current of one straight segment that stays inside cell `cell`; a is its
// start point relative to the cell corner and d its displacement, in cells.
// For the x component, the charge-conserving current on the four x-edges
// (i+1/2, j+s1, k+s2) is the line integral of the CIC weights of the other two
// coordinates along the segment: dx * [W_y(s1) W_z(s2) + sigma dy dz / 12],
// with W(0) = 1 - mid, W(1) = mid, mid = a + d/2, and sigma = +1 when s1 == s2,
// -1 otherwise.  Y and Z follow by cycling the axes.  qfac[c] = q w / (dt *
// product of the two other cell sizes) turns the displacement (in cells) into
// a current density.
template <class T>
void deposit_segment(const or_grid& g, T* J[3], const long long cell[3], const T a[3], const T d[3],
                     const T qfac[3]) {
    T m[3];
    for (int e = 0; e < 3; ++e) m[e] = a[e] + T(0.5) * d[e];
    for (int c = 0; c < 3; ++c) {
        int p = (c + 1) % 3, r = (c + 2) % 3;  // the two transverse axes
        for (int s1 = 0; s1 < 2; ++s1) {
            for (int s2 = 0; s2 < 2; ++s2) {
                T wp = s1 ? m[p] : T(1.0) - m[p];
                T wr = s2 ? m[r] : T(1.0) - m[r];
                double sigma = (s1 == s2) ? 1.0 : -1.0;
                T v = qfac[c] * d[c] * (wp * wr + sigma * d[p] * d[r] / T(12.0));
                long long idx[3] = {cell[0], cell[1], cell[2]};
                idx[p] += s1;
                idx[r] += s2;
                add_at(g, J[c], idx[0], idx[1], idx[2], v);
            }
        }
    }
}

// Villasenor-Buneman deposition (Sec. 3) of the straight move that starts at
// xi0 with displacement d (positions in cells, not wrapped): the move is cut
// at every cell face it crosses (at most one face per axis, since a particle
// moves less than a cell per step), the pieces are taken in order of the
// crossing parameter t in [0,1], and each piece -- start xi0 + t_a d,
// displacement (t_b - t_a) d -- deposits the current of a segment inside the
// cell that holds its midpoint.  The displacement enters as given, never as a
// difference of two rounded positions.
template <class T>
void deposit_vb(const or_grid& g, T* J[3], const T xi0[3], const T d[3], const T qfac[3]) {
    std::vector<T> ts;
    ts.push_back(T(0.0));
    for (int a = 0; a < 3; ++a) {
        double c0 = std::floor(val(xi0[a])), c1 = std::floor(val(xi0[a] + d[a]));
        if (c0 != c1) {
            double face = std::max(c0, c1);
            ts.push_back((T(face) - xi0[a]) / d[a]);
        }
    }
    ts.push_back(T(1.0));
    std::sort(ts.begin(), ts.end(), [](const T& p, const T& q) { return val(p) < val(q); });
    for (size_t s = 0; s + 1 < ts.size(); ++s) {
        T pa[3], ds[3], a[3];
        long long cell[3];
        for (int e = 0; e < 3; ++e) {
            pa[e] = xi0[e] + ts[s] * d[e];
            ds[e] = (ts[s + 1] - ts[s]) * d[e];
            cell[e] = (long long)std::floor(val(pa[e]) + 0.5 * val(ds[e]));
            a[e] = pa[e] - double(cell[e]);
        }
        deposit_segment(g, J, cell, a, ds, qfac);
    }
}

// Esirkepov's charge-conserving current for the TSC form factor, for the
// straight move from xi0 by d (positions in cells, |d_a| < 1).  Per axis the
// old and new 1-D weights S0, S1 live on the 5 nodes base-2 .. base+2 around
// the old position's nearest node base (the new position's three nodes fall
// inside since |d| < 1).  The density change S1x S1y S1z - S0x S0y S0z is split
// into three parts, the x part being
//   W_x = dSx (S0y S0z + dSy S0z / 2 + S0y dSz / 2 + dSy dSz / 3),  dS = S1 - S0,
// (y, z cyclic), and the x current on the edge (i+1/2, j, k) is the running
// sum of -W_x along x from the window's left end: -qfac sum_{i' <= i} W_x, for
// the 4 edges between the 5 nodes (the sum over all 5 vanishes).  qfac is the
// same q w / (dt * product of the two transverse cell sizes) as in the VB path.
// As in the VB path the displacement enters as given: the new offset is taken
// from the old nearest node, s1 = delta0 + d, and when the nearest node stays
// the same the weight changes are the exact factored differences of the
// spline pieces, dS = -d (1 - delta0 - delta1)/2, -d (delta0 + delta1),
// d (1 + delta0 + delta1)/2 on the nodes -1, 0, +1 (no cancellation of two
// rounded weights for small d).
template <class T>
void deposit_esirkepov(const or_grid& g, T* J[3], const T xi0[3], const T d[3], const T qfac[3]) {
    long long base[3];
    T S0[3][5], dS[3][5];
    for (int a = 0; a < 3; ++a) {
        T w0[3], w1[3];
        base[a] = tsc_weights(xi0[a], w0);
        T delta0 = xi0[a] - double(base[a]);
        T s1 = delta0 + d[a];
        long long m1 = tsc_weights(s1, w1);  // nearest node of the new position, relative to base
        for (int k = 0; k < 5; ++k) S0[a][k] = dS[a][k] = T(0.0);
        for (int k = 0; k < 3; ++k) S0[a][1 + k] = w0[k];
        if (m1 == 0) {
            T delta1 = s1;
            dS[a][1] = T(-0.5) * d[a] * (T(1.0) - delta0 - delta1);
            dS[a][2] = T(-1.0) * d[a] * (delta0 + delta1);
            dS[a][3] = T(0.5) * d[a] * (T(1.0) + delta0 + delta1);
        } else {
            T S1[5] = {T(0.0), T(0.0), T(0.0), T(0.0), T(0.0)};
            for (int k = 0; k < 3; ++k) S1[(int)m1 + 1 + k] = w1[k];
            for (int k = 0; k < 5; ++k) dS[a][k] = S1[k] - S0[a][k];
        }
    }
    for (int c = 0; c < 3; ++c) {
        int p = (c + 1) % 3, r = (c + 2) % 3;  // the two transverse axes
        for (int jp = 0; jp < 5; ++jp)
            for (int jr = 0; jr < 5; ++jr) {
                T transverse = S0[p][jp] * S0[r][jr] + T(0.5) * dS[p][jp] * S0[r][jr] +
                               T(0.5) * S0[p][jp] * dS[r][jr] + dS[p][jp] * dS[r][jr] / T(3.0);
                T running = 0.0;
                for (int i = 0; i < 4; ++i) {
                    running += dS[c][i] * transverse;
                    long long idx[3];
                    idx[c] = base[c] - 2 + i;
                    idx[p] = base[p] - 2 + jp;
                    idx[r] = base[r] - 2 + jr;
                    add_at(g, J[c], idx[0], idx[1], idx[2], T(-1.0) * qfac[c] * running);
                }
            }
    }
}

// ------------------------------------------------------------------ Yee FDTD
// Damping factor of the absorbing layer at a lattice position p (in cells)
// along an absorbing axis with n cells: 1 - sigma ((L - dist)/L)^2 inside a
// layer of L cells, 1 elsewhere.
double damp_factor(const or_grid& g, double p, int n) {
    double dist = std::min(p, (double)n - p);
    double L = (double)g.absorb_cells;
    if (g.absorb_cells <= 0 || dist >= L) return 1.0;
    double r = (L - dist) / L;
    return 1.0 - g.absorb_sigma * r * r;
}

template <class T>
void damp(const or_grid& g, T* const F[3], bool isB) {
    for (int a = 0; a < 3; ++a) {
        if (g.bc[a] != BC_ABSORBING) continue;
        for (int c = 0; c < 3; ++c) {
            double off = isB ? stagB(c, a) : stagE(c, a);
            for (int k = 0; k < g.n[2]; ++k)
                for (int j = 0; j < g.n[1]; ++j)
                    for (int i = 0; i < g.n[0]; ++i) {
                        int ijk[3] = {i, j, k};
                        double f = damp_factor(g, ijk[a] + off, g.n[a]);
                        if (f != 1.0) F[c][lin(g, i, j, k)] *= f;
                    }
        }
    }
}

// B <- B - (dt/2) curl E, with forward differences of E onto the B lattice.
template <class T>
void fdtd_b_half(const or_grid& g, T* const E[3], T* B[3]) {
    double h = 0.5 * g.dt;
    double rx = 1.0 / g.d[0], ry = 1.0 / g.d[1], rz = 1.0 / g.d[2];
    for (int k = 0; k < g.n[2]; ++k)
        for (int j = 0; j < g.n[1]; ++j)
            for (int i = 0; i < g.n[0]; ++i) {
                long long o = lin(g, i, j, k);
                T cx = (at(g, E[2], i, j + 1, k) - at(g, E[2], i, j, k)) * ry -
                       (at(g, E[1], i, j, k + 1) - at(g, E[1], i, j, k)) * rz;
                T cy = (at(g, E[0], i, j, k + 1) - at(g, E[0], i, j, k)) * rz -
                       (at(g, E[2], i + 1, j, k) - at(g, E[2], i, j, k)) * rx;
                T cz = (at(g, E[1], i + 1, j, k) - at(g, E[1], i, j, k)) * rx -
                       (at(g, E[0], i, j + 1, k) - at(g, E[0], i, j, k)) * ry;
                B[0][o] -= h * cx;
                B[1][o] -= h * cy;
                B[2][o] -= h * cz;
            }
    damp(g, B, true);
}

// E <- E + dt (curl B - J), with backward differences of B onto the E lattice.
template <class T>
void fdtd_e(const or_grid& g, T* E[3], T* const B[3], T* const J[3]) {
    double dt = g.dt;
    double rx = 1.0 / g.d[0], ry = 1.0 / g.d[1], rz = 1.0 / g.d[2];
    std::vector<T> nE[3];
    long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
    for (int c = 0; c < 3; ++c) nE[c].assign(E[c], E[c] + ncell);
    for (int k = 0; k < g.n[2]; ++k)
        for (int j = 0; j < g.n[1]; ++j)
            for (int i = 0; i < g.n[0]; ++i) {
                long long o = lin(g, i, j, k);
                T cx = (at(g, B[2], i, j, k) - at(g, B[2], i, j - 1, k)) * ry -
                       (at(g, B[1], i, j, k) - at(g, B[1], i, j, k - 1)) * rz;
                T cy = (at(g, B[0], i, j, k) - at(g, B[0], i, j, k - 1)) * rz -
                       (at(g, B[2], i, j, k) - at(g, B[2], i - 1, j, k)) * rx;
                T cz = (at(g, B[1], i, j, k) - at(g, B[1], i - 1, j, k)) * rx -
                       (at(g, B[0], i, j, k) - at(g, B[0], i, j - 1, k)) * ry;
                nE[0][o] = E[0][o] + dt * (cx - J[0][o]);
                nE[1][o] = E[1][o] + dt * (cy - J[1][o]);
                nE[2][o] = E[2][o] + dt * (cz - J[2][o]);
            }
    for (int c = 0; c < 3; ++c) std::copy(nE[c].begin(), nE[c].end(), E[c]);
    damp(g, E, false);
}

// ------------------------------------------------------------------ one step
// Step order (state x^n, u^{n-1/2}, E^n, B^n):
//   1. gather E^n, B^n at x^n           2. Boris u^{n-1/2} -> u^{n+1/2}
//   3. x^{n+1} = x^n + dt u^{n+1/2}/gamma
//   4. Villasenor-Buneman J^{n+1/2} from x^n -> x^{n+1}
//   5. B^{n+1/2} = B^n - dt/2 curl E^n  6. E^{n+1} = E^n + dt (curl B^{n+1/2} - J^{n+1/2})
//   7. B^{n+1} = B^{n+1/2} - dt/2 curl E^{n+1}
template <class T>
struct SpeciesT {
    double q, m;
    int64_t n;
    T *x, *y, *z, *ux, *uy, *uz, *w;
    int8_t* active;
};

template <class T>
void push_and_deposit(const or_grid& g, T* const E[3], T* const B[3], T* J[3], SpeciesT<T>& sp) {
    double L[3] = {g.n[0] * g.d[0], g.n[1] * g.d[1], g.n[2] * g.d[2]};
    for (int64_t p = 0; p < sp.n; ++p) {
        if (!sp.active[p]) continue;
        T* X[3] = {&sp.x[p], &sp.y[p], &sp.z[p]};
        T u[3] = {sp.ux[p], sp.uy[p], sp.uz[p]};
        T xi0[3];
        for (int a = 0; a < 3; ++a) xi0[a] = *X[a] / g.d[a];
        T Ep[3], Bp[3];
        gather_one(g, E, B, xi0, Ep, Bp);
        boris(u, Ep, Bp, sp.q, sp.m, g.dt);
        T gam = sqrt(T(1.0) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        T xn[3], dcell[3];
        for (int a = 0; a < 3; ++a) {
            T disp = g.dt * u[a] / gam;  // x^{n+1} - x^n
            xn[a] = *X[a] + disp;
            dcell[a] = disp / g.d[a];
        }
        if (sp.q != 0.0) {
            T qfac[3];
            for (int c = 0; c < 3; ++c) {
                int p1 = (c + 1) % 3, p2 = (c + 2) % 3;
                qfac[c] = sp.q * sp.w[p] / (g.dt * g.d[p1] * g.d[p2]);
            }
            if (g.form_factor == 2) deposit_esirkepov(g, J, xi0, dcell, qfac);
            else deposit_vb(g, J, xi0, dcell, qfac);
        }
        bool leaves = false;
        for (int a = 0; a < 3; ++a) {
            if (g.bc[a] == BC_PERIODIC) {
                if (val(xn[a]) < 0.0) xn[a] = xn[a] + L[a];
                if (val(xn[a]) >= L[a]) xn[a] = xn[a] - L[a];
            } else if (val(xn[a]) < 0.0 || val(xn[a]) >= L[a]) {
                leaves = true;
            }
        }
        for (int a = 0; a < 3; ++a) *X[a] = xn[a];
        sp.ux[p] = u[0];
        sp.uy[p] = u[1];
        sp.uz[p] = u[2];
        if (leaves) sp.active[p] = 0;
    }
}

#ifdef _OPENMP
// Timing build only (build_oracle.py's threaded variant, which times the oracle
// on all host cores): the particles are split into one contiguous range per
// thread, each range goes through push_and_deposit above -- the same
// statements, particle by particle -- into a thread-private current, and the
// private currents are added into J in thread order.  Only the summation order
// of J differs from the serial build, which compiles without this.
template <class T>
void push_and_deposit_threads(const or_grid& g, T* const E[3], T* const B[3], T* J[3], SpeciesT<T>& sp) {
    const long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
    const int nt = omp_get_max_threads();
    std::vector<T> priv((size_t)nt * 3 * ncell, T(0.0));
#pragma omp parallel num_threads(nt)
    {
        const int t = omp_get_thread_num();
        const int64_t a = sp.n * t / nt, b = sp.n * (t + 1) / nt;
        SpeciesT<T> part = sp;
        part.n = b - a;
        part.x += a, part.y += a, part.z += a, part.ux += a, part.uy += a, part.uz += a, part.w += a;
        part.active += a;
        T* Jt[3] = {&priv[((size_t)t * 3 + 0) * ncell], &priv[((size_t)t * 3 + 1) * ncell],
                    &priv[((size_t)t * 3 + 2) * ncell]};
        push_and_deposit(g, E, B, Jt, part);
    }
    for (int t = 0; t < nt; ++t)
        for (int c = 0; c < 3; ++c)
            for (long long o = 0; o < ncell; ++o) J[c][o] += priv[((size_t)t * 3 + c) * ncell + o];
}
#endif

template <class T>
void step(const or_grid& g, T* E[3], T* B[3], T* J[3], std::vector<SpeciesT<T>>& sps) {
    long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
    for (int c = 0; c < 3; ++c)
        for (long long o = 0; o < ncell; ++o) J[c][o] = T(0.0);
#ifdef _OPENMP
    for (auto& sp : sps) push_and_deposit_threads(g, E, B, J, sp);
#else
    for (auto& sp : sps) push_and_deposit(g, E, B, J, sp);
#endif
    fdtd_b_half(g, E, B);
    fdtd_e(g, E, B, J);
    fdtd_b_half(g, E, B);
}

// ------------------------------------------------------------------ diagnostics
template <class T>
T field_energy(const or_grid& g, T* const E[3], T* const B[3]) {
    long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
    T s = 0.0;
    for (int c = 0; c < 3; ++c)
        for (long long o = 0; o < ncell; ++o) s += E[c][o] * E[c][o] + B[c][o] * B[c][o];
    return T(0.5 * g.d[0] * g.d[1] * g.d[2]) * s;
}

template <class T>
T kinetic_energy(const SpeciesT<T>& sp) {
    T s = 0.0;
    for (int64_t p = 0; p < sp.n; ++p) {
        if (!sp.active[p]) continue;
        T gam = sqrt(T(1.0) + sp.ux[p] * sp.ux[p] + sp.uy[p] * sp.uy[p] + sp.uz[p] * sp.uz[p]);
        s += sp.w[p] * (gam - T(1.0));
    }
    return T(sp.m) * s;
}

SpeciesT<double> as_double(const or_species& s) {
    return SpeciesT<double>{s.q, s.m, s.n, s.x, s.y, s.z, s.ux, s.uy, s.uz, s.w, s.active};
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

// Fields: E[3], B[3], J[3], each n[0]*n[1]*n[2] doubles, x fastest.

// Interpolate E and B to n positions (physical units).  Eout/Bout: 3 x n.
void or_gather(const or_grid* g, double* const* E, double* const* B, int64_t n, const double* x,
               const double* y, const double* z, double* Eout, double* Bout) {
    for (int64_t p = 0; p < n; ++p) {
        double xi[3] = {x[p] / g->d[0], y[p] / g->d[1], z[p] / g->d[2]};
        double Ep[3], Bp[3];
        gather_one(*g, E, B, xi, Ep, Bp);
        for (int c = 0; c < 3; ++c) {
            Eout[c * n + p] = Ep[c];
            Bout[c * n + p] = Bp[c];
        }
    }
}

// Boris-advance n momenta (u: 3 x n, in place) in given particle fields (3 x n).
void or_boris(int64_t n, double* u, const double* Ep, const double* Bp, double q, double m, double dt) {
    for (int64_t p = 0; p < n; ++p) {
        double uu[3] = {u[p], u[n + p], u[2 * n + p]};
        double e[3] = {Ep[p], Ep[n + p], Ep[2 * n + p]};
        double b[3] = {Bp[p], Bp[n + p], Bp[2 * n + p]};
        boris(uu, e, b, q, m, dt);
        u[p] = uu[0];
        u[n + p] = uu[1];
        u[2 * n + p] = uu[2];
    }
}

// Deposit the moves x0 -> x1 (physical units, 3 x n each, x1 unwrapped) of n
// particles of charge q and weights w into J (added to what is there).
void or_deposit(const or_grid* g, double* const* J, int64_t n, const double* x0, const double* x1,
                const double* w, double q) {
    double* Jp[3] = {J[0], J[1], J[2]};
    for (int64_t p = 0; p < n; ++p) {
        double xi0[3], dc[3], qfac[3];
        for (int a = 0; a < 3; ++a) {
            xi0[a] = x0[a * n + p] / g->d[a];
            dc[a] = (x1[a * n + p] - x0[a * n + p]) / g->d[a];
        }
        for (int c = 0; c < 3; ++c)
            qfac[c] = q * w[p] / (g->dt * g->d[(c + 1) % 3] * g->d[(c + 2) % 3]);
        if (g->form_factor == 2) deposit_esirkepov(*g, Jp, xi0, dc, qfac);
        else deposit_vb(*g, Jp, xi0, dc, qfac);
    }
}

void or_fdtd_b_half(const or_grid* g, double* const* E, double* const* B) {
    double* Bp[3] = {B[0], B[1], B[2]};
    fdtd_b_half(*g, E, Bp);
}

void or_fdtd_e(const or_grid* g, double* const* E, double* const* B, double* const* J) {
    double* Ep[3] = {E[0], E[1], E[2]};
    fdtd_e(*g, Ep, B, J);
}

// Full steps.  J holds J^{n+1/2} of the last step on return.
void or_step(const or_grid* g, double* const* E, double* const* B, double* const* J, int nsp,
             const or_species* sp, int nsteps) {
    double* Ep[3] = {E[0], E[1], E[2]};
    double* Bp[3] = {B[0], B[1], B[2]};
    double* Jp[3] = {J[0], J[1], J[2]};
    std::vector<SpeciesT<double>> s;
    for (int i = 0; i < nsp; ++i) s.push_back(as_double(sp[i]));
    for (int t = 0; t < nsteps; ++t) step(*g, Ep, Bp, Jp, s);
}

// Push (gather, Boris, move, deposit) only, for a subset of particles; J is
// added to.  Used to check sampled particles of a large run one by one.
void or_push_deposit(const or_grid* g, double* const* E, double* const* B, double* const* J,
                     const or_species* sp) {
    double* Jp[3] = {J[0], J[1], J[2]};
    SpeciesT<double> s = as_double(*sp);
    push_and_deposit(*g, E, B, Jp, s);
}

// Host threads the particle loop of a whole step uses (1 in the serial build).
int or_threads() {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

double or_field_energy(const or_grid* g, double* const* E, double* const* B) {
    return field_energy(*g, E, B);
}

double or_kinetic_energy(const or_species* sp) { return kinetic_energy(as_double(*sp)); }

// Charge density at the nodes (i,j,k) from CIC weights:
// rho = sum_p q w_p / dV * prod_a (1 - |xi_a - i_a|)_+ , or with form_factor 2
// from the TSC weights on the 27 nearest nodes.  Added into rho.
void or_rho(const or_grid* g, const or_species* sp, double* rho) {
    double dV = g->d[0] * g->d[1] * g->d[2];
    for (int64_t p = 0; p < sp->n; ++p) {
        if (!sp->active[p]) continue;
        double xi[3] = {sp->x[p] / g->d[0], sp->y[p] / g->d[1], sp->z[p] / g->d[2]};
        if (g->form_factor == 2) {
            double w[3][3];
            long long i0[3];
            for (int a = 0; a < 3; ++a) i0[a] = tsc_weights(xi[a], w[a]);
            for (int c = 0; c < 3; ++c)
                for (int b = 0; b < 3; ++b)
                    for (int a = 0; a < 3; ++a)
                        add_at(*g, rho, i0[0] - 1 + a, i0[1] - 1 + b, i0[2] - 1 + c,
                               sp->q * sp->w[p] / dV * (w[0][a] * w[1][b] * w[2][c]));
            continue;
        }
        long long i0[3];
        double f[3];
        for (int a = 0; a < 3; ++a) {
            double fl = std::floor(xi[a]);
            i0[a] = (long long)fl;
            f[a] = xi[a] - fl;
        }
        for (int c = 0; c < 8; ++c) {
            int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
            double wgt = (bx ? f[0] : 1 - f[0]) * (by ? f[1] : 1 - f[1]) * (bz ? f[2] : 1 - f[2]);
            add_at(*g, rho, i0[0] + bx, i0[1] + by, i0[2] + bz, sp->q * sp->w[p] / dV * wgt);
        }
    }
}

// Discrete divergence of an E-lattice vector field at the nodes:
// (Fx(i+1/2) - Fx(i-1/2))/dx + ... .  Writes div (n cells).
void or_div(const or_grid* g, double* const* F, double* div) {
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                div[lin(*g, i, j, k)] = (at(*g, F[0], i, j, k) - at(*g, F[0], i - 1, j, k)) / g->d[0] +
                                        (at(*g, F[1], i, j, k) - at(*g, F[1], i, j - 1, k)) / g->d[1] +
                                        (at(*g, F[2], i, j, k) - at(*g, F[2], i, j, k - 1)) / g->d[2];
            }
}

// Forward-mode (tangent) run: the same steps in Dual arithmetic.  *_t arrays
// carry the tangent of every state array; on return they hold the tangent of
// the final state.  *dwk receives the tangent of the final kinetic energy
// summed over species, *wk its value.
void or_step_tangent(const or_grid* g, double* const* E, double* const* B, double* const* E_t,
                     double* const* B_t, int nsp, const or_species* sp, double* const* ptan, int nsteps,
                     double* wk, double* dwk) {
    long long ncell = (long long)g->n[0] * g->n[1] * g->n[2];
    std::vector<Dual> Ed[3], Bd[3], Jd[3];
    for (int c = 0; c < 3; ++c) {
        Ed[c].resize(ncell);
        Bd[c].resize(ncell);
        Jd[c].assign(ncell, Dual(0.0));
        for (long long o = 0; o < ncell; ++o) {
            Ed[c][o] = Dual(E[c][o], E_t[c][o]);
            Bd[c][o] = Dual(B[c][o], B_t[c][o]);
        }
    }
    // ptan[7*s + k]: tangent of array k (x,y,z,ux,uy,uz,w) of species s.
    std::vector<std::vector<Dual>> store;
    std::vector<SpeciesT<Dual>> sps;
    for (int s = 0; s < nsp; ++s) {
        double* vals[7] = {sp[s].x, sp[s].y, sp[s].z, sp[s].ux, sp[s].uy, sp[s].uz, sp[s].w};
        for (int k = 0; k < 7; ++k) {
            std::vector<Dual> v(sp[s].n);
            for (int64_t p = 0; p < sp[s].n; ++p) v[p] = Dual(vals[k][p], ptan[7 * s + k][p]);
            store.push_back(std::move(v));
        }
    }
    for (int s = 0; s < nsp; ++s) {
        std::vector<Dual>* b = &store[7 * s];
        sps.push_back(SpeciesT<Dual>{sp[s].q, sp[s].m, sp[s].n, b[0].data(), b[1].data(), b[2].data(),
                                     b[3].data(), b[4].data(), b[5].data(), b[6].data(), sp[s].active});
    }
    Dual* Ep[3] = {Ed[0].data(), Ed[1].data(), Ed[2].data()};
    Dual* Bp[3] = {Bd[0].data(), Bd[1].data(), Bd[2].data()};
    Dual* Jp[3] = {Jd[0].data(), Jd[1].data(), Jd[2].data()};
    for (int t = 0; t < nsteps; ++t) step(*g, Ep, Bp, Jp, sps);
    Dual wsum = 0.0;
    for (auto& s : sps) wsum += kinetic_energy(s);
    *wk = wsum.v;
    *dwk = wsum.d;
    for (int c = 0; c < 3; ++c)
        for (long long o = 0; o < ncell; ++o) {
            E[c][o] = Ed[c][o].v;
            E_t[c][o] = Ed[c][o].d;
            B[c][o] = Bd[c][o].v;
            B_t[c][o] = Bd[c][o].d;
        }
    for (int s = 0; s < nsp; ++s) {
        double* vals[7] = {sp[s].x, sp[s].y, sp[s].z, sp[s].ux, sp[s].uy, sp[s].uz, sp[s].w};
        for (int k = 0; k < 7; ++k)
            for (int64_t p = 0; p < sp[s].n; ++p) {
                vals[k][p] = store[7 * s + k][p].v;
                ptan[7 * s + k][p] = store[7 * s + k][p].d;
            }
    }
}

}  // extern "C"
