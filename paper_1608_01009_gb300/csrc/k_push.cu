// Fused FP64 particle kernel: field gather, Boris push, move and
// Villasenor-Buneman current deposition for one species, one supercell chunk
// per CTA iteration (the mixed-precision kernel is k_push32.cu).
//
// Method (arXiv:1608.01009): Sec. 2 lists the stages -- interpolate the field
// to each particle, solve the relativistic equations of motion, compute the
// current density; Sec. 3 fixes the cloud-in-cell form factor, the
// Villasenor-Buneman charge-conserving deposition and double precision; Sec. 4.3
// groups particles by supercells so that a supercell's field and current data
// stay in fast memory (there: L1; here: shared memory).
//
// GB300 design:
//   * persistent CTAs (a multiple of the SM count) stride over a table of
//     chunks (<= CHUNK particles of one supercell), built by the sort;
//   * each chunk's (S+4)^3 x 6 field tile -- the supercell plus 2 cells each
//     side -- arrives in shared memory in ONE 4-D TMA box load from the
//     ghost-padded E|B buffer, completion on an mbarrier (bounded wait);
//   * particles are read and written as coalesced SoA streams; positions are
//     a packed global cell + an offset in the cell, so the path needs no
//     double->int conversion (slower than an FMA on this part);
//   * current goes to an (S+3)^3 shared-memory tile with shared atomics --
//     for S <= 4 the 12 moments per cell that the edge values are linear in,
//     else the 3 edge components -- after the lanes of one cell are summed in
//     the warp, and is merged into the global FP64 J with one RED per non-zero
//     node.
//   The kernel's FP64 instructions are what bound it (GB300 issues FP64 at a
//   small fraction of its FP32 rate); R = double throughout.
#include "push_tile.cuh"

namespace picgb {


// min(v, largest double below 1) for v in [0, 1], on the bit pattern.
__device__ __forceinline__ double below_one_of(double v) {
    const long long b = __double_as_longlong(v), top = __double_as_longlong(0x1.fffffffffffffp-1);
    return __longlong_as_double(b < top ? b : top);
}

// Sum of c[0..11] over the 32 lanes, reduced and scattered by recursive
// halving: five butterfly rounds (partners lane ^ 16, 8, 4, 2, 1) that halve
// the values each lane carries, 13 adds and 13 shuffles per lane instead of
// 12 per round of a full scan.  Lane L ends with the total of value index
// reduce12_index(L); reduce12_owner(L) marks one lane per index.
template <class R>
__device__ __forceinline__ R reduce_scatter12(const R (&c)[12]) {
    const int lane = threadIdx.x & 31;
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
    R x[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) x[i] = (b4 ? c[i + 6] : c[i]) + __shfl_xor_sync(FULL, b4 ? c[i] : c[i + 6], 16);
    R y[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) y[i] = (b3 ? x[i + 3] : x[i]) + __shfl_xor_sync(FULL, b3 ? x[i] : x[i + 3], 8);
    // three values over a pair: lanes without bit 2 keep two, lanes with it one
    const R z0 = (b2 ? y[2] : y[0]) + __shfl_xor_sync(FULL, b2 ? y[0] : y[2], 4);
    const R z1 = y[1] + __shfl_xor_sync(FULL, y[1], 4);
    const R keep = (!b2 && b1) ? z1 : z0;
    const R w = keep + __shfl_xor_sync(FULL, (!b2 && !b1) ? z1 : z0, 2);
    return w + __shfl_xor_sync(FULL, w, 1);
}
__device__ __forceinline__ int reduce12_index(int lane) {
    return 6 * ((lane >> 4) & 1) + 3 * ((lane >> 3) & 1) + ((lane & 4) ? 2 : ((lane >> 1) & 1));
}
__device__ __forceinline__ bool reduce12_owner(int lane) { return (lane & 4) ? (lane & 3) == 0 : (lane & 1) == 0; }

// Moment form of the deposit (FP64 kernel with a coefficient tile).  With p,
// r the transverse axes of component c in the order of (s1, s2) above, the
// four edge values of a segment are linear in four moments,
//   A = Q d_c,  B = A m_p,  C = A m_r,  D = B m_r + Q sigma-term,
//   (0,0): A - B - C + D,  (1,0): B - D,  (0,1): C - D,  (1,1): D,
// so the tile accumulates the 12 moments per cell (5 FP64 operations per
// component instead of 8) and the merge forms each edge value from the four
// cells around it.  Value m of a cell lives at m * TJ^3 + cell key.
template <bool M, int TJ>
__device__ __forceinline__ int value_offset(int m) {
    if constexpr (M) return m * TJ * TJ * TJ;
    else return edge_offset<TJ>(m);
}

// Shared-tile atomic add; the debug build checks the index against the tile
// (12 moments per cell with M, else 3 edge components per cell).
template <class R, int TJ, bool M>
__device__ __forceinline__ void tile_add(R* Jt, int idx, R v) {
    if (in_range(idx, (M ? 12 : 3) * TJ * TJ * TJ)) atomicAdd(Jt + idx, v);
}

// Per distinct key of the warp: the lanes holding it contribute their v, the
// rest zeros, one reduce-scatter, 12 owner lanes add the totals to the tile.
template <class R, int TJ, bool M>
__device__ __forceinline__ void deposit_by_key(R* Jt, int key, const R (&v)[12]) {
    const int lane = threadIdx.x & 31;
    const int eo = value_offset<M, TJ>(reduce12_index(lane));
    const bool owner = reduce12_owner(lane);
    unsigned todo = __ballot_sync(FULL, key >= 0);
    while (todo) {
        const int k = __shfl_sync(FULL, key, __ffs(todo) - 1);
        const bool mine = key == k;
        todo &= ~__ballot_sync(FULL, mine);
        R c[12];
#pragma unroll
        for (int i = 0; i < 12; ++i) c[i] = mine ? v[i] : R(0);
        const R t = reduce_scatter12<R>(c);
        if (owner) tile_add<R, TJ, M>(Jt, k + eo, t);
    }
}

// Which warp reduction is cheaper for the FP64 pipe: one reduce-scatter per
// distinct key (at most nruns of them, 13 adds each) or a segmented scan of
// `rounds` rounds (12 adds each).
#ifndef PICGB_KEYRED
#define PICGB_KEYRED 1  // 0: segmented scan only
#endif
__device__ __forceinline__ bool channels_win(int nruns, int rounds) {
    if constexpr (PICGB_KEYRED == 0) return false;
    else return nruns * 13 <= rounds * 12;
}

// Current of one straight segment per lane, inside the cell whose J-tile
// corner index is `key` (-1: nothing to deposit): start a (cell-relative) and
// displacement d, in cells.  The 12 edge values are the line integrals of the
// two transverse CIC weights, Q d_c [W(s1) W(s2) + sigma d_p d_r / 12]
// (Villasenor-Buneman).  Lanes are ordered by cell, so lanes with the same
// key are summed in the warp before the shared-memory atomics: by one
// reduce-scatter per distinct key when the warp holds few keys, else by a
// segmented scan whose last lane per run adds the run's 12 totals.
template <class R, int TJ, bool M>
__device__ __forceinline__ void deposit_segment(R* Jt, int key, R ax, R ay, R az, R dx, R dy, R dz, R Qx, R Qy,
                                                R Qz) {
    const R h = R(0.5), tw = R(1.0 / 12.0);
    const R mx = fma(h, dx, ax), my = fma(h, dy, ay), mz = fma(h, dz, az);
    const R vol = dx * dy * (dz * tw);  // sigma term d_x d_y d_z / 12, shared by the 3 components
    R v[12];
    if constexpr (M) {  // moments A, B, C, D per component (transverse axes y,z; x,z; x,y)
        const R qx = Qx * dx, bx = qx * my;
        v[0] = qx, v[1] = bx, v[2] = qx * mz, v[3] = fma(bx, mz, Qx * vol);
        const R qy = Qy * dy, by = qy * mx;
        v[4] = qy, v[5] = by, v[6] = qy * mz, v[7] = fma(by, mz, Qy * vol);
        const R qz = Qz * dz, bz = qz * mx;
        v[8] = qz, v[9] = bz, v[10] = qz * my, v[11] = fma(bz, my, Qz * vol);
    } else {
    const R ox = R(1) - mx, oy = R(1) - my, oz = R(1) - mz;
    {  // Jx on edges (i+1/2, j+s1, k+s2)
        const R q = Qx * dx, qc = Qx * vol, qo = q * oy, qm = q * my;
        v[0] = fma(qo, oz, qc);
        v[1] = fma(qm, oz, -qc);
        v[2] = fma(qo, mz, -qc);
        v[3] = fma(qm, mz, qc);
    }
    {  // Jy on edges (i+s1, j+1/2, k+s2)
        const R q = Qy * dy, qc = Qy * vol, qo = q * ox, qm = q * mx;
        v[4] = fma(qo, oz, qc);
        v[5] = fma(qm, oz, -qc);
        v[6] = fma(qo, mz, -qc);
        v[7] = fma(qm, mz, qc);
    }
    {  // Jz on edges (i+s1, j+s2, k+1/2)
        const R q = Qz * dz, qc = Qz * vol, qo = q * ox, qm = q * mx;
        v[8] = fma(qo, oy, qc);
        v[9] = fma(qm, oy, -qc);
        v[10] = fma(qo, my, -qc);
        v[11] = fma(qm, my, qc);
    }
    }
    const int lane = threadIdx.x & 31;
    const int kprev = __shfl_up_sync(FULL, key, 1);
    const int knext = __shfl_down_sync(FULL, key, 1);
    const bool head = lane == 0 || kprev != key;
    const bool tail = lane == 31 || knext != key;
    const unsigned heads = __ballot_sync(FULL, head);
    const int start = 31 - __clz(heads & (FULL >> (31 - lane)));
    // only runs of real keys need summing (lanes with nothing to deposit form -1 runs)
    const int longest = __reduce_max_sync(FULL, key >= 0 ? (unsigned)(lane - start + 1) : 0u);
    const int nruns = __popc(__ballot_sync(FULL, head && key >= 0));
    const int rounds = longest > 1 ? 32 - __clz(longest - 1) : 0;
    if (channels_win(nruns, rounds)) {
        deposit_by_key<R, TJ, M>(Jt, key, v);
        return;
    }
    for (int dd = 1; dd < longest; dd <<= 1) {
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            const R t = __shfl_up_sync(FULL, v[i], dd);
            if (lane - dd >= start) v[i] += t;
        }
    }
    if (tail && key >= 0) {
#pragma unroll
        for (int i = 0; i < 12; ++i) tile_add<R, TJ, M>(Jt, key + value_offset<M, TJ>(i), v[i]);
    }
}

// Current of one piece with plain shared atomics (the deferred crossing moves
// of different lanes belong to different particles, rarely to the same cell).
template <class R, int TJ, bool M>
__device__ __forceinline__ void piece_direct(R* Jt, int b, R ax, R ay, R az, R dx, R dy, R dz, R Qx, R Qy, R Qz) {
    constexpr int TJ2 = TJ * TJ, TJ3 = TJ * TJ * TJ;
    const R h = R(0.5), tw = R(1.0 / 12.0);
    const R mx = fma(h, dx, ax), my = fma(h, dy, ay), mz = fma(h, dz, az);
    const R vol = dx * dy * (dz * tw);  // sigma term d_x d_y d_z / 12, shared by the 3 components
    if constexpr (M) {
        const R qx = Qx * dx, bx = qx * my;
        tile_add<R, TJ, M>(Jt, b, qx);
        tile_add<R, TJ, M>(Jt, b + TJ3, bx);
        tile_add<R, TJ, M>(Jt, b + 2 * TJ3, qx * mz);
        tile_add<R, TJ, M>(Jt, b + 3 * TJ3, fma(bx, mz, Qx * vol));
        const R qy = Qy * dy, by = qy * mx;
        tile_add<R, TJ, M>(Jt, b + 4 * TJ3, qy);
        tile_add<R, TJ, M>(Jt, b + 5 * TJ3, by);
        tile_add<R, TJ, M>(Jt, b + 6 * TJ3, qy * mz);
        tile_add<R, TJ, M>(Jt, b + 7 * TJ3, fma(by, mz, Qy * vol));
        const R qz = Qz * dz, bz = qz * mx;
        tile_add<R, TJ, M>(Jt, b + 8 * TJ3, qz);
        tile_add<R, TJ, M>(Jt, b + 9 * TJ3, bz);
        tile_add<R, TJ, M>(Jt, b + 10 * TJ3, qz * my);
        tile_add<R, TJ, M>(Jt, b + 11 * TJ3, fma(bz, my, Qz * vol));
        return;
    }
    const R ox = R(1) - mx, oy = R(1) - my, oz = R(1) - mz;
    {
        const R q = Qx * dx, qc = Qx * vol, qo = q * oy, qm = q * my;
        tile_add<R, TJ, M>(Jt, b, fma(qo, oz, qc));
        tile_add<R, TJ, M>(Jt, b + TJ, fma(qm, oz, -qc));
        tile_add<R, TJ, M>(Jt, b + TJ2, fma(qo, mz, -qc));
        tile_add<R, TJ, M>(Jt, b + TJ + TJ2, fma(qm, mz, qc));
    }
    {
        const R q = Qy * dy, qc = Qy * vol, qo = q * ox, qm = q * mx;
        tile_add<R, TJ, M>(Jt, TJ3 + b, fma(qo, oz, qc));
        tile_add<R, TJ, M>(Jt, TJ3 + b + 1, fma(qm, oz, -qc));
        tile_add<R, TJ, M>(Jt, TJ3 + b + TJ2, fma(qo, mz, -qc));
        tile_add<R, TJ, M>(Jt, TJ3 + b + 1 + TJ2, fma(qm, mz, qc));
    }
    {
        const R q = Qz * dz, qc = Qz * vol, qo = q * ox, qm = q * mx;
        tile_add<R, TJ, M>(Jt, 2 * TJ3 + b, fma(qo, oy, qc));
        tile_add<R, TJ, M>(Jt, 2 * TJ3 + b + 1, fma(qm, oy, -qc));
        tile_add<R, TJ, M>(Jt, 2 * TJ3 + b + TJ, fma(qo, my, -qc));
        tile_add<R, TJ, M>(Jt, 2 * TJ3 + b + 1 + TJ, fma(qm, my, qc));
    }
}

// Villasenor-Buneman split of a move that leaves its start cell (corner key
// k0 in the J tile, start offset a, displacement d): cut at every face crossed
// (at most one per axis), pieces in order of the crossing parameter, each
// piece deposited in the cell that holds its midpoint.
template <class R, int TJ, bool M>
__device__ void split_direct(R* Jt, int k0, R ax, R ay, R az, R dx, R dy, R dz, R Qx, R Qy, R Qz) {
    const R bx = ax + dx, by = ay + dy, bz = az + dz;
    const int sx = cell_shift(bx), sy = cell_shift(by), sz = cell_shift(bz);
    R t1 = sx ? cross_t(R(sx > 0 ? 1 : 0) - ax, dx) : R(1);
    R t2 = sy ? cross_t(R(sy > 0 ? 1 : 0) - ay, dy) : R(1);
    R t3 = sz ? cross_t(R(sz > 0 ? 1 : 0) - az, dz) : R(1);
    sort3(t1, t2, t3);
    const R ts[5] = {R(0), t1, t2, t3, R(1)};
    const int jx = k0 % TJ, jy = (k0 / TJ) % TJ, jz = k0 / (TJ * TJ);
    for (int s = 0; s < 4; ++s) {
        const R ta = ts[s], tb = ts[s + 1];
        if (!(tb > ta)) continue;
        const R pax = fma(ta, dx, ax), pay = fma(ta, dy, ay), paz = fma(ta, dz, az);
        const R dt = tb - ta;
        const R ddx = dt * dx, ddy = dt * dy, ddz = dt * dz;
        const int ox = cell_shift(fma(R(0.5), ddx, pax)), oy = cell_shift(fma(R(0.5), ddy, pay)),
                  oz = cell_shift(fma(R(0.5), ddz, paz));
        piece_direct<R, TJ, M>(Jt, ((jz + oz) * TJ + (jy + oy)) * TJ + (jx + ox), pax - R(ox), pay - R(oy), paz - R(oz),
                            ddx, ddy, ddz, Qx, Qy, Qz);
    }
}

// One particle per lane; all 32 lanes of the warp call it (lanes without a
// particle pass valid = false).  Returns w (gamma - 1) of the new state.
// CU: cubic cells, so dt/d and the current factor q/(dt d d) are the same on
// every axis (one multiply each instead of three).
// G: the particle in slot p of the sorted order is particle perm[p] of `pin`
// (the sort computed ranks only); its whole record goes to slot p of `ps`.
// Otherwise pin is ps and the particle is updated in place.
template <class R, int S, int NT, bool CU, bool G>
__device__ __forceinline__ R push_lane(const void* __restrict__ Fv, R* Jt, const PStore<R>& ps, const PStore<R>& pin,
                                       const int* __restrict__ perm, int p, bool valid, const PushParams& pp, int c0x,
                                       int c0y, int c0z, int* err, const XQueue<R>& xq, int qbase, int* s_qn) {
    constexpr int T = S + 4, T3 = T * T * T, TJ = S + 3;
    constexpr bool kMom = Tile<R, S>::kMoments;
    const GridDev& g = pp.g;
    const int q = G && valid ? perm[p] : p;  // where the particle is read
    const int cp = valid ? pin.cell[q] : INACTIVE;
    bool act = cp >= 0;  // negative: no particle, or deactivated at an absorbing boundary
    int gx = cell_x(cp), gy = cell_y(cp), gz = cell_z(cp);
    // cell relative to the supercell origin: the periodic image next to the tile
    int lx = gx - c0x, ly = gy - c0y, lz = gz - c0z;
    if (lx < -1) lx += g.n[0]; else if (lx > S) lx -= g.n[0];
    if (ly < -1) ly += g.n[1]; else if (ly > S) ly -= g.n[1];
    if (lz < -1) lz += g.n[2]; else if (lz > S) lz -= g.n[2];
    if (act && ((unsigned)(lx + 1) > (unsigned)(S + 1) || (unsigned)(ly + 1) > (unsigned)(S + 1) ||
                (unsigned)(lz + 1) > (unsigned)(S + 1))) {
        atomicOr(err, ERRBIT_DRIFT);
        act = false;
    }
    if (!act) lx = ly = lz = 0;
    R fx = R(0.25), fy = R(0.25), fz = R(0.25), ux = R(0), uy = R(0), uz = R(0), w = R(0);
    if (act) {
        fx = pin.off[0][q];
        fy = pin.off[1][q];
        fz = pin.off[2][q];
        ux = pin.u[0][q];
        uy = pin.u[1][q];
        uz = pin.u[2][q];
        w = pin.w[q];
    }
    if (G && valid) {
        // the record's constant fields move with it; a particle dropped below
        // keeps its (unused) offsets and momenta
        ps.w[p] = pin.w[q];
        ps.id[p] = pin.id[q];
        if (!act) {
            ps.cell[p] = cp;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                ps.off[a][p] = pin.off[a][q];
                ps.u[a][p] = pin.u[a][q];
            }
        }
    }

    // ---- gather: each component from its own staggered lattice (tile origin = cell c0-2)
    const int tx = lx + 2, ty = ly + 2, tz = lz + 2;
    const R hf = R(0.5);
    const bool sxb = lt_half(fx), syb = lt_half(fy), szb = lt_half(fz);
    const int hx = sxb ? tx - 1 : tx, hy = syb ? ty - 1 : ty, hz = szb ? tz - 1 : tz;
    const R gxf = fx + (sxb ? hf : -hf), gyf = fy + (syb ? hf : -hf), gzf = fz + (szb ? hf : -hf);
    R Ex, Ey, Ez, Bx, By, Bz;
    if constexpr (Tile<R, S>::kCoef) {
        constexpr int NE = Tile<R, S>::NE;
        const Coef<R>* X = static_cast<const Coef<R>*>(Fv);
        Ex = tri_coef<R, T>(X + 0 * NE, hx, ty, tz, gxf, fy, fz);
        Ey = tri_coef<R, T>(X + 1 * NE, tx, hy, tz, fx, gyf, fz);
        Ez = tri_coef<R, T>(X + 2 * NE, tx, ty, hz, fx, fy, gzf);
        Bx = tri_coef<R, T>(X + 3 * NE, tx, hy, hz, fx, gyf, gzf);
        By = tri_coef<R, T>(X + 4 * NE, hx, ty, hz, gxf, fy, gzf);
        Bz = tri_coef<R, T>(X + 5 * NE, hx, hy, tz, gxf, gyf, fz);
    } else {
        const R* F = static_cast<const R*>(Fv);
        Ex = tri_raw<R, T>(F + 0 * T3, hx, ty, tz, gxf, fy, fz);
        Ey = tri_raw<R, T>(F + 1 * T3, tx, hy, tz, fx, gyf, fz);
        Ez = tri_raw<R, T>(F + 2 * T3, tx, ty, hz, fx, fy, gzf);
        Bx = tri_raw<R, T>(F + 3 * T3, tx, hy, hz, fx, gyf, gzf);
        By = tri_raw<R, T>(F + 4 * T3, hx, ty, hz, gxf, fy, gzf);
        Bz = tri_raw<R, T>(F + 5 * T3, hx, hy, tz, gxf, gyf, fz);
    }

    // ---- Boris: half electric kick, rotation, half electric kick
    const R h = pp.qdt2m;
    const R umx = fma(h, Ex, ux), umy = fma(h, Ey, uy), umz = fma(h, Ez, uz);
    const R hg = h * rsqrt_ge1(fma(umx, umx, fma(umy, umy, fma(umz, umz, R(1)))));
    const R tbx = hg * Bx, tby = hg * By, tbz = hg * Bz;
    const R sf = R(2) * rcp_ge1(fma(tbx, tbx, fma(tby, tby, fma(tbz, tbz, R(1)))));
    const R sbx = sf * tbx, sby = sf * tby, sbz = sf * tbz;
    const R upx = fma(umy, tbz, fma(-umz, tby, umx));
    const R upy = fma(umz, tbx, fma(-umx, tbz, umy));
    const R upz = fma(umx, tby, fma(-umy, tbx, umz));
    ux = fma(h, Ex, fma(upy, sbz, fma(-upz, sby, umx)));
    uy = fma(h, Ey, fma(upz, sbx, fma(-upx, sbz, umy)));
    uz = fma(h, Ez, fma(upx, sby, fma(-upy, sbx, umz)));

    // ---- move: displacement in cells, x^{n+1} = x^n + dt u / gamma
    const R u2p1 = fma(ux, ux, fma(uy, uy, fma(uz, uz, R(1))));
    const R gi = rsqrt_ge1(u2p1);
    R dx, dy, dz;
    if constexpr (CU) {
        const R gd = gi * pp.dtd[0];
        dx = ux * gd, dy = uy * gd, dz = uz * gd;
    } else {
        dx = ux * (gi * pp.dtd[0]), dy = uy * (gi * pp.dtd[1]), dz = uz * (gi * pp.dtd[2]);
    }
    const R bx = fx + dx, by = fy + dy, bz = fz + dz;  // end point in the start cell's frame
    const int sx = cell_shift(bx), sy = cell_shift(by), sz = cell_shift(bz);
    if (act && ((unsigned)(lx + sx + 1) > (unsigned)(S + 1) || (unsigned)(ly + sy + 1) > (unsigned)(S + 1) ||
                (unsigned)(lz + sz + 1) > (unsigned)(S + 1))) {
        // cannot happen while K * max(dt/d) < 1; record it, drop the particle, touch no tile
        atomicOr(err, ERRBIT_DRIFT);
        ps.cell[p] = INACTIVE | cp;
        if (G) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                ps.off[a][p] = pin.off[a][q];
                ps.u[a][p] = pin.u[a][q];
            }
        }
        act = false;
    }

    // ---- Villasenor-Buneman deposit into the shared J tile (tile origin = cell c0-1)
    const bool dep = act && w != R(0);
    const R wq = dep ? w : R(0);
    const R Qx = pp.cq[0] * wq;
    const R Qy = CU ? Qx : pp.cq[1] * wq, Qz = CU ? Qx : pp.cq[2] * wq;
    const int key0 = ((lz + 1) * TJ + (ly + 1)) * TJ + (lx + 1);
    {
        // a crossing lane would make its whole warp execute the split on the FP64
        // pipe, so crossing moves are queued and split after the chunk by full
        // warps; moves that stay in their cell deposit one segment each, summed per
        // cell run
        const bool cross = dep && (sx | sy | sz) != 0;
        deposit_segment<R, TJ, kMom>(Jt, dep && !cross ? key0 : -1, fx, fy, fz, dx, dy, dz, Qx, Qy, Qz);
        const unsigned cm = __ballot_sync(FULL, cross);
        if (cm) {
            const int lane = threadIdx.x & 31, first = __ffs(cm) - 1;
            int base = 0;
            if (lane == first) base = atomicAdd(s_qn, __popc(cm));
            base = __shfl_sync(FULL, base, first);
            const int slot = base + __popc(cm & ((1u << lane) - 1u));
            if (cross && slot >= CHUNK) atomicOr(err, ERRBIT_DRIFT);  // a chunk longer than CHUNK: dropped
            if (cross && slot < CHUNK && in_range(qbase + slot, (long long)gridDim.x * CHUNK)) {
                const int q = qbase + slot;
                xq.key[q] = key0;
                xq.a[0][q] = fx;
                xq.a[1][q] = fy;
                xq.a[2][q] = fz;
                xq.d[0][q] = dx;
                xq.d[1][q] = dy;
                xq.d[2][q] = dz;
                xq.w[q] = wq;
            }
        }
    }
    if (!act) return R(0);

    // ---- new cell and offset
    R nfx = bx, nfy = by, nfz = bz;
    // the shifted offsets lie in [0, 1] (non-negative, so their bit patterns
    // order like integers) and are clamped below 1 on the integer ALU; a warp
    // with no crossing lane skips the block (FP64-pipe issue is what bounds
    // this kernel)
    if (__any_sync(__activemask(), (sx | sy | sz) != 0)) {
        if (sx) nfx = below_one_of(bx - R(sx));
        if (sy) nfy = below_one_of(by - R(sy));
        if (sz) nfz = below_one_of(bz - R(sz));
    }
    int ng[3] = {gx + sx, gy + sy, gz + sz};
    bool gone = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (ng[a] < 0 || ng[a] >= g.n[a]) {
            if (g.bc[a] == 0) ng[a] += ng[a] < 0 ? g.n[a] : -g.n[a];
            else gone = true;
        }
    }
    ps.cell[p] = gone ? (INACTIVE | cp) : pack_cell(ng[0], ng[1], ng[2]);
    ps.off[0][p] = nfx;
    ps.off[1][p] = nfy;
    ps.off[2][p] = nfz;
    ps.u[0][p] = ux;
    ps.u[1][p] = uy;
    ps.u[2][p] = uz;
    // kinetic energy of the new state: w (gamma - 1), gamma = (1 + u^2) / sqrt(1 + u^2)
    return gone ? R(0) : w * fma(u2p1, gi, R(-1));
}

// Two resident CTAs of 256 threads per SM (the kernel needs about 100
// registers; its shared tile is 106 KB at S = 4).
template <class R, int S, int NT, bool CU, bool G>
__global__ void __launch_bounds__(NT, 2) k_push(const __grid_constant__ CUtensorMap tmEB, PushParams pp, PStore<R> ps,
                                            PStore<R> pin, const int* __restrict__ perm, XQueue<R> xq,
                                            const Chunk* __restrict__ chunks, const int* __restrict__ nchunks,
                                            double* __restrict__ J, double* __restrict__ ek_part,
                                            int* __restrict__ err) {
    constexpr int T = S + 4, T3 = T * T * T, TJ = S + 3, TJ3 = TJ * TJ * TJ;
    constexpr bool kCoef = Tile<R, S>::kCoef;
    extern __shared__ unsigned char smem_raw[];
    // smem: raw TMA tile (re-used as the J tile once the coefficients are built) | coefficient tile
    R* F = reinterpret_cast<R*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    constexpr bool kMom = Tile<R, S>::kMoments;
    constexpr int ACC = Tile<R, S>::ACC, RAW = Tile<R, S>::RAW;
    R* Jt = kCoef ? F : F + 6 * T3;
    Coef<R>* X = reinterpret_cast<Coef<R>*>(F + RAW);
    const void* Fuse = kCoef ? static_cast<const void*>(X) : static_cast<const void*>(F);
    __shared__ uint64_t bar;
    __shared__ double red[NT / 32];
    __shared__ int s_qn;  // entries in this CTA's crossing queue
    const GridDev& g = pp.g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int qbase = blockIdx.x * CHUNK;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        s_qn = 0;
    }
    __syncthreads();
    uint32_t phase = 0;
    double ek = 0.0;
    const int nch = *nchunks;
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const Chunk ch = chunks[c];
        const int sx = ch.sc % g.nsc[0], sy = (ch.sc / g.nsc[0]) % g.nsc[1], sz = ch.sc / (g.nsc[0] * g.nsc[1]);
        const int c0x = sx * S, c0y = sy * S, c0z = sz * S;
        if (threadIdx.x == 0) {
            fence_proxy_async();
            mbar_expect_tx(&bar, 6u * T3 * (uint32_t)sizeof(R));
            // field tile: cells c0-2 .. c0+S+1, i.e. padded index c0 .. c0+S+3
            tma_load_4d(F, &tmEB, c0x, c0y, c0z, 0, &bar);
        }
        const int end = ch.start + ch.count;
        if (!kCoef)
            for (int i = threadIdx.x; i < 3 * TJ3; i += NT) Jt[i] = R(0);
        const bool ok = mbar_wait_bounded(&bar, phase, WAIT_LIMIT, WAIT_LIMIT_NS);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(err, ERRBIT_TIMEOUT);
                ek_part[blockIdx.x] = 0.0;  // no stale partial of an earlier launch survives
            }
            return;
        }
        phase ^= 1u;
        if (kCoef) {
            build_coef<R, T, NT>(F, X);
            __syncthreads();
            for (int i = threadIdx.x; i < ACC; i += NT) Jt[i] = R(0);  // J tile over the raw tile
            __syncthreads();
        }
        R ek_chunk = R(0);  // at most CHUNK / NT particles per lane
        for (int base = ch.start + warp * 32; base < end; base += NT) {
            const int p = base + lane;
            ek_chunk += push_lane<R, S, NT, CU, G>(Fuse, Jt, ps, pin, perm, p, p < end, pp, c0x, c0y, c0z, err, xq,
                                                   qbase, &s_qn);
        }
        ek += (double)ek_chunk;
        __syncthreads();
        // the deferred crossing moves, split by every thread of the CTA
        const int nq = min(s_qn, CHUNK);
        for (int i = threadIdx.x; i < nq; i += NT) {
            const int q = qbase + i;
            if (!in_range(q, (long long)gridDim.x * CHUNK)) continue;  // debug build only
            const R w = xq.w[q];
            split_direct<R, TJ, kMom>(Jt, xq.key[q], xq.a[0][q], xq.a[1][q], xq.a[2][q], xq.d[0][q], xq.d[1][q],
                                      xq.d[2][q], pp.cq[0] * w, pp.cq[1] * w, pp.cq[2] * w);
        }
        __syncthreads();
        if (threadIdx.x == 0) s_qn = 0;
        // merge: J tile cell t is domain cell c0 - 1 + t, padded index c0 + 1 + t
        for (int i = threadIdx.x; i < 3 * TJ3; i += NT) {
            const int comp = i / TJ3, r = i - comp * TJ3;
            const int tz = r / (TJ * TJ), ty = (r / TJ) % TJ, tx = r % TJ;
            R v;
            if constexpr (kMom) {
                // edge value from the moments of the (up to) four cells around it:
                // (0,0) A - B - C + D of the cell, (1,0) B - D of the cell one step
                // down the first transverse axis, (0,1) C - D down the second, (1,1) D
                const R* Mc = Jt + 4 * comp * TJ3;
                const int sp = comp == 0 ? TJ : 1, sr = comp == 2 ? TJ : TJ * TJ;
                const bool hp = (comp == 0 ? ty : tx) > 0, hr = (comp == 2 ? ty : tz) > 0;
                v = (Mc[r] - Mc[TJ3 + r]) + (Mc[3 * TJ3 + r] - Mc[2 * TJ3 + r]);
                if (hp) v += Mc[TJ3 + r - sp] - Mc[3 * TJ3 + r - sp];
                if (hr) v += Mc[2 * TJ3 + r - sr] - Mc[3 * TJ3 + r - sr];
                if (hp && hr) v += Mc[3 * TJ3 + r - sp - sr];
            } else {
                v = Jt[i];
            }
            if (v != R(0)) {
                const long long o = (long long)comp * g.P + (c0x + 1 + tx) +
                                    (long long)g.np[0] * ((c0y + 1 + ty) + (long long)g.np[1] * (c0z + 1 + tz));
                if (in_range(o, 3 * g.P)) atomicAdd(&J[o], (double)v);
            }
        }
        __syncthreads();
    }
    const double s = block_sum<NT>(ek, red);
    if (threadIdx.x == 0) ek_part[blockIdx.x] = s * pp.mass;
}

// ------------------------------------------------------------------ launchers
#ifndef PICGB_PUSH_NT
#define PICGB_PUSH_NT 256
#endif
constexpr int PUSH_NT = PICGB_PUSH_NT;

template <class R, int S>
size_t push_smem_bytes() {
    constexpr int T = S + 4;
    if (Tile<R, S>::kCoef) return 128 + sizeof(R) * Tile<R, S>::RAW + sizeof(Coef<R>) * 6 * Tile<R, S>::NE;
    return 128 + sizeof(R) * (6 * T * T * T + Tile<R, S>::ACC);
}

template <class R, int S>
cudaError_t push_setup(int* blocks_per_sm) {
    const int sm = (int)push_smem_bytes<R, S>();
    cudaError_t e = cudaSuccess;
    for (auto f : {k_push<R, S, PUSH_NT, true, false>, k_push<R, S, PUSH_NT, false, false>,
                   k_push<R, S, PUSH_NT, true, true>, k_push<R, S, PUSH_NT, false, true>})
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_push<R, S, PUSH_NT, false, false>, PUSH_NT,
                                                         sm);
}

// perm null: the particles are updated in place in ps.  Otherwise slot i of
// ps receives particle perm[i] of pin, updated (pin and ps are the store's
// two buffers; the sort computed ranks only).
template <class R, int S>
cudaError_t push_launch(int grid, cudaStream_t st, const CUtensorMap& tm, const PushParams& pp, const PStore<R>& ps,
                        const PStore<R>& pin, const int* perm, const XQueue<R>& xq, const Chunk* chunks,
                        const int* nchunks, double* J, double* ek_part, int* err) {
    const bool cubic = pp.g.d[0] == pp.g.d[1] && pp.g.d[1] == pp.g.d[2];
    const size_t sm = push_smem_bytes<R, S>();
    if (cubic && perm)
        k_push<R, S, PUSH_NT, true, true><<<grid, PUSH_NT, sm, st>>>(tm, pp, ps, pin, perm, xq, chunks, nchunks, J,
                                                                    ek_part, err);
    else if (cubic)
        k_push<R, S, PUSH_NT, true, false><<<grid, PUSH_NT, sm, st>>>(tm, pp, ps, ps, nullptr, xq, chunks, nchunks, J,
                                                                     ek_part, err);
    else if (perm)
        k_push<R, S, PUSH_NT, false, true><<<grid, PUSH_NT, sm, st>>>(tm, pp, ps, pin, perm, xq, chunks, nchunks, J,
                                                                     ek_part, err);
    else
        k_push<R, S, PUSH_NT, false, false><<<grid, PUSH_NT, sm, st>>>(tm, pp, ps, ps, nullptr, xq, chunks, nchunks,
                                                                      J, ek_part, err);
    return cudaGetLastError();
}

#define PICGB_PUSH_INST(R, S)                                                                                   \
    template cudaError_t push_setup<R, S>(int*);                                                                \
    template cudaError_t push_launch<R, S>(int, cudaStream_t, const CUtensorMap&, const PushParams&,            \
                                           const PStore<R>&, const PStore<R>&, const int*, const XQueue<R>&,    \
                                           const Chunk*, const int*, double*, double*, int*);
PICGB_PUSH_INST(double, 2)
PICGB_PUSH_INST(double, 4)
PICGB_PUSH_INST(double, 8)

PICGB_INDEX_FLAG_READER(push_index_flags)

}  // namespace picgb
