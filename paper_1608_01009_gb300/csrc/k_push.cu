// Fused particle kernel: field gather, Boris push, move and Villasenor-Buneman
// current deposition for one species, one supercell chunk per CTA iteration.
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
//     a packed global cell + an offset in the cell, so the FP64 path needs no
//     double->int conversion (slower than an FMA on this part);
//   * current goes to an (S+3)^3 shared-memory tile with shared atomics --
//     3 edge components per cell, or for FP64 with S <= 4 the 12 moments per
//     cell that the edge values are linear in -- and is merged into the
//     global FP64 J with one RED per non-zero node.
//   R = double: every value in FP64.  R = float (mixed): offsets, momenta,
//   field tile (from the FP32 field copy), interpolation and the shared J tile
//   in FP32; the merge into J and the kinetic-energy sum in FP64.
#include <type_traits>

#include "pic_internal.cuh"

namespace picgb {



template <class R>
__device__ __forceinline__ R prm(double d, float f);
template <>
__device__ __forceinline__ double prm<double>(double d, float) {
    return d;
}
template <>
__device__ __forceinline__ float prm<float>(double, float f) {
    return f;
}

template <class R>
__device__ __forceinline__ R lerp(R a, R b, R t) {
    return fma(t, b - a, a);
}

// Shared-memory field tile.  TMA lands the raw (S+4)^3 x 6 box.  For S <= 4 it
// is then rebuilt as per-cell bilinear coefficients of every z plane,
//   f(a, b) = F00 + a Dx + b (Dy + a Dxy)        (a, b = x, y fractions),
// over lattice cells i, j in [0, T-2], k in [0, T-1]: one trilinear
// interpolation is then 2 vector loads and 2 x 3 FMAs + 1 lerp, instead of 8
// scalar loads and 7 lerps (14 operations).  FP32: one float4 per cell; FP64:
// two double2.  S = 8 keeps the raw tile (its coefficient tile would not fit).
#ifndef PICGB_MOMENTS
#define PICGB_MOMENTS 1
#endif
template <class R, int S>
struct Tile {
    static constexpr int T = S + 4, T3 = T * T * T, TJ = S + 3, TJ3 = TJ * TJ * TJ;
    static constexpr int NE = (T - 1) * (T - 1) * T;  // coefficient cells per component
    static constexpr bool kCoef = S <= 4;
    // FP64 with a coefficient tile accumulates the deposit's 12 moments per
    // cell (see value_offset) instead of the 3 edge components
    static constexpr bool kMoments = PICGB_MOMENTS && sizeof(R) == 8 && kCoef;
    static constexpr int ACC = kMoments ? 12 * TJ3 : 3 * TJ3;         // accumulation tile (elements)
    static constexpr int RAW = 6 * T3 > ACC ? 6 * T3 : ACC;           // raw tile region, re-used for it
};

template <class R>
struct Coef;
template <>
struct Coef<float> {
    float4 v;  // F00, Dx, Dy, Dxy
};
template <>
struct Coef<double> {
    double2 a, b;  // (F00, Dx), (Dy, Dxy)
};

__device__ __forceinline__ float bil(const Coef<float>& q, float a, float b) {
    return fmaf(b, fmaf(a, q.v.w, q.v.z), fmaf(a, q.v.y, q.v.x));
}
__device__ __forceinline__ double bil(const Coef<double>& q, double a, double b) {
    return fma(b, fma(a, q.b.y, q.b.x), fma(a, q.a.y, q.a.x));
}

template <class R, int T>
__device__ __forceinline__ R tri_raw(const R* __restrict__ F, int i, int j, int k, R a, R b, R c) {
    const R* q = F + (k * T + j) * T + i;
    R c00 = lerp(q[0], q[1], a);
    R c10 = lerp(q[T], q[T + 1], a);
    R c01 = lerp(q[T * T], q[T * T + 1], a);
    R c11 = lerp(q[T * T + T], q[T * T + T + 1], a);
    return lerp(lerp(c00, c10, b), lerp(c01, c11, b), c);
}

template <class R, int T>
__device__ __forceinline__ R tri_coef(const Coef<R>* __restrict__ X, int i, int j, int k, R a, R b, R c) {
    const int o = (k * (T - 1) + j) * (T - 1) + i;
    const R v0 = bil(X[o], a, b), v1 = bil(X[o + (T - 1) * (T - 1)], a, b);
    return lerp(v0, v1, c);
}

// Build the coefficient tile X from the raw tile F.
template <class R, int T, int NT>
__device__ __forceinline__ void build_coef(const R* __restrict__ F, Coef<R>* __restrict__ X) {
    constexpr int NE = (T - 1) * (T - 1) * T;
    for (int e = threadIdx.x; e < 6 * NE; e += NT) {
        const int comp = e / NE, r = e - comp * NE;
        const int i = r % (T - 1), j = (r / (T - 1)) % (T - 1), k = r / ((T - 1) * (T - 1));
        const R* f = F + comp * T * T * T + (k * T + j) * T + i;
        const R f00 = f[0], f10 = f[1], f01 = f[T], f11 = f[T + 1];
        const R dx = f10 - f00, dy = f01 - f00, dxy = (f11 - f10) - dy;
        if constexpr (sizeof(R) == 4) {
            X[e].v = make_float4(f00, dx, dy, dxy);
        } else {
            X[e].a = make_double2(f00, dx);
            X[e].b = make_double2(dy, dxy);
        }
    }
}

constexpr unsigned FULL = 0xffffffffu;

// Comparisons of cell offsets on their bit patterns (integer ALU, not the FP64
// pipe).  Offsets lie in [0,1); end points b = offset + displacement lie in
// (-1, 2) and are never -0.
__device__ __forceinline__ bool lt_half(double x) { return __double2hiint(x) < 0x3FE00000; }
__device__ __forceinline__ bool lt_half(float x) { return __float_as_int(x) < 0x3F000000; }
__device__ __forceinline__ int cell_shift(double b) {
    const int h = __double2hiint(b);
    return h < 0 ? -1 : (h >= 0x3FF00000 ? 1 : 0);
}
__device__ __forceinline__ int cell_shift(float b) {
    const int h = __float_as_int(b);
    return h < 0 ? -1 : (h >= 0x3F800000 ? 1 : 0);
}

template <class R>
__device__ __forceinline__ R below_one();
template <>
__device__ __forceinline__ double below_one<double>() {
    return 0x1.fffffffffffffp-1;
}
template <>
__device__ __forceinline__ float below_one<float>() {
    return 0x1.fffffep-1f;
}

// min(v, largest double below 1) for v in [0, 1], on the bit pattern.
__device__ __forceinline__ double below_one_of(double v) {
    const long long b = __double_as_longlong(v), top = __double_as_longlong(0x1.fffffffffffffp-1);
    return __longlong_as_double(b < top ? b : top);
}

// Crossing parameter (face - a) / d: IEEE division in FP64; in the FP32 kernel
// the fast divide (its 2-ulp error is far below the FP32 state's own rounding).
__device__ __forceinline__ double cross_t(double num, double d) { return num / d; }
__device__ __forceinline__ float cross_t(float num, float d) { return __fdividef(num, d); }

template <class R>
__device__ __forceinline__ void sort3(R& a, R& b, R& c) {
    R lo = fmin(a, b), hi = fmax(a, b);
    a = lo;
    b = hi;
    lo = fmin(b, c);
    hi = fmax(b, c);
    b = lo;
    c = hi;
    lo = fmin(a, b);
    hi = fmax(a, b);
    a = lo;
    b = hi;
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

// The 12 edge values of one cell, v[0..11] = Jx (i+1/2, j+s1, k+s2), Jy
// (i+s1, j+1/2, k+s2), Jz (i+s1, j+s2, k+1/2) with (s1, s2) = (0,0), (1,0),
// (0,1), (1,1): offset of value m from the cell's corner in the J tile.
template <int TJ>
__device__ __forceinline__ int edge_offset(int m) {
    const int comp = m >> 2, e = m & 3;
    return comp * TJ * TJ * TJ + (e & 1) * (comp == 0 ? TJ : 1) + (e >> 1) * (comp == 2 ? TJ : TJ * TJ);
}

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
        if (owner) atomicAdd(Jt + k + eo, t);
    }
}

// Which warp reduction is cheaper for the FP64 pipe: one reduce-scatter per
// distinct key (at most nruns of them, 13 adds each) or a segmented scan of
// `rounds` rounds (12 adds each).  The FP32 kernel is bound by instruction
// issue, not by its adds, and the per-key path issues more instructions
// (selects, ballots, shuffles): it keeps the scan.
#ifndef PICGB_KEYRED
#define PICGB_KEYRED 1  // 0: segmented scan only
#endif
#ifndef PICGB_F32_PAIRED
#define PICGB_F32_PAIRED 1  // FP32 kernel: packed two-wide FP32 adds in the warp scan
#endif
template <class R>
struct DepositCost {
    __device__ static bool channels_win(int nruns, int rounds) {
        if constexpr (PICGB_KEYRED == 0 || sizeof(R) == 4) return false;
        else return nruns * 13 <= rounds * 12;
    }
};

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
    } else if constexpr (sizeof(R) == 4 && PICGB_F32_PAIRED) {
        // the same edge values, two at a time with packed two-wide FP32 instructions
        const float ox = 1.0f - mx, oy = 1.0f - my, oz = 1.0f - mz;
        const auto edges = [](float* out, float q, float qc, float o1, float m1, float o2, float m2) {
            const float2 a = __fmul2_rn(make_float2(q, q), make_float2(o1, m1));        // (q o1, q m1)
            const float2 lo = __ffma2_rn(a, make_float2(o2, o2), make_float2(qc, -qc));  // s2 = 0
            const float2 hi = __ffma2_rn(a, make_float2(m2, m2), make_float2(-qc, qc));  // s2 = 1
            out[0] = lo.x, out[1] = lo.y, out[2] = hi.x, out[3] = hi.y;
        };
        edges(v + 0, Qx * dx, Qx * vol, oy, my, oz, mz);
        edges(v + 4, Qy * dy, Qy * vol, ox, mx, oz, mz);
        edges(v + 8, Qz * dz, Qz * vol, ox, mx, oy, my);
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
    if (DepositCost<R>::channels_win(nruns, rounds)) {
        deposit_by_key<R, TJ, M>(Jt, key, v);
        return;
    }
    if constexpr (sizeof(R) == 4 && PICGB_F32_PAIRED) {
        // FP32: the adds of value pairs as packed two-wide FP32 instructions
        for (int dd = 1; dd < longest; dd <<= 1) {
            const bool add = lane - dd >= start;
#pragma unroll
            for (int i = 0; i < 12; i += 2) {
                const float2 t = make_float2(__shfl_up_sync(FULL, v[i], dd), __shfl_up_sync(FULL, v[i + 1], dd));
                if (add) {
                    const float2 s2 = __fadd2_rn(make_float2(v[i], v[i + 1]), t);
                    v[i] = s2.x;
                    v[i + 1] = s2.y;
                }
            }
        }
    } else {
        for (int dd = 1; dd < longest; dd <<= 1) {
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                const R t = __shfl_up_sync(FULL, v[i], dd);
                if (lane - dd >= start) v[i] += t;
            }
        }
    }
    if (tail && key >= 0) {
#pragma unroll
        for (int i = 0; i < 12; ++i) atomicAdd(Jt + key + value_offset<M, TJ>(i), v[i]);
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
        R* J = Jt + b;
        const R qx = Qx * dx, bx = qx * my;
        atomicAdd(J, qx);
        atomicAdd(J + TJ3, bx);
        atomicAdd(J + 2 * TJ3, qx * mz);
        atomicAdd(J + 3 * TJ3, fma(bx, mz, Qx * vol));
        const R qy = Qy * dy, by = qy * mx;
        atomicAdd(J + 4 * TJ3, qy);
        atomicAdd(J + 5 * TJ3, by);
        atomicAdd(J + 6 * TJ3, qy * mz);
        atomicAdd(J + 7 * TJ3, fma(by, mz, Qy * vol));
        const R qz = Qz * dz, bz = qz * mx;
        atomicAdd(J + 8 * TJ3, qz);
        atomicAdd(J + 9 * TJ3, bz);
        atomicAdd(J + 10 * TJ3, qz * my);
        atomicAdd(J + 11 * TJ3, fma(bz, my, Qz * vol));
        return;
    }
    const R ox = R(1) - mx, oy = R(1) - my, oz = R(1) - mz;
    {
        const R q = Qx * dx, qc = Qx * vol, qo = q * oy, qm = q * my;
        R* J = Jt + b;
        atomicAdd(J, fma(qo, oz, qc));
        atomicAdd(J + TJ, fma(qm, oz, -qc));
        atomicAdd(J + TJ2, fma(qo, mz, -qc));
        atomicAdd(J + TJ + TJ2, fma(qm, mz, qc));
    }
    {
        const R q = Qy * dy, qc = Qy * vol, qo = q * ox, qm = q * mx;
        R* J = Jt + TJ3 + b;
        atomicAdd(J, fma(qo, oz, qc));
        atomicAdd(J + 1, fma(qm, oz, -qc));
        atomicAdd(J + TJ2, fma(qo, mz, -qc));
        atomicAdd(J + 1 + TJ2, fma(qm, mz, qc));
    }
    {
        const R q = Qz * dz, qc = Qz * vol, qo = q * ox, qm = q * mx;
        R* J = Jt + 2 * TJ3 + b;
        atomicAdd(J, fma(qo, oy, qc));
        atomicAdd(J + 1, fma(qm, oy, -qc));
        atomicAdd(J + TJ, fma(qo, my, -qc));
        atomicAdd(J + 1 + TJ, fma(qm, my, qc));
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

// FP32 kernel with a coefficient tile: each warp keeps the moves that leave
// their start cell in a small shared-memory queue (WQ entries of key, start
// offset, displacement and weight, SoA) carved from the raw tile's space
// behind the J tile, and splits them with all lanes once the queue is full
// and at the end of the chunk.  A warp whose lanes cross in bulk splits them
// at once.
#ifndef PICGB_F32_QUEUE
#define PICGB_F32_QUEUE 1
#endif
#ifndef PICGB_F32_GQ
#define PICGB_F32_GQ 0  // 1: FP32 crossing moves through the per-CTA global queue, as FP64
#endif
constexpr int WQ = 31;
template <class R, int S, int NT>
struct WarpQueue {
    static constexpr int TJ = S + 3, T = S + 4;
    static constexpr int OFF = (3 * TJ * TJ * TJ + 7) & ~7;  // floats behind the J tile
    static constexpr bool kOn = PICGB_F32_QUEUE && sizeof(R) == 4 && Tile<R, S>::kCoef &&
                                OFF + (NT / 32) * 8 * WQ <= 6 * T * T * T;
};

template <class R, int TJ>
__device__ __forceinline__ void warp_queue_flush(R* Jt, const R* q, int n, const PushParams& pp) {
    __syncwarp();
    const int lane = threadIdx.x & 31;
    if (lane < n) {
        const R w = q[7 * WQ + lane];
        split_direct<R, TJ, false>(Jt, __float_as_int(q[lane]), q[WQ + lane], q[2 * WQ + lane], q[3 * WQ + lane],
                            q[4 * WQ + lane], q[5 * WQ + lane], q[6 * WQ + lane], pp.cq_f[0] * w, pp.cq_f[1] * w,
                            pp.cq_f[2] * w);
    }
    __syncwarp();
}

// Prefetch of the next batch's particle records into registers, per kernel:
// 0 none, 1 cell and offsets, 2 the whole record, loaded one batch ahead so
// that their latency overlaps the current batch's work (the warp's first
// batch of a chunk is loaded while the field tile is fetched and built).
// Mixed 128^3 x 32 particle kernel: 3.85 ms without, 3.71 ms at level 1,
// 3.62 ms at level 2; the FP64 kernel (FP64-pipe bound) gains nothing at
// level 1 and loses 2.4% at level 2.  An additional L2 prefetch of the batch
// after the next cost 1%.
#ifndef PICGB_PREFETCH_F32
#define PICGB_PREFETCH_F32 2
#endif
#ifndef PICGB_PREFETCH_F64
#define PICGB_PREFETCH_F64 0
#endif
template <class R>
struct Prefetch {
    static constexpr int level = sizeof(R) == 4 ? PICGB_PREFETCH_F32 : PICGB_PREFETCH_F64;
};

template <class R>
struct PIn {
    int cell;
    R off[3], u[3], w;
};
template <class R>
__device__ __forceinline__ void load_head(PIn<R>& in, const PStore<R>& ps, int p, bool valid) {
    in.cell = valid ? ps.cell[p] : INACTIVE;
    if (valid) {
#pragma unroll
        for (int a = 0; a < 3; ++a) in.off[a] = ps.off[a][p];
    }
}
template <class R>
__device__ __forceinline__ void load_tail(PIn<R>& in, const PStore<R>& ps, int p, bool valid) {
    if (valid) {
#pragma unroll
        for (int a = 0; a < 3; ++a) in.u[a] = ps.u[a][p];
        in.w = ps.w[p];
    }
}

// One particle per lane; all 32 lanes of the warp call it (lanes without a
// particle pass valid = false).  Returns w (gamma - 1) of the new state.
// CU: cubic cells, so dt/d and the current factor q/(dt d d) are the same on
// every axis (one multiply each instead of three).
template <class R, int S, int NT, bool CU>
__device__ __forceinline__ R push_lane(const void* __restrict__ Fv, R* Jt, const PStore<R>& ps, int p, bool valid,
                                       const PushParams& pp, int c0x, int c0y, int c0z, int* err,
                                       const XQueue<R>& xq, int qbase, int* s_qn, R* wqueue, int& wq_n,
                                       const PIn<R>& in) {
    constexpr int T = S + 4, T3 = T * T * T, TJ = S + 3;
    constexpr bool kMom = Tile<R, S>::kMoments;
    const GridDev& g = pp.g;
    int cp;
    if constexpr (Prefetch<R>::level >= 1) cp = in.cell;
    else cp = valid ? ps.cell[p] : INACTIVE;
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
        if constexpr (Prefetch<R>::level >= 1) {
            fx = in.off[0];
            fy = in.off[1];
            fz = in.off[2];
        } else {
            fx = ps.off[0][p];
            fy = ps.off[1][p];
            fz = ps.off[2][p];
        }
        if constexpr (Prefetch<R>::level >= 2) {
            ux = in.u[0];
            uy = in.u[1];
            uz = in.u[2];
            w = in.w;
        } else {
            ux = ps.u[0][p];
            uy = ps.u[1][p];
            uz = ps.u[2][p];
            w = ps.w[p];
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
    const R h = prm<R>(pp.qdt2m, pp.qdt2m_f);
    const R umx = fma(h, Ex, ux), umy = fma(h, Ey, uy), umz = fma(h, Ez, uz);
    const R hg = h * rsqrt(fma(umx, umx, fma(umy, umy, fma(umz, umz, R(1)))));
    const R tbx = hg * Bx, tby = hg * By, tbz = hg * Bz;
    const R sf = R(2) / fma(tbx, tbx, fma(tby, tby, fma(tbz, tbz, R(1))));
    const R sbx = sf * tbx, sby = sf * tby, sbz = sf * tbz;
    const R upx = fma(umy, tbz, fma(-umz, tby, umx));
    const R upy = fma(umz, tbx, fma(-umx, tbz, umy));
    const R upz = fma(umx, tby, fma(-umy, tbx, umz));
    ux = fma(h, Ex, fma(upy, sbz, fma(-upz, sby, umx)));
    uy = fma(h, Ey, fma(upz, sbx, fma(-upx, sbz, umy)));
    uz = fma(h, Ez, fma(upx, sby, fma(-upy, sbx, umz)));

    // ---- move: displacement in cells, x^{n+1} = x^n + dt u / gamma
    const R u2p1 = fma(ux, ux, fma(uy, uy, fma(uz, uz, R(1))));
    const R gi = rsqrt(u2p1);
    R dx, dy, dz;
    if constexpr (CU) {
        const R gd = gi * prm<R>(pp.dtd[0], pp.dtd_f[0]);
        dx = ux * gd, dy = uy * gd, dz = uz * gd;
    } else {
        dx = ux * (gi * prm<R>(pp.dtd[0], pp.dtd_f[0])), dy = uy * (gi * prm<R>(pp.dtd[1], pp.dtd_f[1])),
        dz = uz * (gi * prm<R>(pp.dtd[2], pp.dtd_f[2]));
    }
    const R bx = fx + dx, by = fy + dy, bz = fz + dz;  // end point in the start cell's frame
    const int sx = cell_shift(bx), sy = cell_shift(by), sz = cell_shift(bz);
    if (act && ((unsigned)(lx + sx + 1) > (unsigned)(S + 1) || (unsigned)(ly + sy + 1) > (unsigned)(S + 1) ||
                (unsigned)(lz + sz + 1) > (unsigned)(S + 1))) {
        // cannot happen while K * max(dt/d) < 1; record it, drop the particle, touch no tile
        atomicOr(err, ERRBIT_DRIFT);
        ps.cell[p] = INACTIVE | cp;
        act = false;
    }

    // ---- Villasenor-Buneman deposit into the shared J tile (tile origin = cell c0-1)
    const bool dep = act && w != R(0);
    const R wq = dep ? w : R(0);
    const R Qx = prm<R>(pp.cq[0], pp.cq_f[0]) * wq;
    const R Qy = CU ? Qx : prm<R>(pp.cq[1], pp.cq_f[1]) * wq, Qz = CU ? Qx : prm<R>(pp.cq[2], pp.cq_f[2]) * wq;
    const int key0 = ((lz + 1) * TJ + (ly + 1)) * TJ + (lx + 1);
    if constexpr (sizeof(R) == 8 || PICGB_F32_GQ) {
        // FP64: a crossing lane would make its whole warp execute the split on the
        // FP64 pipe, so crossing moves are queued and split after the chunk by full
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
            if (cross && slot < CHUNK) {
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
    } else if constexpr (WarpQueue<R, S, NT>::kOn) {
        const bool cross = dep && (sx | sy | sz) != 0;
        deposit_segment<R, TJ, kMom>(Jt, dep && !cross ? key0 : -1, fx, fy, fz, dx, dy, dz, Qx, Qy, Qz);
        const unsigned cm = __ballot_sync(FULL, cross);
        if (cm) {
            const int cnt = __popc(cm), lane = threadIdx.x & 31;
            if (cnt >= 16) {
                if (cross) split_direct<R, TJ, false>(Jt, key0, fx, fy, fz, dx, dy, dz, Qx, Qy, Qz);
            } else {
                if (wq_n + cnt > WQ) {
                    warp_queue_flush<R, TJ>(Jt, wqueue, wq_n, pp);
                    wq_n = 0;
                }
                if (cross) {
                    const int q = wq_n + __popc(cm & ((1u << lane) - 1u));
                    wqueue[q] = __int_as_float(key0);
                    wqueue[WQ + q] = fx;
                    wqueue[2 * WQ + q] = fy;
                    wqueue[3 * WQ + q] = fz;
                    wqueue[4 * WQ + q] = dx;
                    wqueue[5 * WQ + q] = dy;
                    wqueue[6 * WQ + q] = dz;
                    wqueue[7 * WQ + q] = wq;
                }
                wq_n += cnt;
            }
        }
    } else {
        // FP32: the split runs in the warp (its arithmetic is cheap); each piece is
        // summed per cell run like a whole move
        const int nseg = 1 + (sx != 0) + (sy != 0) + (sz != 0);
        if (!__any_sync(FULL, dep && nseg > 1)) {
            deposit_segment<R, TJ, false>(Jt, dep ? key0 : -1, fx, fy, fz, dx, dy, dz, Qx, Qy, Qz);
        } else {
            R t1 = R(1), t2 = R(1), t3 = R(1);
            if (sx) t1 = cross_t(R(sx > 0 ? 1 : 0) - fx, dx);
            if (sy) t2 = cross_t(R(sy > 0 ? 1 : 0) - fy, dy);
            if (sz) t3 = cross_t(R(sz > 0 ? 1 : 0) - fz, dz);
            sort3(t1, t2, t3);
            // first piece [0, t1]: starts at the offset itself and stays in the start cell
            deposit_segment<R, TJ, false>(Jt, dep ? key0 : -1, fx, fy, fz, t1 * dx, t1 * dy, t1 * dz, Qx, Qy, Qz);
            const int jx = lx + 1, jy = ly + 1, jz = lz + 1;
#pragma unroll
            for (int s = 1; s < 4; ++s) {
                if (!__any_sync(FULL, dep && s < nseg)) break;
                const R ta = s == 1 ? t1 : (s == 2 ? t2 : t3);
                const R tb = s == 1 ? t2 : (s == 2 ? t3 : R(1));
                const bool on = dep && s < nseg && tb > ta;
                const R pax = fma(ta, dx, fx), pay = fma(ta, dy, fy), paz = fma(ta, dz, fz);
                const R dt = tb - ta;
                const R ddx = dt * dx, ddy = dt * dy, ddz = dt * dz;
                const int ox = cell_shift(fma(R(0.5), ddx, pax)), oy = cell_shift(fma(R(0.5), ddy, pay)),
                          oz = cell_shift(fma(R(0.5), ddz, paz));
                deposit_segment<R, TJ, false>(Jt, on ? ((jz + oz) * TJ + (jy + oy)) * TJ + (jx + ox) : -1, pax - R(ox),
                                       pay - R(oy), paz - R(oz), ddx, ddy, ddz, Qx, Qy, Qz);
            }
        }
    }
    if (!act) return R(0);

    // ---- new cell and offset
    R nfx = bx, nfy = by, nfz = bz;
    if constexpr (sizeof(R) == 8) {
        // FP64: the shifted offsets lie in [0, 1] (non-negative, so their bit
        // patterns order like integers) and are clamped below 1 on the integer
        // ALU; a warp with no crossing lane skips the block (FP64-pipe issue is
        // what bounds this kernel)
        if (__any_sync(__activemask(), (sx | sy | sz) != 0)) {
            if (sx) nfx = below_one_of(bx - R(sx));
            if (sy) nfy = below_one_of(by - R(sy));
            if (sz) nfz = below_one_of(bz - R(sz));
        }
    } else {
        nfx = sx ? fmin(bx - R(sx), below_one<R>()) : bx;
        nfy = sy ? fmin(by - R(sy), below_one<R>()) : by;
        nfz = sz ? fmin(bz - R(sz), below_one<R>()) : bz;
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

// Resident CTAs per SM the register budget is cut for (FP32: 4 CTAs of 256
// threads at 64 registers; the FP64 kernel needs ~100 registers, i.e. 2).
#ifndef PICGB_PUSH_MINB_F32
#define PICGB_PUSH_MINB_F32 4
#endif
template <class R>
constexpr int push_min_blocks() {
    return sizeof(R) == 4 ? PICGB_PUSH_MINB_F32 : 2;
}

template <class R, int S, int NT, bool CU>
__global__ void __launch_bounds__(NT, push_min_blocks<R>()) k_push(const __grid_constant__ CUtensorMap tmEB, PushParams pp, PStore<R> ps,
                                            XQueue<R> xq, const Chunk* __restrict__ chunks, const int* __restrict__ nchunks,
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
    R* wqueue = F + WarpQueue<R, S, NT>::OFF + warp * 8 * WQ;  // used only where WarpQueue<..>::kOn
    int wq_n = 0;
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
        constexpr int PF = Prefetch<R>::level;
        PIn<R> nx;  // the warp's first batch: loaded while the field tile is fetched and built
        if constexpr (PF >= 1) {
            load_head(nx, ps, ch.start + warp * 32 + lane, ch.start + warp * 32 + lane < end);
            if constexpr (PF >= 2) load_tail(nx, ps, ch.start + warp * 32 + lane, ch.start + warp * 32 + lane < end);
        }
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
            PIn<R> in;
            if constexpr (PF >= 1) {
                in = nx;
                const int pn = p + NT;
                load_head(nx, ps, pn, pn < end);
                if constexpr (PF >= 2) load_tail(nx, ps, pn, pn < end);
            }
            ek_chunk += push_lane<R, S, NT, CU>(Fuse, Jt, ps, p, p < end, pp, c0x, c0y, c0z, err, xq, qbase, &s_qn,
                                            wqueue, wq_n, in);
        }
        if constexpr (WarpQueue<R, S, NT>::kOn) {
            if (wq_n > 0) warp_queue_flush<R, TJ>(Jt, wqueue, wq_n, pp);
            wq_n = 0;
        }
        ek += (double)ek_chunk;
        __syncthreads();
        // the deferred crossing moves (FP64), split by every thread of the CTA
        const int nq = (sizeof(R) == 8 || PICGB_F32_GQ) ? min(s_qn, CHUNK) : 0;
        for (int i = threadIdx.x; i < nq; i += NT) {
            const int q = qbase + i;
            const R w = xq.w[q];
            split_direct<R, TJ, kMom>(Jt, xq.key[q], xq.a[0][q], xq.a[1][q], xq.a[2][q], xq.d[0][q], xq.d[1][q], xq.d[2][q],
                                prm<R>(pp.cq[0], pp.cq_f[0]) * w, prm<R>(pp.cq[1], pp.cq_f[1]) * w,
                                prm<R>(pp.cq[2], pp.cq_f[2]) * w);
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
                atomicAdd(&J[o], (double)v);
            }
        }
        __syncthreads();
    }
    const double s = block_sum<NT>(ek, red);
    if (threadIdx.x == 0) ek_part[blockIdx.x] = s * pp.mass;
}

// ------------------------------------------------------------------ FP32, four particles per thread
// The mixed-precision kernel is bound by instruction issue and latency, not by
// memory (its store traffic is 60 B per particle-step).  Particles are sorted
// by cell (about 30 per cell), so this kernel gives each thread G = 4
// consecutive particles, read and written with 16-byte vector accesses:
//   * the thread sums its particles' 12 edge currents in registers while
//     they share a cell, adding the sum to the shared tile when the cell
//     changes;
//   * after its four particles, one segmented scan over the warp's 32 lanes
//     (runs of about 8 lanes: 3 rounds) combines the lanes that hold the same
//     cell, and the last lane of each run adds the run's 12 totals;
//   * moves that leave their start cell are queued per CTA (global memory,
//     one slot per particle of the chunk) and split into Villasenor-Buneman
//     pieces by all threads after the chunk.
// A chunk may start at any particle: the groups overlapping its ends mask the
// particles outside it and store element by element.
#ifndef PICGB_F32_GROUP
#define PICGB_F32_GROUP 1  // 0: the one-particle-per-lane FP32 kernel
#endif
#ifndef PICGB_PUSHG_MINB
#define PICGB_PUSHG_MINB 4
#endif
#ifndef PICGB_PG
#define PICGB_PG 2
#endif
constexpr int PG = PICGB_PG;  // particles per thread: 2 (8-byte accesses) or 4 (16-byte accesses)
template <int G>
struct GVec;
template <>
struct GVec<4> {
    using F = float4;
    using I = int4;
};
template <>
struct GVec<2> {
    using F = float2;
    using I = int2;
};
using VecF = GVec<PG>::F;
using VecI = GVec<PG>::I;

__device__ __forceinline__ float& el(float4& v, int j) { return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w)); }
__device__ __forceinline__ int& el(int4& v, int j) { return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w)); }
__device__ __forceinline__ float& el(float2& v, int j) { return j == 0 ? v.x : v.y; }
__device__ __forceinline__ int& el(int2& v, int j) { return j == 0 ? v.x : v.y; }

// The 12 edge currents of a straight move inside one cell (Villasenor-Buneman),
// two at a time with packed two-wide FP32 instructions; order as edge_offset.
__device__ __forceinline__ void vb_edges32(float (&v)[12], float ax, float ay, float az, float dx, float dy, float dz,
                                           float Qx, float Qy, float Qz) {
    const float mx = fmaf(0.5f, dx, ax), my = fmaf(0.5f, dy, ay), mz = fmaf(0.5f, dz, az);
    const float vol = dx * dy * (dz * (1.0f / 12.0f));
    const float ox = 1.0f - mx, oy = 1.0f - my, oz = 1.0f - mz;
    const auto edges = [](float* out, float q, float qc, float o1, float m1, float o2, float m2) {
        const float2 a = __fmul2_rn(make_float2(q, q), make_float2(o1, m1));
        const float2 lo = __ffma2_rn(a, make_float2(o2, o2), make_float2(qc, -qc));
        const float2 hi = __ffma2_rn(a, make_float2(m2, m2), make_float2(-qc, qc));
        out[0] = lo.x, out[1] = lo.y, out[2] = hi.x, out[3] = hi.y;
    };
    edges(v + 0, Qx * dx, Qx * vol, oy, my, oz, mz);
    edges(v + 4, Qy * dy, Qy * vol, ox, mx, oz, mz);
    edges(v + 8, Qz * dz, Qz * vol, ox, mx, oy, my);
}

template <int TJ>
__device__ __forceinline__ void add12(float* Jt, int key, const float (&a)[12]) {
#pragma unroll
    for (int i = 0; i < 12; ++i) atomicAdd(Jt + key + edge_offset<TJ>(i), a[i]);
}

// Lanes holding the same cell key (consecutive lanes; key -1 holds nothing)
// are summed by a segmented scan; the last lane of each run adds the totals.
template <int TJ>
__device__ __forceinline__ void warp_runs_add(float* Jt, int key, float (&v)[12]) {
    const int lane = threadIdx.x & 31;
    const int kprev = __shfl_up_sync(FULL, key, 1);
    const int knext = __shfl_down_sync(FULL, key, 1);
    const bool head = lane == 0 || kprev != key;
    const bool tail = lane == 31 || knext != key;
    const unsigned heads = __ballot_sync(FULL, head);
    const int start = 31 - __clz(heads & (FULL >> (31 - lane)));
    const int longest = __reduce_max_sync(FULL, key >= 0 ? (unsigned)(lane - start + 1) : 0u);
    for (int dd = 1; dd < longest; dd <<= 1) {
        const bool add = lane - dd >= start;
#pragma unroll
        for (int i = 0; i < 12; i += 2) {
            const float2 t = make_float2(__shfl_up_sync(FULL, v[i], dd), __shfl_up_sync(FULL, v[i + 1], dd));
            if (add) {
                const float2 s2 = __fadd2_rn(make_float2(v[i], v[i + 1]), t);
                v[i] = s2.x;
                v[i + 1] = s2.y;
            }
        }
    }
    if (tail && key >= 0) add12<TJ>(Jt, key, v);
}

template <int S, int NT, bool CU>
__global__ void __launch_bounds__(NT, PICGB_PUSHG_MINB)
    k_push_g(const __grid_constant__ CUtensorMap tmEB, PushParams pp, PStore<float> ps, XQueue<float> xq,
             const Chunk* __restrict__ chunks, const int* __restrict__ nchunks, double* __restrict__ J,
             double* __restrict__ ek_part, int* __restrict__ err) {
    constexpr int T = S + 4, T3 = T * T * T, TJ = S + 3, TJ3 = TJ * TJ * TJ;
    constexpr bool kCoef = Tile<float, S>::kCoef;
    constexpr int RAW = Tile<float, S>::RAW;
    extern __shared__ unsigned char smem_raw[];
    float* F = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float* Jt = kCoef ? F : F + 6 * T3;
    Coef<float>* X = reinterpret_cast<Coef<float>*>(F + RAW);
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
    const float h = pp.qdt2m_f;
    const float dtdx = pp.dtd_f[0], dtdy = CU ? dtdx : pp.dtd_f[1], dtdz = CU ? dtdx : pp.dtd_f[2];
    const float cqx = pp.cq_f[0], cqy = CU ? cqx : pp.cq_f[1], cqz = CU ? cqx : pp.cq_f[2];
    uint32_t phase = 0;
    double ek = 0.0;
    const int nch = *nchunks;
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const Chunk ch = chunks[c];
        const int scx = ch.sc % g.nsc[0], scy = (ch.sc / g.nsc[0]) % g.nsc[1], scz = ch.sc / (g.nsc[0] * g.nsc[1]);
        const int c0x = scx * S, c0y = scy * S, c0z = scz * S;
        if (threadIdx.x == 0) {
            fence_proxy_async();
            mbar_expect_tx(&bar, 6u * T3 * (uint32_t)sizeof(float));
            tma_load_4d(F, &tmEB, c0x, c0y, c0z, 0, &bar);
        }
        if (!kCoef)
            for (int i = threadIdx.x; i < 3 * TJ3; i += NT) Jt[i] = 0.0f;
        const bool ok = mbar_wait_bounded(&bar, phase, WAIT_LIMIT, WAIT_LIMIT_NS);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(err, ERRBIT_TIMEOUT);
                ek_part[blockIdx.x] = 0.0;
            }
            return;
        }
        phase ^= 1u;
        if (kCoef) {
            build_coef<float, T, NT>(F, X);
            __syncthreads();
            for (int i = threadIdx.x; i < 3 * TJ3; i += NT) Jt[i] = 0.0f;
            __syncthreads();
        }
        const int start = ch.start, end = ch.start + ch.count;
        const int ga = start / PG, gb = (end + PG - 1) / PG;
        float ek_chunk = 0.0f;
        for (int gw = ga + warp * 32; gw < gb; gw += NT) {
            const int gq = gw + lane, p0 = gq * PG;
            const bool gv = gq < gb;
            VecI c4;
#pragma unroll
            for (int j = 0; j < PG; ++j) el(c4, j) = INACTIVE;
            VecF fx4{}, fy4{}, fz4{}, ux4{}, uy4{}, uz4{}, w4{};
            if (gv) {
                c4 = *reinterpret_cast<const VecI*>(ps.cell + p0);
                fx4 = *reinterpret_cast<const VecF*>(ps.off[0] + p0);
                fy4 = *reinterpret_cast<const VecF*>(ps.off[1] + p0);
                fz4 = *reinterpret_cast<const VecF*>(ps.off[2] + p0);
                ux4 = *reinterpret_cast<const VecF*>(ps.u[0] + p0);
                uy4 = *reinterpret_cast<const VecF*>(ps.u[1] + p0);
                uz4 = *reinterpret_cast<const VecF*>(ps.u[2] + p0);
                w4 = *reinterpret_cast<const VecF*>(ps.w + p0);
            }
            // Phase A, free of side effects so that the four particles' chains can
            // interleave: the start cell inside the tile, the gather and the Boris
            // push (u^{n+1/2} replaces u in place).  kinfo: the J-tile key of the
            // start cell, and bits for a start cell on the tile's slack layer (a
            // move further out would leave the tile); -1 for no particle.
            int kinfo[PG];
            bool bad = false;
#pragma unroll
            for (int j = 0; j < PG; ++j) {
                const int p = p0 + j;
                const bool valid = gv && p >= start && p < end;
                const int cp = valid ? el(c4, j) : INACTIVE;
                bool act = cp >= 0;
                int lx = cell_x(cp) - c0x, ly = cell_y(cp) - c0y, lz = cell_z(cp) - c0z;
                if (lx < -1) lx += g.n[0]; else if (lx > S) lx -= g.n[0];
                if (ly < -1) ly += g.n[1]; else if (ly > S) ly -= g.n[1];
                if (lz < -1) lz += g.n[2]; else if (lz > S) lz -= g.n[2];
                if (act && ((unsigned)(lx + 1) > (unsigned)(S + 1) || (unsigned)(ly + 1) > (unsigned)(S + 1) ||
                            (unsigned)(lz + 1) > (unsigned)(S + 1))) {
                    bad = true;
                    act = false;
                }
                if (!act) lx = ly = lz = 0;
                const float fx = act ? el(fx4, j) : 0.25f, fy = act ? el(fy4, j) : 0.25f,
                            fz = act ? el(fz4, j) : 0.25f;
                const float ux = act ? el(ux4, j) : 0.0f, uy = act ? el(uy4, j) : 0.0f, uz = act ? el(uz4, j) : 0.0f;
                // gather: each component from its own staggered lattice (tile origin = cell c0-2)
                const int tx = lx + 2, ty = ly + 2, tz = lz + 2;
                const bool sxb = lt_half(fx), syb = lt_half(fy), szb = lt_half(fz);
                const int hx = sxb ? tx - 1 : tx, hy = syb ? ty - 1 : ty, hz = szb ? tz - 1 : tz;
                const float gxf = fx + (sxb ? 0.5f : -0.5f), gyf = fy + (syb ? 0.5f : -0.5f),
                            gzf = fz + (szb ? 0.5f : -0.5f);
                float Ex, Ey, Ez, Bx, By, Bz;
                if constexpr (kCoef) {
                    constexpr int NE = Tile<float, S>::NE;
                    const Coef<float>* Xc = static_cast<const Coef<float>*>(Fuse);
                    Ex = tri_coef<float, T>(Xc + 0 * NE, hx, ty, tz, gxf, fy, fz);
                    Ey = tri_coef<float, T>(Xc + 1 * NE, tx, hy, tz, fx, gyf, fz);
                    Ez = tri_coef<float, T>(Xc + 2 * NE, tx, ty, hz, fx, fy, gzf);
                    Bx = tri_coef<float, T>(Xc + 3 * NE, tx, hy, hz, fx, gyf, gzf);
                    By = tri_coef<float, T>(Xc + 4 * NE, hx, ty, hz, gxf, fy, gzf);
                    Bz = tri_coef<float, T>(Xc + 5 * NE, hx, hy, tz, gxf, gyf, fz);
                } else {
                    const float* Fr = static_cast<const float*>(Fuse);
                    Ex = tri_raw<float, T>(Fr + 0 * T3, hx, ty, tz, gxf, fy, fz);
                    Ey = tri_raw<float, T>(Fr + 1 * T3, tx, hy, tz, fx, gyf, fz);
                    Ez = tri_raw<float, T>(Fr + 2 * T3, tx, ty, hz, fx, fy, gzf);
                    Bx = tri_raw<float, T>(Fr + 3 * T3, tx, hy, hz, fx, gyf, gzf);
                    By = tri_raw<float, T>(Fr + 4 * T3, hx, ty, hz, gxf, fy, gzf);
                    Bz = tri_raw<float, T>(Fr + 5 * T3, hx, hy, tz, gxf, gyf, fz);
                }
                // Boris: half electric kick, rotation, half electric kick
                const float umx = fmaf(h, Ex, ux), umy = fmaf(h, Ey, uy), umz = fmaf(h, Ez, uz);
                const float hg = h * rsqrtf(fmaf(umx, umx, fmaf(umy, umy, fmaf(umz, umz, 1.0f))));
                const float tbx = hg * Bx, tby = hg * By, tbz = hg * Bz;
                const float sf = __fdividef(2.0f, fmaf(tbx, tbx, fmaf(tby, tby, fmaf(tbz, tbz, 1.0f))));
                const float sbx = sf * tbx, sby = sf * tby, sbz = sf * tbz;
                const float upx = fmaf(umy, tbz, fmaf(-umz, tby, umx));
                const float upy = fmaf(umz, tbx, fmaf(-umx, tbz, umy));
                const float upz = fmaf(umx, tby, fmaf(-umy, tbx, umz));
                if (act) {
                    el(ux4, j) = fmaf(h, Ex, fmaf(upy, sbz, fmaf(-upz, sby, umx)));
                    el(uy4, j) = fmaf(h, Ey, fmaf(upz, sbx, fmaf(-upx, sbz, umy)));
                    el(uz4, j) = fmaf(h, Ez, fmaf(upx, sby, fmaf(-upy, sbx, umz)));
                }
                const int edge = (lx == -1 ? 1 : 0) | (lx == S ? 2 : 0) | (ly == -1 ? 4 : 0) | (ly == S ? 8 : 0) |
                                 (lz == -1 ? 16 : 0) | (lz == S ? 32 : 0);
                kinfo[j] = act ? (((lz + 1) * TJ + (ly + 1)) * TJ + (lx + 1)) | (edge << 16) : -1;
            }
            // Phase B: move, Villasenor-Buneman deposit (a move inside its start
            // cell joins the thread's running sum; a move that leaves it is
            // queued), new cell and offset, kinetic energy
            float acc[12];
#pragma unroll
            for (int i = 0; i < 12; ++i) acc[i] = 0.0f;
            int kacc = -1;
#pragma unroll
            for (int j = 0; j < PG; ++j) {
                const int ki = kinfo[j];
                bool act = ki >= 0;
                const int key0 = ki & 0xFFFF, edge = ki >> 16;
                const float fx = el(fx4, j), fy = el(fy4, j), fz = el(fz4, j);
                const float ux = el(ux4, j), uy = el(uy4, j), uz = el(uz4, j);
                const float w = act ? el(w4, j) : 0.0f;
                const float u2p1 = fmaf(ux, ux, fmaf(uy, uy, fmaf(uz, uz, 1.0f)));
                const float gi = rsqrtf(u2p1);
                const float dx = ux * (gi * dtdx), dy = uy * (gi * dtdy), dz = uz * (gi * dtdz);
                const float bx = fx + dx, by = fy + dy, bz = fz + dz;
                const int sx = cell_shift(bx), sy = cell_shift(by), sz = cell_shift(bz);
                if (act && ((sx < 0 && (edge & 1)) || (sx > 0 && (edge & 2)) || (sy < 0 && (edge & 4)) ||
                            (sy > 0 && (edge & 8)) || (sz < 0 && (edge & 16)) || (sz > 0 && (edge & 32)))) {
                    // cannot happen while K * max(dt/d) < 1; record it, drop the particle, touch no tile
                    bad = true;
                    el(c4, j) = INACTIVE | el(c4, j);
                    act = false;
                }
                const bool dep = act && w != 0.0f;
                const bool cross = dep && (sx | sy | sz) != 0;
                const int kdep = dep && !cross ? key0 : -1;
                const float Qx = cqx * w, Qy = cqy * w, Qz = cqz * w;
                if (kdep >= 0 && kdep != kacc) {
                    if (kacc >= 0) add12<TJ>(Jt, kacc, acc);
#pragma unroll
                    for (int i = 0; i < 12; ++i) acc[i] = 0.0f;
                    kacc = kdep;
                }
                if (kdep >= 0) {
                    float v[12];
                    vb_edges32(v, fx, fy, fz, dx, dy, dz, Qx, Qy, Qz);
#pragma unroll
                    for (int i = 0; i < 12; i += 2) {
                        const float2 s2 = __fadd2_rn(make_float2(acc[i], acc[i + 1]), make_float2(v[i], v[i + 1]));
                        acc[i] = s2.x;
                        acc[i + 1] = s2.y;
                    }
                }
                const unsigned cm = __ballot_sync(FULL, cross);
                if (cm) {
                    const int first = __ffs(cm) - 1;
                    int base = 0;
                    if (lane == first) base = atomicAdd(&s_qn, __popc(cm));
                    base = __shfl_sync(FULL, base, first);
                    const int slot = base + __popc(cm & ((1u << lane) - 1u));
                    if (cross && slot >= CHUNK) bad = true;
                    if (cross && slot < CHUNK) {
                        const int q = qbase + slot;
                        xq.key[q] = key0;
                        xq.a[0][q] = fx;
                        xq.a[1][q] = fy;
                        xq.a[2][q] = fz;
                        xq.d[0][q] = dx;
                        xq.d[1][q] = dy;
                        xq.d[2][q] = dz;
                        xq.w[q] = w;
                    }
                }
                if (act) {
                    // new cell and offset
                    const int cp = el(c4, j);
                    int ng[3] = {cell_x(cp) + sx, cell_y(cp) + sy, cell_z(cp) + sz};
                    bool gone = false;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        if (ng[a] < 0 || ng[a] >= g.n[a]) {
                            if (g.bc[a] == 0) ng[a] += ng[a] < 0 ? g.n[a] : -g.n[a];
                            else gone = true;
                        }
                    }
                    el(c4, j) = gone ? (INACTIVE | cp) : pack_cell(ng[0], ng[1], ng[2]);
                    el(fx4, j) = sx ? fminf(bx - (float)sx, below_one<float>()) : bx;
                    el(fy4, j) = sy ? fminf(by - (float)sy, below_one<float>()) : by;
                    el(fz4, j) = sz ? fminf(bz - (float)sz, below_one<float>()) : bz;
                    // kinetic energy of the new state: w (gamma - 1)
                    if (!gone) ek_chunk += w * fmaf(u2p1, gi, -1.0f);
                }
            }
            if (bad) atomicOr(err, ERRBIT_DRIFT);
            warp_runs_add<TJ>(Jt, kacc, acc);
            if (gv) {
                if (p0 >= start && p0 + PG <= end) {
                    *reinterpret_cast<VecI*>(ps.cell + p0) = c4;
                    *reinterpret_cast<VecF*>(ps.off[0] + p0) = fx4;
                    *reinterpret_cast<VecF*>(ps.off[1] + p0) = fy4;
                    *reinterpret_cast<VecF*>(ps.off[2] + p0) = fz4;
                    *reinterpret_cast<VecF*>(ps.u[0] + p0) = ux4;
                    *reinterpret_cast<VecF*>(ps.u[1] + p0) = uy4;
                    *reinterpret_cast<VecF*>(ps.u[2] + p0) = uz4;
                } else {
#pragma unroll
                    for (int j = 0; j < PG; ++j) {
                        const int p = p0 + j;
                        if (p >= start && p < end) {
                            ps.cell[p] = el(c4, j);
                            ps.off[0][p] = el(fx4, j);
                            ps.off[1][p] = el(fy4, j);
                            ps.off[2][p] = el(fz4, j);
                            ps.u[0][p] = el(ux4, j);
                            ps.u[1][p] = el(uy4, j);
                            ps.u[2][p] = el(uz4, j);
                        }
                    }
                }
            }
        }
        ek += (double)ek_chunk;
        __syncthreads();
        // the queued moves that leave their start cell, split by every thread
        const int nq = min(s_qn, CHUNK);
        for (int i = threadIdx.x; i < nq; i += NT) {
            const int q = qbase + i;
            const float w = xq.w[q];
            split_direct<float, TJ, false>(Jt, xq.key[q], xq.a[0][q], xq.a[1][q], xq.a[2][q], xq.d[0][q], xq.d[1][q],
                                           xq.d[2][q], cqx * w, cqy * w, cqz * w);
        }
        __syncthreads();
        if (threadIdx.x == 0) s_qn = 0;
        // merge: J tile cell t is domain cell c0 - 1 + t, padded index c0 + 1 + t
        for (int i = threadIdx.x; i < 3 * TJ3; i += NT) {
            const float v = Jt[i];
            if (v != 0.0f) {
                const int comp = i / TJ3, r = i - comp * TJ3;
                const int tz = r / (TJ * TJ), ty = (r / TJ) % TJ, tx = r % TJ;
                const long long o = (long long)comp * g.P + (c0x + 1 + tx) +
                                    (long long)g.np[0] * ((c0y + 1 + ty) + (long long)g.np[1] * (c0z + 1 + tz));
                atomicAdd(&J[o], (double)v);
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
    constexpr int T = S + 4, TJ = S + 3;
    if (Tile<R, S>::kCoef) return 128 + sizeof(R) * Tile<R, S>::RAW + sizeof(Coef<R>) * 6 * Tile<R, S>::NE;
    return 128 + sizeof(R) * (6 * T * T * T + 3 * TJ * TJ * TJ);
}

template <class R, int S>
cudaError_t push_setup(int* blocks_per_sm) {
    const int sm = (int)push_smem_bytes<R, S>();
    if constexpr (sizeof(R) == 4 && PICGB_F32_GROUP) {
        cudaError_t e = cudaFuncSetAttribute(k_push_g<S, PUSH_NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_push_g<S, PUSH_NT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_push_g<S, PUSH_NT, false>, PUSH_NT, sm);
    }
    cudaError_t e = cudaFuncSetAttribute(k_push<R, S, PUSH_NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_push<R, S, PUSH_NT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_push<R, S, PUSH_NT, false>, PUSH_NT, sm);
}

template <class R, int S>
cudaError_t push_launch(int grid, cudaStream_t st, const CUtensorMap& tm, const PushParams& pp, const PStore<R>& ps,
                        const XQueue<R>& xq, const Chunk* chunks, const int* nchunks, double* J, double* ek_part,
                        int* err) {
    const bool cubic = pp.g.d[0] == pp.g.d[1] && pp.g.d[1] == pp.g.d[2];
    if constexpr (sizeof(R) == 4 && PICGB_F32_GROUP) {
        if (cubic)
            k_push_g<S, PUSH_NT, true><<<grid, PUSH_NT, push_smem_bytes<R, S>(), st>>>(tm, pp, ps, xq, chunks, nchunks,
                                                                                    J, ek_part, err);
        else
            k_push_g<S, PUSH_NT, false><<<grid, PUSH_NT, push_smem_bytes<R, S>(), st>>>(tm, pp, ps, xq, chunks,
                                                                                     nchunks, J, ek_part, err);
        return cudaGetLastError();
    }
    if (cubic)
        k_push<R, S, PUSH_NT, true><<<grid, PUSH_NT, push_smem_bytes<R, S>(), st>>>(tm, pp, ps, xq, chunks, nchunks, J,
                                                                               ek_part, err);
    else
        k_push<R, S, PUSH_NT, false><<<grid, PUSH_NT, push_smem_bytes<R, S>(), st>>>(tm, pp, ps, xq, chunks, nchunks,
                                                                                J, ek_part, err);
    return cudaGetLastError();
}

#define PICGB_PUSH_INST(R, S)                                                                                   \
    template cudaError_t push_setup<R, S>(int*);                                                                \
    template cudaError_t push_launch<R, S>(int, cudaStream_t, const CUtensorMap&, const PushParams&,            \
                                           const PStore<R>&, const XQueue<R>&, const Chunk*, const int*, double*, \
                                           double*, int*);                                                      \
    template size_t push_smem_bytes<R, S>();
PICGB_PUSH_INST(double, 2)
PICGB_PUSH_INST(double, 4)
PICGB_PUSH_INST(double, 8)
PICGB_PUSH_INST(float, 4)
PICGB_PUSH_INST(float, 8)

}  // namespace picgb
