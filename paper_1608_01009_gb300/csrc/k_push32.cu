// Fused mixed-precision particle kernel: field gather, Boris push, move and
// Villasenor-Buneman current deposition with cell-relative FP32 offsets, FP32
// momenta, FP32 interpolation from the FP32 field copy and FP32 current
// values, summed in a 32-bit fixed-point shared tile and merged into the
// global FP64 current (the FP64 kernel is k_push.cu).
//
// Method (arXiv:1608.01009): the stages of Sec. 2 with the schemes of Sec. 3,
// particles processed by supercells (Sec. 4.3); the precision split is this
// library's mixed mode.  The field tile, its TMA load and coefficient form,
// the chunk table and the crossing queue are those of the FP64 kernel.
#include "push_tile.cuh"

namespace picgb {

// The mixed-precision kernel is bound by instruction issue and latency, not by
// memory (its store traffic is 60 B per particle-step), and its deposit was
// most of its work (timing-only builds on the 128^3 x 32 workload: 2.1 of
// 3.4 ms, of which 0.9 ms in the warp reduction of the per-cell sums).  So:
//   * each thread takes G = 2 consecutive particles (cell-sorted, about 30 per
//     cell), read and written with 8-byte vector accesses; their gathers and
//     pushes form two independent chains (phase A, free of side effects);
//   * the thread sums its particles' 12 edge currents in registers while they
//     share a cell and adds the sum to the shared tile when the cell changes
//     and after its group (phase B);
//   * the shared tile is fixed point (see fx_split): 32-bit integer atomic adds
//     combine lanes that hit one address, so no warp reduction is needed;
//   * moves that leave their start cell are queued per CTA (global memory,
//     one slot per particle of the chunk) and split into Villasenor-Buneman
//     pieces by all threads after the chunk.
//   * 32-bit integer atomics to one address still serialise (about one cycle
//     per lane), so each thread sums two consecutive groups (4 particles)
//     before it adds: a cell's run covers half as many lanes and each lane
//     adds half as often.
// Measured on the 128^3 x 32 workload (67.1 M particles): 3.62 ms per launch
// with one particle per lane and a warp scan, 3.38 ms with two per thread,
// 2.82 ms with the fixed-point tile, 2.38 ms with two groups per thread
// between adds (one group: 2.78, four: 2.70, eight: 3.15 ms; 4 CTAs per SM at
// 64 registers: 3.10 ms; the lanes of a cell summed by the hardware integer
// reduction before one lane adds: 3.97 ms).  On the 134 M-particle laser
// ramp (64 per cell) after 450 steps: 7.16 ms with one group, 4.58 ms with two.
//   * lanes add to two copies of the tile (lane parity), which halves the lanes
//     of one cell that meet at one address: 2.36 -> 2.27 ms (four copies: 2.46
//     ms, the copies' zeroing and merge outweigh it); laser ramp 4.55 -> 4.04 ms.
// A chunk may start at any particle: the groups overlapping its ends mask the
// particles outside it and store element by element.
#ifndef PICGB_PUSHG_MINB
#define PICGB_PUSHG_MINB 3  // resident CTAs per SM the register budget is cut for (80 registers)
#endif
#ifndef PICGB_PG
#define PICGB_PG 2
#endif
#ifndef PICGB_GM
#define PICGB_GM 2  // consecutive groups per thread between flushes of its register sums
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

// Fixed-point current tile.  Shared-memory FP32 atomic adds serialise the
// lanes of a warp that hit one address (measured on this part: about 28
// cycles per warp instruction at 8 lanes per address and 110 at 32, against
// 6.5 without conflicts), while 32-bit integer atomic adds combine them (1 to
// 2 cycles per warp instruction), so the tile sums integers and no warp
// reduction is needed.  A value v enters as two integers, hi = round(v s) and
// lo = round((v s - hi) 2^19), with s a power of two fixed per launch so that
// |v s| <= 2^18 for any move (|d| < dt/d cells and |w| <= the species' largest
// weight): the CHUNK = 4096 particles of a chunk cannot overflow either sum
// (|hi|, |lo| <= 2^18 per contribution), and hi 2^19 + lo resolves 2^-37 of
// the largest single contribution, so that even a current component many
// orders of magnitude below that bound keeps FP32-level relative accuracy.
constexpr float FX_MAGIC = 12582912.0f;  // 1.5 * 2^23: x + FX_MAGIC holds round(x) in its low bits (|x| < 2^22)
constexpr int FX_LO_BITS = 19;
constexpr int FX_RANGE_BITS = 18;

__device__ __forceinline__ void fx_split(float v, float s, int& hi, int& lo) {
    const float x = v * s;  // exact: s is a power of two
    const float t = x + FX_MAGIC;
    hi = __float_as_int(t) - __float_as_int(FX_MAGIC);
    const float r = x - (t - FX_MAGIC);  // exact, |r| <= 1/2
    lo = __float_as_int(fmaf(r, (float)(1 << FX_LO_BITS), FX_MAGIC)) - __float_as_int(FX_MAGIC);
}

// The same split for a pair of values with packed two-wide FP32 instructions.
__device__ __forceinline__ void fx_split2(float v0, float v1, float s, int (&hi)[2], int (&lo)[2]) {
    const float2 M = make_float2(FX_MAGIC, FX_MAGIC);
    const float2 x = __fmul2_rn(make_float2(v0, v1), make_float2(s, s));
    const float2 t = __fadd2_rn(x, M);
    const float2 d = __fadd2_rn(t, make_float2(-FX_MAGIC, -FX_MAGIC));  // round(x), exact
    const float2 r = __fadd2_rn(x, make_float2(-d.x, -d.y));
    const float2 t2 = __ffma2_rn(r, make_float2((float)(1 << FX_LO_BITS), (float)(1 << FX_LO_BITS)), M);
    const int m = __float_as_int(FX_MAGIC);
    hi[0] = __float_as_int(t.x) - m;
    hi[1] = __float_as_int(t.y) - m;
    lo[0] = __float_as_int(t2.x) - m;
    lo[1] = __float_as_int(t2.y) - m;
}

template <int TJ>
__device__ __forceinline__ void add12i(int* Ji, int key, const float (&a)[12], float s) {
    constexpr int LO = 3 * TJ * TJ * TJ;
#pragma unroll
    for (int i = 0; i < 12; i += 2) {
        int hi[2], lo[2];
        fx_split2(a[i], a[i + 1], s, hi, lo);
        const int o0 = key + edge_offset<TJ>(i), o1 = key + edge_offset<TJ>(i + 1);
        if (in_range(o0, LO)) {  // debug build only: the hi and lo halves of one tile copy
            atomicAdd(Ji + o0, hi[0]);
            atomicAdd(Ji + LO + o0, lo[0]);
        }
        if (in_range(o1, LO)) {
            atomicAdd(Ji + o1, hi[1]);
            atomicAdd(Ji + LO + o1, lo[1]);
        }
    }
}

// Villasenor-Buneman split of a move that leaves its start cell (corner key k0
// in the J tile), each piece added to the fixed-point tile: cut at every face
// crossed, pieces in order of the crossing parameter, each piece deposited in
// the cell that holds its midpoint.
template <int TJ>
__device__ void split_fx(int* Ji, int k0, float ax, float ay, float az, float dx, float dy, float dz, float Qx,
                         float Qy, float Qz, float s) {
    const float bx = ax + dx, by = ay + dy, bz = az + dz;
    const int sx = cell_shift(bx), sy = cell_shift(by), sz = cell_shift(bz);
    float t1 = sx ? cross_t((sx > 0 ? 1.0f : 0.0f) - ax, dx) : 1.0f;
    float t2 = sy ? cross_t((sy > 0 ? 1.0f : 0.0f) - ay, dy) : 1.0f;
    float t3 = sz ? cross_t((sz > 0 ? 1.0f : 0.0f) - az, dz) : 1.0f;
    sort3(t1, t2, t3);
    const float ts[5] = {0.0f, t1, t2, t3, 1.0f};
    const int jx = k0 % TJ, jy = (k0 / TJ) % TJ, jz = k0 / (TJ * TJ);
    for (int p = 0; p < 4; ++p) {
        const float ta = ts[p], tb = ts[p + 1];
        if (!(tb > ta)) continue;
        const float pax = fmaf(ta, dx, ax), pay = fmaf(ta, dy, ay), paz = fmaf(ta, dz, az);
        const float dt = tb - ta;
        const float ddx = dt * dx, ddy = dt * dy, ddz = dt * dz;
        const int ox = cell_shift(fmaf(0.5f, ddx, pax)), oy = cell_shift(fmaf(0.5f, ddy, pay)),
                  oz = cell_shift(fmaf(0.5f, ddz, paz));
        float v[12];
        vb_edges32(v, pax - (float)ox, pay - (float)oy, paz - (float)oz, ddx, ddy, ddz, Qx, Qy, Qz);
        add12i<TJ>(Ji, ((jz + oz) * TJ + (jy + oy)) * TJ + (jx + ox), v, s);
    }
}

// G: slot p of the sorted order holds particle perm[p] of `pin` (the sort
// computed ranks only); its updated record goes to slot p of `ps`, read with
// element loads.  Otherwise pin is ps and the groups are updated in place.
template <int S, int NT, bool CU, bool G>
__global__ void __launch_bounds__(NT, PICGB_PUSHG_MINB)
    k_push_g(const __grid_constant__ CUtensorMap tmEB, PushParams pp, PStore<float> ps, PStore<float> pin,
             const int* __restrict__ perm, XQueue<float> xq,
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
    const int nch = *nchunks;
    // the raw field tile of chunk cc (supercell origin), loaded by TMA; thread 0 only
    const auto issue = [&](int cc) {
        const int sc = chunks[cc].sc;
        fence_proxy_async();
        mbar_expect_tx(&bar, 6u * T3 * (uint32_t)sizeof(float));
        tma_load_4d(F, &tmEB, (sc % g.nsc[0]) * S, ((sc / g.nsc[0]) % g.nsc[1]) * S, (sc / (g.nsc[0] * g.nsc[1])) * S,
                    0, &bar);
    };
    __syncthreads();
    const float h = pp.qdt2m_f;
    const float dtdx = pp.dtd_f[0], dtdy = CU ? dtdx : pp.dtd_f[1], dtdz = CU ? dtdx : pp.dtd_f[2];
    const float cqx = pp.cq_f[0], cqy = CU ? cqx : pp.cq_f[1], cqz = CU ? cqx : pp.cq_f[2];
    // this lane's copy of the fixed-point tile: lanes next to each other (often of
    // one cell) add to different copies, so fewer of them hit one address
    constexpr int NCP = Tile<float, S>::FX_COPIES;
    int* const Jall = reinterpret_cast<int*>(Jt);
    int* const Ji = Jall + (lane % NCP) * 6 * TJ3;
    // scale of the fixed-point tile: the largest value a move can deposit is below
    // max|cq| w_max max(dt/d) (1 + max(dt/d)^2 / 12) < 1.25 max|cq| w_max max(dt/d)
    float fxs = 1.0f;
    double fxinv = 1.0 / (1 << FX_LO_BITS);
    {
        const float vmax = 1.25f * fmaxf(fabsf(cqx), fmaxf(fabsf(cqy), fabsf(cqz))) * fmaxf(dtdx, fmaxf(dtdy, dtdz)) *
                           *pp.wmax;
        if (vmax > 0.0f && vmax < 3.0e38f) {
            int ex;
            frexpf(vmax, &ex);  // vmax < 2^ex
            const int e = max(-120, min(120, FX_RANGE_BITS - ex));
            fxs = ldexpf(1.0f, e);
            fxinv = ldexp(1.0, -e - FX_LO_BITS);
        }
    }
    uint32_t phase = 0;
    double ek = 0.0;
    float g2max = 0.0f;  // largest gamma^2 = 1 + u^2 of the pushed particles (their speed bound)
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const Chunk ch = chunks[c];
        const int scx = ch.sc % g.nsc[0], scy = (ch.sc / g.nsc[0]) % g.nsc[1], scz = ch.sc / (g.nsc[0] * g.nsc[1]);
        const int c0x = scx * S, c0y = scy * S, c0z = scz * S;
        if (threadIdx.x == 0) issue(c);
        if (!kCoef)
            for (int i = threadIdx.x; i < NCP * 6 * TJ3; i += NT) Jall[i] = 0;
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
            for (int i = threadIdx.x; i < NCP * 6 * TJ3; i += NT) Jall[i] = 0;  // the tile over the raw tile
            __syncthreads();
        }
        const int start = ch.start, end = ch.start + ch.count;
        const int ga = start / PG, gb = (end + PG - 1) / PG;
        float ek_chunk = 0.0f;
        for (int gw = ga + warp * 32 * PICGB_GM; gw < gb; gw += NT * PICGB_GM) {
          float acc[12];
#pragma unroll
          for (int i = 0; i < 12; ++i) acc[i] = 0.0f;
          int kacc = -1;
#pragma unroll 1
          for (int gm = 0; gm < PICGB_GM; ++gm) {
            const int gq = gw + lane * PICGB_GM + gm, p0 = gq * PG;
            const bool gv = gq < gb;
            VecI c4;
#pragma unroll
            for (int j = 0; j < PG; ++j) el(c4, j) = INACTIVE;
            VecF fx4{}, fy4{}, fz4{}, ux4{}, uy4{}, uz4{}, w4{};
            VecI id4{};
            if (G && gv) {
#pragma unroll
                for (int j = 0; j < PG; ++j) {
                    const int p = p0 + j;
                    if (p >= start && p < end) {
                        const int q = perm[p];
                        el(c4, j) = pin.cell[q];
                        el(fx4, j) = pin.off[0][q];
                        el(fy4, j) = pin.off[1][q];
                        el(fz4, j) = pin.off[2][q];
                        el(ux4, j) = pin.u[0][q];
                        el(uy4, j) = pin.u[1][q];
                        el(uz4, j) = pin.u[2][q];
                        el(w4, j) = pin.w[q];
                        el(id4, j) = pin.id[q];
                    }
                }
            } else if (gv) {
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
                    if (kacc >= 0) add12i<TJ>(Ji, kacc, acc, fxs);
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
                    if (cross && slot < CHUNK && in_range(qbase + slot, (long long)gridDim.x * CHUNK)) {
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
                    g2max = fmaxf(g2max, u2p1);
                }
            }
            if (bad) atomicOr(err, ERRBIT_DRIFT);
            if (gv) {
                if (p0 >= start && p0 + PG <= end) {
                    *reinterpret_cast<VecI*>(ps.cell + p0) = c4;
                    *reinterpret_cast<VecF*>(ps.off[0] + p0) = fx4;
                    *reinterpret_cast<VecF*>(ps.off[1] + p0) = fy4;
                    *reinterpret_cast<VecF*>(ps.off[2] + p0) = fz4;
                    *reinterpret_cast<VecF*>(ps.u[0] + p0) = ux4;
                    *reinterpret_cast<VecF*>(ps.u[1] + p0) = uy4;
                    *reinterpret_cast<VecF*>(ps.u[2] + p0) = uz4;
                    if (G) {
                        *reinterpret_cast<VecF*>(ps.w + p0) = w4;
                        *reinterpret_cast<VecI*>(ps.id + p0) = id4;
                    }
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
                            if (G) {
                                ps.w[p] = el(w4, j);
                                ps.id[p] = el(id4, j);
                            }
                        }
                    }
                }
            }
        }  // groups of this thread
          if (kacc >= 0) add12i<TJ>(Ji, kacc, acc, fxs);

        }
        ek += (double)ek_chunk;
        __syncthreads();
        // the queued moves that leave their start cell, split by every thread
        const int nq = min(s_qn, CHUNK);
        for (int i = threadIdx.x; i < nq; i += NT) {
            const int q = qbase + i;
            if (!in_range(q, (long long)gridDim.x * CHUNK)) continue;  // debug build only
            const float w = xq.w[q];
            split_fx<TJ>(Ji, xq.key[q], xq.a[0][q], xq.a[1][q], xq.a[2][q], xq.d[0][q], xq.d[1][q], xq.d[2][q],
                         cqx * w, cqy * w, cqz * w, fxs);
        }
        __syncthreads();
        if (threadIdx.x == 0) s_qn = 0;
        // merge: J tile cell t is domain cell c0 - 1 + t, padded index c0 + 1 + t
        for (int i = threadIdx.x; i < 3 * TJ3; i += NT) {
            int hi = 0, lo = 0;
#pragma unroll
            for (int cpy = 0; cpy < NCP; ++cpy) {
                hi += Jall[cpy * 6 * TJ3 + i];
                lo += Jall[cpy * 6 * TJ3 + 3 * TJ3 + i];
            }
            if ((hi | lo) != 0) {
                const int comp = i / TJ3, r = i - comp * TJ3;
                const int tz = r / (TJ * TJ), ty = (r / TJ) % TJ, tx = r % TJ;
                const long long o = (long long)comp * g.P + (c0x + 1 + tx) +
                                    (long long)g.np[0] * ((c0y + 1 + ty) + (long long)g.np[1] * (c0z + 1 + tz));
                if (in_range(o, 3 * g.P)) atomicAdd(&J[o], (double)(((long long)hi << FX_LO_BITS) + lo) * fxinv);
            }
        }
        __syncthreads();
    }
    const double s = block_sum<NT>(ek, red);
    if (threadIdx.x == 0) ek_part[blockIdx.x] = s * pp.mass;
    if (pp.drift) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g2max = fmaxf(g2max, __shfl_xor_sync(FULL, g2max, o));
        if (lane == 0) atomicMax(pp.drift, __float_as_uint(g2max));  // non-negative floats order like their bits
    }
}

// ------------------------------------------------------------------ launchers
constexpr int PUSH32_NT = 256;

template <int S>
size_t push32_smem_bytes() {
    constexpr int T = S + 4;
    using TL = Tile<float, S>;
    if (TL::kCoef) return 128 + sizeof(float) * TL::RAW + sizeof(Coef<float>) * 6 * TL::NE;
    return 128 + sizeof(float) * (6 * T * T * T + TL::ACC);
}

template <int S>
cudaError_t push32_setup(int* blocks_per_sm) {
    const int sm = (int)push32_smem_bytes<S>();
    cudaError_t e = cudaSuccess;
    for (auto f : {k_push_g<S, PUSH32_NT, true, false>, k_push_g<S, PUSH32_NT, false, false>,
                   k_push_g<S, PUSH32_NT, true, true>, k_push_g<S, PUSH32_NT, false, true>})
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_push_g<S, PUSH32_NT, false, false>,
                                                         PUSH32_NT, sm);
}

// perm null: the particles are updated in place in ps.  Otherwise slot i of
// ps receives particle perm[i] of pin, updated (the store's two buffers).
template <int S>
cudaError_t push32_launch(int grid, cudaStream_t st, const CUtensorMap& tm, const PushParams& pp,
                          const PStore<float>& ps, const PStore<float>& pin, const int* perm,
                          const XQueue<float>& xq, const Chunk* chunks, const int* nchunks, double* J,
                          double* ek_part, int* err) {
    const bool cubic = pp.g.d[0] == pp.g.d[1] && pp.g.d[1] == pp.g.d[2];
    const size_t sm = push32_smem_bytes<S>();
    if (cubic && perm)
        k_push_g<S, PUSH32_NT, true, true><<<grid, PUSH32_NT, sm, st>>>(tm, pp, ps, pin, perm, xq, chunks, nchunks, J,
                                                                       ek_part, err);
    else if (cubic)
        k_push_g<S, PUSH32_NT, true, false><<<grid, PUSH32_NT, sm, st>>>(tm, pp, ps, ps, nullptr, xq, chunks, nchunks,
                                                                        J, ek_part, err);
    else if (perm)
        k_push_g<S, PUSH32_NT, false, true><<<grid, PUSH32_NT, sm, st>>>(tm, pp, ps, pin, perm, xq, chunks, nchunks,
                                                                        J, ek_part, err);
    else
        k_push_g<S, PUSH32_NT, false, false><<<grid, PUSH32_NT, sm, st>>>(tm, pp, ps, ps, nullptr, xq, chunks,
                                                                         nchunks, J, ek_part, err);
    return cudaGetLastError();
}

#define PICGB_PUSH32_INST(S)                                                                                     \
    template cudaError_t push32_setup<S>(int*);                                                                  \
    template cudaError_t push32_launch<S>(int, cudaStream_t, const CUtensorMap&, const PushParams&,              \
                                          const PStore<float>&, const PStore<float>&, const int*,                \
                                          const XQueue<float>&, const Chunk*, const int*, double*, double*, int*);
PICGB_PUSH32_INST(4)
PICGB_PUSH32_INST(8)

PICGB_INDEX_FLAG_READER(push32_index_flags)

}  // namespace picgb
