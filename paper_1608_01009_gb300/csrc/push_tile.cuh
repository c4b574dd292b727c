// Shared-memory field tile and the cell arithmetic of the particle kernels
// (FP64: k_push.cu; mixed FP32: k_push32.cu).
#pragma once
#include "pic_internal.cuh"

namespace picgb {

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
#ifndef PICGB_FX_COPIES
#define PICGB_FX_COPIES 2
#endif
template <class R, int S>
struct Tile {
    static constexpr int T = S + 4, T3 = T * T * T, TJ = S + 3, TJ3 = TJ * TJ * TJ;
    static constexpr int NE = (T - 1) * (T - 1) * T;  // coefficient cells per component
    static constexpr bool kCoef = S <= 4;
    // FP64 with a coefficient tile accumulates the deposit's 12 moments per
    // cell (see value_offset) instead of the 3 edge components
    static constexpr bool kMoments = PICGB_MOMENTS && sizeof(R) == 8 && kCoef;
    // accumulation tile (elements): FP64 12 moments per cell, or the 3 edge
    // components per cell without a coefficient tile;
    // FP32: FX_COPIES copies of the 3 edge components per cell as two 32-bit
    // fixed-point parts (lanes spread over the copies; one copy without a
    // coefficient tile, whose raw tile is kept)
    static constexpr int FX_COPIES = sizeof(R) == 4 && kCoef ? PICGB_FX_COPIES : 1;
    static constexpr int ACC = kMoments ? 12 * TJ3 : (sizeof(R) == 4 ? FX_COPIES * 6 * TJ3 : 3 * TJ3);
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
    if (!in_range((k * T + j) * T + i, T * T * T - T * T - T - 1)) return R(0);  // debug build only
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
    if (!in_range(o, (T - 1) * (T - 1) * (T - 1))) return R(0);  // debug build only: o + (T-1)^2 < (T-1)^2 T
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

// The 12 edge values of one cell, v[0..11] = Jx (i+1/2, j+s1, k+s2), Jy
// (i+s1, j+1/2, k+s2), Jz (i+s1, j+s2, k+1/2) with (s1, s2) = (0,0), (1,0),
// (0,1), (1,1): offset of value m from the cell's corner in the J tile.
template <int TJ>
__device__ __forceinline__ int edge_offset(int m) {
    const int comp = m >> 2, e = m & 3;
    return comp * TJ * TJ * TJ + (e & 1) * (comp == 0 ? TJ : 1) + (e >> 1) * (comp == 2 ? TJ : TJ * TJ);
}

}  // namespace picgb
