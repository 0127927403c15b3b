// Exact fixed-point geometry and the simulation-of-simplicity predicates of the projection.
//
// Every vertex position is held as a signed 64-bit integer in units of 2^-CDP_Q grid cells
// ("fixed point").  Inside one simplex all coordinates are taken relative to an integer cell, so
// differences of vertex coordinates and of grid nodes fit in 54 bits, 2x2 minors in 128 bits
// and 3x3 determinants are evaluated exactly with a split 192-bit accumulation.  Every
// combinatorial decision of the projection (which cell holds a vertex, which cells an edge
// crosses and in which order, which grid lines cross a facet, which grid nodes lie inside a
// simplex) is the sign of one of two exact predicates with a grid point as one argument:
//
//   side2 : orient2d of a projected grid point against a projected simplex edge
//           (eq. raytraceMin is this predicate in the plane of two axes),
//   side3 : orientation of a grid point against a simplex facet (eq. orientation).
//
// Degenerate ties are broken by simulation of simplicity (eq. sos): every grid point g is moved
// to g - (eps^2, eps^3, eps^4).  Both predicates are affine in g, so the perturbed sign is the
// sign of the first non-zero term of D0, then the eps^2, eps^3, eps^4 coefficients (the
// expansion of eq. orientation_sos reduces to the facet normal's components because the same
// offset is applied to the point only).  Because all decisions come from these exact signs of
// one perturbed configuration, they are mutually consistent (Sect. 3.3, Fig. degenerate).
#pragma once

#include <stdint.h>

#ifndef CDP_HD
#define CDP_HD __host__ __device__ __forceinline__
#endif
// rarely executed or once-per-simplex code: kept out of line so that the hot loops stay small
// enough for the instruction cache
#ifndef CDP_COLD
#define CDP_COLD inline __host__ __device__ __noinline__
#endif

namespace cdp {

typedef long long i64;
typedef unsigned long long u64;
typedef __int128 i128;
typedef unsigned __int128 u128;

// fractional bits of the fixed-point coordinates (grid units)
constexpr int CDP_Q = 40;
// largest simplex extent (cells per axis) for which the exact arithmetic is guaranteed
constexpr int CDP_MAX_EXTENT = 2048;

CDP_HD int sgn_i64(i64 v) { return (v > 0) - (v < 0); }
CDP_HD int sgn_i128(i128 v) { return (v > 0) - (v < 0); }

CDP_HD i128 mul64(i64 a, i64 b) { return (i128)a * (i128)b; }

// Sign of a.b for a: three 128-bit integers (|a_i| < 2^110), b: three 64-bit integers
// (|b_i| < 2^55).  The sum needs up to ~168 bits: each a_i is split as ah*2^64 + al (al
// unsigned) and the two partial sums are recombined exactly.
struct Wide {
    i128 hi;  // value = hi * 2^64 + lo, 0 <= lo < 2^64
    u64 lo;
};

CDP_HD Wide dot3_wide(const i128 a[3], const i64 b[3]) {
    i128 hi = 0, lo = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        i64 ah = (i64)(a[i] >> 64);
        u64 al = (u64)a[i];
        hi += (i128)ah * (i128)b[i];
        u64 bb = b[i] < 0 ? (u64)0 - (u64)b[i] : (u64)b[i];
        u128 p = (u128)al * (u128)bb;  // < 2^119
        lo += b[i] < 0 ? -(i128)p : (i128)p;
    }
    i128 q = lo >> 64;  // floor(lo / 2^64)
    Wide w;
    w.hi = hi + q;
    w.lo = (u64)lo;
    return w;
}

CDP_HD int sgn_wide(const Wide& w) {
    if (w.hi != 0) return w.hi > 0 ? 1 : -1;
    return w.lo != 0 ? 1 : 0;
}

// |v| < 2^127 converted with one rounding per 64-bit half (each component keeps its own
// relative accuracy; no cancellation because the halves are taken of |v|)
template <typename R>
CDP_HD R i128_to_real(i128 v, int scale);

template <>
CDP_HD double i128_to_real<double>(i128 v, int scale) {
    bool neg = v < 0;
    u128 a = neg ? (u128)0 - (u128)v : (u128)v;
    double f = (double)(u64)(a >> 64) * 18446744073709551616.0 + (double)(u64)a;
    f = ldexp(f, -scale);
    return neg ? -f : f;
}

template <>
CDP_HD float i128_to_real<float>(i128 v, int scale) {
    bool neg = v < 0;
    u128 a = neg ? (u128)0 - (u128)v : (u128)v;
    u64 hi = (u64)(a >> 64), lo = (u64)a;
    // hi < 2^47 here: scale both halves into float range first
    float f = ldexpf((float)hi, 64 - scale) + ldexpf((float)lo, -scale);
    return neg ? -f : f;
}

// (w.hi * 2^64 + w.lo) * 2^-scale in double, converted from sign and magnitude so that a
// small negative value is not lost to cancellation between the two halves
CDP_HD double wide_to_double(const Wide& w, int scale) {
    bool neg = w.hi < 0;
    u128 mh;
    u64 ml;
    if (!neg) {
        mh = (u128)w.hi;
        ml = w.lo;
    } else if (w.lo != 0) {
        mh = (u128)(-(w.hi + 1));
        ml = (u64)0 - w.lo;
    } else {
        mh = (u128)(-w.hi);
        ml = 0;
    }
    double hi = (double)(u64)(mh >> 64) * 18446744073709551616.0 + (double)(u64)mh;
    double v = ldexp(hi, 64 - scale) + ldexp((double)ml, -scale);
    return neg ? -v : v;
}

template <typename R>
CDP_HD R i64_to_real(i64 v, int scale);
template <>
CDP_HD double i64_to_real<double>(i64 v, int scale) { return ldexp((double)v, -scale); }
template <>
CDP_HD float i64_to_real<float>(i64 v, int scale) { return ldexpf((float)v, -scale); }

// Exact cross product of two 3-vectors of 64-bit integers (|components| < 2^54).
CDP_HD void cross_exact(const i64 a[3], const i64 b[3], i128 out[3]) {
    out[0] = mul64(a[1], b[2]) - mul64(a[2], b[1]);
    out[1] = mul64(a[2], b[0]) - mul64(a[0], b[2]);
    out[2] = mul64(a[0], b[1]) - mul64(a[1], b[0]);
}

// ------------------------------------------------------------------------------------------
// Perturbed predicates.  The grid point is g - delta, delta = (eps^2, eps^3, eps^4): along axis
// u its perturbation dominates that of axis v whenever u < v.
// ------------------------------------------------------------------------------------------

// side2: sign of orient2d(a, b, p - delta) in the plane of axes (u, v), u < v:
//   (b_u - a_u)(p_v - a_v) - (b_v - a_v)(p_u - a_u)
//   - delta_v (b_u - a_u) + delta_u (b_v - a_v).
// au, av, bu, bv, pu, pv are fixed-point coordinates in one frame.
CDP_COLD int side2_exact(i64 au, i64 av, i64 bu, i64 bv, i64 pu, i64 pv) {
    i64 du = bu - au, dv = bv - av;
    i128 d0 = mul64(du, pv - av) - mul64(dv, pu - au);
    if (d0 != 0) return d0 > 0 ? 1 : -1;
    if (dv != 0) return dv > 0 ? 1 : -1;
    return du > 0 ? -1 : (du < 0 ? 1 : 0);
}

// side3: sign of n.(g - delta - a) for the exact facet normal n (any vertex a of the facet):
//   D0 = n.(g - a); perturbation -n.delta, dominated by the first non-zero component of n.
CDP_COLD int side3_exact(const i128 n[3], const i64 a[3], const i64 g[3]) {
    i64 d[3] = {g[0] - a[0], g[1] - a[1], g[2] - a[2]};
    int s = sgn_wide(dot3_wide(n, d));
    if (s != 0) return s;
    if (n[0] != 0) return n[0] > 0 ? -1 : 1;
    if (n[1] != 0) return n[1] > 0 ? -1 : 1;
    return n[2] > 0 ? -1 : (n[2] < 0 ? 1 : 0);
}

// parity of a permutation of (0, 1, 2, 3): +1 even, -1 odd
CDP_HD int parity4(int a, int b, int c, int d) {
    int p[4] = {a, b, c, d}, inv = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = i + 1; j < 4; ++j) inv += p[i] > p[j];
    return (inv & 1) ? -1 : 1;
}

}  // namespace cdp
