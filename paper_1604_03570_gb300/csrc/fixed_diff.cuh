// fixed_diff.cuh -- exact fixed-point time stepping for FP64 storage (MF_FIXED_DIFF).
//
// The flux-form update u_new = u + lam * div F(u) of Sec. 4.1 is linear in u.  On GB300 the FP64
// pipe, and the FP64 <-> FP32 conversions with it, issue about 2 operations per clock per SM
// while the memory system delivers about 1.4 FP64 cells per clock per SM: the plain FP64 stencil
// (9 FP64 operations per cell at radius 1) is bound by FP64 issue, far below the memory roofline.
// This path does no FP64 arithmetic inside the time loop:
//
//   1. before the first step the level's valid cells are mapped in place from FP64 to 64-bit
//      integers K = u / 2^E, truncated toward zero, on a grid 2^E per component chosen from the
//      largest exponent present so that |K| < 2^(B - H);
//   2. every step forms the Laplacian L = sum_j w_j K_j of the direct form, with the operator's
//      coefficients scaled to integers w_j (denominator den), in exact 64-bit integer arithmetic
//      (exact arithmetic makes the direct form and the flux form of Sec. 4.1 the same number),
//      and writes K' = round((K 2^64 + L * Lq) / 2^t) on the next step's grid 2^E', where
//      Lq = round(lam / den * 2^64) and t = 64 - (E - E'); E' follows the level maximum the
//      step before reduced, so the precision follows a decaying solution.  A step that keeps
//      the grid (t = 64, the common case) takes L Lq / 2^64 from three 32-bit partial products
//      of |L|, within -2 .. +1 units in magnitude and odd in L (fix_incr);
//   3. after the last step the valid cells are mapped back to FP64, rounded to nearest.
//
// Error: step 1 and every rounding in step 2 are at most two units 2^E of the grid; with
// max|u| >= 2^(E + B - H - 2) that is <= 2^(3 + H - B) max|u| per step.  The rounding of Lq adds
// at most |L| 2^-65 <= 1/8 unit per step whatever lam is, and step 3 the FP64 rounding.
// Headroom: one step grows max|u| by less than 2^H (the forward-Euler update's infinity norm is
// at most 1.25 at the stability limit for R <= 4); choosing E' = E + b + H - B, with 2^b above
// the largest |K| on grid E, keeps |K| < 2^B on every grid, so |L| <= sum |w| 2^B < 2^63.
#pragma once

#include <cstdint>

#include "mf_internal.h"

namespace mfk {

// Arithmetic tag of the fixed-point path (storage: 64-bit fixed point inside an advance).
struct FixA {};

constexpr int kFixH = 1;  // headroom bits for one step's growth

// Integer weights of the direct-form (2R+1)-point Laplacian per direction, scaled by den:
// w0 (centre, already summed over the three directions) and w(m) for the pair at distance m.
//   R = 1: (1, -2, 1)                                     -> w0 = -6,     w1 = 1
//   R = 2: (-1, 16, -30, 16, -1) / 12                     -> w0 = -90,    w = 16, -1
//   R = 4: (-9, 128, -1008, 8064, -14350, ...) / 5040     -> w0 = -43050, w = 8064, -1008, 128, -9
// B: bits of |K|; sum |w| * 2^B < 2^63 (R = 1: 12; R = 2: 192; R = 4: 98304 = 3 * 2^15).
template <int R> struct FixW;
template <> struct FixW<1> {
    static constexpr int B = 58;
    static __device__ __forceinline__ long long w0() { return -6; }
    static __device__ __forceinline__ long long w(int) { return 1; }
};
template <> struct FixW<2> {
    static constexpr int B = 55;
    static __device__ __forceinline__ long long w0() { return -90; }
    static __device__ __forceinline__ long long w(int m) { return m == 1 ? 16 : -1; }
};
template <> struct FixW<4> {
    static constexpr int B = 46;
    static __device__ __forceinline__ long long w0() { return -43050; }
    static __device__ __forceinline__ long long w(int m) { return m == 1 ? 8064 : m == 2 ? -1008 : m == 3 ? 128 : -9; }
};

// High word of |v|'s encoding: its order is the order of |v| for finite v (the reduction key of
// the FP64 level maximum that gives the first grid).
__device__ __forceinline__ uint32_t fix_key(double v) { return (uint32_t)__double2hiint(v) & 0x7fffffffu; }

// The first grid exponent E of a level whose largest |u| has the key wmax: u < 2^(e - 1022)
// for the biased exponent e = wmax >> 20, so E = e - 1022 - (B - H) gives |K| < 2^(B - H).
__device__ __forceinline__ int fix_first_grid(uint32_t wmax, int B) { return (int)(wmax >> 20) - 1022 - (B - kFixH); }

// K = u / 2^E truncated toward zero, for FP64 u: with the 64-bit significand
// M = 2^63 + (mantissa << 11) and the biased exponent e, u = M 2^(e - 1086) and
// K = M >> (1086 + E - e) (PTX clamps a shift of 64 or more to a result of 0).  Zeros and
// subnormals map to 0.
__device__ __forceinline__ long long fix_from_f64(double v, int E) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const unsigned int e = (unsigned int)(bits >> 52) & 0x7ffu;
    const unsigned long long m = (bits << 11) | 0x8000000000000000ull;
    const unsigned int t = (unsigned int)(1086 + E) - e;
    unsigned long long k;
    asm("shr.b64 %0, %1, %2;" : "=l"(k) : "l"(m), "r"(t));
    if (e == 0u) k = 0ull;
    return (long long)bits < 0 ? -(long long)k : (long long)k;
}

// K 2^E as FP64, rounded to nearest (ties away from zero).  |K| = n 2^-lz with n in [2^63, 2^64)
// gives the biased exponent E + 1086 - lz; adding the rounded (n >> 11), whose leading one lands
// in bit 52, to (E + 1085 - lz) << 52 assembles exponent and significand (a carry out of the
// significand raises the exponent, as it should).  Results below the normal range flush to 0.
__device__ __forceinline__ double fix_to_f64(long long K, int E) {
    const unsigned long long s = (unsigned long long)(K >> 63);
    const unsigned long long a = ((unsigned long long)K ^ s) - s;
    if (a == 0ull) return 0.0;
    const int lz = __clzll((long long)a);
    const unsigned long long n = a << lz;
    const int be = E + 1086 - lz;
    if (be <= 0) return 0.0;
    const unsigned long long sig = (n >> 11) + ((n >> 10) & 1ull);
    const unsigned long long bits = (((unsigned long long)(unsigned int)(be - 1) << 52) + sig) | (s << 63);
    return __longlong_as_double((long long)bits);
}

// Signed 128-bit product L * q (q unsigned): {hi, lo}.
__device__ __forceinline__ void fix_mul128(long long L, unsigned long long q, long long &hi, unsigned long long &lo) {
    const unsigned long long ul = (unsigned long long)L;
    lo = ul * q;
    unsigned long long h = __umul64hi(ul, q);
    if (L < 0) h -= q;  // two's complement: L = ul - 2^64
    hi = (long long)h;
}

// An upper bound on the bit length of the largest |K| of a level from the OR M of its |K| values:
// the stencil ORs the high words of |K| in ones' complement (-K - 1 for K < 0) shifted up by 32
// bits, so every |K| <= M + 2^32.
__device__ __forceinline__ int fix_bits(unsigned long long M) { return 64 - __clzll((long long)(M + (1ull << 32))); }

// The increment of a step that keeps the grid (t = 64): L q / 2^64, formed on |L| and given L's
// sign, so that L and -L get increments of opposite sign and equal size (a field and its
// negative evolve alike, as they do under rounding to nearest).  With |L| = ah 2^32 + al and
// q = qh 2^32 + ql, the three partial products that reach bit 64 are each truncated (the fourth,
// al ql, is below 2^64): |L| q / 2^64 - 3 < ah qh + floor(ah ql / 2^32) + floor(al qh / 2^32)
// <= |L| q / 2^64, and the + 1 centres the magnitude error on (-2, 1].
__device__ __forceinline__ long long fix_incr(unsigned long long L, uint32_t qh, uint32_t ql) {
    const unsigned long long s = (unsigned long long)((long long)L >> 63);
    const unsigned long long a = (L ^ s) - s;  // |L| < 2^63
    const uint32_t ah = (uint32_t)(a >> 32), al = (uint32_t)a;
    const unsigned long long m = (unsigned long long)ah * qh + (((unsigned long long)ah * ql) >> 32) +
                                 (((unsigned long long)al * qh) >> 32) + 1ull;
    return (long long)((m ^ s) - s);
}

// One cell of a fixed-point step: K' = round((K 2^64 + L q) / 2^t), 0 < t <= 65 (launch-uniform).
// The 128-bit numerator is exact: |K| < 2^B and |L q| < 2^126.
__device__ __forceinline__ long long fix_update(long long K, long long L, unsigned long long q, int t) {
    long long hi;
    unsigned long long lo;
    fix_mul128(L, q, hi, lo);
    hi += K;
    if (t >= 65) {  // round (add 2^(t-1) = 2^64 * 2^(t-65)), then shift
        hi += 1ll << (t - 65);
        return hi >> (t - 64);
    }
    const unsigned long long l2 = lo + (1ull << (t - 1));
    hi += l2 < lo ? 1 : 0;
    if (t == 64) return hi;
    return (long long)(((unsigned long long)hi << (64 - t)) | (l2 >> t));
}

}  // namespace mfk
