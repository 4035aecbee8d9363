// fixed_diff.cuh -- exact fixed-point differences for FP64 storage (MF_FIXED_DIFF).
//
// The flux-form update u_new = u + lam * div F(u) of Sec. 4.1 is linear in u.  On GB300 the FP64
// pipe, and the FP64 <-> FP32 conversions with it, issue about 2 operations per clock per SM,
// while the memory system delivers about 1.4 FP64 cells per clock per SM: the plain FP64 stencil
// (9 FP64 operations per cell at radius 1) is bound by FP64 issue, far below the memory
// roofline.  This path keeps FP64 storage and does one FP64 operation per cell:
//
//   1. every value u read is mapped to a 64-bit integer K = u / Q, truncated toward zero, on a
//      grid Q = 2^(T0 - 1086) fixed per level and component, with T0 chosen from the largest
//      exponent present so that |K| < 2^B;  only integer instructions are used (bit fields of
//      the IEEE-754 encoding, a 64-bit shift);
//   2. the Laplacian L = sum_j w_j K_j of the direct form, with the operator's coefficients
//      scaled to integers w_j (denominator den), is formed in exact 64-bit integer arithmetic;
//      exact arithmetic makes the direct form and the flux form of Sec. 4.1 the same number;
//   3. D = L * Q is turned into an FP64 value with integer instructions (leading-zero count,
//      shift, exponent assembly; truncated to 53 bits);
//   4. u_new = fma(lam / den, D, u) in FP64, the one FP64 operation.
//
// Error: each K differs from u / Q by less than 1, so L * Q differs from den * Lap(u) by less than
// sum_j |w_j| * Q, with Q <= 2^(1 - B) max|u|; step 3 adds a relative 2^-52.  B leaves room for the
// integer sum: sum_j |w_j| * 2^B < 2^63.
#pragma once

#include <cstdint>

namespace mfk {

// Arithmetic tag of the fixed-point path (storage FP64).
struct FixA {};

// Integer weights of the direct-form (2R+1)-point Laplacian per direction, scaled by den:
// w0 (centre, already summed over the three directions) and w[m] for the pair at distance m.
//   R = 1: (1, -2, 1)                                     -> w0 = -6,     w1 = 1
//   R = 2: (-1, 16, -30, 16, -1) / 12                     -> w0 = -90,    w = 16, -1
//   R = 4: (-9, 128, -1008, 8064, -14350, ...) / 5040     -> w0 = -43050, w = 8064, -1008, 128, -9
// B: bits of |K|; sum |w| * 2^B < 2^63 (R = 1: 12; R = 2: 192; R = 4: 98304 = 3 * 2^15).
template <int R> struct FixW;
template <> struct FixW<1> {
    static constexpr int B = 58;
    static constexpr double den = 1.0;
    static __device__ __forceinline__ long long w0() { return -6; }
    static __device__ __forceinline__ long long w(int) { return 1; }
};
template <> struct FixW<2> {
    static constexpr int B = 55;
    static constexpr double den = 12.0;
    static __device__ __forceinline__ long long w0() { return -90; }
    static __device__ __forceinline__ long long w(int m) { return m == 1 ? 16 : -1; }
};
template <> struct FixW<4> {
    static constexpr int B = 46;
    static constexpr double den = 5040.0;
    static __device__ __forceinline__ long long w0() { return -43050; }
    static __device__ __forceinline__ long long w(int m) { return m == 1 ? 8064 : m == 2 ? -1008 : m == 3 ? 128 : -9; }
};

// The grid constant of a level (component) whose largest |u| has the high word wmax (sign bit
// cleared, as reduced by the stencil and by k_fix_emax): T0 = 64 - B + max(E, B), E the biased
// exponent of that value.  Then |u| < 2^(E - 1022) gives |K| < 2^B, and zeros, subnormals and
// values below the grid map to K = 0.
template <int R> __device__ __forceinline__ int fix_t0(uint32_t wmax) {
    const int E = (int)(wmax >> 20);
    return 64 - FixW<R>::B + (E > FixW<R>::B ? E : FixW<R>::B);
}

// K = u / Q truncated toward zero.  u = M * 2^(e - 1086) with the 64-bit significand
// M = 2^63 + (mantissa << 11) and e the biased exponent, so K = M >> (T0 - e); PTX clamps a shift
// of 64 or more to a result of 0.  A value above the level's maximum (e > E, possible only in
// cells whose result is not used) wraps the shift count to a large unsigned number: K = 0.
__device__ __forceinline__ long long fix_of(double v, int T0) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const unsigned long long m = (bits << 11) | 0x8000000000000000ull;
    const unsigned int t = (unsigned int)T0 - ((unsigned int)(bits >> 52) & 0x7ffu);
    unsigned long long k;
    asm("shr.b64 %0, %1, %2;" : "=l"(k) : "l"(m), "r"(t));
    return (long long)bits < 0 ? -(long long)k : (long long)k;
}

// D = L * Q as an FP64 value, truncated to 53 significant bits.  |L| = n * 2^-lz with
// n in [2^63, 2^64) gives the biased exponent T0 - lz; adding (n >> 11), which carries the
// leading one into bit 52, to (T0 - lz - 1) << 52 assembles exponent and significand.
__device__ __forceinline__ double fix_to_f64(long long L, int T0) {
    const unsigned long long s = (unsigned long long)(L >> 63);  // 0 or all ones
    const unsigned long long a = ((unsigned long long)L ^ s) - s;
    const int lz = __clzll((long long)a);
    const unsigned long long n = a << (lz & 63);
    const unsigned long long bits = (((unsigned long long)(unsigned int)(T0 - lz - 1) << 52) + (n >> 11)) | (s << 63);
    return a ? __longlong_as_double((long long)bits) : 0.0;
}

// High word of |v|'s encoding: its order is the order of |v| for finite v (the reduction key of
// the level maximum).
__device__ __forceinline__ uint32_t fix_key(double v) { return (uint32_t)__double2hiint(v) & 0x7fffffffu; }

}  // namespace mfk
