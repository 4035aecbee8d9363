// stencil_common.cuh -- scalar helpers and the per-cell flux-form update shared by the
// stencil kernels (global-memory and TMA-staged variants), so that every variant evaluates
// the same expression in the same order.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace mfk {

// ------------------------------------------------------------------ scalar helpers

template <typename A> struct Ar;
template <> struct Ar<double> {
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
};
template <> struct Ar<float> {
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
};

// The arithmetic type of a storage type when the path computes natively: FP64 for FP64
// storage, FP32 for FP32 and BF16 storage.
template <typename S> struct NativeArith { using T = S; };
template <> struct NativeArith<__nv_bfloat16> { using T = float; };

template <typename S, typename A> __device__ __forceinline__ A ld(const S *p);
template <> __device__ __forceinline__ double ld<double, double>(const double *p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld<float, float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ double ld<float, double>(const float *p) { return (double)__ldg(p); }
template <> __device__ __forceinline__ float ld<__nv_bfloat16, float>(const __nv_bfloat16 *p) {
    return __bfloat162float(__ldg(p));
}
template <> __device__ __forceinline__ double ld<__nv_bfloat16, double>(const __nv_bfloat16 *p) {
    return (double)__bfloat162float(__ldg(p));
}

__device__ __forceinline__ void st(double *p, double v) { *p = v; }
__device__ __forceinline__ void st(long long *p, long long v) { *p = v; }
__device__ __forceinline__ void st(float *p, float v) { *p = v; }
__device__ __forceinline__ void st(float *p, double v) { *p = __double2float_rn(v); }
__device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void st(__nv_bfloat16 *p, double v) { *p = __double2bfloat16(v); }

__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return (double)v; }
__device__ __forceinline__ double to_f64(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
__device__ __forceinline__ void from_f64(double *p, double v) { *p = v; }
__device__ __forceinline__ void from_f64(float *p, double v) { *p = __double2float_rn(v); }
__device__ __forceinline__ void from_f64(__nv_bfloat16 *p, double v) { *p = __double2bfloat16(v); }

// Face-flux weights b_m of the centred (2R+1)-point Laplacian of order 2R written as a flux
// difference, F_{i+1/2} = sum_m b_m (u_{i+m} - u_{i+1-m}), b_m = sum_{j>=m} c_j with the
// classical centred second-derivative weights c_j (R=1: c=(-2,1); R=2: (-5/2,4/3,-1/12);
// R=4: (-205/72, 8/5, -1/5, 8/315, -1/560)).
template <int R> struct FluxW;
template <> struct FluxW<1> { static __device__ __forceinline__ double b(int) { return 1.0; } };
template <> struct FluxW<2> {
    static __device__ __forceinline__ double b(int m) { return m == 1 ? 15.0 / 12.0 : -1.0 / 12.0; }
};
template <> struct FluxW<4> {
    static __device__ __forceinline__ double b(int m) {
        return m == 1 ? 205.0 / 144.0 : m == 2 ? -127.0 / 720.0 : m == 3 ? 17.0 / 720.0 : -1.0 / 560.0;
    }
};

// Flux at the face between q[c] and q[c+1] of a line of values q (index c = centre - 1 for
// the lower face): F = b_1 (q[c+1] - q[c]) + sum_{m>=2} b_m (q[c+m] - q[c+1-m]).
template <typename A, int R>
__device__ __forceinline__ A face_flux(const A *q, int c) {
    if constexpr (R == 1) return Ar<A>::sub(q[c + 1], q[c]);  // b_1 = 1: the product is exact
    A f = Ar<A>::mul((A)FluxW<R>::b(1), Ar<A>::sub(q[c + 1], q[c]));
#pragma unroll
    for (int m = 2; m <= R; ++m) f = Ar<A>::fma((A)FluxW<R>::b(m), Ar<A>::sub(q[c + m], q[c + 1 - m]), f);
    return f;
}

// Packed pairs of FP32 values for Blackwell's add/sub/fma.rn.f32x2: each lane is rounded
// exactly as the scalar _rn operation, so paired and scalar code give identical bits.
struct F2 {
    float x, y;
};
__device__ __forceinline__ F2 sub2(F2 a, F2 b) {
    F2 r;
    asm("{\n\t.reg .b64 a, b, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "sub.rn.f32x2 d, a, b;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ F2 add2(F2 a, F2 b) {
    F2 r;
    asm("{\n\t.reg .b64 a, b, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "add.rn.f32x2 d, a, b;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {
    F2 r;
    asm("{\n\t.reg .b64 a, b, c, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "mov.b64 c, {%6, %7};\n\tfma.rn.f32x2 d, a, b, c;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}

__device__ __forceinline__ F2 mul2(F2 a, F2 b) {
    F2 r;
    asm("{\n\t.reg .b64 a, b, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "mul.rn.f32x2 d, a, b;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

// face_flux<float, R> of two lines at once (qa, qb; the same face index c): the same operations
// in the same order, each lane rounded as the scalar code rounds it.
template <int R>
__device__ __forceinline__ F2 face_flux2(const float *qa, const float *qb, int c) {
    if constexpr (R == 1) return sub2(F2{qa[c + 1], qb[c + 1]}, F2{qa[c], qb[c]});
    const float b1 = (float)FluxW<R>::b(1);
    F2 f = mul2(F2{b1, b1}, sub2(F2{qa[c + 1], qb[c + 1]}, F2{qa[c], qb[c]}));
#pragma unroll
    for (int m = 2; m <= R; ++m) {
        const float bm = (float)FluxW<R>::b(m);
        f = fma2(F2{bm, bm}, sub2(F2{qa[c + m], qb[c + m]}, F2{qa[c + 1 - m], qb[c + 1 - m]}), f);
    }
    return f;
}

// Runge-Kutta stage combination a * u0 + b * e of the state at the start of the step (u0) and
// the forward-Euler value e: one rounding of the product b * e, one of the fused multiply-add.
template <typename A> __device__ __forceinline__ A rk_combine(A e, A u0, A a, A b) {
    return Ar<A>::fma(a, u0, Ar<A>::mul(b, e));
}

template <typename S, typename A> __device__ __forceinline__ A ld_smem(const S *p);
template <> __device__ __forceinline__ double ld_smem<double, double>(const double *p) { return *p; }
template <> __device__ __forceinline__ float ld_smem<float, float>(const float *p) { return *p; }
template <> __device__ __forceinline__ double ld_smem<float, double>(const float *p) { return (double)*p; }
template <> __device__ __forceinline__ float ld_smem<__nv_bfloat16, float>(const __nv_bfloat16 *p) {
    return __bfloat162float(*p);
}
template <> __device__ __forceinline__ double ld_smem<__nv_bfloat16, double>(const __nv_bfloat16 *p) {
    return (double)__bfloat162float(*p);
}

// One cell's update from the lines through it: x line qx, y line qy (2R+1 values each,
// centre at R) and the z fluxes below/above.  Order: ((Dx + Dy) + Dz), then u + lam*div.
template <typename A, int R>
__device__ __forceinline__ A update_cell(const A *qx, const A *qy, A fzm, A fzp, A u, A lam) {
    A dxv = Ar<A>::sub(face_flux<A, R>(qx, R), face_flux<A, R>(qx, R - 1));
    A dyv = Ar<A>::sub(face_flux<A, R>(qy, R), face_flux<A, R>(qy, R - 1));
    A dzv = Ar<A>::sub(fzp, fzm);
    A div = Ar<A>::add(Ar<A>::add(dxv, dyv), dzv);
    return Ar<A>::fma(lam, div, u);
}

// The same update with the two x-face fluxes given (computed once per face and shared by
// the two cells beside it: the identical expression on identical operands).
template <typename A, int R>
__device__ __forceinline__ A update_cell_fx(A fxp, A fxm, const A *qy, A fzm, A fzp, A u, A lam) {
    A dxv = Ar<A>::sub(fxp, fxm);
    A dyv = Ar<A>::sub(face_flux<A, R>(qy, R), face_flux<A, R>(qy, R - 1));
    A dzv = Ar<A>::sub(fzp, fzm);
    A div = Ar<A>::add(Ar<A>::add(dxv, dyv), dzv);
    return Ar<A>::fma(lam, div, u);
}

// The same update with every face flux given: (Dx + Dy) + Dz, then u + lam * div.
template <typename A>
__device__ __forceinline__ A update_cell_f(A fxp, A fxm, A fyp, A fym, A fzp, A fzm, A u, A lam) {
    A div = Ar<A>::add(Ar<A>::add(Ar<A>::sub(fxp, fxm), Ar<A>::sub(fyp, fym)), Ar<A>::sub(fzp, fzm));
    return Ar<A>::fma(lam, div, u);
}

}  // namespace mfk
