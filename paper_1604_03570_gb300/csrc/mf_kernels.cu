// mf_kernels.cu -- CUDA kernels of the MultiFab sweep for sm_103a (GB300).
//
//   k_fill          FillBoundary (Sec. 3.1): one persistent copy kernel over the precomputed
//                   list of box-box intersections (periodic images included) of every level.
//   k_stencil       the heat-equation kernel of Sec. 4.1 in flux form (face fluxes, then
//                   their divergence), out of place, over the device work list of logical
//                   tiles (Sec. 3.2 MFIter / tilebox()); one persistent launch for all boxes.
//                   Each thread owns an (x, y) column of the tile and marches along z with
//                   a register queue of 2R+1 values, so the z-face flux of the previous
//                   cell is reused; x and y neighbours come through L1.
//   k_stencil_plain the untiled per-box baseline of Sec. 3.1 (one launch per box).
//   k_reduce_*      whole-level reductions (Sec. 3.1: the sum, mf.max(0) and norms): FP64
//                   Neumaier-compensated sums, exact max / min, a fixed reduction tree over
//                   the box layout's rows, so the result depends on neither tiles nor timing.
//   k_interp / k_avgdown   inter-level operations of a refined level (Sec. 3).
//   k_scatter / k_gather   dense host layout <-> FArrayBoxes with dtype conversion.
//
// Per-cell floating-point order is fixed (explicit _rn intrinsics, no contraction left to
// the compiler), so every tile shape and every box layout gives identical bits.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <type_traits>

#include "mf_internal.h"
#include "stencil_common.cuh"
#include "reduce_common.cuh"

namespace mfk {

// ------------------------------------------------------------------ FillBoundary

__device__ __forceinline__ uint32_t fdiv(uint32_t n, FastDiv d) { return (__umulhi(n, d.m) + n) >> d.s; }

// A warp copies one task of 256 cells or 16-byte vectors (8 per lane, every load issued
// before the stores).  Lanes 0..11 load one 8-byte word of the 96-byte task header each and
// the warp shares them by shuffle, so warps never wait for one another.
constexpr int kFillCellsPerLane = 8;
union FbTaskWords {
    FbTask t;
    unsigned long long w[sizeof(FbTask) / 8];
};

// Cells off + lane + 32 u, u < U, of the task.
template <typename E, int U>
__device__ __forceinline__ void fill_copy(E *base, const FbTask &tk, int lane, int off) {
    const E *sb = base + tk.src;
    E *db = base + tk.dst;
    E v[U];
    uint32_t dof[U];  // offsets within the destination FArrayBox
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int i = off + lane + 32 * u;
        const uint32_t l = (uint32_t)(tk.first + i);
        const uint32_t r0 = fdiv(l, tk.f0);
        const uint32_t x = l - r0 * (uint32_t)tk.n0;
        const uint32_t r1 = fdiv(r0, tk.f1);
        const uint32_t y = r0 - r1 * (uint32_t)tk.n1;
        const uint32_t c = fdiv(r1, tk.f2);
        const uint32_t z = r1 - c * (uint32_t)tk.n2;
        dof[u] = c * (uint32_t)tk.d_cs + z * (uint32_t)tk.d_pl + y * (uint32_t)tk.d_px + x;
        if (i < tk.count) v[u] = __ldg(sb + (c * (uint32_t)tk.s_cs + z * (uint32_t)tk.s_pl + y * (uint32_t)tk.s_px + x));
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
        if (off + lane + 32 * u < tk.count) db[dof[u]] = v[u];
}

// Jobs: the work of one kernel, run by a range of a launch's blocks.  run(b, nb) does what block
// b of an nb-block launch of that kernel does, so one kernel body serves its own launch and a
// shared one (k_pair: two jobs that neither read what the other writes nor write the same
// cells, in one launch).

template <typename E>
struct FillJob {
    LevelPtrs lv;
    const FbTask *tasks;
    int ntasks;
    __device__ __forceinline__ void run(int b, int nb) const {
        constexpr int W = (int)(sizeof(FbTask) / 8);
        const int lane = threadIdx.x & 31;
        const int nwarps = (int)(((unsigned)nb * blockDim.x) >> 5);
        for (int t = (int)(((unsigned)b * blockDim.x + threadIdx.x) >> 5); t < ntasks; t += nwarps) {
            unsigned long long word = 0;
            if (lane < W) word = __ldg((const unsigned long long *)(tasks + t) + lane);
            FbTaskWords h;
#pragma unroll
            for (int i = 0; i < W; ++i) h.w[i] = __shfl_sync(0xffffffffu, word, i);
            if (h.t.vec) {  // two halves of 4 vectors per lane (registers)
                fill_copy<uint4, kFillCellsPerLane / 2>((uint4 *)lv.base[h.t.level], h.t, lane, 0);
                fill_copy<uint4, kFillCellsPerLane / 2>((uint4 *)lv.base[h.t.level], h.t, lane, 16 * kFillCellsPerLane);
            } else {
                fill_copy<E, kFillCellsPerLane>((E *)lv.base[h.t.level], h.t, lane, 0);
            }
        }
    }
};

template <typename E>
__global__ void __launch_bounds__(256) k_fill(LevelPtrs lv, const FbTask *__restrict__ tasks, int ntasks) {
    FillJob<E>{lv, tasks, ntasks}.run(blockIdx.x, gridDim.x);
}

// Two jobs in one launch: blocks [0, na) run a, the rest run b.
template <typename J1, typename J2>
__global__ void __launch_bounds__(256) k_pair(J1 a, int na, J2 b) {
    if ((int)blockIdx.x < na) a.run(blockIdx.x, na);
    else b.run((int)blockIdx.x - na, (int)gridDim.x - na);
}

// Per-box baseline: the entries of one destination box, one thread per cell.
template <typename E>
__global__ void k_fill_plain(E *base, const FabInfo *__restrict__ ftab, const FbEntry *__restrict__ ent, int count,
                             long long total, const int *__restrict__ cbeg) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    int lo = 0, hi = count - 1;
    while (lo < hi) {  // last entry with cbeg <= g
        int mid = (lo + hi + 1) >> 1;
        if (cbeg[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const FbEntry e = ent[lo];
    const FabInfo &sf = ftab[e.sfab];
    const FabInfo &df = ftab[e.dfab];
    unsigned l = (unsigned)(g - cbeg[lo]);
    unsigned x = l % e.n[0];
    l /= e.n[0];
    unsigned y = l % e.n[1];
    l /= e.n[1];
    unsigned z = l % e.n[2];
    unsigned c = l / e.n[2];
    base[e.dst + c * df.cstride + z * df.plane + (long long)y * df.px + x] =
        base[e.src + c * sf.cstride + z * sf.plane + (long long)y * sf.px + x];
}

// ------------------------------------------------------------------ stencil

template <typename S, typename A, int R>
__global__ void __launch_bounds__(256) k_stencil(StencilParams p) {
    for (int w = blockIdx.x; w < p.ntiles; w += gridDim.x) {
        const Tile t = p.tiles[w];
        const FabInfo f = p.ftab[t.fab];
        const long long pl = f.plane;
        const int px = f.px;
        const S *src = (const S *)p.src[f.level] + f.org + t.comp * f.cstride;
        S *dst = (S *)p.dst[f.level] + f.org + t.comp * f.cstride;
        const S *u0 = p.u0[f.level] ? (const S *)p.u0[f.level] + f.org + t.comp * f.cstride : nullptr;
        const A lam = (A)p.lam[f.level][t.comp];
        const A rka = (A)p.rk_a, rkb = (A)p.rk_b;
        for (int yy = threadIdx.y; yy < t.ty; yy += blockDim.y) {
            for (int xx = threadIdx.x; xx < t.tx; xx += blockDim.x) {
                const int x = t.x0 + xx, y = t.y0 + yy;
                const S *col = src + (long long)y * px + x;
                S *ocol = dst + (long long)y * px + x;
                A q[2 * R + 1];  // q[j] = u(x, y, z - R + j)
                int z = t.z0;
#pragma unroll
                for (int j = 0; j < 2 * R + 1; ++j) q[j] = ld<S, A>(col + (long long)(z - R + j) * pl);
                A fzm = face_flux<A, R>(q, R - 1);
                for (int k = 0; k < t.tz; ++k) {
                    z = t.z0 + k;
                    const S *c0 = col + (long long)z * pl;
                    A qx[2 * R + 1], qy[2 * R + 1];
#pragma unroll
                    for (int j = 0; j < 2 * R + 1; ++j) {
                        qx[j] = (j == R) ? q[R] : ld<S, A>(c0 + (j - R));
                        qy[j] = (j == R) ? q[R] : ld<S, A>(c0 + (long long)(j - R) * px);
                    }
                    const A fzp = face_flux<A, R>(q, R);
                    A v = update_cell<A, R>(qx, qy, fzm, fzp, q[R], lam);
                    if (u0) v = rk_combine<A>(v, ld<S, A>(u0 + (long long)z * pl + (long long)y * px + x), rka, rkb);
                    st(ocol + (long long)z * pl, v);
                    fzm = fzp;
                    if (k + 1 < t.tz) {
#pragma unroll
                        for (int j = 0; j < 2 * R; ++j) q[j] = q[j + 1];
                        q[2 * R] = ld<S, A>(col + (long long)(z + 1 + R) * pl);
                    }
                }
            }
        }
    }
}

// Untiled per-box baseline: one thread per cell, every neighbour loaded, every flux
// computed on its own (same formulas and order, hence the same bits).
template <typename S, typename A, int R>
__global__ void k_stencil_plain(const S *__restrict__ src, S *__restrict__ dst, FabInfo f, A lam) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= f.n[0] || y >= f.n[1]) return;
    const long long pl = f.plane;
    const int px = f.px;
    const S *c0 = src + f.org + (long long)z * pl + (long long)y * px + x;
    A qx[2 * R + 1], qy[2 * R + 1], qz[2 * R + 1];
#pragma unroll
    for (int j = 0; j < 2 * R + 1; ++j) {
        qx[j] = ld<S, A>(c0 + (j - R));
        qy[j] = ld<S, A>(c0 + (long long)(j - R) * px);
        qz[j] = ld<S, A>(c0 + (long long)(j - R) * pl);
    }
    const A fzm = face_flux<A, R>(qz, R - 1);
    const A fzp = face_flux<A, R>(qz, R);
    st(dst + f.org + (long long)z * pl + (long long)y * px + x, update_cell<A, R>(qx, qy, fzm, fzp, qz[R], lam));
}

// ------------------------------------------------------------------ reduction

// ------------------------------------------------------------------ refluxing
// Berger-Colella flux correction of the two-level advance, in FP64 whatever the storage:
// reg_c = lam_c * F_c per coarse face, reg_f = sum over substeps of lam_f / r^3 * (sum of the
// r^2 fine face fluxes), and every uncovered coarse cell next to the interface adds
// sum over its faces of sc * (reg_f - reg_c).  One thread per (face or cell, component), the
// sums in a fixed order.

template <typename S, int R>
__device__ __forceinline__ double line_flux(const S *low, long long dstride) {
    double q[2 * R];  // q[j] = u(low + (j - R + 1) e_d)
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) q[j] = to_f64(low[(long long)(j - R + 1) * dstride]);
    return face_flux<double, R>(q, R - 1);
}

template <typename S, int R>
struct CFluxJob {
    const S *base;
    const CFace *faces;
    int n, ncomp;
    RefluxW w;
    double *reg;
    __device__ __forceinline__ void run(int b, int nb) const {
        for (int i = b * blockDim.x + threadIdx.x; i < n * ncomp; i += nb * blockDim.x) {
            const int e = i / ncomp, c = i - e * ncomp;
            const CFace f = faces[e];
            reg[i] = __dmul_rn(w.w[c], line_flux<S, R>(base + f.c_low + c * f.cstride, f.dstride));
        }
    }
};

template <typename S, int R>
__global__ void __launch_bounds__(256) k_cf_coarse_flux(const S *__restrict__ base, const CFace *__restrict__ faces,
                                                        int n, int ncomp, RefluxW w, double *reg) {
    CFluxJob<S, R>{base, faces, n, ncomp, w, reg}.run(blockIdx.x, gridDim.x);
}

// NFF = r^2 fine faces per coarse face, a compile-time count so that all their loads issue
// before the ordered sum.
template <typename S, int R, int NFF>
__global__ void __launch_bounds__(256) k_cf_fine_flux(const S *__restrict__ base, const CFace *__restrict__ faces,
                                                      const FFace *__restrict__ ff, int n, int ncomp, RefluxW w,
                                                      double *reg, int first) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * ncomp; i += gridDim.x * blockDim.x) {
        const int e = i / ncomp, c = i - e * ncomp;
        const int f0 = faces[e].ffirst;
        double fl[NFF];
#pragma unroll
        for (int k = 0; k < NFF; ++k) {
            const FFace g = ff[f0 + k];
            fl[k] = line_flux<S, R>(base + g.f_low + c * g.cstride, g.dstride);
        }
        double sum = 0.0;
#pragma unroll
        for (int k = 0; k < NFF; ++k) sum = __dadd_rn(sum, fl[k]);
        const double v = __dmul_rn(w.w[c], sum);
        reg[i] = first ? v : __dadd_rn(reg[i], v);
    }
}

template <typename S>
struct RefluxJob {
    S *base;
    const CCell *cells;
    int ncell;
    const CFace *faces;
    int ncomp;
    const double *regc, *regf;
    __device__ __forceinline__ void run(int b, int nb) const {
        for (int i = b * blockDim.x + threadIdx.x; i < ncell * ncomp; i += nb * blockDim.x) {
            const int j = i / ncomp, c = i - j * ncomp;
            const CCell cl = cells[j];
            double corr = 0.0;
            for (int e = cl.efirst; e < cl.efirst + cl.ecount; ++e) {
                const double d = __dsub_rn(regf[(long long)e * ncomp + c], regc[(long long)e * ncomp + c]);
                corr = __dadd_rn(corr, faces[e].sc > 0 ? d : -d);
            }
            S *p = base + cl.c_elem + c * cl.cstride;
            from_f64(p, __dadd_rn(to_f64(*p), corr));
        }
    }
};

template <typename S>
__global__ void __launch_bounds__(256) k_reflux_apply(S *base, const CCell *__restrict__ cells, int ncell,
                                                      const CFace *__restrict__ faces, int ncomp,
                                                      const double *__restrict__ regc, const double *__restrict__ regf) {
    RefluxJob<S>{base, cells, ncell, faces, ncomp, regc, regf}.run(blockIdx.x, gridDim.x);
}

static int blocks_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 65535)); }

template <typename S>
static cudaError_t cf_coarse_s(int R, const void *base, const CFace *faces, int n, int ncomp, const RefluxW &w,
                               double *reg, cudaStream_t s) {
    const int g = blocks_for((long long)n * ncomp);
    switch (R) {
        case 1: k_cf_coarse_flux<S, 1><<<g, 256, 0, s>>>((const S *)base, faces, n, ncomp, w, reg); break;
        case 2: k_cf_coarse_flux<S, 2><<<g, 256, 0, s>>>((const S *)base, faces, n, ncomp, w, reg); break;
        case 4: k_cf_coarse_flux<S, 4><<<g, 256, 0, s>>>((const S *)base, faces, n, ncomp, w, reg); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S, int NFF>
static cudaError_t cf_fine_t(int R, const void *base, const CFace *faces, const FFace *ff, int n, int ncomp,
                             const RefluxW &w, double *reg, bool first, cudaStream_t s) {
    const int g = blocks_for((long long)n * ncomp);
    switch (R) {
        case 1: k_cf_fine_flux<S, 1, NFF><<<g, 256, 0, s>>>((const S *)base, faces, ff, n, ncomp, w, reg, first); break;
        case 2: k_cf_fine_flux<S, 2, NFF><<<g, 256, 0, s>>>((const S *)base, faces, ff, n, ncomp, w, reg, first); break;
        case 4: k_cf_fine_flux<S, 4, NFF><<<g, 256, 0, s>>>((const S *)base, faces, ff, n, ncomp, w, reg, first); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S>
static cudaError_t cf_fine_s(int R, const void *base, const CFace *faces, const FFace *ff, int n, int nff, int ncomp,
                             const RefluxW &w, double *reg, bool first, cudaStream_t s) {
    if (nff == 4) return cf_fine_t<S, 4>(R, base, faces, ff, n, ncomp, w, reg, first, s);
    if (nff == 16) return cf_fine_t<S, 16>(R, base, faces, ff, n, ncomp, w, reg, first, s);
    return cudaErrorInvalidValue;  // ratio 2 or 4
}

cudaError_t launch_cf_coarse_flux(int dtype, int R, const void *base, const CFace *faces, int n, int ncomp,
                                  const RefluxW &w, double *reg, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    switch (dtype) {
        case F64: return cf_coarse_s<double>(R, base, faces, n, ncomp, w, reg, s);
        case F32: return cf_coarse_s<float>(R, base, faces, n, ncomp, w, reg, s);
        case BF16: return cf_coarse_s<__nv_bfloat16>(R, base, faces, n, ncomp, w, reg, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_cf_fine_flux(int dtype, int R, const void *base, const CFace *faces, const FFace *ff, int n,
                                int nff, int ncomp, const RefluxW &w, double *reg, bool first, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    switch (dtype) {
        case F64: return cf_fine_s<double>(R, base, faces, ff, n, nff, ncomp, w, reg, first, s);
        case F32: return cf_fine_s<float>(R, base, faces, ff, n, nff, ncomp, w, reg, first, s);
        case BF16: return cf_fine_s<__nv_bfloat16>(R, base, faces, ff, n, nff, ncomp, w, reg, first, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_reflux_apply(int dtype, void *base, const CCell *cells, int ncell, const CFace *faces, int ncomp,
                                const double *regc, const double *regf, cudaStream_t s) {
    if (ncell == 0) return cudaSuccess;
    const int g = blocks_for((long long)ncell * ncomp);
    switch (dtype) {
        case F64: k_reflux_apply<<<g, 256, 0, s>>>((double *)base, cells, ncell, faces, ncomp, regc, regf); break;
        case F32: k_reflux_apply<<<g, 256, 0, s>>>((float *)base, cells, ncell, faces, ncomp, regc, regf); break;
        case BF16: k_reflux_apply<<<g, 256, 0, s>>>((__nv_bfloat16 *)base, cells, ncell, faces, ncomp, regc, regf); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Whole-level reductions of one component (Sec. 3.1: the MultiFab's sum, max and norms).  The
// valid rows of all FArrayBoxes form one list (rowpre[b] = first row of box b); warp w of the
// grid takes rows w, w + warps, ... with its lanes along x, so the accumulation order, hence the
// bits, depends only on the box layout and the fixed grid -- not on tiles or timing.
// Sums (sum, sum |u|, sum u^2) accumulate in FP64 with Neumaier compensation; max, min and
// max |u| are exact (FP64 holds every stored value; NaN values are skipped).
template <int OP> struct RedOp;
template <> struct RedOp<RED_SUM> {
    static constexpr bool sum = true;
    static __device__ __forceinline__ double val(double x) { return x; }
};
template <> struct RedOp<RED_NORM1> {
    static constexpr bool sum = true;
    static __device__ __forceinline__ double val(double x) { return ::fabs(x); }
};
template <> struct RedOp<RED_NORM2> {
    static constexpr bool sum = true;
    static __device__ __forceinline__ double val(double x) { return __dmul_rn(x, x); }
};
template <> struct RedOp<RED_MAX> {
    static constexpr bool sum = false;
    static constexpr double init = -__builtin_huge_val();
    static __device__ __forceinline__ double val(double x) { return x; }
    static __device__ __forceinline__ double pick(double a, double b) { return ::fmax(a, b); }
};
template <> struct RedOp<RED_MIN> {
    static constexpr bool sum = false;
    static constexpr double init = __builtin_huge_val();
    static __device__ __forceinline__ double val(double x) { return x; }
    static __device__ __forceinline__ double pick(double a, double b) { return ::fmin(a, b); }
};
template <> struct RedOp<RED_NORM0> {
    static constexpr bool sum = false;
    static constexpr double init = 0.0;
    static __device__ __forceinline__ double val(double x) { return ::fabs(x); }
    static __device__ __forceinline__ double pick(double a, double b) { return ::fmax(a, b); }
};

__device__ __forceinline__ double block_pick_max(double m, bool is_min) {
    for (int off = 16; off > 0; off >>= 1) {
        const double o = __shfl_down_sync(0xffffffffu, m, off);
        m = is_min ? ::fmin(m, o) : ::fmax(m, o);
    }
    __shared__ double sm[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) sm[wid] = m;
    __syncthreads();
    if (wid == 0) {
        m = lane < nw ? sm[lane] : sm[0];
        for (int off = 16; off > 0; off >>= 1) {
            const double o = __shfl_down_sync(0xffffffffu, m, off);
            m = is_min ? ::fmin(m, o) : ::fmax(m, o);
        }
    }
    return m;
}

template <typename S, int OP>
__global__ void __launch_bounds__(256) k_reduce_partial(const S *__restrict__ base, const FabInfo *__restrict__ ftab,
                                                        const long long *__restrict__ rowpre, int nfab, int comp,
                                                        double2 *partials) {
    using O = RedOp<OP>;
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long nrows = rowpre[nfab];
    double s, c = 0.0;
    if constexpr (O::sum) s = 0.0; else s = O::init;
    for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows; r += nw) {
        int lo = 0, hi = nfab - 1;  // the box holding row r: last lo with rowpre[lo] <= r
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (rowpre[mid] <= r) lo = mid; else hi = mid - 1;
        }
        const FabInfo f = ftab[lo];
        const int rr = (int)(r - rowpre[lo]);
        const int y = rr % f.n[1], z = rr / f.n[1];
        const S *p = base + f.org + comp * f.cstride + (long long)z * f.plane + (long long)y * f.px;
        for (int x = lane; x < f.n[0]; x += 32) {
            const double v = O::val(to_f64(p[x]));
            if constexpr (O::sum) neu_add(s, c, v); else s = O::pick(s, v);
        }
    }
    if constexpr (O::sum) {
        block_reduce(s, c);
    } else {
        s = block_pick_max(s, OP == RED_MIN);
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = make_double2(s, c);
}

template <int OP>
__global__ void __launch_bounds__(256) k_reduce_final(const double2 *partials, int n, double *out) {
    using O = RedOp<OP>;
    if constexpr (O::sum) {
        double s = 0.0, c = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) neu_merge(s, c, partials[i].x, partials[i].y);
        block_reduce(s, c);
        if (threadIdx.x == 0) out[0] = OP == RED_NORM2 ? __dsqrt_rn(__dadd_rn(s, c)) : __dadd_rn(s, c);
    } else {
        double m = O::init;
        for (int i = threadIdx.x; i < n; i += blockDim.x) m = O::pick(m, partials[i].x);
        m = block_pick_max(m, OP == RED_MIN);
        if (threadIdx.x == 0) out[0] = m;
    }
}

// ------------------------------------------------------------------ dense staging

__global__ void k_fill_nan(double *p, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = __longlong_as_double(0x7ff8000000000000LL);
}

struct DenseChunk {
    int dlo[3], dn[3];
    int z0, z1;       // global z range [z0, z1) held by the stage
    int comp, nc;     // components [comp, comp + nc) held by the stage
};

template <typename S, bool kScatter>
__global__ void k_dense(S *base, const FabInfo *__restrict__ ftab, double *stage, DenseChunk d) {
    const FabInfo f = ftab[blockIdx.y];
    const int zlo = max(f.lo[2], d.z0), zhi = min(f.lo[2] + f.n[2], d.z1);
    if (zlo >= zhi) return;
    const int nz = zhi - zlo, ny = f.n[1];
    const long long rows = (long long)nz * ny * d.nc;
    const long long zs = (long long)(d.z1 - d.z0) * d.dn[1] * d.dn[0];
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        const int y = (int)(r % ny);
        const int z = (int)((r / ny) % nz) + zlo;
        const int cc = (int)(r / ((long long)ny * nz));
        S *frow = base + f.org + (long long)(d.comp + cc) * f.cstride + (long long)(z - f.lo[2]) * f.plane +
                  (long long)y * f.px;
        double *srow = stage + cc * zs + ((long long)(z - d.z0) * d.dn[1] + (y + f.lo[1] - d.dlo[1])) * d.dn[0] +
                       (f.lo[0] - d.dlo[0]);
        for (int x = threadIdx.x; x < f.n[0]; x += blockDim.x) {
            if (kScatter) from_f64(frow + x, srow[x]);
            else srow[x] = to_f64(frow[x]);
        }
    }
}

// ------------------------------------------------------------------ AMR

template <typename A, typename S> __device__ __forceinline__ A to_arith(S v) {
    if constexpr (std::is_same<S, __nv_bfloat16>::value) return (A)__bfloat162float(v);
    else return (A)v;
}

// Cells numbered 0..ncells-1 form consecutive non-empty segments (runs, regions); segment q
// holds [start[q], start[q+1]) and start[nseg] = ncells.  first is the segment holding cell
// c0 = 32 w.  For the calling lane's cell c0 + lane this returns its segment and its offset in
// it, with one coalesced load and one warp reduction: the lanes mark, in a 32-bit mask, the
// window positions where a segment starts; a lane's segment is first plus the number of marks
// at or below it, less one.  Whole-warp call.
__device__ __forceinline__ void warp_segment(const int *__restrict__ start, int first, int nseg, int ncells, int c0,
                                             int &seg, int &off) {
    const int lane = threadIdx.x & 31;
    const int s = first + lane <= nseg ? __ldg(start + first + lane) : ncells;
    const unsigned bit = lane == 0 ? 1u : (s - c0 < 32 ? 1u << (s - c0) : 0u);
    const unsigned m = __reduce_or_sync(0xffffffffu, bit);
    const unsigned le = m & (0xffffffffu >> (31 - lane));
    const int k = __popc(le) - 1;
    const int s0 = __shfl_sync(0xffffffffu, s, 0);
    seg = first + k;
    off = k == 0 ? c0 + lane - s0 : lane - (31 - __clz(le));
}

// Linear-interpolation stencil of fine index i at ratio r: coarse k0 and weight of k0+1
// from the cell-centre position x = (2i + 1 - r) / (2r) in coarse index units.  The weight
// is a multiple of 1/(2r), exact in FP32 and FP64.
template <typename A>
__device__ __forceinline__ void lin_w(int i, int r, int &k0, A &w1) {
    const int num = 2 * i + 1 - r, den = 2 * r;
    int q = num / den;
    if (num % den != 0 && num < 0) --q;
    k0 = q;
    w1 = (A)(num - den * q) / (A)den;
}

// Coarse-to-fine ghost interpolation (Sec. 2.3): one thread per fine ghost cell of the work
// list, trilinear in space and linear in time, (1 - alpha) cold + alpha cnew at each of the 8
// coarse points, accumulated z, y, x ascending with the weight product (wz wy) wx -- the
// arithmetic of the storage type's native precision (FP64 for FP64, FP32 otherwise).
template <typename S>
struct InterpJob {
    S *fbase;
    const S *cold, *cnew;
    const InterpRun *runs;
    const int *rstart, *wfirst;
    int nruns, ncells, ncomp, ratio;
    double alpha;
    __device__ __forceinline__ void run(int b, int nb) const {
        using A = typename NativeArith<S>::T;
        using O = Ar<A>;
        const A a1 = (A)alpha, a0 = (A)(1.0 - alpha);
        // at alpha = 0 the new coarse level is not read: the first substep of a coarse step may
        // run while that level is being computed (its value would only be scaled by 0)
        const bool tnew = alpha != 0.0;
        const int nw = (ncells + 31) >> 5;
        const int lane = threadIdx.x & 31;
        for (int w = (b * blockDim.x + threadIdx.x) >> 5; w < nw; w += (nb * blockDim.x) >> 5) {
            int q, t;
            warp_segment(rstart, __ldg(wfirst + w), nruns, ncells, w << 5, q, t);
            if ((w << 5) + lane >= ncells) continue;
            const InterpRun run = runs[q];
            int ix[3] = {run.I, run.J, run.K};
            ix[run.axis] += t;
            int kx, ky, kz;
            A wx1, wy1, wz1;
            lin_w(ix[0], ratio, kx, wx1);
            lin_w(ix[1], ratio, ky, wy1);
            lin_w(ix[2], ratio, kz, wz1);
            const A wx[2] = {O::sub((A)1, wx1), wx1}, wy[2] = {O::sub((A)1, wy1), wy1},
                    wz[2] = {O::sub((A)1, wz1), wz1};
            const long long cb = run.cbase + (long long)kz * run.cplane + (long long)ky * run.cpx + kx;
            S *fo = fbase + run.fdst + (long long)t * run.fstep;
            for (int c = 0; c < ncomp; ++c) {
                const S *po = cold + cb + (long long)c * run.ccs, *pn = cnew + cb + (long long)c * run.ccs;
                A v = (A)0;
#pragma unroll
                for (int dz = 0; dz < 2; ++dz)
#pragma unroll
                    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                        for (int dx = 0; dx < 2; ++dx) {
                            const int o = dz * run.cplane + dy * run.cpx + dx;
                            const A tv = tnew ? O::add(O::mul(a0, ld<S, A>(po + o)), O::mul(a1, ld<S, A>(pn + o)))
                                              : O::mul(a0, ld<S, A>(po + o));
                            v = O::add(v, O::mul(O::mul(O::mul(wz[dz], wy[dy]), wx[dx]), tv));
                        }
                st(fo + (long long)c * run.fcs, v);
            }
        }
    }
};

template <typename S>
__global__ void __launch_bounds__(256) k_interp(S *__restrict__ fbase, const S *__restrict__ cold,
                                                const S *__restrict__ cnew, const InterpRun *__restrict__ runs,
                                                const int *__restrict__ rstart, const int *__restrict__ wfirst,
                                                int nruns, int ncells, int ncomp, int ratio, double alpha) {
    InterpJob<S>{fbase, cold, cnew, runs, rstart, wfirst, nruns, ncells, ncomp, ratio, alpha}.run(blockIdx.x,
                                                                                                   gridDim.x);
}

// Vector load of the RR consecutive fine children along x (RR * sizeof(S) bytes, aligned to
// that size, or to 16 bytes above it), or RR scalar loads.
template <int B> struct LdVec;
template <> struct LdVec<2> { using T = unsigned short; };
template <> struct LdVec<4> { using T = unsigned int; };
template <> struct LdVec<8> { using T = uint2; };
template <> struct LdVec<16> { using T = uint4; };

template <typename S, int RR, bool VEC>
__device__ __forceinline__ void ld_children(const S *p, S (&v)[RR]) {
    constexpr int B = RR * (int)sizeof(S);
    if constexpr (!VEC) {
#pragma unroll
        for (int i = 0; i < RR; ++i) v[i] = __ldg(p + i);
    } else if constexpr (B <= 16) {
        const typename LdVec<B>::T t = __ldg(reinterpret_cast<const typename LdVec<B>::T *>(p));
        memcpy(v, &t, B);
    } else {
        uint4 t[B / 16];
#pragma unroll
        for (int i = 0; i < B / 16; ++i) t[i] = __ldg(reinterpret_cast<const uint4 *>(p) + i);
        memcpy(v, t, B);
    }
}

// Average-down (Sec. 2.3): one thread per coarse cell of the work list, the mean of its RR^3
// fine children summed z, y, x ascending, times 1/RR^3 (a power of two: the same value as
// the division), in the storage type's native precision.  Consecutive lanes take consecutive
// coarse x, so each fine row is read as one contiguous span per warp.  A warp takes U
// consecutive 32-cell chunks at a time with all their loads issued before the sums.
template <typename S, int RR, bool VEC, int U>
struct AvgJob {
    const S *fbase;
    S *cbase;
    const AvgRegion *regs;
    const int *rstart, *wfirst;
    int nregs, ncells, ncomp;
    __device__ __forceinline__ void run(int b, int nb) const {
        using A = typename NativeArith<S>::T;
        using O = Ar<A>;
        const A inv = (A)(1.0 / (double)(RR * RR * RR));
        const int nw = (ncells + 31) >> 5;
        const int lane = threadIdx.x & 31;
        const int nwarps = (nb * blockDim.x) >> 5;
        for (int w0 = ((b * blockDim.x + threadIdx.x) >> 5) * U; w0 < nw; w0 += nwarps * U) {
            bool act[U];
            const S *fp[U];
            S *cp[U];
            int fpl[U], fpx[U], fcs[U], ccs[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int w = w0 + u;
                act[u] = false;
                if (w >= nw) continue;  // warp-uniform
                int q, t;
                warp_segment(rstart, __ldg(wfirst + w), nregs, ncells, w << 5, q, t);
                if ((w << 5) + lane >= ncells) continue;
                const AvgRegion rg = regs[q];
                const int x = t % rg.n[0], yz = t / rg.n[0];
                const int y = yz % rg.n[1], z = yz / rg.n[1];
                fp[u] = fbase + rg.fsrc + (long long)z * RR * rg.fplane + (long long)y * RR * rg.fpx + x * RR;
                cp[u] = cbase + rg.cdst + (long long)z * rg.cplane + (long long)y * rg.cpx + x;
                fpl[u] = rg.fplane;
                fpx[u] = rg.fpx;
                fcs[u] = rg.fcs;
                ccs[u] = rg.ccs;
                act[u] = true;
            }
            for (int c = 0; c < ncomp; ++c) {
                S v[U][RR * RR][RR];
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (act[u]) {
                        const S *fc = fp[u] + (long long)c * fcs[u];
#pragma unroll
                        for (int r = 0; r < RR * RR; ++r)
                            ld_children<S, RR, VEC>(fc + (long long)(r / RR) * fpl[u] + (long long)(r % RR) * fpx[u],
                                                    v[u][r]);
                    }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (act[u]) {
                        A sum = (A)0;
#pragma unroll
                        for (int r = 0; r < RR * RR; ++r)
#pragma unroll
                            for (int dx = 0; dx < RR; ++dx) sum = O::add(sum, to_arith<A>(v[u][r][dx]));
                        st(cp[u] + (long long)c * ccs[u], O::mul(sum, inv));
                    }
            }
        }
    }
};

template <typename S, int RR, bool VEC, int U>
__global__ void __launch_bounds__(256) k_avgdown(const S *__restrict__ fbase, S *__restrict__ cbase,
                                                 const AvgRegion *__restrict__ regs, const int *__restrict__ rstart,
                                                 const int *__restrict__ wfirst, int nregs, int ncells, int ncomp) {
    AvgJob<S, RR, VEC, U>{fbase, cbase, regs, rstart, wfirst, nregs, ncells, ncomp}.run(blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------------ launchers

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    }
    return n;
}

template <typename K>
static int persistent_grid(K kernel, int block, int work) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    long long g = (long long)per_sm * sm_count();
    if (work < g) g = work;
    return g < 1 ? 1 : (int)g;
}

cudaError_t launch_fill(int dtype, const LevelPtrs &lv, const FbTask *tasks, int ntasks, int grid, cudaStream_t s) {
    if (ntasks == 0) return cudaSuccess;
    switch (dtype_size(dtype)) {
        case 8: {
            int g = grid > 0 ? grid : persistent_grid(k_fill<unsigned long long>, 256, (ntasks + 7) / 8);
            k_fill<unsigned long long><<<g, 256, 0, s>>>(lv, tasks, ntasks);
            break;
        }
        case 4: {
            int g = grid > 0 ? grid : persistent_grid(k_fill<unsigned int>, 256, (ntasks + 7) / 8);
            k_fill<unsigned int><<<g, 256, 0, s>>>(lv, tasks, ntasks);
            break;
        }
        default: {
            int g = grid > 0 ? grid : persistent_grid(k_fill<unsigned short>, 256, (ntasks + 7) / 8);
            k_fill<unsigned short><<<g, 256, 0, s>>>(lv, tasks, ntasks);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_fill_plain(int dtype, void *base, const FabInfo *ftab, const FbEntry *ent, int count,
                              long long total, const int *cbeg, cudaStream_t s) {
    if (total == 0) return cudaSuccess;
    const int blocks = (int)((total + 255) / 256);
    switch (dtype_size(dtype)) {
        case 8: k_fill_plain<<<blocks, 256, 0, s>>>((unsigned long long *)base, ftab, ent, count, total, cbeg); break;
        case 4: k_fill_plain<<<blocks, 256, 0, s>>>((unsigned int *)base, ftab, ent, count, total, cbeg); break;
        default: k_fill_plain<<<blocks, 256, 0, s>>>((unsigned short *)base, ftab, ent, count, total, cbeg);
    }
    return cudaGetLastError();
}

template <typename S, typename A, int R>
static cudaError_t stencil_t(const StencilParams &p, int bx, int by, int grid, cudaStream_t s) {
    dim3 block(bx, by);
    int g = grid > 0 ? grid : persistent_grid(k_stencil<S, A, R>, bx * by, p.ntiles);
    k_stencil<S, A, R><<<g, block, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename S, typename A>
static cudaError_t stencil_r(int R, const StencilParams &p, int bx, int by, int grid, cudaStream_t s) {
    switch (R) {
        case 1: return stencil_t<S, A, 1>(p, bx, by, grid, s);
        case 2: return stencil_t<S, A, 2>(p, bx, by, grid, s);
        case 4: return stencil_t<S, A, 4>(p, bx, by, grid, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_stencil(int dtype, int R, bool fp64diff, const StencilParams &p, int bx, int by, int grid,
                           cudaStream_t s) {
    if (p.ntiles == 0) return cudaSuccess;
    if (bx * by > 256 || bx <= 0 || by <= 0) return cudaErrorInvalidValue;
    switch (dtype) {
        case F64: return stencil_r<double, double>(R, p, bx, by, grid, s);
        case F32: return fp64diff ? stencil_r<float, double>(R, p, bx, by, grid, s)
                                  : stencil_r<float, float>(R, p, bx, by, grid, s);
        case BF16: return fp64diff ? stencil_r<__nv_bfloat16, double>(R, p, bx, by, grid, s)
                                   : stencil_r<__nv_bfloat16, float>(R, p, bx, by, grid, s);
    }
    return cudaErrorInvalidValue;
}

template <typename S, typename A, int R>
static cudaError_t plain_t(const void *src, void *dst, const FabInfo &f, double lam, int comp, cudaStream_t s) {
    dim3 block(32, 4);
    dim3 grid((f.n[0] + 31) / 32, (f.n[1] + 3) / 4, f.n[2]);
    const long long off = (long long)comp * f.cstride;
    k_stencil_plain<S, A, R><<<grid, block, 0, s>>>((const S *)src + off, (S *)dst + off, f, (A)lam);
    return cudaGetLastError();
}

template <typename S, typename A>
static cudaError_t plain_r(int R, const void *src, void *dst, const FabInfo &f, double lam, int comp,
                           cudaStream_t s) {
    switch (R) {
        case 1: return plain_t<S, A, 1>(src, dst, f, lam, comp, s);
        case 2: return plain_t<S, A, 2>(src, dst, f, lam, comp, s);
        case 4: return plain_t<S, A, 4>(src, dst, f, lam, comp, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_stencil_plain(int dtype, int R, const void *src, void *dst, const FabInfo &f, double lam, int comp,
                                 cudaStream_t s) {
    switch (dtype) {
        case F64: return plain_r<double, double>(R, src, dst, f, lam, comp, s);
        case F32: return plain_r<float, float>(R, src, dst, f, lam, comp, s);
        case BF16: return plain_r<__nv_bfloat16, float>(R, src, dst, f, lam, comp, s);
    }
    return cudaErrorInvalidValue;
}

template <typename S, int OP>
static cudaError_t reduce_t(const void *base, const FabInfo *ftab, const long long *rowpre, int nfab, int comp,
                            double2 *partials, int grid, double *out_dev, cudaStream_t s) {
    k_reduce_partial<S, OP><<<grid, 256, 0, s>>>((const S *)base, ftab, rowpre, nfab, comp, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<OP><<<1, 256, 0, s>>>(partials, grid, out_dev);
    return cudaGetLastError();
}

template <typename S>
static cudaError_t reduce_s(int op, const void *base, const FabInfo *ftab, const long long *rowpre, int nfab,
                            int comp, double2 *partials, int grid, double *out_dev, cudaStream_t s) {
    switch (op) {
        case RED_SUM: return reduce_t<S, RED_SUM>(base, ftab, rowpre, nfab, comp, partials, grid, out_dev, s);
        case RED_MAX: return reduce_t<S, RED_MAX>(base, ftab, rowpre, nfab, comp, partials, grid, out_dev, s);
        case RED_MIN: return reduce_t<S, RED_MIN>(base, ftab, rowpre, nfab, comp, partials, grid, out_dev, s);
        case RED_NORM0: return reduce_t<S, RED_NORM0>(base, ftab, rowpre, nfab, comp, partials, grid, out_dev, s);
        case RED_NORM1: return reduce_t<S, RED_NORM1>(base, ftab, rowpre, nfab, comp, partials, grid, out_dev, s);
        case RED_NORM2: return reduce_t<S, RED_NORM2>(base, ftab, rowpre, nfab, comp, partials, grid, out_dev, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_reduce(int dtype, int op, const void *base, const FabInfo *ftab, const long long *rowpre, int nfab,
                          int comp, double2 *partials, int grid, double *out_dev, cudaStream_t s) {
    switch (dtype) {
        case F64: return reduce_s<double>(op, base, ftab, rowpre, nfab, comp, partials, grid, out_dev, s);
        case F32: return reduce_s<float>(op, base, ftab, rowpre, nfab, comp, partials, grid, out_dev, s);
        case BF16: return reduce_s<__nv_bfloat16>(op, base, ftab, rowpre, nfab, comp, partials, grid, out_dev, s);
    }
    return cudaErrorInvalidValue;
}

static cudaError_t dense_common(bool scatter, int dtype, void *base, const FabInfo *ftab, int nfab, double *stage,
                                const int dlo[3], const int dn[3], int z0, int z1, int comp, int nc, cudaStream_t s) {
    DenseChunk d;
    for (int i = 0; i < 3; ++i) { d.dlo[i] = dlo[i]; d.dn[i] = dn[i]; }
    d.z0 = z0; d.z1 = z1; d.comp = comp; d.nc = nc;
    if (!scatter) {
        long long n = (long long)nc * (z1 - z0) * dn[1] * dn[0];
        k_fill_nan<<<4 * sm_count(), 256, 0, s>>>(stage, n);
    }
    dim3 grid(64, nfab);
    switch (dtype) {
        case F64:
            if (scatter) k_dense<double, true><<<grid, 128, 0, s>>>((double *)base, ftab, stage, d);
            else k_dense<double, false><<<grid, 128, 0, s>>>((double *)base, ftab, stage, d);
            break;
        case F32:
            if (scatter) k_dense<float, true><<<grid, 128, 0, s>>>((float *)base, ftab, stage, d);
            else k_dense<float, false><<<grid, 128, 0, s>>>((float *)base, ftab, stage, d);
            break;
        default:
            if (scatter) k_dense<__nv_bfloat16, true><<<grid, 128, 0, s>>>((__nv_bfloat16 *)base, ftab, stage, d);
            else k_dense<__nv_bfloat16, false><<<grid, 128, 0, s>>>((__nv_bfloat16 *)base, ftab, stage, d);
    }
    return cudaGetLastError();
}

cudaError_t launch_scatter_dense(int dtype, void *base, const FabInfo *ftab, int nfab, const double *stage,
                                 const int dlo[3], const int dn[3], int z0, int z1, int comp, int nc, cudaStream_t s) {
    return dense_common(true, dtype, base, ftab, nfab, const_cast<double *>(stage), dlo, dn, z0, z1, comp, nc, s);
}

cudaError_t launch_gather_dense(int dtype, const void *base, const FabInfo *ftab, int nfab, double *stage,
                                const int dlo[3], const int dn[3], int z0, int z1, int comp, int nc, cudaStream_t s) {
    return dense_common(false, dtype, const_cast<void *>(base), ftab, nfab, stage, dlo, dn, z0, z1, comp, nc, s);
}

cudaError_t launch_interp(int dtype, void *fbase, const void *cold, const void *cnew, const InterpRun *runs,
                          const int *rstart, const int *wfirst, int nruns, int ncells, int ncomp, int ratio,
                          double alpha, cudaStream_t s) {
    if (ncells == 0) return cudaSuccess;
    const int blocks = (int)(((long long)ncells + 255) / 256);
    switch (dtype) {
        case F64: {
            const int g = persistent_grid(k_interp<double>, 256, blocks);
            k_interp<double><<<g, 256, 0, s>>>((double *)fbase, (const double *)cold, (const double *)cnew,
                                                         runs, rstart, wfirst, nruns, ncells, ncomp, ratio, alpha);
            break;
        }
        case F32: {
            const int g = persistent_grid(k_interp<float>, 256, blocks);
            k_interp<float><<<g, 256, 0, s>>>((float *)fbase, (const float *)cold, (const float *)cnew, runs,
                                                        rstart, wfirst, nruns, ncells, ncomp, ratio, alpha);
            break;
        }
        default: {
            const int g = persistent_grid(k_interp<__nv_bfloat16>, 256, blocks);
            k_interp<__nv_bfloat16><<<g, 256, 0, s>>>((__nv_bfloat16 *)fbase, (const __nv_bfloat16 *)cold,
                                                                (const __nv_bfloat16 *)cnew, runs, rstart, wfirst,
                                                                nruns, ncells, ncomp, ratio, alpha);
        }
    }
    return cudaGetLastError();
}

template <typename S, int RR, bool VEC>
static void avgdown_t(const void *fbase, void *cbase, const AvgRegion *regs, const int *rstart, const int *wfirst,
                      int nregs, int ncells, int ncomp, cudaStream_t s) {
    const int blocks = (int)(((long long)ncells + 255) / 256);
    constexpr int U = RR == 2 ? 2 : 1;
    const int g = persistent_grid(k_avgdown<S, RR, VEC, U>, 256, blocks);
    k_avgdown<S, RR, VEC, U><<<g, 256, 0, s>>>((const S *)fbase, (S *)cbase, regs, rstart, wfirst, nregs, ncells,
                                               ncomp);
}

template <typename S>
static void avgdown_s(const void *fbase, void *cbase, const AvgRegion *regs, const int *rstart, const int *wfirst,
                      int nregs, int ncells, int ncomp, int ratio, bool vec, cudaStream_t s) {
    if (ratio == 2) {
        if (vec) avgdown_t<S, 2, true>(fbase, cbase, regs, rstart, wfirst, nregs, ncells, ncomp, s);
        else avgdown_t<S, 2, false>(fbase, cbase, regs, rstart, wfirst, nregs, ncells, ncomp, s);
    } else {
        if (vec) avgdown_t<S, 4, true>(fbase, cbase, regs, rstart, wfirst, nregs, ncells, ncomp, s);
        else avgdown_t<S, 4, false>(fbase, cbase, regs, rstart, wfirst, nregs, ncells, ncomp, s);
    }
}

cudaError_t launch_avgdown(int dtype, const void *fbase, void *cbase, const AvgRegion *regs, const int *rstart,
                           const int *wfirst, int nregs, int ncells, int ncomp, int ratio, bool vec, cudaStream_t s) {
    if (ncells == 0) return cudaSuccess;
    if (ratio != 2 && ratio != 4) return cudaErrorInvalidValue;
    switch (dtype) {
        case F64: avgdown_s<double>(fbase, cbase, regs, rstart, wfirst, nregs, ncells, ncomp, ratio, vec, s); break;
        case F32: avgdown_s<float>(fbase, cbase, regs, rstart, wfirst, nregs, ncells, ncomp, ratio, vec, s); break;
        default:
            avgdown_s<__nv_bfloat16>(fbase, cbase, regs, rstart, wfirst, nregs, ncells, ncomp, ratio, vec, s);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ paired launches
// Two independent jobs of the two-level advance in one launch, each with the block count its
// own launch would have; an empty job leaves the other to its own launcher.

template <typename K>
static int job_grid(K kernel, int blocks) {
    return persistent_grid(kernel, 256, blocks);
}

template <typename J1, typename J2>
static cudaError_t launch_pair(const J1 &a, int na, const J2 &b, int nb, cudaStream_t s) {
    k_pair<J1, J2><<<na + nb, 256, 0, s>>>(a, na, b);
    return cudaGetLastError();
}

template <typename E, typename S>
static cudaError_t fill_interp_t(const LevelPtrs &lv, const FbTask *tasks, int ntasks, const InterpArgs &ia,
                                 cudaStream_t s) {
    const FillJob<E> a{lv, tasks, ntasks};
    const InterpJob<S> b{(S *)ia.fbase, (const S *)ia.cold, (const S *)ia.cnew, ia.runs, ia.rstart, ia.wfirst,
                         ia.nruns, ia.ncells, ia.ncomp, ia.ratio, ia.alpha};
    return launch_pair(a, job_grid(k_fill<E>, (ntasks + 7) / 8), b,
                       job_grid(k_interp<S>, (int)(((long long)ia.ncells + 255) / 256)), s);
}

cudaError_t launch_fill_interp(int dtype, const LevelPtrs &lv, const FbTask *tasks, int ntasks, const InterpArgs &ia,
                               cudaStream_t s) {
    if (ntasks == 0)
        return launch_interp(dtype, ia.fbase, ia.cold, ia.cnew, ia.runs, ia.rstart, ia.wfirst, ia.nruns, ia.ncells,
                             ia.ncomp, ia.ratio, ia.alpha, s);
    if (ia.ncells == 0) return launch_fill(dtype, lv, tasks, ntasks, 0, s);
    switch (dtype) {
        case F64: return fill_interp_t<unsigned long long, double>(lv, tasks, ntasks, ia, s);
        case F32: return fill_interp_t<unsigned int, float>(lv, tasks, ntasks, ia, s);
        case BF16: return fill_interp_t<unsigned short, __nv_bfloat16>(lv, tasks, ntasks, ia, s);
    }
    return cudaErrorInvalidValue;
}

template <typename E, typename S, int R>
static cudaError_t fill_cflux_t(const LevelPtrs &lv, const FbTask *tasks, int ntasks, const void *cbase,
                                const CFace *faces, int nface, int ncomp, const RefluxW &w, double *reg,
                                cudaStream_t s) {
    const FillJob<E> a{lv, tasks, ntasks};
    const CFluxJob<S, R> b{(const S *)cbase, faces, nface, ncomp, w, reg};
    return launch_pair(a, job_grid(k_fill<E>, (ntasks + 7) / 8), b, blocks_for((long long)nface * ncomp), s);
}

template <typename E, typename S>
static cudaError_t fill_cflux_s(int R, const LevelPtrs &lv, const FbTask *tasks, int ntasks, const void *cbase,
                                const CFace *faces, int nface, int ncomp, const RefluxW &w, double *reg,
                                cudaStream_t s) {
    switch (R) {
        case 1: return fill_cflux_t<E, S, 1>(lv, tasks, ntasks, cbase, faces, nface, ncomp, w, reg, s);
        case 2: return fill_cflux_t<E, S, 2>(lv, tasks, ntasks, cbase, faces, nface, ncomp, w, reg, s);
        case 4: return fill_cflux_t<E, S, 4>(lv, tasks, ntasks, cbase, faces, nface, ncomp, w, reg, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_fill_cflux(int dtype, int R, const LevelPtrs &lv, const FbTask *tasks, int ntasks,
                              const void *cbase, const CFace *faces, int nface, int ncomp, const RefluxW &w,
                              double *reg, cudaStream_t s) {
    if (ntasks == 0) return launch_cf_coarse_flux(dtype, R, cbase, faces, nface, ncomp, w, reg, s);
    if (nface == 0) return launch_fill(dtype, lv, tasks, ntasks, 0, s);
    switch (dtype) {
        case F64: return fill_cflux_s<unsigned long long, double>(R, lv, tasks, ntasks, cbase, faces, nface, ncomp, w, reg, s);
        case F32: return fill_cflux_s<unsigned int, float>(R, lv, tasks, ntasks, cbase, faces, nface, ncomp, w, reg, s);
        case BF16:
            return fill_cflux_s<unsigned short, __nv_bfloat16>(R, lv, tasks, ntasks, cbase, faces, nface, ncomp, w, reg, s);
    }
    return cudaErrorInvalidValue;
}

template <typename S, int RR, bool VEC>
static cudaError_t avg_reflux_t(const AvgArgs &aa, const RefluxArgs &ra, cudaStream_t s) {
    constexpr int U = RR == 2 ? 2 : 1;
    const AvgJob<S, RR, VEC, U> a{(const S *)aa.fbase, (S *)aa.cbase, aa.regs, aa.rstart, aa.wfirst, aa.nregs,
                                  aa.ncells, aa.ncomp};
    const RefluxJob<S> b{(S *)ra.base, ra.cells, ra.ncell, ra.faces, ra.ncomp, ra.regc, ra.regf};
    return launch_pair(a, job_grid(k_avgdown<S, RR, VEC, U>, (int)(((long long)aa.ncells + 255) / 256)), b,
                       blocks_for((long long)ra.ncell * ra.ncomp), s);
}

template <typename S>
static cudaError_t avg_reflux_s(const AvgArgs &aa, const RefluxArgs &ra, cudaStream_t s) {
    if (aa.ratio == 2) return aa.vec ? avg_reflux_t<S, 2, true>(aa, ra, s) : avg_reflux_t<S, 2, false>(aa, ra, s);
    return aa.vec ? avg_reflux_t<S, 4, true>(aa, ra, s) : avg_reflux_t<S, 4, false>(aa, ra, s);
}

cudaError_t launch_avg_reflux(int dtype, const AvgArgs &aa, const RefluxArgs &ra, cudaStream_t s) {
    if (ra.ncell == 0)
        return launch_avgdown(dtype, aa.fbase, aa.cbase, aa.regs, aa.rstart, aa.wfirst, aa.nregs, aa.ncells, aa.ncomp,
                              aa.ratio, aa.vec, s);
    if (aa.ncells == 0)
        return launch_reflux_apply(dtype, ra.base, ra.cells, ra.ncell, ra.faces, ra.ncomp, ra.regc, ra.regf, s);
    if (aa.ratio != 2 && aa.ratio != 4) return cudaErrorInvalidValue;
    switch (dtype) {
        case F64: return avg_reflux_s<double>(aa, ra, s);
        case F32: return avg_reflux_s<float>(aa, ra, s);
        case BF16: return avg_reflux_s<__nv_bfloat16>(aa, ra, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace mfk
