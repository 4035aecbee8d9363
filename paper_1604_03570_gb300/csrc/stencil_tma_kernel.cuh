// stencil_tma_kernel.cuh -- the flux-form stencil sweep (Sec. 4.1) over the logical-tile work list
// (Sec. 3.2), staged through shared memory by the Tensor Memory Accelerator.
//
// One persistent CTA takes tiles (box, component, x/y/z extent) from the work list.  For a
// tile it streams the z-planes of the tile plus R halo planes on each side: plane p is one
// cp.async.bulk.tensor load of (BX x (ty + 2R)) elements -- the tile's rows with their x/y
// halo, read from the FArrayBox (ghost cells included) -- into a ring of NS shared-memory
// slots, completion signalled on one mbarrier per slot.  Thread 0 keeps NS planes in flight;
// every thread owns up to CPT (x, y) cells of the tile and marches them along z with a
// register queue of 2R+1 values, so the lower z-face flux is the previous cell's upper one.
// x and y neighbours come from the centre plane in shared memory.  The per-cell arithmetic
// (face fluxes, then their divergence, then u + lam * div) is the same expression, in the
// same order, as the untiled kernel, so every tile shape gives identical bits.
//
// Every mbarrier wait is bounded (about one second of clock64 cycles); on expiry the CTA
// sets the error word, drains its own copies (again bounded) and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "fixed_diff.cuh"
#include "mf_internal.h"
#include "stencil_common.cuh"

namespace mfk {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false after ~kWaitCycles without completion.
constexpr long long kWaitCycles = 2000000000LL;
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z,
                                            int c) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(c), "r"(smem_u32(bar))
        : "memory");
}

// 16-byte vectors of the storage type: VX elements, converted to the arithmetic type.
template <typename S> struct V16;
template <> struct V16<double> {
    static constexpr int n = 2;
    template <typename A> static __device__ __forceinline__ void ld(const double *p, A *o) {
        const double2 v = *(const double2 *)p;
        o[0] = (A)v.x; o[1] = (A)v.y;
    }
    static __device__ __forceinline__ void st(double *p, const double *v) { *(double2 *)p = make_double2(v[0], v[1]); }
};
template <> struct V16<float> {
    static constexpr int n = 4;
    template <typename A> static __device__ __forceinline__ void ld(const float *p, A *o) {
        const float4 v = *(const float4 *)p;
        o[0] = (A)v.x; o[1] = (A)v.y; o[2] = (A)v.z; o[3] = (A)v.w;
    }
    static __device__ __forceinline__ void st(float *p, const float *v) {
        *(float4 *)p = make_float4(v[0], v[1], v[2], v[3]);
    }
    static __device__ __forceinline__ void st(float *p, const double *v) {
        *(float4 *)p = make_float4(__double2float_rn(v[0]), __double2float_rn(v[1]), __double2float_rn(v[2]),
                                   __double2float_rn(v[3]));
    }
};
template <> struct V16<__nv_bfloat16> {
    static constexpr int n = 8;
    template <typename A> static __device__ __forceinline__ void ld(const __nv_bfloat16 *p, A *o) {
        const uint4 v = *(const uint4 *)p;
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            o[2 * i] = (A)__uint_as_float(w[i] << 16);
            o[2 * i + 1] = (A)__uint_as_float(w[i] & 0xffff0000u);
        }
    }
    template <typename A> static __device__ __forceinline__ void st(__nv_bfloat16 *p, const A *v) {
        __nv_bfloat16 b[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) mfk::st(&b[i], v[i]);
        *(uint4 *)p = *(const uint4 *)b;
    }
};

template <> struct V16<long long> {  // the fixed-point path's 64-bit integers
    static constexpr int n = 2;
    template <typename A> static __device__ __forceinline__ void ld(const long long *p, A *o) {
        const longlong2 v = *(const longlong2 *)p;
        o[0] = (A)v.x; o[1] = (A)v.y;
    }
    static __device__ __forceinline__ void st(long long *p, const long long *v) {
        *(longlong2 *)p = make_longlong2(v[0], v[1]);
    }
};

// Groups of a thread's row: GB = 16 bytes (V16), or GB = 32 bytes -- one whole 32-byte
// sector, stored with one 256-bit store -- for FP32 and FP64 storage.
template <typename S, int GB> struct VG;
template <typename S> struct VG<S, 16> : V16<S> {};
template <> struct VG<float, 32> {
    static constexpr int n = 8;
    template <typename A> static __device__ __forceinline__ void ld(const float *p, A *o) {
        V16<float>::ld(p, o);
        V16<float>::ld(p + 4, o + 4);
    }
    static __device__ __forceinline__ void st8(float *p, float a0, float a1, float a2, float a3, float a4, float a5,
                                               float a6, float a7) {
        asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(a0), "f"(a1), "f"(a2),
                     "f"(a3), "f"(a4), "f"(a5), "f"(a6), "f"(a7)
                     : "memory");
    }
    static __device__ __forceinline__ void st(float *p, const float *v) {
        st8(p, v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7]);
    }
    static __device__ __forceinline__ void st(float *p, const double *v) {
        st8(p, __double2float_rn(v[0]), __double2float_rn(v[1]), __double2float_rn(v[2]), __double2float_rn(v[3]),
            __double2float_rn(v[4]), __double2float_rn(v[5]), __double2float_rn(v[6]), __double2float_rn(v[7]));
    }
};
template <> struct VG<double, 32> {
    static constexpr int n = 4;
    template <typename A> static __device__ __forceinline__ void ld(const double *p, A *o) {
        V16<double>::ld(p, o);
        V16<double>::ld(p + 2, o + 2);
    }
    static __device__ __forceinline__ void st(double *p, const double *v) {
        asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(v[0]), "d"(v[1]), "d"(v[2]), "d"(v[3])
                     : "memory");
    }
};

template <> struct VG<long long, 32> {
    static constexpr int n = 4;
    template <typename A> static __device__ __forceinline__ void ld(const long long *p, A *o) {
        V16<long long>::ld(p, o);
        V16<long long>::ld(p + 2, o + 2);
    }
    static __device__ __forceinline__ void st(long long *p, const long long *v) {
        asm volatile("st.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(v[0]), "l"(v[1]), "l"(v[2]), "l"(v[3])
                     : "memory");
    }
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Warp 0 is the producer: its first lane issues the TMA loads of every plane of every tile of
// this CTA, in order, into the ring of NS slots, each time waiting for the slot's "empty"
// barrier (all consumer warps done with the plane that last used it).  The other warps are
// consumers: each thread owns one 16-byte group (element e = VX * gx, cells x = e - g + c) in
// ROWS consecutive rows of the tile and marches it along z with a register queue.  There is
// no CTA-wide barrier inside the loop, so consumers run ahead as far as the loaded planes
// allow, and the producer starts on the next tile while the consumers finish this one.
// Where the tile's new values are also ghost cells of neighbouring boxes (ghost push), each
// consumer warp keeps the tile's push pieces in a small shared-memory table, written once per
// tile, and tests a piece's z range before touching it.
// The CTA has 32 + (consumer groups rounded up to a warp) threads.
// Launch bounds and registers: ptxas gives a kernel bounded to w warps per CTA at most
// 16384 / ceil(w / 4) / 32 registers per thread, rounded down to a multiple of 8 (17 warps: 96,
// 13-16: 128, 9-12: 168, up to 8: 255).  At radius 1 and 2 the 17-warp bound keeps the kernels
// at 96 registers, so that two 9-warp CTAs share an SM; the 25-point stencil, the
// fixed-point path's 64-bit queues and BF16 storage's unpacked 8-cell groups take 168 (12
// warps) or 128 (13 warps).
template <int R, typename A = float> struct TmaBounds { static constexpr int threads = R == 4 ? 384 : 544; };
template <int R> struct TmaBounds<R, FixA> { static constexpr int threads = R == 4 ? 384 : 416; };
template <typename S, int R, typename A, int ROWS, int GB> struct TmaThreads {
    static constexpr int value = std::is_same<S, __nv_bfloat16>::value ? 384 : TmaBounds<R, A>::threads;
};
// the fixed-point path's 2-row, 32-byte-group schedule keeps eight 64-bit cells per thread
template <> struct TmaThreads<long long, 1, FixA, 2, 32> { static constexpr int value = 384; };

// One ghost-push piece as a consumer warp keeps it (see the tile prologue).
struct PushRec {
    unsigned long long base;  // byte address of tile cell (0, 0, 0) in the destination
    long long plane;          // destination plane stride (elements)
    int px;                   // destination row pitch (elements)
    uint32_t zr, yr, xr;      // [lo, hi) ranges relative to the tile, packed lo | hi << 16
};


template <typename S, typename A, int R, int ROWS, int GB, bool RK>
__global__ void __launch_bounds__(TmaThreads<S, R, A, ROWS, GB>::value) k_stencil_tma(const __grid_constant__ StencilTmaParams p) {
    using V = VG<S, GB>;
    constexpr int VX = V::n;  // cells per group: one GB-byte vector of a row
    // FP32 arithmetic at radius 1: pairs of cells through the packed f32x2 instructions
    constexpr bool kPair = std::is_same<A, float>::value && R == 1 && VX % 2 == 0;
    // FP32 arithmetic at radius 2 and 4: the y and z face fluxes and the update of pairs of cells
    // through the packed instructions (face_flux2), the operations and order of the scalar code
    constexpr bool kPairR = std::is_same<A, float>::value && R > 1 && VX % 2 == 0;
    // exact fixed-point steps on 64-bit integers (fixed_diff.cuh)
    constexpr bool kFix = std::is_same<A, FixA>::value;
    static_assert(!kFix || (std::is_same<S, long long>::value && !RK), "fixed-point steps: 64-bit storage, plain steps");
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages];
    unsigned char *slots = (unsigned char *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    const int NS = p.nstages;  // power of two
    const int tid = threadIdx.x;
    const int ncw = (int)(blockDim.x >> 5) - 1;  // consumer warps
    __shared__ PushRec ptab[TmaThreads<S, R, A, ROWS, GB>::value / 32 - 1][kMaxPush];  // per consumer warp
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], (uint32_t)ncw);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    // Programmatic dependent launch: the next launch in the stream may start its CTAs (which
    // only find room as this grid's CTAs exit) and set up; before touching level data or the
    // error word every thread waits for the previous grid to complete.  Both are no-ops for a
    // launch without the attribute.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (*(volatile int *)p.err) return;  // an earlier launch already failed: do nothing
    if constexpr (kFix) {
        // grid bookkeeping, once per launch: the output grid of each component from its input
        // grid and the largest |K| of the input level (fixed_diff.cuh), and the clearing of the
        // set the launch after this one accumulates into (read by the launch before this one,
        // complete now; touched by no other thread of this one)
        if (blockIdx.x == 0 && tid < kMaxComp) {
            p.fix_out->E[tid] = p.fix_in->E[tid] + fix_bits(p.fix_in->M[tid]) + kFixH - FixW<R>::B;
            p.fix_clear->M[tid] = 0ull;
        }
    }
    // this CTA's tiles: its own range of a balanced schedule, else every gridDim.x-th tile
    int w0 = blockIdx.x, w1 = p.ntiles, ws = gridDim.x;
    if (p.cta_tiles) {
        w0 = p.cta_tiles[blockIdx.x];
        w1 = p.cta_tiles[blockIdx.x + 1];
        ws = 1;
    }

    if (tid < 32) {
        // ------------------------------------------------------------------ producer
        if (tid != 0) return;
        uint32_t seq = 0;
        for (int w = w0; w < w1; w += ws) {
            const Tile t = p.tiles[w];
            const TmaFab tf = p.tfab[t.fab];
            TileStrip ts;
            ts.lfab = ts.rfab = -1;
            if (p.strips) ts = p.strips[w];
            const CUtensorMap *map = p.maps + t.fab;
            const uint32_t plane_bytes = (uint32_t)(tf.bx * tf.by * (int)sizeof(S));
            const int ycoord = tf.ngrow + t.y0 - R, zcoord = tf.ngrow + t.z0 - R;
            const int ntot = t.tz + 2 * R;
            for (int pl = 0; pl < ntot; ++pl, ++seq) {
                const uint32_t sl = seq & (uint32_t)(NS - 1);
                if (seq >= (uint32_t)NS && !mbar_wait(&empty[sl], ((seq >> p.nstages_log2) - 1) & 1u)) {
                    atomicOr(p.err, 1);
                    return;  // consumers give up on their own bounded waits
                }
                unsigned char *sp = slots + (size_t)sl * p.slot_bytes;
                // centre planes (the x neighbours of the tile's cells) also take the x halo strips
                const bool centre = pl >= R && pl < R + t.tz;
                const bool ls = centre && ts.lfab >= 0, rs = centre && ts.rfab >= 0;
                mbar_expect_tx(&full[sl], plane_bytes + (ls ? p.strip_bytes : 0) + (rs ? p.strip_bytes : 0));
                tma_load_4d(sp, map, &full[sl], tf.xs, ycoord, zcoord + pl, t.comp);
                if (ls) tma_load_4d(sp + p.strip_off, p.smaps + ts.lfab, &full[sl], ts.lx, ts.ly, ts.lz + pl - R, t.comp);
                if (rs)
                    tma_load_4d(sp + p.strip_off + p.strip_pitch, p.smaps + ts.rfab, &full[sl], ts.rx, ts.ry,
                                ts.rz + pl - R, t.comp);
            }
        }
        // drain: the last NS planes must have landed before the CTA may exit
        for (uint32_t k = seq > (uint32_t)NS ? seq - NS : 0; k < seq; ++k)
            if (!mbar_wait(&full[k & (uint32_t)(NS - 1)], (k >> p.nstages_log2) & 1u)) {
                atomicOr(p.err, 1);
                return;
            }
        return;
    }

    // ------------------------------------------------------------------ consumers
    const int ctid = tid - 32;
    const int cw = ctid >> 5;  // consumer warp
    const int lane = tid & 31;
    uint32_t seq = 0;
    auto wait_seq = [&](uint32_t sq) -> bool {
        return mbar_wait(&full[sq & (uint32_t)(NS - 1)], (sq >> p.nstages_log2) & 1u);
    };
    auto slot_ptr = [&](uint32_t sq) -> const S * {
        return (const S *)(slots + (size_t)(sq & (uint32_t)(NS - 1)) * p.slot_bytes);
    };
    auto release = [&](uint32_t sq) {  // this warp is done with plane sq
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[sq & (uint32_t)(NS - 1)]);
    };
    for (int w = w0; w < w1; w += ws) {
        const Tile t = p.tiles[w];
        const TmaFab tf = p.tfab[t.fab];
        const FabInfo f = p.ftab[t.fab];
        const int xv = tf.xv;   // element of valid x = 0 in a loaded row
        const int bx = tf.bx;   // elements of a loaded row
        const int xvg = xv + tf.xs;  // row element of valid x = 0 in the FArrayBox
        TileStrip ts;
        ts.lfab = ts.rfab = -1;
        ts.pcount = 0;
        if (p.strips) ts = p.strips[w];
        if (!p.push) ts.pcount = 0;

        // groups of valid cells: x0c = VX * gx .. + VX - 1 at row element xv + x0c
        const int ngx = (f.n[0] + VX - 1) / VX;
        const int nset = (t.ty + ROWS - 1) / ROWS;
        const bool act = ctid < ngx * nset;
        const int x0c = act ? (ctid % ngx) * VX : 0;
        const int y0 = act ? ROWS * (ctid / ngx) : 0;
        const int nrow = act ? min(ROWS, t.ty - y0) : 0;  // rows of the set that exist
        const int soff = (y0 + R) * bx + xv + x0c;       // smem offset of the first row's group

        // Ghost-push pieces of the tile, in the warp's own table: lane i writes piece i
        // (destination address of tile cell (0, 0, 0), plane stride, row pitch, and the piece's
        // z, y and x ranges relative to the tile, x packed with the full-row flag in bit 31).
        // pmask: the pieces touching this thread's cells, wm: the union over the warp.
        PushRec *ptw = ptab[cw];
        __syncwarp();  // the warp's previous tile is done with the table
        if (lane < ts.pcount) {
            const PushPiece pp = p.push[ts.pfirst + lane];
            const FabInfo df = p.ftab[pp.dfab];
            const long long off = pp.dst + t.comp * df.cstride - pp.z0 * df.plane - pp.y0 * (long long)df.px - pp.x0;
            PushRec pr;
            pr.base = (unsigned long long)(uintptr_t)p.dst[df.level] + (unsigned long long)off * sizeof(S);
            pr.plane = df.plane;
            pr.px = df.px;
            pr.zr = (uint32_t)pp.z0 | (uint32_t)(pp.z0 + pp.nz) << 16;
            pr.yr = (uint32_t)pp.y0 | (uint32_t)(pp.y0 + pp.ny) << 16;
            pr.xr = (uint32_t)pp.x0 | (uint32_t)(pp.x0 + pp.nx) << 16 | (pp.full_row ? 0x80000000u : 0u);
            ptw[lane] = pr;
        }
        __syncwarp();
        uint32_t pmask = 0u;
        for (int pi = 0; pi < ts.pcount; ++pi) {
            const uint32_t yr = ptw[pi].yr, xr = ptw[pi].xr;
            const int py0 = (int)(yr & 0xffffu), py1 = (int)(yr >> 16);
            const int px0 = (int)(xr & 0xffffu), px1 = (int)((xr >> 16) & 0x7fffu);
            const bool hit = act && y0 + nrow > py0 && y0 < py1 && ((xr >> 31) || (x0c < px1 && x0c + VX > px0));
            if (hit) pmask |= 1u << pi;
        }

        // fixed for the tile: output pointer (advanced one plane per step) and the shared-memory
        // offset of every x-halo cell -- the loaded row for cells of the box (and for filled
        // ghost columns), the neighbour strip outside a strip-served face; cells that only feed
        // don't-care outputs (ghost and padding positions) read their own row
        int hl[ROWS][R], hr[ROWS][R];
        // Groups start at valid x >= 0, so only cells past the right face (x >= n0) can sit in a
        // group; where that face is strip-served, cell c of row r reads strip offset
        // cob + r * strip_w + c instead of its own row.
        uint32_t cov = 0;  // bit c: cell c of the group takes its value from a strip (every row)
        int cob = 0;
        {
            const int lso = p.strip_off / (int)sizeof(S), rso = (p.strip_off + p.strip_pitch) / (int)sizeof(S);
            const int xw = p.strip_w;
            const int n0 = f.n[0];
            auto src = [&](int x, int r) -> int {
                if (x < 0 && x >= -R && ts.lfab >= 0) return lso + (y0 + r) * xw + ts.lidx0 + x;
                if (x >= n0 && x < n0 + R && ts.rfab >= 0) return rso + (y0 + r) * xw + ts.ridx0 + (x - n0);
                return (y0 + r + R) * bx + min(max(x + xv, 0), bx - 1);
            };
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    hl[r][i] = src(x0c - R + i, r);
                    hr[r][i] = src(x0c + VX + i, r);
                }
            }
#pragma unroll
            for (int c = 0; c < VX; ++c) {
                const int x = x0c + c;
                if (x >= n0 && x < n0 + R && ts.rfab >= 0) cov |= 1u << c;
            }
            cob = rso + y0 * xw + ts.ridx0 + x0c - n0;
        }
        // Where R cells are a whole number of 16-byte vectors (R = 4 in FP32, R >= 2 in FP64), the
        // x halo of a row is usually R consecutive, aligned shared-memory elements on each side
        // (box widths and row pitches multiples of 16 bytes): then it is read as vectors.  The
        // whole warp takes the vector path or the per-cell one.
        constexpr int kHV = (R * (int)sizeof(S)) % 16 == 0 ? R * (int)sizeof(S) / 16 : 0;  // vectors per side
        bool hvec = false;
        if constexpr (kHV > 0) {
            bool ok = true;
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                ok = ok && (hl[r][0] * (int)sizeof(S)) % 16 == 0 && (hr[r][0] * (int)sizeof(S)) % 16 == 0;
#pragma unroll
                for (int i = 1; i < R; ++i) ok = ok && hl[r][i] == hl[r][0] + i && hr[r][i] == hr[r][0] + i;
            }
            hvec = __all_sync(0xffffffffu, ok);
        }
        const long long ooff = f.org + t.comp * f.cstride + (long long)t.z0 * f.plane + (long long)(t.y0 + y0) * f.px + x0c;
        S *op = (S *)p.dst[f.level] + ooff;
        // Runge-Kutta stage: the state at the start of the step, at the output's position
        const S *u0p = RK ? (const S *)p.u0[f.level] + ooff : nullptr;
        // a group at a row end that fills only half of a 32-byte sector also writes the other
        // half (ghost / padding cells, don't-care values there: strips, not those cells, feed
        // the stencil), so that no sector is written in part
        const bool full = x0c + VX <= f.n[0];
        const bool lpad = act && x0c == 0 && xvg >= VX && (f.org * (long long)sizeof(S)) % 32 == 16;
        const bool rpad = act && full && x0c + VX == f.n[0] && xvg + f.n[0] + VX <= f.px &&
                          ((f.org + f.n[0]) * (long long)sizeof(S)) % 32 == 16;
        const int xo = lpad ? -VX : VX;  // the extra store of a row-end group
        const bool both = __any_sync(0xffffffffu, lpad && rpad);  // one group spans the whole row
        // the common case for the whole warp: every thread active with all its rows, whole groups,
        // no row-end completion store -- each plane is then ROWS vector stores
        const bool plain_st = __all_sync(0xffffffffu, act && nrow == ROWS && full && !lpad && !rpad);
        using LT = typename std::conditional<kFix, double, A>::type;
        const LT lam = (LT)p.lam[f.level][t.comp];  // fixed-point path: lam / den

        // Pieces that cover every plane of the tile and whole rows (the y faces) become one
        // destination pointer per row of this thread, advanced a plane per step; the rest (z faces,
        // one or two planes per tile, and irregular pieces) take the general loop below.
        S *fyp[ROWS];
        uint32_t fmask = 0u;  // bit r: row r is also stored at fyp[r]
        long long fdp = 0;    // their common plane stride
        uint32_t slow = pmask;
#pragma unroll
        for (int r = 0; r < ROWS; ++r) fyp[r] = nullptr;
        for (int pi = 0; pi < ts.pcount; ++pi) {
            if (!(pmask & (1u << pi))) continue;
            const uint32_t zr = ptw[pi].zr, yr = ptw[pi].yr, xr = ptw[pi].xr;
            const long long dplane = ptw[pi].plane;
            if ((zr & 0xffffu) != 0u || (int)(zr >> 16) < t.tz || !(xr >> 31) || !full) continue;
            if (fdp != 0 && fdp != dplane) continue;
            const int py0 = (int)(yr & 0xffffu), py1 = (int)(yr >> 16);
            const unsigned long long b = ptw[pi].base;
            const int dpx = ptw[pi].px;
            bool ok = true;
            uint32_t take = 0u;
            S *gp[ROWS];
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const int yy = y0 + r;
                gp[r] = nullptr;
                if (r >= nrow || yy < py0 || yy >= py1) continue;
                gp[r] = (S *)(uintptr_t)(b + (unsigned long long)((long long)yy * dpx + x0c) * sizeof(S));
                if ((fmask & (1u << r)) || ((uintptr_t)gp[r] & (GB - 1)) != 0) ok = false;
                take |= 1u << r;
            }
            if (!ok || !take) continue;
#pragma unroll
            for (int r = 0; r < ROWS; ++r)
                if (take & (1u << r)) fyp[r] = gp[r];
            fmask |= take;
            fdp = dplane;
            slow &= ~(1u << pi);
        }
        const uint32_t wm = __reduce_or_sync(0xffffffffu, slow);

        // stores of output plane k at o: the tile's rows (with row-end completion stores where a
        // group fills half a sector) and the ghost push into neighbour boxes
        auto store_plane = [&](auto &out, int k, S *o) {
            if (plain_st) {
#pragma unroll
                for (int r = 0; r < ROWS; ++r) V::st(o + r * f.px, out[r]);
            } else if (act) {
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    if (r >= nrow) continue;
                    S *orow = o + r * f.px;
                    if (full) {
                        V::st(orow, out[r]);
                    } else {
#pragma unroll
                        for (int c = 0; c < VX; ++c)
                            if (x0c + c < f.n[0]) st(orow + c, out[r][c]);
                    }
                    if (lpad || rpad) V::st(orow + xo, out[r]);
                    if (both && lpad && rpad) V::st(orow + VX, out[r]);
                }
            }
            // ghost push: the same values into the neighbour boxes whose ghost faces hold them
            if (fmask) {
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    if (fmask & (1u << r)) V::st(fyp[r], out[r]);
                    fyp[r] += fdp;
                }
            }
            if (wm) {
                uint32_t m = wm;
                while (m) {
                    const int pi = __ffs(m) - 1;
                    m &= m - 1;
                    const uint32_t zr = ptw[pi].zr;
                    if (k < (int)(zr & 0xffffu) || k >= (int)(zr >> 16) || !(slow & (1u << pi))) continue;
                    const unsigned long long b = ptw[pi].base;
                    const long long dplane = ptw[pi].plane;
                    const int dpx = ptw[pi].px;
                    const uint32_t yr = ptw[pi].yr, xr = ptw[pi].xr;
                    const int py0 = (int)(yr & 0xffffu), py1 = (int)(yr >> 16);
                    const int px0 = (int)(xr & 0xffffu), px1 = (int)((xr >> 16) & 0x7fffu);
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) {
                        const int yy = y0 + r;
                        if (r >= nrow || yy < py0 || yy >= py1) continue;
                        S *gp = (S *)(uintptr_t)(b + (unsigned long long)(k * dplane + (long long)yy * dpx + x0c) *
                                                         sizeof(S));
                        if ((xr >> 31) && full && ((uintptr_t)gp & (GB - 1)) == 0) {
                            V::st(gp, out[r]);
                        } else {
#pragma unroll
                            for (int c = 0; c < VX; ++c) {
                                const int x = x0c + c;
                                if (x >= px0 && x < px1) st(gp + c, out[r][c]);
                            }
                        }
                    }
                }
            }
        };
        if constexpr (kFix) {
            // this component's grid change: t = 64 - (E - E') from the largest |K| of the input
            // level (volatile: written by the previous launch, which this one may have overlapped)
            const unsigned long long M = *(volatile const unsigned long long *)&p.fix_in->M[t.comp];
            const int tt = 64 - FixW<R>::B + kFixH + fix_bits(M);
            const unsigned long long lq = p.fix_q[t.comp];
            const uint32_t qh = (uint32_t)(lq >> 32), ql = (uint32_t)lq;
            const bool same_grid = tt == 64;  // the common case: K' = K + L q / 2^64
            // the OR of the high words of |K'| (ones' complement) over this thread's valid cells
            // (bit r * VX + c of vbits) bounds the largest |K'| (fix_bits)
            uint32_t omax = 0u;
            uint32_t vbits = 0u;
#pragma unroll
            for (int r = 0; r < ROWS; ++r)
#pragma unroll
                for (int c = 0; c < VX; ++c)
                    if (act && r < nrow && x0c + c < f.n[0]) vbits |= 1u << (r * VX + c);
            long long q[ROWS][VX][2 * R + 1];  // z queue per cell: q[r][c][i] = K(z - R + i)
            bool ok = true;
#pragma unroll
            for (int pl = 0; pl < 2 * R; ++pl) {
                ok = ok && wait_seq(seq + pl);
                const S *sp = slot_ptr(seq + pl);
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    long long v[VX];
                    V::template ld<long long>(sp + soff + r * bx, v);
#pragma unroll
                    for (int c = 0; c < VX; ++c) q[r][c][pl] = v[c];
                }
            }
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) atomicOr(p.err, 1);
                return;
            }
            for (int pl = 0; pl < 2 * R; ++pl)
                if (pl < R || pl >= t.tz + R) release(seq + pl);
            // as in the plain path below: a copy of the plane loop for the warp's common case (no
            // strip cell inside a group, whole-row stores), one basic block per plane (a third copy
            // for tiles that push nothing measured slower here)
            const bool fast = (kHV == 0 || hvec) && plain_st && !__any_sync(0xffffffffu, cov != 0u);
            auto plane_loop = [&](auto fast_t) -> bool {
                constexpr bool FAST = decltype(fast_t)::value;
#pragma unroll(2 * R + 1)
            for (int k = 0; k < t.tz; ++k) {
                if (!__all_sync(0xffffffffu, wait_seq(seq + k + 2 * R))) {
                    if (lane == 0) atomicOr(p.err, 1);
                    return false;
                }
                const S *newp = slot_ptr(seq + k + 2 * R);
                const S *cp = slot_ptr(seq + k + R);
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    long long v[VX];
                    V::template ld<long long>(newp + soff + r * bx, v);
#pragma unroll
                    for (int c = 0; c < VX; ++c) q[r][c][2 * R] = v[c];
                }
                // y window per column: wy[m][c] = K(x + c, y0 - R + m)
                long long wy[2 * R + ROWS][VX];
                const S *cc = cp + soff;
#pragma unroll
                for (int m = 0; m < 2 * R + ROWS; ++m) {
                    if (m >= R && m < R + ROWS) continue;
                    V::template ld<long long>(cc + (m - R) * bx, wy[m]);
                }
#pragma unroll
                for (int r = 0; r < ROWS; ++r)
#pragma unroll
                    for (int c = 0; c < VX; ++c) wy[R + r][c] = q[r][c][R];
                long long out[ROWS][VX];
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    long long wx[VX + 2 * R];  // x window: wx[i] = K(x0 - R + i)
                    if (kHV > 0 && (FAST || hvec)) {
#pragma unroll
                        for (int j = 0; j < kHV; ++j) {
                            V16<S>::template ld<long long>(cp + hl[r][0] + j * V16<S>::n, wx + j * V16<S>::n);
                            V16<S>::template ld<long long>(cp + hr[r][0] + j * V16<S>::n, wx + R + VX + j * V16<S>::n);
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < R; ++i) {
                            wx[i] = cp[hl[r][i]];
                            wx[R + VX + i] = cp[hr[r][i]];
                        }
                    }
#pragma unroll
                    for (int c = 0; c < VX; ++c) wx[R + c] = q[r][c][R];
                    if (!FAST && cov) {  // the box face is inside this group: x neighbours from the strips
#pragma unroll
                        for (int c = 0; c < VX; ++c)
                            if (cov & (1u << c)) wx[R + c] = cp[cob + r * p.strip_w + c];
                    }
#pragma unroll
                    for (int c = 0; c < VX; ++c) {
                        // direct form in exact integer arithmetic (wrapping unsigned sums: only the
                        // unused results of ghost or padding positions can exceed the headroom)
                        unsigned long long L = (unsigned long long)(FixW<R>::w0() * q[r][c][R]);
#pragma unroll
                        for (int m = 1; m <= R; ++m) {
                            const unsigned long long pair =
                                ((unsigned long long)wx[R + c + m] + (unsigned long long)wx[R + c - m]) +
                                ((unsigned long long)wy[R + r + m][c] + (unsigned long long)wy[R + r - m][c]) +
                                ((unsigned long long)q[r][c][R + m] + (unsigned long long)q[r][c][R - m]);
                            L += (unsigned long long)FixW<R>::w(m) * pair;
                        }
                        out[r][c] = same_grid ? q[r][c][R] + fix_incr(L, qh, ql)
                                              : fix_update(q[r][c][R], (long long)L, lq, tt);
                        const int hw = (int)(out[r][c] >> 32);
                        if (vbits & (1u << (r * VX + c))) omax |= (uint32_t)(hw ^ (hw >> 31));
                    }
                }
#pragma unroll
                for (int r = 0; r < ROWS; ++r)
#pragma unroll
                    for (int c = 0; c < VX; ++c)
#pragma unroll
                        for (int i = 0; i < 2 * R; ++i) q[r][c][i] = q[r][c][i + 1];
                // every read of the centre plane (and of the last R planes) is done
                release(seq + k + R);
                if (k >= t.tz - R) release(seq + k + 2 * R);
                S *o = op;
                op += f.plane;
                store_plane(out, k, o);
            }
                return true;
            };
            // (one-row schedules keep the single loop: the second copy slowed their general loop,
            // which the many small tiles of a many-box level mostly take)
            bool ok_loop;
            if constexpr (ROWS > 1) ok_loop = fast ? plane_loop(std::true_type{}) : plane_loop(std::false_type{});
            else ok_loop = plane_loop(std::false_type{});
            if (!ok_loop) return;
            // the bit length of the largest |K'| of the output, per component, for the next
            // launch's grid: an OR over the warp, then an atomic OR
            omax = __reduce_or_sync(0xffffffffu, omax);
            if (lane == 0 && omax) atomicOr(&p.fix_out->M[t.comp], (unsigned long long)omax << 32);
        } else {
            A q[ROWS][VX][2 * R + 1];  // z queue per cell: q[r][c][i] = u(z - R + i)
            A fzm[ROWS][VX];
            bool ok = true;
#pragma unroll
            for (int pl = 0; pl < 2 * R; ++pl) {
                ok = ok && wait_seq(seq + pl);
                const S *sp = slot_ptr(seq + pl);
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    A v[VX];
                    V::ld(sp + soff + r * bx, v);
#pragma unroll
                    for (int c = 0; c < VX; ++c) q[r][c][pl] = v[c];
                }
            }
            if (!__all_sync(0xffffffffu, ok)) {  // the whole warp leaves together
                if (lane == 0) atomicOr(p.err, 1);
                return;
            }
#pragma unroll
            for (int r = 0; r < ROWS; ++r)
#pragma unroll
                for (int c = 0; c < VX; ++c) fzm[r][c] = face_flux<A, R>(q[r][c], R - 1);
            // planes 0 .. R-1 live on in the queues only; so do planes tz + R .. 2R - 1 of a tile
            // thinner than R (never a centre plane, and below the planes the z loop releases)
            for (int pl = 0; pl < 2 * R; ++pl)
                if (pl < R || pl >= t.tz + R) release(seq + pl);

            // Three copies of the plane loop: the common case for the whole warp (x halos as
            // vectors where R cells fill them, no strip cell inside a group, whole-row stores)
            // without the per-row tests,
            // so that each plane is one basic block, once with plain row stores for warps that push
            // nothing and once through the push; and the general one.
            const bool fast = (kHV == 0 || hvec) && plain_st && !__any_sync(0xffffffffu, cov != 0u);
            const bool nopush = !__any_sync(0xffffffffu, fmask != 0u) && wm == 0u;
            auto plane_loop = [&](auto mode_t) -> bool {
                constexpr int MODE = decltype(mode_t)::value;  // 0 general, 1 fast, 2 fast without push
                constexpr bool FAST = MODE > 0;
            // unrolled by two at radius 1 (packed pairs) and 4, so that half the queue shifts become
            // register renames (at radius 2 the unrolled loop spills)
#pragma unroll(kPair || R == 4 ? 2 : 1)
            for (int k = 0; k < t.tz; ++k) {
                if (!__all_sync(0xffffffffu, wait_seq(seq + k + 2 * R))) {
                    if (lane == 0) atomicOr(p.err, 1);
                    return false;
                }
                const S *newp = slot_ptr(seq + k + 2 * R);
                const S *cp = slot_ptr(seq + k + R);
                // Runge-Kutta stage: the state at the start of the step at this plane's cells, read
                // from global memory before the arithmetic that hides its latency
                A u0v[RK ? ROWS : 1][VX];
                if constexpr (RK) {
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) {
                        if (!FAST && r >= nrow) continue;
                        const S *urow = u0p + r * f.px;
                        if (FAST || full) {
                            V::ld(urow, u0v[r]);
                        } else {
#pragma unroll
                            for (int c = 0; c < VX; ++c) u0v[r][c] = x0c + c < f.n[0] ? ld<S, A>(urow + c) : (A)0;
                        }
                    }
                    u0p += f.plane;
                }
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    A v[VX];
                    V::ld(newp + soff + r * bx, v);
#pragma unroll
                    for (int c = 0; c < VX; ++c) q[r][c][2 * R] = v[c];
                }
                // y window per column: wy[m][c] = u(x + c, y0 - R + m), m = 0 .. 2R+ROWS-1 (the set's
                // own rows from the queues, the rest from the centre plane)
                A wy[2 * R + ROWS][VX];
                const S *cc = cp + soff;
#pragma unroll
                for (int m = 0; m < 2 * R + ROWS; ++m) {
                    if (m >= R && m < R + ROWS) continue;
                    V::ld(cc + (m - R) * bx, wy[m]);
                }
#pragma unroll
                for (int r = 0; r < ROWS; ++r)
#pragma unroll
                    for (int c = 0; c < VX; ++c) wy[R + r][c] = q[r][c][R];
                // y-face fluxes at y0 - 1/2 + r, r = 0 .. ROWS (inner faces shared by two rows)
                A fy[ROWS + 1][VX];
                if constexpr (kPair) {  // radius 1: the flux is a difference, two cells per instruction
#pragma unroll
                    for (int r = 0; r <= ROWS; ++r)
#pragma unroll
                        for (int c = 0; c < VX; c += 2) {
                            const F2 d = sub2(F2{wy[r + 1][c], wy[r + 1][c + 1]}, F2{wy[r][c], wy[r][c + 1]});
                            fy[r][c] = d.x;
                            fy[r][c + 1] = d.y;
                        }
                } else if constexpr (kPairR) {
#pragma unroll
                    for (int c = 0; c < VX; c += 2) {
                        float ca[2 * R + ROWS], cb[2 * R + ROWS];
#pragma unroll
                        for (int m = 0; m < 2 * R + ROWS; ++m) {
                            ca[m] = wy[m][c];
                            cb[m] = wy[m][c + 1];
                        }
#pragma unroll
                        for (int r = 0; r <= ROWS; ++r) {
                            const F2 fyr = face_flux2<R>(ca, cb, R - 1 + r);
                            fy[r][c] = fyr.x;
                            fy[r][c + 1] = fyr.y;
                        }
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < VX; ++c) {
                        A col[2 * R + ROWS];
#pragma unroll
                        for (int m = 0; m < 2 * R + ROWS; ++m) col[m] = wy[m][c];
#pragma unroll
                        for (int r = 0; r <= ROWS; ++r) fy[r][c] = face_flux<A, R>(col, R - 1 + r);
                    }
                }
                A out[ROWS][VX];
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    // x window: w[i] = u(x0 - R + i), i = 0 .. VX + 2R - 1
                    A wx[VX + 2 * R];
                    if (kHV > 0 && (FAST || hvec)) {
#pragma unroll
                        for (int j = 0; j < kHV; ++j) {
                            V16<S>::ld(cp + hl[r][0] + j * V16<S>::n, wx + j * V16<S>::n);
                            V16<S>::ld(cp + hr[r][0] + j * V16<S>::n, wx + R + VX + j * V16<S>::n);
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < R; ++i) {
                            wx[i] = ld_smem<S, A>(cp + hl[r][i]);
                            wx[R + VX + i] = ld_smem<S, A>(cp + hr[r][i]);
                        }
                    }
#pragma unroll
                    for (int c = 0; c < VX; ++c) wx[R + c] = q[r][c][R];
                    if (!FAST && cov) {  // the box face is inside this group: x neighbours from the strips
#pragma unroll
                        for (int c = 0; c < VX; ++c)
                            if (cov & (1u << c)) wx[R + c] = ld_smem<S, A>(cp + cob + r * p.strip_w + c);
                    }
                    // x-face fluxes: fx[c] is the face left of cell c (scalar: the packed form would
                    // pair neighbouring window values, which sit in unaligned register pairs, and
                    // measured slower)
                    A fx[VX + 1];
#pragma unroll
                    for (int c = 0; c <= VX; ++c) fx[c] = face_flux<A, R>(wx, c + R - 1);
                    if constexpr (kPair) {
                        // the same operations as update_cell_f in the same order, two cells at a time:
                        // ((fxp - fxm) + (fyp - fym)) + (fzp - fzm), then u + lam * div
#pragma unroll
                        for (int c = 0; c < VX; c += 2) {
                            const F2 u = F2{q[r][c][1], q[r][c + 1][1]};
                            const F2 fzp = sub2(F2{q[r][c][2], q[r][c + 1][2]}, u);
                            const F2 dx = F2{Ar<A>::sub(fx[c + 1], fx[c]), Ar<A>::sub(fx[c + 2], fx[c + 1])};
                            const F2 dy = sub2(F2{fy[r + 1][c], fy[r + 1][c + 1]}, F2{fy[r][c], fy[r][c + 1]});
                            const F2 dz = sub2(fzp, F2{fzm[r][c], fzm[r][c + 1]});
                            const F2 o = fma2(F2{lam, lam}, add2(add2(dx, dy), dz), u);
                            out[r][c] = o.x;
                            out[r][c + 1] = o.y;
                            fzm[r][c] = fzp.x;
                            fzm[r][c + 1] = fzp.y;
                            q[r][c][0] = q[r][c][1];
                            q[r][c][1] = q[r][c][2];
                            q[r][c + 1][0] = q[r][c + 1][1];
                            q[r][c + 1][1] = q[r][c + 1][2];
                        }
                    } else if constexpr (kPairR) {
                        // update_cell_f's operations in its order, two cells at a time
#pragma unroll
                        for (int c = 0; c < VX; c += 2) {
                            const F2 fzp = face_flux2<R>(q[r][c], q[r][c + 1], R);
                            const F2 u = F2{q[r][c][R], q[r][c + 1][R]};
                            const F2 dx = sub2(F2{fx[c + 1], fx[c + 2]}, F2{fx[c], fx[c + 1]});
                            const F2 dy = sub2(F2{fy[r + 1][c], fy[r + 1][c + 1]}, F2{fy[r][c], fy[r][c + 1]});
                            const F2 dz = sub2(fzp, F2{fzm[r][c], fzm[r][c + 1]});
                            const F2 o = fma2(F2{lam, lam}, add2(add2(dx, dy), dz), u);
                            out[r][c] = o.x;
                            out[r][c + 1] = o.y;
                            fzm[r][c] = fzp.x;
                            fzm[r][c + 1] = fzp.y;
#pragma unroll
                            for (int i = 0; i < 2 * R; ++i) {
                                q[r][c][i] = q[r][c][i + 1];
                                q[r][c + 1][i] = q[r][c + 1][i + 1];
                            }
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < VX; ++c) {
                            const A fzp = face_flux<A, R>(q[r][c], R);
                            out[r][c] = update_cell_f<A>(fx[c + 1], fx[c], fy[r + 1][c], fy[r][c], fzp, fzm[r][c],
                                                         q[r][c][R], lam);
                            fzm[r][c] = fzp;
#pragma unroll
                            for (int i = 0; i < 2 * R; ++i) q[r][c][i] = q[r][c][i + 1];
                        }
                    }
                }
                // every read of the centre plane (and of the last R planes) is done
                release(seq + k + R);
                if (k >= t.tz - R) release(seq + k + 2 * R);
                S *o = op;
                op += f.plane;
                if constexpr (RK) {  // a Runge-Kutta stage: rk_a * u0 + rk_b * (forward-Euler value)
                    const A rka = (A)p.rk_a, rkb = (A)p.rk_b;
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) {
                        if (!FAST && r >= nrow) continue;
#pragma unroll
                        for (int c = 0; c < VX; ++c) out[r][c] = rk_combine<A>(out[r][c], u0v[r][c], rka, rkb);
                    }
                }
                if constexpr (MODE == 2) {
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) V::st(o + r * f.px, out[r]);
                } else {
                    store_plane(out, k, o);
                }
            }
                return true;
            };
            const bool ok_loop = !fast    ? plane_loop(std::integral_constant<int, 0>{})
                                 : nopush ? plane_loop(std::integral_constant<int, 2>{})
                                          : plane_loop(std::integral_constant<int, 1>{});
            if (!ok_loop) return;
        }
        seq += (uint32_t)(t.tz + 2 * R);
    }
}

// Raise the kernel's dynamic shared-memory limit to at least smem (never lowers it).
template <typename S, typename A, int R, int ROWS, int GB, bool RK>
static cudaError_t tma_configure(int smem) {
    static int configured = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(k_stencil_tma<S, A, R, ROWS, GB, RK>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    return cudaSuccess;
}

template <typename S, typename A, int R, int ROWS, int GB, bool RK>
static cudaError_t tma_t(int nt, const StencilTmaParams &p, int grid, cudaStream_t s) {
    if (nt < 64 || nt > TmaThreads<S, R, A, ROWS, GB>::value || nt % 32) return cudaErrorInvalidValue;
    const int smem = p.nstages * p.slot_bytes + 128;
    auto kern = k_stencil_tma<S, A, R, ROWS, GB, RK>;
    cudaError_t e = tma_configure<S, A, R, ROWS, GB, RK>(smem);
    if (e != cudaSuccess) return e;
    int g = grid;
    if (g <= 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        long long gg = (long long)per_sm * sm_count();
        g = (int)(gg < p.ntiles ? gg : p.ntiles);
        if (g < 1) g = 1;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g);
    cfg.blockDim = dim3((unsigned)nt);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, p);
}

// The instantiated schedules: (R, rows, group bytes).  32-byte groups exist for FP32 and FP64
// storage with one row per thread and R <= 2 (registers).
template <typename S> constexpr bool kHasWide = !std::is_same<S, __nv_bfloat16>::value;

// Calls f.template run<R, ROWS, GB>() for the instantiated schedule, else returns fallback.
template <typename S, typename F, typename T>
static T tma_dispatch(int R, int rows, int gb, F &&f, T fallback) {
    switch ((R * 4 + rows) * 2 + (gb == 32 ? 1 : 0)) {
        case (1 * 4 + 1) * 2: return f.template run<1, 1, 16>();
        case (1 * 4 + 2) * 2: return f.template run<1, 2, 16>();
        case (2 * 4 + 1) * 2: return f.template run<2, 1, 16>();
        case (2 * 4 + 2) * 2: return f.template run<2, 2, 16>();
        case (4 * 4 + 1) * 2: return f.template run<4, 1, 16>();
        case (4 * 4 + 2) * 2:  // the 25-point stencil, two rows per thread: FP32 and FP64 storage
            if constexpr (kHasWide<S> && !std::is_same<S, long long>::value) return f.template run<4, 2, 16>();
            break;
        case (1 * 4 + 1) * 2 + 1:
            if constexpr (kHasWide<S>) return f.template run<1, 1, 32>();
            break;
        case (2 * 4 + 1) * 2 + 1:
            if constexpr (kHasWide<S>) return f.template run<2, 1, 32>();
            break;
        case (1 * 4 + 2) * 2 + 1:
            if constexpr (std::is_same<S, long long>::value) return f.template run<1, 2, 32>();
            break;
    }
    return fallback;
}

template <typename S, typename A, bool RK>
struct LaunchF {
    int nt;
    const StencilTmaParams &p;
    int grid;
    cudaStream_t s;
    template <int R, int ROWS, int GB> cudaError_t run() { return tma_t<S, A, R, ROWS, GB, RK>(nt, p, grid, s); }
};

// Launch of one schedule for a storage type, Runge-Kutta stage or not (instantiated in
// stencil_tma.cu for plain steps and in stencil_tma_rk.cu for stages).
template <bool RK>
cudaError_t launch_tma_variant(int dtype, int R, bool fp64diff, int rows, int gb, int nt, const StencilTmaParams &p,
                               int grid, cudaStream_t s) {
    switch (dtype) {
        case F64: return tma_dispatch<double>(R, rows, gb, LaunchF<double, double, RK>{nt, p, grid, s}, cudaErrorInvalidValue);
        case F32:
            return fp64diff ? tma_dispatch<float>(R, rows, gb, LaunchF<float, double, RK>{nt, p, grid, s}, cudaErrorInvalidValue)
                            : tma_dispatch<float>(R, rows, gb, LaunchF<float, float, RK>{nt, p, grid, s}, cudaErrorInvalidValue);
        case BF16:
            return fp64diff ? tma_dispatch<__nv_bfloat16>(R, rows, gb, LaunchF<__nv_bfloat16, double, RK>{nt, p, grid, s},
                                                          cudaErrorInvalidValue)
                            : tma_dispatch<__nv_bfloat16>(R, rows, gb, LaunchF<__nv_bfloat16, float, RK>{nt, p, grid, s},
                                                          cudaErrorInvalidValue);
    }
    return cudaErrorInvalidValue;
}

}  // namespace mfk
