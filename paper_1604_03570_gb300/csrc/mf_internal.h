// mf_internal.h -- device-side tables and kernel launchers shared by mf_host.cpp and the
// CUDA translation units.  Not part of the public ABI (see include/mf.h).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace mfk {

constexpr int kMaxComp = 16;
constexpr int kMaxLev = 2;

enum DType { F64 = 0, F32 = 1, BF16 = 2 };

inline int dtype_size(int dt) { return dt == F64 ? 8 : dt == F32 ? 4 : 2; }

// One FArrayBox.  Element (x, y, z, c) of the box, in coordinates relative to the valid
// lower corner (x in [-g, n0 + g)), lives at  org + c*cstride + z*plane + y*px + x.
struct FabInfo {
    long long org;      // element offset of valid cell (0,0,0), comp 0, within a time level
    long long plane;    // px * py
    long long cstride;  // plane * (n2 + 2g)
    int px;             // row pitch in elements (multiple of 16 bytes)
    int n[3];           // valid extents
    int lo[3];          // valid lower corner, global index
    int level;          // level slot in merged launches
};

// One FillBoundary copy region: extents n, src/dst element offsets of the region's first
// cell (comp 0) within a time level, and the FArrayBoxes whose strides apply.
struct FbEntry {
    long long src, dst;
    int n[3];
    int sfab, dfab;
    int level;
};

// Division by a runtime constant d >= 1 for numerators below 2^31 (round-up multiplier,
// Granlund & Montgomery 1994): q = (umulhi(n, m) + n) >> s with s = ceil(log2 d),
// m = floor(2^32 (2^s - d) / d) + 1.
struct FastDiv {
    uint32_t m, s;
};
inline FastDiv make_fastdiv(uint32_t d) {
    uint32_t s = 0;
    while ((1ull << s) < d) ++s;
    return FastDiv{(uint32_t)(((1ull << 32) * ((1ull << s) - d)) / d + 1), s};
}

// Work unit of the fill kernel (one warp), self-contained so that a warp needs one load to start:
// cells [first, first + count) of one copy region in the linear order (comp, z, y, x).
// With vec != 0 every offset, stride and the x extent n0 count 16-byte vectors instead of
// elements (a region whose rows start and end on 16-byte boundaries on both sides).
struct FbTask {
    long long src, dst;    // offsets of the region's first cell, comp 0
    int s_pl, d_pl;        // plane strides (an FArrayBox has fewer than 2^31 elements)
    int s_cs, d_cs;        // component strides
    int s_px, d_px;        // row pitches
    int n0, n1, n2;        // region extents
    int first, count;
    int level;
    FastDiv f0, f1, f2;    // division by n0, n1, n2
    int vec;               // units: 0 elements, 1 16-byte vectors
    int pad_;
};
static_assert(sizeof(FbTask) % 8 == 0, "the fill kernel copies its task header in 8-byte words");

// Stencil work list entry: a logical tile of one box and one component (Sec. 3.2 tilebox()).
struct Tile {
    int fab;
    int comp;
    short x0, y0, z0;   // tile lower corner relative to the box's valid lower corner
    short tx, ty, tz;   // tile extents
};

// Coarse-fine interpolation (Sec. 2.3, mf_interp_cf): a run of fine ghost cells along one
// direction whose coarse cells floor(i/r) lie in one coarse box under one periodic shift.  The
// cells of all runs are numbered in one sequence; run q holds cells [rstart[q], rstart[q+1]).
struct InterpRun {
    long long fdst;     // fine element offset of the first cell (comp 0) within a time level
    long long cbase;    // element offset, in the owning coarse FAB, of global coarse index (0,0,0)
                        // after the run's periodic shift (may lie outside the FAB; only
                        // cbase + the offsets of the cells read are inside)
    int I, J, K;        // global fine index of the first cell
    int axis;           // direction the run advances in: 0 x, 1 y, 2 z
    int fstep;          // fine element stride along axis
    int fcs, ccs;       // component strides of the fine and coarse FABs (elements)
    int cpx, cplane;    // coarse row and plane pitch (elements; a FAB holds < 2^31 elements)
};

// Average-down region (Sec. 2.3): coarse valid cells [clo, clo + n) of one coarse FAB from one
// fine FAB, with every offset and stride the kernel needs.  The cells of all regions are
// numbered in one sequence, x fastest; region q holds cells [rstart[q], rstart[q+1]).
struct AvgRegion {
    long long fsrc;     // fine element offset of the first child of coarse cell clo (comp 0)
    long long cdst;     // coarse element offset of cell clo (comp 0)
    int fpx, fplane;    // fine row and plane pitch
    int cpx, cplane;    // coarse row and plane pitch
    int fcs, ccs;       // component strides
    int n[3];
    int pad_;
};

struct LevelPtrs {
    void *base[kMaxLev];
};

struct StencilParams {
    const void *src[kMaxLev];
    void *dst[kMaxLev];
    const void *u0[kMaxLev];  // Runge-Kutta stage: state at the start of the step (nullptr: plain step)
    double rk_a, rk_b;        // the stage writes rk_a * u0 + rk_b * (forward-Euler value)
    const FabInfo *ftab;
    const Tile *tiles;
    int ntiles;
    double lam[kMaxLev][kMaxComp];
};

// TMA-staged stencil: per FArrayBox, the shared-memory plane geometry of its tensor map.

constexpr int kMaxStages = 16;
constexpr int kMaxPush = 16;  // ghost-push pieces per tile
constexpr int kTileClasses = 5;  // box-size classes of the tile shapes (the host's tile_class)

struct TmaFab {
    int bx, by;   // box of one plane load: bx elements of each of by rows
    int ngrow;
    int xv;       // element of valid x = 0 within the loaded row
    int xs;       // row element where the loaded row starts (16-byte aligned): 0 for the whole
                  // row, or valid x = 0 when strips serve both x faces (valid cells only)
    int pad_;
};

// x halo of a tile taken straight from the neighbouring box (its valid cells), or -1 when
// the tile's own ghost columns hold it.  Coordinates are the neighbour tensor's (x, y, z) of
// the strip for the tile's first z plane.
struct TileStrip {
    int lfab, rfab;
    int lx, ly, lz;
    int rx, ry, rz;
    int lidx0, ridx0;    // strip column of the neighbour cell next to the face (x = -1 and x = n0, plus 1)
    int pfirst, pcount;  // this tile's ghost-push pieces
};

// Ghost push: cells [x0, x0+nx) x [y0, y0+ny) x [z0, z0+nz) of a tile (tile coordinates) are
// ghost cells of box dfab; dst is the element offset (comp 0) of the piece's first cell there.
struct PushPiece {
    long long dst;
    int x0, y0, z0, nx, ny, nz;
    int dfab;
    int full_row;  // the piece spans the tile's whole row and the destination rows match it
    int pad_;
};

struct StencilTmaParams {
    const CUtensorMap *maps;   // one per FArrayBox, over the source time level
    const CUtensorMap *smaps;  // strip maps (box XH x strip_rows), over the source time level
    const TileStrip *strips;   // per tile, or nullptr
    int strip_rows;            // rows of a strip load
    int strip_off;             // byte offset of the left strip in a slot; right strip follows
    int strip_bytes;           // bytes of one strip load (right strip at strip_off + strip_pitch)
    int strip_pitch;
    int strip_w;               // elements per strip row
    const TmaFab *tfab;
    const FabInfo *ftab;
    const Tile *tiles;
    const int *cta_tiles;      // CTA b takes tiles [cta_tiles[b], cta_tiles[b+1]); nullptr: tiles b, b + grid, ...
    int ntiles;
    int nstages;               // shared-memory ring slots (power of two)
    int nstages_log2;
    int slot_bytes;            // bytes per slot (multiple of 128)
    int pad_;
    void *dst[kMaxLev];
    int *err;                  // set non-zero when a bounded wait expires
    const PushPiece *push;     // ghost-push pieces (nullptr: no push)
    const void *u0[kMaxLev];   // Runge-Kutta stage: state at the start of the step (nullptr: plain step)
    double rk_a, rk_b;         // the stage writes rk_a * u0 + rk_b * (forward-Euler value)
    double lam[kMaxLev][kMaxComp];
    // fixed-point steps (MF_FIXED_DIFF; the level holds 64-bit fixed point): the grid state of
    // the input level (read), of the output level (written), and a third set cleared for the
    // launch after this one (see FixSet and mf_advance), and per component
    // fix_q = round(lam / den * 2^64)
    const struct FixSet *fix_in;
    struct FixSet *fix_out;
    struct FixSet *fix_clear;
    unsigned long long fix_q[kMaxComp];
};

// Grid state of one level in the fixed-point path, per component: M the OR of all |K| (its bit
// length is that of the largest |K|; 64-bit atomicOr), E the grid exponent (the level holds K = u / 2^E), key the high word of the largest
// |u| of an FP64 level (the first grid).  Three sets rotate over the steps of an advance.
struct FixSet {
    unsigned long long M[kMaxComp];
    int E[kMaxComp];
    unsigned int key[kMaxComp];
};

// Denominator of the integer weights of the fixed-point path at radius R (fixed_diff.cuh FixW).
inline int fix_den(int R) { return R == 1 ? 1 : R == 2 ? 12 : 5040; }

// ---- launchers (mf_kernels.cu, stencil_tma.cu); all asynchronous on `s`
cudaError_t launch_stencil_tma(int dtype, int R, bool fp64diff, int rows, int gb, int nt, const StencilTmaParams &p,
                               int grid, cudaStream_t s);
// the fixed-point-difference variant (FP64 storage, p.fix_* set; stencil_tma_fix.cu)
cudaError_t launch_stencil_tma_fix(int R, int rows, int gb, int nt, const StencilTmaParams &p, int grid, cudaStream_t s);
int tma_ctas_per_sm_fix(int R, int rows, int gb, int nt, int smem);
int tma_max_threads_fix(int R, int rows, int gb);  // largest CTA of a fixed-point schedule
bool tma_has_group_fix(int R, int rows, int gb);   // whether the fixed-point path has that schedule
// The conversion passes of a fixed-point advance over the valid cells of one level (in place):
// the largest |u| of every component of an FP64 level into set->key (atomicMax; set cleared by the
// caller); FP64 -> fixed point on the first grid, recording set->E and set->M (err |= 2 for a
// non-finite maximum); fixed point on grid set->E -> FP64.
cudaError_t launch_fix_emax(const void *base, const FabInfo *ftab, int nfab, int ncomp, int maxz, FixSet *set,
                            cudaStream_t s);
cudaError_t launch_fix_in(int R, void *base, const FabInfo *ftab, int nfab, int ncomp, int maxz, FixSet *set, int *err,
                          cudaStream_t s);
cudaError_t launch_fix_out(void *base, const FabInfo *ftab, int nfab, int ncomp, int maxz, const FixSet *set,
                           cudaStream_t s);
// the Runge-Kutta-stage variant (p.u0 set); launch_stencil_tma dispatches to it
cudaError_t launch_stencil_tma_rk(int dtype, int R, bool fp64diff, int rows, int gb, int nt, const StencilTmaParams &p,
                                  int grid, cudaStream_t s);
// whether the TMA stencil has a schedule with rows rows of gb-byte groups per thread
bool tma_has_group(int dtype, int R, int rows, int gb);
int tma_max_threads(int dtype, int R);  // largest CTA of the TMA stencil for a storage type and radius R
int tma_max_rows(int R);         // most rows of 16-byte groups a TMA stencil thread may compute
// resident CTAs per SM of the TMA stencil with nt threads and smem dynamic shared bytes (0: none)
int tma_ctas_per_sm(int dtype, int R, int rows, int gb, int nt, int smem);
cudaError_t launch_fill(int dtype, const LevelPtrs &lv, const FbTask *tasks, int ntasks, int grid, cudaStream_t s);
cudaError_t launch_stencil(int dtype, int R, bool fp64diff, const StencilParams &p, int bx, int by, int grid,
                           cudaStream_t s);
// untiled per-box baseline (one box per launch)
cudaError_t launch_stencil_plain(int dtype, int R, const void *src, void *dst, const FabInfo &f, double lam,
                                 int comp, cudaStream_t s);
cudaError_t launch_fill_plain(int dtype, void *base, const FabInfo *ftab, const FbEntry *ent, int count,
                              long long total, const int *cbeg, cudaStream_t s);
// Refluxing of the two-level advance (Berger-Colella flux correction).  A coarse face of the
// coarse-fine interface: the coarse cell C next to it lies in no fine box; the fine region is on
// C's high side (sc = +1) or low side (sc = -1) along direction d.
struct CFace {
    long long c_low;    // element offset (coarse level, comp 0) of the face's lower cell, in C's FArrayBox
    long long cstride;  // component stride of that FArrayBox
    long long dstride;  // its element stride along d
    int ffirst;         // the face's r^2 fine faces: FFace[ffirst .. ffirst + r^2)
    int sc;
};
// A fine face on the interface, seen from the fine box inside (its ghost cells hold the outside).
struct FFace {
    long long f_low;    // element offset (fine level, comp 0) of the face's lower cell
    long long cstride;
    long long dstride;
};
// An uncovered coarse cell next to the interface and its coarse faces CFace[efirst .. + ecount).
struct CCell {
    long long c_elem;
    long long cstride;
    int efirst, ecount;
};
struct RefluxW {
    double w[kMaxComp];  // per component: lam_c (coarse fluxes) or lam_f / r^3 (fine fluxes)
};
cudaError_t launch_cf_coarse_flux(int dtype, int R, const void *base, const CFace *faces, int n, int ncomp,
                                  const RefluxW &w, double *reg, cudaStream_t s);
cudaError_t launch_cf_fine_flux(int dtype, int R, const void *base, const CFace *faces, const FFace *ff, int n,
                                int nff, int ncomp, const RefluxW &w, double *reg, bool first, cudaStream_t s);
cudaError_t launch_reflux_apply(int dtype, void *base, const CCell *cells, int ncell, const CFace *faces, int ncomp,
                                const double *regc, const double *regf, cudaStream_t s);

// whole-level reduction of one component (RED_*), result written to out_dev (device)
enum { RED_SUM = 0, RED_MAX = 1, RED_MIN = 2, RED_NORM0 = 3, RED_NORM1 = 4, RED_NORM2 = 5 };
cudaError_t launch_reduce(int dtype, int op, const void *base, const FabInfo *ftab, const long long *rowpre, int nfab,
                          int comp, double2 *partials, int grid, double *out_dev, cudaStream_t s);
cudaError_t launch_scatter_dense(int dtype, void *base, const FabInfo *ftab, int nfab, const double *stage,
                                 const int dlo[3], const int dn[3], int z0, int z1, int comp, int ncomp_chunk,
                                 cudaStream_t s);
cudaError_t launch_gather_dense(int dtype, const void *base, const FabInfo *ftab, int nfab, double *stage,
                                const int dlo[3], const int dn[3], int z0, int z1, int comp, int ncomp_chunk,
                                cudaStream_t s);
// runs/rstart (nruns + 1 entries, rstart[nruns] = ncells)/wfirst (the run holding cell 32 w,
// one entry per 32 cells): the interpolation work list.
cudaError_t launch_interp(int dtype, void *fbase, const void *cold, const void *cnew, const InterpRun *runs,
                          const int *rstart, const int *wfirst, int nruns, int ncells, int ncomp, int ratio,
                          double alpha, cudaStream_t s);
// vec: every region's fine offsets and pitches are multiples of ratio (vector loads of r children)
cudaError_t launch_avgdown(int dtype, const void *fbase, void *cbase, const AvgRegion *regs, const int *rstart,
                           const int *wfirst, int nregs, int ncells, int ncomp, int ratio, bool vec, cudaStream_t s);

// Paired launches of the two-level advance (two independent jobs, one launch each would take).
struct InterpArgs {
    void *fbase;
    const void *cold, *cnew;
    const InterpRun *runs;
    const int *rstart, *wfirst;
    int nruns, ncells, ncomp, ratio;
    double alpha;
};
struct AvgArgs {
    const void *fbase;
    void *cbase;
    const AvgRegion *regs;
    const int *rstart, *wfirst;
    int nregs, ncells, ncomp, ratio;
    bool vec;
};
struct RefluxArgs {
    void *base;
    const CCell *cells;
    int ncell;
    const CFace *faces;
    int ncomp;
    const double *regc, *regf;
};
// a fine level's ghost fill and its coarse-fine interpolation (disjoint ghost cells)
cudaError_t launch_fill_interp(int dtype, const LevelPtrs &lv, const FbTask *tasks, int ntasks, const InterpArgs &ia,
                               cudaStream_t s);
// a fill of the new coarse level and the coarse face fluxes of the old one
cudaError_t launch_fill_cflux(int dtype, int R, const LevelPtrs &lv, const FbTask *tasks, int ntasks,
                              const void *cbase, const CFace *faces, int nface, int ncomp, const RefluxW &w,
                              double *reg, cudaStream_t s);
// the average-down (covered coarse cells) and the flux correction (uncovered ones)
cudaError_t launch_avg_reflux(int dtype, const AvgArgs &aa, const RefluxArgs &ra, cudaStream_t s);

int sm_count();

// Sets the message mf_last_error() returns on this thread; returns code.
int set_error(int code, const char *msg);

}  // namespace mfk
