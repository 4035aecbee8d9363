/*
 * mf.h -- C ABI of the GB300 MultiFab time-step sweep (libmf.so).
 *
 * The objects follow arXiv 1604.03570 ("BoxLib with Tiling"):
 *   Box        a rectangle of cells in index space, six integers (Sec. 3.1).
 *   FArrayBox  the data of one box grown by the ghost width, ncomp components, stored with
 *              x fastest, then y, z, component (Sec. 3.1).
 *   MultiFab   all FArrayBoxes of one level (Sec. 3.1, Fig. 1); here one handle per level,
 *              living on one GPU.
 *   MFIter     the loop over boxes, or over logical tiles of boxes (Sec. 3.2); here a
 *              device work list of (box, component, tile) entries consumed by persistent kernels.
 *
 * Conventions for every call:
 *   - Boxes are int[6] = {lo0, lo1, lo2, hi0, hi1, hi2}, inclusive bounds, in the index space
 *     of the level's domain.  The domain is periodic in x, y and z.  Cells are cubes of side
 *     dx = 1/N_x (N_x cells along x), so an N^3 domain is the unit cube.
 *   - Return 0 on success, a negative MF_E* code on error; mf_last_error() then gives a
 *     message (thread-local).  No call aborts the process.
 *   - Field memory is owned by the caller (e.g. allocated by PyTorch) and attached with
 *     mf_attach; it must outlive the handle.  The library allocates small device metadata
 *     (intersection and work lists, reduction partials) inside mf_attach and never again
 *     while advancing, so mf_advance can be captured and replayed as a CUDA graph.
 *   - Every call that touches field data is asynchronous on the attached stream, except
 *     mf_sum, mf_copy_to_host and mf_copy_fab_to_host, which synchronise that stream.
 *   - Host pointers passed in are only read during the call.
 */
#ifndef MF_H
#define MF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mf mf_t;

/* Storage type of the field.  F64 computes in FP64; F32 and BF16 compute in FP32. */
typedef enum { MF_F64 = 0, MF_F32 = 1, MF_BF16 = 2 } mf_dtype;

/* Centred (2R+1)-point Laplacian of order 2R per direction; the value is the radius R.
 * R = 1 is the paper's second-order heat kernel (Sec. 4.1, 7-point star); R = 4 is the
 * 9-cell-wide 8th-order stencil of the SMC code (Sec. 4.2, 25-point star). */
typedef enum { MF_LAP2_7PT = 1, MF_LAP4_13PT = 2, MF_LAP8_25PT = 4 } mf_stencil_kind;

/* mf_stencil.flags */
enum {
    MF_FP64_DIFF = 1,     /* FP32/BF16 storage: compute the flux differences in FP64 */
    MF_PLAIN_PER_BOX = 2, /* the untiled baseline of Sec. 3.1: one launch per box per phase,
                             launched eagerly, no work list, no graph */
    MF_REFLUX = 4,        /* mf_amr_advance only: Berger-Colella refluxing (see there) */
    MF_FIXED_DIFF = 8     /* mf_advance, FP64 storage, TMA kernel: the steps in exact 64-bit
                             fixed-point integer arithmetic (see mf_advance) */
};

typedef struct {
    int kind;                  /* mf_stencil_kind */
    const double *diffusivity; /* [ncomp] D_c > 0 */
    int flags;                 /* MF_FP64_DIFF | MF_PLAIN_PER_BOX | MF_REFLUX | MF_FIXED_DIFF */
} mf_stencil;

/* Error codes */
enum {
    MF_OK = 0,
    MF_EINVAL = -1,     /* bad argument: box outside the domain, overlapping boxes, bad sizes */
    MF_ENOMEM = -2,     /* host or device allocation failed */
    MF_ECUDA = -3,      /* a CUDA runtime call failed (message has the CUDA error string) */
    MF_EUNSTABLE = -4,  /* lam * 3 * |sigma_R(pi)| > 2: forward Euler would blow up */
    MF_EALIGN = -5,     /* attached pointer not 256-byte aligned or buffer too small */
    MF_ESTATE = -6      /* operation needs an attached handle (or a missing setup step) */
};

/*
 * mf_create -- a level whose boxes chop the domain [domain_lo, domain_hi] into pieces of
 * max_grid_size cells per side (the last piece along a direction takes the remainder).
 * Box order: x fastest, then y, then z.  Sec. 3: a level is a union of non-intersecting
 * grids; Sec. 3.1: MultiFab.  ngrow >= 0 ghost cells per side, 1 <= ncomp <= 16.
 * The handle is created on the host only; no CUDA call is made.
 */
int mf_create(mf_t **out, const int domain_lo[3], const int domain_hi[3], int max_grid_size,
              int ncomp, int ngrow, int dtype);

/*
 * mf_create_boxes -- a level from an explicit box list (nboxes * 6 ints).  Boxes must lie in
 * the domain and must not overlap; they need not cover the domain, nor be of one size or shape
 * (a refined level, Sec. 3).
 */
int mf_create_boxes(mf_t **out, const int domain_lo[3], const int domain_hi[3], const int *boxes,
                    int nboxes, int ncomp, int ngrow, int dtype);

/*
 * mf_create_regional -- a level from a box list, as mf_create_boxes, stored in regions.
 * Sec. 2 (TiDA, Fig. 2): a grid's data may be allocated as several regions, each one contiguous
 * block, and the tiles of the iteration space are logical, independent of that layout.  Here
 * the level's boxes are grouped into regions, rectangles that their boxes cover exactly with
 * sides of at most max_region cells (1 <= max_region <= 240), found by cutting the boxes'
 * bounding box along planes that cross no box (mf_box_regions); the FArrayBoxes, their ghost
 * cells and FillBoundary belong to the regions, and the boxes stay the level's cells and
 * logical tiles.  A level of many small boxes then keeps ghost cells only around its regions:
 * no fill between the boxes of one region.  Every computation gives the same bits as the
 * same boxes stored one FArrayBox each.
 * mf_nboxes, mf_get_boxes and mf_copy_fab_to_host / _from_host address the boxes as given:
 * the box grown by ngrow is read from its region, and only the box's own cells are written (its
 * ghost frame there is other boxes' cells or the region's ghost cells); mf_fb_regions, mf_get_fb_regions, mf_interp_cells,
 * mf_avgdown_cells, mf_reflux_faces, mf_step_bytes and mf_bytes describe the regions' storage.
 */
int mf_create_regional(mf_t **out, const int domain_lo[3], const int domain_hi[3], const int *boxes,
                       int nboxes, int ncomp, int ngrow, int dtype, int max_region);

/* The regions mf_create_regional makes from a box list (host only; boxes as for
 * mf_create_boxes, assumed disjoint): returns their number, writes region_of[i], the region
 * of box i, and, when regions_out is not NULL (room for nboxes * 6 ints), the regions as
 * {lo[3], hi[3]}.  A region is either a rectangle its boxes cover exactly, every side at most
 * max_region, or a single box that no cut separates from the others.  Sec. 2 (Fig. 2): regions
 * are the contiguous blocks a grid's data is allocated in. */
int mf_box_regions(const int *boxes, int nboxes, int max_region, int *regions_out, int *region_of);
/* The storage of a level (Sec. 2, Sec. 3.1): its FArrayBoxes (the regions of a regional level,
 * the boxes otherwise) as {lo[3], hi[3]} into regions_out (room for mf_nregions * 6 ints), and
 * the FArrayBox of each box into region_of (room for mf_nboxes ints); either may be NULL. */
int mf_nregions(const mf_t *mf);
int mf_get_regions(const mf_t *mf, int *regions_out, int *region_of);

/* Releases the handle (metadata, device work lists, graphs), after waiting for the work it queued
 * on its attached stream.  The field memory stays the caller's.  Sec. 3.1 gives a MultiFab no
 * explicit lifetime call; this is the end of the handle that mf_create made.  A NULL handle is
 * ignored. */
void mf_destroy(mf_t *mf);

/* Layout queries (host only): the level's boxes, the grids of Sec. 3 (the BoxArray of
 * Sec. 3.1), as {lo[3], hi[3]} each. */
int mf_nboxes(const mf_t *mf);
int mf_get_boxes(const mf_t *mf, int *boxes /* nboxes*6 */);
/* Bytes of device memory mf_attach needs: two time levels of all FArrayBoxes, each
 * FArrayBox 256-byte aligned, rows padded so that every valid row starts 16-byte aligned.
 * Sec. 3.1: an FArrayBox holds its grid's data, grown by the ghost cells, as one contiguous
 * array; here all FArrayBoxes of a level follow each other in one caller-owned allocation,
 * two time levels because the forward-Euler update of Sec. 4.1 is read out of place.
 * 0 for a NULL handle. */
size_t mf_bytes(const mf_t *mf);
/* Number of FillBoundary copy regions (box-box intersections incl. periodic images; Sec. 3.1's
 * ghost exchange) and the number of ghost cells per component they write. */
long long mf_fb_regions(const mf_t *mf, long long *ghost_cells_out);
/* Copies up to max regions (Sec. 3.1's intersection list) as 11 ints each: {dst box, src box, dst lo[3] (global index,
 * may lie outside the domain), src lo[3] (inside the domain), extent[3]}. */
long long mf_get_fb_regions(const mf_t *mf, int *out, long long max);

/*
 * mf_attach -- give the handle its field memory (mf_bytes(mf) bytes, 256-byte aligned, device
 * memory of the current device) and the CUDA stream (cudaStream_t, may be NULL for the
 * legacy stream) every later call runs on.  Builds and uploads the FillBoundary list and the
 * tile work list.  May be called again to move the handle to another buffer or stream.
 * Sec. 3.1: the FArrayBox data of a MultiFab are contiguous arrays, and every process holds
 * the list of all grids for communication within a level; here the caller allocates the
 * arrays and the library precomputes the box-box intersection list of FillBoundary once,
 * from that grid list.  MF_EALIGN for a misaligned or short buffer; MF_ENOMEM when the
 * metadata allocation fails.
 */
int mf_attach(mf_t *mf, void *dev_ptr, size_t bytes, void *cuda_stream);

/* Tile shape of the stencil sweep (Sec. 3.2 MFIter(mf, tilesize)); tile[d] <= 0 along a
 * direction means "whole box".  tile == NULL selects the autotuner on the next advance.
 * Synchronises the stream; may grow the device work list (the one allocation after attach,
 * never made while advancing). */
int mf_set_tile(mf_t *mf, const int tile[3]);
int mf_get_tile(const mf_t *mf, int tile[3]);

/* Stencil kernel variant (how the Sec. 4.1 kernel reads its neighbours; the paper has one CPU
 * kernel, so no counterpart of the choice).  MF_KERNEL_TMA (default): tile planes staged into shared memory by
 * TMA bulk-tensor copies (used whenever the tile shape fits, else the next one).
 * MF_KERNEL_GLOBAL: neighbours read through L1 from global memory.  Both give identical bits. */
enum { MF_KERNEL_TMA = 0, MF_KERNEL_GLOBAL = 1 };
int mf_set_kernel(mf_t *mf, int variant);

/* Schedule of the TMA stencil besides the tile shape (Sec. 3.2's tiling, GPU-side parameters): in[0] rows per thread (1 or 2; 0 = 2),
 * in[1] shared-memory ring slots (a power of two up to 16; 0 = by radius), in[2] bytes per
 * row group of a thread (16 or 32; 0 = 16).  Where a radius or storage type lacks the
 * combination the launch falls back to 16-byte groups and the rows the radius allows.
 * Results do not depend on the schedule (identical bits).  The autotuner, when on, overrides
 * it; MF_EINVAL for values out of range. */
int mf_set_schedule(mf_t *mf, const int in[3]);

/* The schedule in use (Sec. 3.2; after the autotuner, if it ran): {tile x, y, z, rows per thread, ring
 * slots, kernel variant in use (MF_KERNEL_*), bytes per row group of a thread (16 or 32)}.
 * A tile z extent of 0 means whole boxes, which the TMA kernel splits in z evenly over one
 * wave of CTAs. */
int mf_get_schedule(const mf_t *mf, int out[7]);

/* Tile shapes per box-size class (Sec. 3.2: the tile size may change from loop to loop; here it
 * may also change with the size of the box, within one launch).  A box's class is its y extent:
 * up to 8, 16, 32 or 64 cells, or above (classes 0-4).  mf_set_class_tile gives the boxes of
 * class cls the tile y extent ty and, where the level's tile has a z extent, the z extent tz
 * (0 = the whole box, -1 = the level's tile shape); it turns the autotuner off, and mf_set_tile
 * resets every class to -1.  mf_get_class_tiles writes per class {1 if the level has boxes of
 * that class else 0, ty, tz}.  Results do not depend on the tile shapes (identical bits).  The
 * autotuner, after choosing the level's schedule, times other shapes for each class holding at
 * least 5% of the cells and keeps those that make the launch faster by more than 2%.
 * MF_EINVAL for a class or extent out of range. */
int mf_set_class_tile(mf_t *mf, int cls, int ty, int tz);
int mf_get_class_tiles(const mf_t *mf, int out[15]);

/* The autotuner (Sec. 3.2 and Table 1: the tile size is a parameter whose best value depends on
 * the machine and the loop) keeps its choice per level geometry, storage type, components, ghost
 * width, radius, arithmetic, kernel and GPU for the life of the process.  When the environment variable
 * MF_AUTOTUNE_CACHE names a file, choices are also read from that file and appended to it, one
 * text line each (the key, then tile[3], rows, ring slots, group bytes, push, and the per-class
 * y and z extents), so that a later process skips the timing runs; unreadable lines are
 * ignored.  mf_autotune_cache_reset forgets the process's choices (the file, if any, is read
 * again at the next lookup).  Host only; always returns 0. */
int mf_autotune_cache_reset(void);

/*
 * Dense host arrays are (ncomp, Nz, Ny, Nx) doubles over the whole domain, x fastest.
 * mf_copy_from_host writes the valid cells of every box of the current time level
 * (ghosts unchanged); cells of the dense array outside every box are ignored.
 * mf_copy_to_host writes every dense cell: valid data where a box covers it, NaN elsewhere.
 * Both convert to/from the storage type on the GPU and stage through the non-current time
 * level, which they overwrite.  Sec. 3.1: an FArrayBox's index-space information turns its
 * 1-D array into a multi-dimensional one (component slowest, x fastest, the Fortran order the
 * paper's kernels see); these calls apply that map between the boxes and one dense array.
 * FP64 to BF16 rounds to nearest even; FP64 to FP32 rounds to nearest.
 */
int mf_copy_from_host(mf_t *mf, const double *dense);
int mf_copy_to_host(mf_t *mf, double *dense);

/* One box including ghosts, (ncomp, nz+2g, ny+2g, nx+2g) doubles, current time level: the
 * box's FArrayBox (Sec. 3.1), or on a regional level the box's window of its region (see
 * mf_create_regional: there _from_host writes the box's own cells only). */
int mf_copy_fab_to_host(mf_t *mf, int box, double *out);
int mf_copy_fab_from_host(mf_t *mf, int box, const double *in);

/*
 * mf_fill_boundary -- Sec. 3.1 mf.FillBoundary(): every ghost cell of every FArrayBox of the
 * current time level (faces, edges and corners) takes the value of the valid cell that owns
 * the same point of the periodic domain.  One fused copy kernel over the precomputed
 * intersection list.  Ghost cells no box owns are left unchanged.
 */
int mf_fill_boundary(mf_t *mf);

/*
 * mf_interp_cf -- coarse-to-fine ghost interpolation between AMR levels (Sec. 3; ratio 2 or
 * 4).  Every ghost cell of the fine level's current time level whose point lies in no fine
 * box gets the trilinear interpolant of the coarse data, each coarse value taken as
 * (1 - alpha) * crse_old + alpha * crse_new (current time levels of the two handles, which
 * may be the same handle).  The coarse level must cover its domain, have ngrow >= 1, have
 * its ghosts filled, and fine domain = ratio * coarse domain.  Runs on the fine handle's stream.
 * Arithmetic: FP64 for FP64 levels (the definition's order of operations, the weight product
 * (wz wy) wx, terms summed z, y, x ascending); FP32 for FP32 and BF16 levels, same order.
 */
int mf_interp_cf(mf_t *fine, const mf_t *crse_old, const mf_t *crse_new, double alpha, int ratio);

/* mf_interp_cells -- (Sec. 3, the interpolation of mf_interp_cf) the number of fine ghost cells
 * (per component) that mf_interp_cf writes:
 * the ghost cells of the fine boxes whose point lies in no fine box.  *runs_out (may be NULL)
 * gets the number of runs of the interpolation work list.  Host lists only: needs no attached
 * memory.  Negative error code (MF_EINVAL) for a bad ratio or layouts that do not nest. */
long long mf_interp_cells(const mf_t *fine, const mf_t *crse, int ratio, long long *runs_out);

/* mf_avgdown_cells -- (Sec. 3, the average-down of mf_average_down) the number of coarse cells
 * (per component) mf_average_down writes: the
 * coarse valid cells under the fine boxes.  *regions_out (may be NULL) gets the number of
 * (fine box, coarse box) regions of its work list.  Host lists only: needs no attached memory.
 * MF_EINVAL for a bad ratio, fine boxes not aligned to the ratio, or levels that do not nest. */
long long mf_avgdown_cells(const mf_t *fine, const mf_t *crse, int ratio, long long *regions_out);

/* mf_reflux_faces -- (Sec. 3's subcycled levels, the refluxing of mf_amr_advance) the number of
 * coarse faces of the coarse-fine interface that the
 * refluxing of mf_amr_advance (MF_REFLUX) corrects across: faces of coarse cells in no fine box
 * whose other side is covered by the fine level (periodic images included).  *cells_out (may
 * be NULL) gets the number of coarse cells corrected.  Host lists only: needs no attached
 * memory.  MF_EINVAL for a bad ratio, fine boxes not made of whole coarse cells, or levels that
 * do not nest. */
long long mf_reflux_faces(const mf_t *fine, const mf_t *crse, int ratio, long long *cells_out);

/* mf_average_down -- every coarse valid cell whose children are all fine valid cells becomes
 * their mean (current time levels): the r^3 children summed z, y, x ascending, times 1/r^3, in
 * FP64 for FP64 levels and FP32 for FP32/BF16 levels.  ratio 2 or 4; fine boxes must start and
 * end on multiples of ratio (MF_EINVAL otherwise).  Runs on the coarse handle's stream.
 * Sec. 3 (levels of a nested hierarchy whose mesh spacings differ by a ratio of 2 or 4) and
 * Sec. 1 (subcycled AMR time stepping) use the coarse data under a fine level without
 * defining how they are set; the reading taken here is the conservative one, the mean of the
 * children. */
int mf_average_down(const mf_t *fine, mf_t *crse, int ratio);

/*
 * mf_advance -- nsteps forward-Euler steps of u_t = D_c Lap u (Sec. 4.1): each step is
 * FillBoundary on the current level, then the flux-form stencil (face fluxes, then their
 * divergence) from the current into the other time level, then the two swap.  All boxes and
 * tiles go through one persistent launch per phase; the whole advance is captured once as a
 * CUDA graph and replayed.  With MF_PLAIN_PER_BOX it runs the untiled per-box baseline.
 * lam_c = D_c dt / dx^2 = D_c dt N_x^2.  Returns MF_EUNSTABLE if max_c lam_c * 3 |sigma_R(pi)| > 2.
 * Only the ghost cells the stencil reads are exchanged: x halos may be read straight from the
 * neighbour box, and the stencil may write the y/z face ghosts of the level it produces (the
 * autotuner times both ways).  The ghost cells of the result are therefore not all current:
 * call mf_fill_boundary before reading them.
 *
 * MF_FIXED_DIFF (FP64 storage; TMA kernel; not with MF_PLAIN_PER_BOX): the same operator
 * stepped in exact 64-bit integer arithmetic, with no FP64 arithmetic inside the time loop.  The
 * advance maps the level's valid cells once from FP64 to fixed point, K = u / 2^E on a grid per
 * component taken from the largest exponent present; every step forms the integer Laplacian L
 * exactly and writes K' = round((K 2^64 + L q) / 2^t), q = round(lam / den * 2^64) with den
 * the operator's common denominator (1, 12, 5040 for R = 1, 2, 4), on the next step's grid
 * (t = 64 - (E - E'), E' from the level maximum the step before reduced, so the precision
 * follows a decaying solution); after the last step the valid cells are mapped back to FP64.
 * |K| stays below 2^B, B = 58, 55, 46 bits for R = 1, 2, 4, so each step's error is a few units
 * of 2^E, about 2^(3 - B) max|u|.  The grids come from level-wide maxima, so the results are
 * bitwise independent of tiles and box layout.  After such an advance the ghost cells hold
 * fixed-point bit patterns, not FP64 values: call mf_fill_boundary before reading them.  A
 * non-finite value in the level makes the next synchronising call fail with MF_ECUDA.  FP64
 * arithmetic is slow next to memory bandwidth on some GPUs (GB300 issues about 2 FP64
 * operations per clock per SM); this path needs none per cell.
 */
int mf_advance(mf_t *mf, const mf_stencil *st, double dt, int nsteps);

/*
 * mf_amr_advance -- two-level subcycled advance (fine = crse refined by ratio).  Sec. 1 states
 * that BoxLib supports several time-subcycling modes for AMR and Sec. 3 that levels differ by a
 * ratio of 2 or 4, without defining a scheme; the reading taken here is the standard
 * Berger-Oliger subcycling below (coarse step first, then nsub fine substeps with coarse ghost
 * data linear in time, then the average-down).  Per coarse step,
 * FillBoundary + stencil on the coarse level; then nsub fine substeps of dt/nsub, each
 * FillBoundary + coarse-fine interpolation at alpha = s/nsub + stencil; then average-down
 * onto the new coarse level.  Both levels must have the same dtype and ncomp.
 * With MF_REFLUX in st->flags (Berger-Colella flux correction, which makes the two-level
 * advance conservative): every coarse cell that lies in no fine box but shares a face with the
 * fine region is corrected after the average-down by
 *   sc * (lam_f / r^3 * sum over substeps and the r^2 fine faces of F_f - lam_c * F_c),
 * F the face flux of the stencil (sum_m b_m (u_{i+m} - u_{i+1-m})), sc = +1 when the fine
 * region is on the cell's high side, -1 on its low side; fluxes in FP64 from the coarse state at
 * the start of the step and from each substep's fine state after its fill and interpolation.
 * The fine boxes must consist of whole coarse cells (MF_EINVAL otherwise).
 * Inside the advance each level exchanges only the ghost cells that are read (the coarse level:
 * the stencil's faces and the cells the interpolation and the flux registers read); the ghost
 * cells of the results are not all current.
 */
int mf_amr_advance(mf_t *crse, mf_t *fine, const mf_stencil *st, double dt_crse, int ncrse_steps, int nsub,
                   int ratio);

/* Runge-Kutta advance (Sec. 4.2: SMC integrates its 8th-order operator with a third-order
 * Runge-Kutta method; read as the three-stage SSP scheme of Shu and Osher):
 *   u1 = E(u),  u2 = 3/4 u + 1/4 E(u1),  u_new = 1/3 u + 2/3 E(u2),
 * E(v) = v + lam * div F(v) being one FillBoundary + forward-Euler flux-form step (mf_advance).
 * The stages need a third level of the handle's layout: mf_stage_bytes() bytes of device
 * memory, 256-byte aligned, owned by the caller and attached once with mf_attach_stage (it must
 * outlive the handle; MF_EALIGN if misaligned or too small, MF_ESTATE before mf_attach).
 * mf_rk3_advance runs nsteps steps (3 stencil launches each) as one CUDA graph on the attached
 * stream, asynchronously; the result is the current level.  Same stencils, flags (except
 * MF_PLAIN_PER_BOX: MF_EINVAL) and stability check as mf_advance; MF_ESTATE without a stage
 * level. */
size_t mf_stage_bytes(const mf_t *mf);
int mf_attach_stage(mf_t *mf, void *dev_ptr, size_t bytes);
int mf_rk3_advance(mf_t *mf, const mf_stencil *st, double dt, int nsteps);

/* mf_sum -- sum of component comp over all valid cells of the current time level, FP64 with
 * compensated (Neumaier) accumulation; synchronises the stream.  Sec. 3.1 whole-level
 * reduction (the paper's example is mf.max(0)). */
int mf_sum(mf_t *mf, int comp, double *out);

/* mf_reduce -- whole-level reduction of component comp over all valid cells of the current time
 * level (Sec. 3.1: a MultiFab answers sum, max and norm queries; the paper's example is
 * mf.max(0)); synchronises the stream and writes the result to *out.
 *   MF_RED_SUM    sum of u            (FP64, Neumaier-compensated; = mf_sum)
 *   MF_RED_MAX    max u               (exact)
 *   MF_RED_MIN    min u               (exact)
 *   MF_RED_NORM0  max |u|             (exact)
 *   MF_RED_NORM1  sum |u|             (FP64, compensated)
 *   MF_RED_NORM2  sqrt(sum u^2)       (squares rounded to FP64, sum compensated, then sqrt)
 * NaN values are skipped by MAX, MIN and NORM0.  The rows of the boxes are reduced in a fixed
 * order and tree, so the bits depend only on the box layout.  MF_EINVAL for a bad component or
 * operation, MF_ESTATE before mf_attach. */
enum { MF_RED_SUM = 0, MF_RED_MAX = 1, MF_RED_MIN = 2, MF_RED_NORM0 = 3, MF_RED_NORM1 = 4, MF_RED_NORM2 = 5 };
int mf_reduce(mf_t *mf, int comp, int op, double *out);

/* Algorithmic bytes per step of the sweep (Sec. 4.1's fill and kernel): S*C*(2V + 2G + G_face)
 * (valid cells read and written, ghost cells copied, face ghosts read by the stencil of radius
 * R). */
double mf_step_bytes(const mf_t *mf, int R);

/* Phase timing (Sec. 4.1 times the ghost fill and the kernel separately): when on, the
 * graph of mf_advance also records a CUDA event wherever the kind of launch changes (fill to
 * stencil or back; consecutive stencil launches have no event between them).  mf_phase_ms
 * then returns the summed device time of the FillBoundary phases (out[0]) and of the stencil
 * phases (out[1]) of the last mf_advance on this handle, waiting for it to finish;
 * MF_ESTATE when that advance was not timed. */
int mf_set_timing(mf_t *mf, int on);
int mf_phase_ms(mf_t *mf, double out[2]);

/* Kernel launches of the last mf_advance (or, on the coarse handle, mf_amr_advance) call
 * (measurement support; the paper counts threads, not launches, so no counterpart):
 * out[0] ghost-fill (and, with MF_FIXED_DIFF, the three conversion passes), out[1] stencil,
 * out[2] coarse-fine interpolation and flux-register,
 * out[3] average-down and reflux launches.  Launches whose work list is empty are not made and not counted. */
int mf_launch_count(const mf_t *mf, int out[4]);

/* Measured FP64 fused multiply-add throughput of the current GPU in TFLOP/s (2 flops per
 * FMA): 8 independent FMA chains per thread, 8 CTAs of 256 threads per SM, best of three
 * timed launches on `stream` (cudaStream_t; NULL = legacy stream).  The ceiling of the FP64
 * sweep on parts whose FP64 rate is low next to their memory bandwidth.  Measurement support,
 * not part of the method (no counterpart in the paper); allocates and frees 8 bytes of device memory and synchronises. */
int mf_fp64_fma_rate(double *tflops, void *stream);

/* Which time level (0 or 1) is current (Sec. 4.1's out-of-place update alternates them). */
int mf_current(const mf_t *mf);

/* The thread-local message of the last failing call (error reporting: no counterpart in the
 * paper). */
const char *mf_last_error(void);

/*
 * mf_sum_strided_noalloc -- the compensated FP64 sum of mf_sum for one strided 3-D device
 * array, for callers that cannot allocate device memory: code running while another component
 * owns every device allocation (a caching allocator or a fixed memory pool), real-time loops
 * where an allocation could stall or fail, plug-ins in processes that forbid new allocations.
 * It calls no cudaMalloc, cudaFree or allocating library routine and needs no mf_t handle.
 * The paper has no counterpart of this entry point.
 *
 * data   device pointer (current device) to element (0,0,0); element (x, y, z) is at
 *        data + x + y*sy + z*sz (strides in elements, sy >= nx, sz >= sy*ny); dtype MF_F64,
 *        MF_F32 or MF_BF16.  nx*ny*nz <= 268,435,456 cells, else MF_EINVAL.
 * out    host pointer receiving the sum.  stream: cudaStream_t (NULL = legacy stream); the
 *        call enqueues two kernels and a copy on it and then waits for that stream, so it
 *        returns MF_ESTATE, enqueueing nothing, when the stream is capturing a graph.
 * Scratch: a file-scope device array of 1 MiB (65,536 block partials), present on every GPU
 * that loads the library until the process exits.  The first call on a device looks up the
 * array's device address (with that device current) and caches it.  Every call reuses the
 * same array, so calls whose kernels overlap on the GPU (other streams, other host threads)
 * race and must be serialised by the caller.
 */
int mf_sum_strided_noalloc(const void *data, int dtype, int nx, int ny, int nz, long long sy, long long sz,
                           double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MF_H */
