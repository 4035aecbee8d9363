/*
 * mf_oracle.c -- plain, slow, FP64 CPU oracle for the MultiFab time-step sweep of
 * "BoxLib with Tiling" (arXiv 1604.03570).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or calls
 * this file; only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code, header, table or constant with the CUDA path.
 *
 * Every routine is the plain definition of one step of the method, written for a
 * reader to check by eye against the paper:
 *   - Box / FArrayBox: a grid is a Box of six integers (Sec. 3.1); an FArrayBox holds
 *     ncomp components over the Box grown by the ghost width, stored contiguously with
 *     x fastest, then y, z and component (Fortran order, Sec. 3.1 listing of f(lo,hi,a,...)).
 *   - FillBoundary (Sec. 3.1, mf.FillBoundary(); Sec. 3.3 local copies): every ghost cell
 *     of every FArrayBox takes the value of the valid cell that owns the same point of the
 *     periodic domain.  The owner is found by linear search, no intersection lists.
 *   - Heat-equation kernel (Sec. 4.1): forward Euler with centred differences computed
 *     in two steps -- one loop per direction for the face fluxes, then one loop for the
 *     divergence of the flux.  The update is out of place (old -> new).
 *   - The direct (non-flux) form of the same operator, used only as a cross-check.
 *   - Coarse-to-fine ghost interpolation and average-down between AMR levels (Sec. 3,
 *     levels with refinement ratio 2 or 4; the paper names the inter-level copy but not
 *     its formula -- the readings are trilinear in space, linear in time, and the mean of
 *     the children).
 *
 * The paper's threaded loop (Sec. 3.3: the iterations over tiles shared among OpenMP threads) is
 * orc_advance_omp: the same per-box work, distributed over the boxes of a level with an OpenMP
 * parallel loop, giving the same bits as orc_advance (a reported CPU baseline, not part of the
 * compared method).
 *
 * Compile with -O2 -ffp-contract=off so that every product and sum is rounded on its own.
 * All arrays are double precision.  Boxes are passed as int[6] = {lo0,lo1,lo2,hi0,hi1,hi2}
 * with inclusive bounds.  The FArrayBoxes of a level are stored back to back in box order.
 */
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- boxes and layout */

static long box_len(const int *b, int d, int g) { return (long)b[3 + d] - b[d] + 1 + 2L * g; }

static long fab_cells(const int *b, int g) { return box_len(b, 0, g) * box_len(b, 1, g) * box_len(b, 2, g); }

/* Offset (in doubles) of each FArrayBox of the level in the back-to-back storage. */
long orc_fab_offset(int nbox, const int *boxes, int g, int ncomp, int ib)
{
    long off = 0;
    for (int b = 0; b < ib && b < nbox; ++b) off += fab_cells(boxes + 6 * b, g) * ncomp;
    return off;
}

long orc_level_size(int nbox, const int *boxes, int g, int ncomp)
{
    return orc_fab_offset(nbox, boxes, g, ncomp, nbox);
}

/* Offsets of all FArrayBoxes (caller frees). */
static long *fab_offsets(int nbox, const int *boxes, int g, int ncomp)
{
    long *off = (long *)malloc(sizeof(long) * (nbox + 1));
    off[0] = 0;
    for (int b = 0; b < nbox; ++b) off[b + 1] = off[b] + fab_cells(boxes + 6 * b, g) * ncomp;
    return off;
}

/* Index of global cell (i,j,k), component c inside the FArrayBox of box b (grown by g). */
static long fab_index(const int *b, int g, int i, int j, int k, int c)
{
    long nx = box_len(b, 0, g), ny = box_len(b, 1, g), nz = box_len(b, 2, g);
    long x = i - (b[0] - g), y = j - (b[1] - g), z = k - (b[2] - g);
    return ((c * nz + z) * ny + y) * nx + x;
}

static int box_contains(const int *b, int i, int j, int k)
{
    return i >= b[0] && i <= b[3] && j >= b[1] && j <= b[4] && k >= b[2] && k <= b[5];
}

/* First box of the list whose valid region holds (i,j,k); -1 if none. */
static int find_owner(int nbox, const int *boxes, int i, int j, int k)
{
    for (int a = 0; a < nbox; ++a)
        if (box_contains(boxes + 6 * a, i, j, k)) return a;
    return -1;
}

/* Floor division and periodic wrap of an index into [lo, hi]. */
static int floor_div(int a, int b) { int q = a / b; if ((a % b != 0) && ((a < 0) != (b < 0))) --q; return q; }
static int wrap(int i, int lo, int hi) { int L = hi - lo + 1; int r = (i - lo) % L; if (r < 0) r += L; return lo + r; }

/*
 * Domain chopped into boxes of max_grid_size per side; the last box along a direction
 * takes the remainder.  Box index runs x fastest, then y, then z.  Returns the number of
 * boxes; writes at most maxbox of them.
 */
int orc_chop(const int *dlo, const int *dhi, int mgs, int *boxes, int maxbox)
{
    int n[3];
    for (int d = 0; d < 3; ++d) n[d] = (dhi[d] - dlo[d] + 1 + mgs - 1) / mgs;
    int count = 0;
    for (int bz = 0; bz < n[2]; ++bz)
        for (int by = 0; by < n[1]; ++by)
            for (int bx = 0; bx < n[0]; ++bx) {
                int idx[3] = {bx, by, bz};
                if (count < maxbox) {
                    int *b = boxes + 6 * count;
                    for (int d = 0; d < 3; ++d) {
                        b[d] = dlo[d] + idx[d] * mgs;
                        b[3 + d] = b[d] + mgs - 1;
                        if (b[3 + d] > dhi[d]) b[3 + d] = dhi[d];
                    }
                }
                ++count;
            }
    return count;
}

/* ---------------------------------------------------------------- dense <-> FArrayBoxes */

/* Copy the valid region of every box out of a dense domain array (ncomp, Nz, Ny, Nx); ghost
 * cells are set to NaN so that a read of an unfilled ghost cannot go unnoticed. */
void orc_fabs_from_dense(int nbox, const int *boxes, const int *dlo, const int *dhi, int g, int ncomp,
                         const double *dense, double *fabs)
{
    long Nx = dhi[0] - dlo[0] + 1, Ny = dhi[1] - dlo[1] + 1, Nz = dhi[2] - dlo[2] + 1;
    long off = 0;
    for (int b = 0; b < nbox; ++b) {
        const int *B = boxes + 6 * b;
        long cells = fab_cells(B, g) * ncomp;
        for (long q = 0; q < cells; ++q) fabs[off + q] = NAN;
        for (int c = 0; c < ncomp; ++c)
            for (int k = B[2]; k <= B[5]; ++k)
                for (int j = B[1]; j <= B[4]; ++j)
                    for (int i = B[0]; i <= B[3]; ++i)
                        fabs[off + fab_index(B, g, i, j, k, c)] =
                            dense[((c * Nz + (k - dlo[2])) * Ny + (j - dlo[1])) * Nx + (i - dlo[0])];
        off += cells;
    }
}

void orc_dense_from_fabs(int nbox, const int *boxes, const int *dlo, const int *dhi, int g, int ncomp,
                         const double *fabs, double *dense)
{
    long Nx = dhi[0] - dlo[0] + 1, Ny = dhi[1] - dlo[1] + 1, Nz = dhi[2] - dlo[2] + 1;
    long off = 0;
    for (int b = 0; b < nbox; ++b) {
        const int *B = boxes + 6 * b;
        for (int c = 0; c < ncomp; ++c)
            for (int k = B[2]; k <= B[5]; ++k)
                for (int j = B[1]; j <= B[4]; ++j)
                    for (int i = B[0]; i <= B[3]; ++i)
                        dense[((c * Nz + (k - dlo[2])) * Ny + (j - dlo[1])) * Nx + (i - dlo[0])] =
                            fabs[off + fab_index(B, g, i, j, k, c)];
        off += fab_cells(B, g) * ncomp;
    }
}

/* ---------------------------------------------------------------- FillBoundary */

/*
 * Sec. 3.1 mf.FillBoundary(): every ghost cell of every FArrayBox (faces, edges and
 * corners of the grown box) takes the value of the valid cell that owns the same point of
 * the periodic domain.  Ghost cells whose point no box owns (a level that does not cover
 * the domain) are left untouched.  Returns the number of ghost cells written per component.
 */
/* the ghost cells of box b (writes only them; reads valid cells of other boxes) */
static long fill_box(int b, int nbox, const int *boxes, const int *dlo, const int *dhi, int g, int ncomp,
                     const long *off, double *data)
{
    long written = 0;
    const int *B = boxes + 6 * b;
    long offb = off[b];
    for (int k = B[2] - g; k <= B[5] + g; ++k)
        for (int j = B[1] - g; j <= B[4] + g; ++j)
            for (int i = B[0] - g; i <= B[3] + g; ++i) {
                if (box_contains(B, i, j, k)) continue;
                int wi = wrap(i, dlo[0], dhi[0]), wj = wrap(j, dlo[1], dhi[1]), wk = wrap(k, dlo[2], dhi[2]);
                int a = find_owner(nbox, boxes, wi, wj, wk);
                if (a < 0) continue;
                const int *A = boxes + 6 * a;
                long offa = off[a];
                for (int c = 0; c < ncomp; ++c)
                    data[offb + fab_index(B, g, i, j, k, c)] = data[offa + fab_index(A, g, wi, wj, wk, c)];
                ++written;
            }
    return written;
}

long orc_fill_boundary(int nbox, const int *boxes, const int *dlo, const int *dhi, int g, int ncomp, double *data)
{
    long written = 0;
    long *off = fab_offsets(nbox, boxes, g, ncomp);
    for (int b = 0; b < nbox; ++b) written += fill_box(b, nbox, boxes, dlo, dhi, g, ncomp, off, data);
    free(off);
    return written;
}

/* ---------------------------------------------------------------- stencils */

/*
 * Sec. 4.1 heat-equation kernel, flux form, out of place:
 *   face flux   F_{i+1/2} = sum_{m=1..R} b_m (u_{i+m} - u_{i+1-m})      (one loop per direction,
 *                                                                        over the nodal face box)
 *   divergence  u_new_i = u_i + lam_c * sum_d (F^d_{i+1/2} - F^d_{i-1/2}) (one loop)
 * b[0..R-1] holds b_1..b_R; lam[c] = D_c dt / dx^2.  Reads the ghost cells of src
 * (FillBoundary must have run) and writes the valid cells of dst only.
 */
/* the valid cells of box b of dst */
static void stencil_flux_box(int b, const int *boxes, int g, int ncomp, int R, const double *bcoef, const double *lam,
                             const long *offs, const double *src, double *dst)
{
    {
        const int *B = boxes + 6 * b;
        long off = offs[b];
        long n[3] = {B[3] - B[0] + 1, B[4] - B[1] + 1, B[5] - B[2] + 1};
        /* one face array per direction: extent n+1 along that direction */
        double *F[3];
        long fn[3][3];
        for (int d = 0; d < 3; ++d) {
            for (int e = 0; e < 3; ++e) fn[d][e] = n[e] + (e == d ? 1 : 0);
            F[d] = (double *)malloc(sizeof(double) * fn[d][0] * fn[d][1] * fn[d][2]);
        }
        for (int c = 0; c < ncomp; ++c) {
            /* flux loops: face f along direction d lies between cells f-1 and f */
            for (int d = 0; d < 3; ++d) {
                for (long z = 0; z < fn[d][2]; ++z)
                    for (long y = 0; y < fn[d][1]; ++y)
                        for (long x = 0; x < fn[d][0]; ++x) {
                            int p[3] = {B[0] + (int)x, B[1] + (int)y, B[2] + (int)z};
                            double flux = 0.0;
                            for (int m = 1; m <= R; ++m) {
                                int hi_[3] = {p[0], p[1], p[2]}, lo_[3] = {p[0], p[1], p[2]};
                                hi_[d] = p[d] - 1 + m; /* u_{i+m}   with i = f-1 */
                                lo_[d] = p[d] - m;     /* u_{i+1-m} with i = f-1 */
                                double diff = src[off + fab_index(B, g, hi_[0], hi_[1], hi_[2], c)] -
                                              src[off + fab_index(B, g, lo_[0], lo_[1], lo_[2], c)];
                                flux = flux + bcoef[m - 1] * diff;
                            }
                            F[d][(z * fn[d][1] + y) * fn[d][0] + x] = flux;
                        }
            }
            /* divergence loop over the valid cells */
            for (long z = 0; z < n[2]; ++z)
                for (long y = 0; y < n[1]; ++y)
                    for (long x = 0; x < n[0]; ++x) {
                        long q[3] = {x, y, z};
                        double div = 0.0;
                        for (int d = 0; d < 3; ++d) {
                            long up[3] = {q[0], q[1], q[2]};
                            up[d] += 1;
                            double fp = F[d][(up[2] * fn[d][1] + up[1]) * fn[d][0] + up[0]];
                            double fm = F[d][(q[2] * fn[d][1] + q[1]) * fn[d][0] + q[0]];
                            div = div + (fp - fm);
                        }
                        int i = B[0] + (int)x, j = B[1] + (int)y, k = B[2] + (int)z;
                        long at = off + fab_index(B, g, i, j, k, c);
                        dst[at] = src[at] + lam[c] * div;
                    }
        }
        for (int d = 0; d < 3; ++d) free(F[d]);
    }
}

void orc_stencil_flux(int nbox, const int *boxes, int g, int ncomp, int R, const double *bcoef, const double *lam,
                      const double *src, double *dst)
{
    long *offs = fab_offsets(nbox, boxes, g, ncomp);
    for (int b = 0; b < nbox; ++b) stencil_flux_box(b, boxes, g, ncomp, R, bcoef, lam, offs, src, dst);
    free(offs);
}

/*
 * The same operator in direct form, u_new = u + lam_c * sum_d (c_0 u + sum_m c_m (u_{+m} + u_{-m})),
 * with ccoef[0..R] = c_0..c_R.  A cross-check of the flux form, not part of the method.
 */
void orc_stencil_direct(int nbox, const int *boxes, int g, int ncomp, int R, const double *ccoef, const double *lam,
                        const double *src, double *dst)
{
    long *offs = fab_offsets(nbox, boxes, g, ncomp);
    for (int b = 0; b < nbox; ++b) {
        const int *B = boxes + 6 * b;
        long off = offs[b];
        for (int c = 0; c < ncomp; ++c)
            for (int k = B[2]; k <= B[5]; ++k)
                for (int j = B[1]; j <= B[4]; ++j)
                    for (int i = B[0]; i <= B[3]; ++i) {
                        double u = src[off + fab_index(B, g, i, j, k, c)];
                        double lap = 0.0;
                        for (int d = 0; d < 3; ++d) {
                            double s = ccoef[0] * u;
                            for (int m = 1; m <= R; ++m) {
                                int pp[3] = {i, j, k}, pm[3] = {i, j, k};
                                pp[d] += m;
                                pm[d] -= m;
                                s = s + ccoef[m] * (src[off + fab_index(B, g, pp[0], pp[1], pp[2], c)] +
                                                    src[off + fab_index(B, g, pm[0], pm[1], pm[2], c)]);
                            }
                            lap = lap + s;
                        }
                        dst[off + fab_index(B, g, i, j, k, c)] = u + lam[c] * lap;
                    }
    }
    free(offs);
}

/*
 * nsteps forward-Euler steps: FillBoundary(old), flux-form stencil old -> new, swap.
 * Returns 0 when the result is in a, 1 when it is in b.
 */
int orc_advance(int nbox, const int *boxes, const int *dlo, const int *dhi, int g, int ncomp, int R,
                const double *bcoef, const double *lam, int nsteps, double *a, double *b)
{
    double *cur = a, *nxt = b;
    for (int s = 0; s < nsteps; ++s) {
        orc_fill_boundary(nbox, boxes, dlo, dhi, g, ncomp, cur);
        orc_stencil_flux(nbox, boxes, g, ncomp, R, bcoef, lam, cur, nxt);
        double *t = cur; cur = nxt; nxt = t;
    }
    return cur == a ? 0 : 1;
}

/* The threads orc_advance_omp uses (1 when the library was built without OpenMP). */
int orc_omp_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * orc_advance with the paper's threaded loop (Sec. 3.3): in each phase the boxes are shared among
 * OpenMP threads.  Every box's ghost fill writes only that box's ghost cells and reads only valid
 * cells, and every box's stencil writes only that box's valid cells, so the bits equal orc_advance's.
 */
int orc_advance_omp(int nbox, const int *boxes, const int *dlo, const int *dhi, int g, int ncomp, int R,
                    const double *bcoef, const double *lam, int nsteps, double *a, double *b)
{
    double *cur = a, *nxt = b;
    long *off = fab_offsets(nbox, boxes, g, ncomp);
    for (int s = 0; s < nsteps; ++s) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
        for (int i = 0; i < nbox; ++i) fill_box(i, nbox, boxes, dlo, dhi, g, ncomp, off, cur);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
        for (int i = 0; i < nbox; ++i) stencil_flux_box(i, boxes, g, ncomp, R, bcoef, lam, off, cur, nxt);
        double *t = cur; cur = nxt; nxt = t;
    }
    free(off);
    return cur == a ? 0 : 1;
}

/* ---------------------------------------------------------------- AMR: interpolation, average-down */

/*
 * Position of fine cell i_f, refinement ratio r, in coarse index units: x = (2 i_f + 1 - r) / (2 r)
 * (cell centres: (i_f + 1/2)/r - 1/2).  Linear interpolation uses coarse cells k0 = floor(x) and
 * k0 + 1 with weights 1 - t and t, t = x - k0.  For r = 2 this gives {1/4, 3/4} on {k-1, k} for
 * i_f = 2k and {3/4, 1/4} on {k, k+1} for i_f = 2k + 1.
 */
static void lin_weights(int i_f, int r, int *k0, double *w0, double *w1)
{
    int num = 2 * i_f + 1 - r, den = 2 * r;
    *k0 = floor_div(num, den);
    double t = (double)(num - den * (*k0)) / (double)den;
    *w0 = 1.0 - t;
    *w1 = t;
}

/*
 * Coarse-to-fine ghost interpolation: every ghost cell of a fine FArrayBox whose point of
 * the periodic fine domain lies in no fine box (fine-fine copies take precedence) gets
 * the trilinear interpolant of the coarse data, each coarse value taken linearly in time,
 * (1 - alpha) * cold + alpha * cnew.  The coarse level must cover its domain; coarse
 * indices wrap periodically.  Returns the number of fine ghost cells written per component.
 */
long orc_interp_cf(int nf, const int *fboxes, const int *fdlo, const int *fdhi, int gf,
                   int nc, const int *cboxes, const int *cdlo, const int *cdhi, int gc,
                   int ncomp, int ratio, double alpha, const double *cold, const double *cnew, double *fdata)
{
    long written = 0;
    long *foff = fab_offsets(nf, fboxes, gf, ncomp);
    long *coff = fab_offsets(nc, cboxes, gc, ncomp);
    for (int b = 0; b < nf; ++b) {
        const int *B = fboxes + 6 * b;
        long offb = foff[b];
        for (int k = B[2] - gf; k <= B[5] + gf; ++k)
            for (int j = B[1] - gf; j <= B[4] + gf; ++j)
                for (int i = B[0] - gf; i <= B[3] + gf; ++i) {
                    if (box_contains(B, i, j, k)) continue;
                    int wi = wrap(i, fdlo[0], fdhi[0]), wj = wrap(j, fdlo[1], fdhi[1]), wk = wrap(k, fdlo[2], fdhi[2]);
                    if (find_owner(nf, fboxes, wi, wj, wk) >= 0) continue;
                    int kx, ky, kz;
                    double wx[2], wy[2], wz[2];
                    lin_weights(i, ratio, &kx, &wx[0], &wx[1]);
                    lin_weights(j, ratio, &ky, &wy[0], &wy[1]);
                    lin_weights(k, ratio, &kz, &wz[0], &wz[1]);
                    for (int c = 0; c < ncomp; ++c) {
                        double v = 0.0;
                        for (int dz = 0; dz < 2; ++dz)
                            for (int dy = 0; dy < 2; ++dy)
                                for (int dx = 0; dx < 2; ++dx) {
                                    int ci = wrap(kx + dx, cdlo[0], cdhi[0]);
                                    int cj = wrap(ky + dy, cdlo[1], cdhi[1]);
                                    int ck = wrap(kz + dz, cdlo[2], cdhi[2]);
                                    int a = find_owner(nc, cboxes, ci, cj, ck);
                                    if (a < 0) { written = -1; goto done; } /* coarse level must cover the domain */
                                    const int *A = cboxes + 6 * a;
                                    long at = coff[a] + fab_index(A, gc, ci, cj, ck, c);
                                    double tv = (1.0 - alpha) * cold[at] + alpha * cnew[at];
                                    v = v + (wz[dz] * wy[dy] * wx[dx]) * tv;
                                }
                        fdata[offb + fab_index(B, gf, i, j, k, c)] = v;
                    }
                    ++written;
                }
    }
done:
    free(foff);
    free(coff);
    return written;
}

/*
 * Average-down: every coarse valid cell whose ratio^3 children lie in a fine box becomes
 * the mean of those children, summed z, y, x ascending.  Returns the number of coarse cells
 * written per component.
 */
long orc_average_down(int nf, const int *fboxes, int gf, int nc, const int *cboxes, int gc,
                      int ncomp, int ratio, const double *fdata, double *cdata)
{
    long written = 0;
    long *foff = fab_offsets(nf, fboxes, gf, ncomp);
    long *coff = fab_offsets(nc, cboxes, gc, ncomp);
    for (int a = 0; a < nc; ++a) {
        const int *A = cboxes + 6 * a;
        long offa = coff[a];
        for (int k = A[2]; k <= A[5]; ++k)
            for (int j = A[1]; j <= A[4]; ++j)
                for (int i = A[0]; i <= A[3]; ++i) {
                    int f = find_owner(nf, fboxes, i * ratio, j * ratio, k * ratio);
                    if (f < 0) continue;
                    const int *B = fboxes + 6 * f;
                    long offb = foff[f];
                    for (int c = 0; c < ncomp; ++c) {
                        double s = 0.0;
                        for (int z = 0; z < ratio; ++z)
                            for (int y = 0; y < ratio; ++y)
                                for (int x = 0; x < ratio; ++x)
                                    s = s + fdata[offb + fab_index(B, gf, i * ratio + x, j * ratio + y, k * ratio + z, c)];
                        cdata[offa + fab_index(A, gc, i, j, k, c)] = s / (double)(ratio * ratio * ratio);
                    }
                    ++written;
                }
    }
    free(foff);
    free(coff);
    return written;
}
