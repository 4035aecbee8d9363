// mf_host.cpp -- host side of libmf: Box algebra, FArrayBox layout, FillBoundary
// intersection lists, tile work lists, coarse-fine lists, CUDA-graph capture and the
// extern "C" entry points declared in include/mf.h.
//
// Correspondence with arXiv 1604.03570:
//   Box / BoxArray chop          Sec. 3 (levels of non-intersecting grids), Sec. 3.1 (Box)
//   FArrayBox layout             Sec. 3.1 (contiguous, x fastest, ghost cells around the box)
//   FillBoundary metadata        Sec. 3.1 / 3.3: box-box intersections with every periodic
//                                image, computed once per BoxArray (their cost grows with the
//                                number of boxes, Sec. 3.3), via a uniform bin hash
//   MFIter / tilebox()           Sec. 3.2: tiles of a given size from each box's lower corner,
//                                the last tile along a direction smaller; flattened into one
//                                device work list for all boxes
//   thread-private arenas        Sec. 3.3: nothing allocates while advancing; every list and
//                                scratch buffer is sized at attach
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mf.h"
#include "mf_internal.h"

using namespace mfk;

// ------------------------------------------------------------------ errors

static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int mfk::set_error(int code, const char *msg) {
    g_err = msg;
    return code;
}

#define CU(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return fail(MF_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

// ------------------------------------------------------------------ boxes

struct Box {
    int lo[3], hi[3];
    bool empty() const { return lo[0] > hi[0] || lo[1] > hi[1] || lo[2] > hi[2]; }
    long long cells() const {
        return empty() ? 0 : (long long)(hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
    }
    int len(int d) const { return hi[d] - lo[d] + 1; }
    bool contains(int i, int j, int k) const {
        return i >= lo[0] && i <= hi[0] && j >= lo[1] && j <= hi[1] && k >= lo[2] && k <= hi[2];
    }
};

static Box intersect(const Box &a, const Box &b) {
    Box r;
    for (int d = 0; d < 3; ++d) {
        r.lo[d] = std::max(a.lo[d], b.lo[d]);
        r.hi[d] = std::min(a.hi[d], b.hi[d]);
    }
    return r;
}
static Box grow(const Box &a, int g) {
    Box r = a;
    for (int d = 0; d < 3; ++d) { r.lo[d] -= g; r.hi[d] += g; }
    return r;
}
static Box shift(const Box &a, const int s[3]) {
    Box r = a;
    for (int d = 0; d < 3; ++d) { r.lo[d] += s[d]; r.hi[d] += s[d]; }
    return r;
}
static int floor_div(int a, int b) {
    int q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}
static Box coarsen(const Box &a, int r) {
    Box c;
    for (int d = 0; d < 3; ++d) { c.lo[d] = floor_div(a.lo[d], r); c.hi[d] = floor_div(a.hi[d], r); }
    return c;
}

// Uniform bin hash over the domain: each box is registered in every bin it touches.
struct BinHash {
    Box dom;
    int bs = 1, nb[3] = {1, 1, 1};
    std::vector<std::vector<int>> bins;
    void build(const Box &domain, const std::vector<Box> &boxes) {
        dom = domain;
        int maxlen = 1;
        for (auto &b : boxes) for (int d = 0; d < 3; ++d) maxlen = std::max(maxlen, b.len(d));
        bs = std::max(8, maxlen);
        for (int d = 0; d < 3; ++d) nb[d] = (dom.len(d) + bs - 1) / bs;
        bins.assign((size_t)nb[0] * nb[1] * nb[2], {});
        for (int i = 0; i < (int)boxes.size(); ++i) {
            Box c = intersect(boxes[i], dom);
            if (c.empty()) continue;
            int l[3], h[3];
            for (int d = 0; d < 3; ++d) {
                l[d] = (c.lo[d] - dom.lo[d]) / bs;
                h[d] = (c.hi[d] - dom.lo[d]) / bs;
            }
            for (int z = l[2]; z <= h[2]; ++z)
                for (int y = l[1]; y <= h[1]; ++y)
                    for (int x = l[0]; x <= h[0]; ++x) bins[((size_t)z * nb[1] + y) * nb[0] + x].push_back(i);
        }
    }
    // Boxes that may intersect q (q clipped to the domain), each once.
    void query(const Box &q, std::vector<int> &out, std::vector<int> &stamp, int tag) const {
        out.clear();
        Box c = intersect(q, dom);
        if (c.empty()) return;
        int l[3], h[3];
        for (int d = 0; d < 3; ++d) {
            l[d] = (c.lo[d] - dom.lo[d]) / bs;
            h[d] = (c.hi[d] - dom.lo[d]) / bs;
        }
        for (int z = l[2]; z <= h[2]; ++z)
            for (int y = l[1]; y <= h[1]; ++y)
                for (int x = l[0]; x <= h[0]; ++x)
                    for (int i : bins[((size_t)z * nb[1] + y) * nb[0] + x])
                        if (stamp[i] != tag) { stamp[i] = tag; out.push_back(i); }
    }
};

// ------------------------------------------------------------------ device buffers

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    ~DevBuf() { if (p) cudaFree(p); }
    int ensure(size_t n) {
        if (n <= bytes && p) return 0;
        if (p) { cudaFree(p); p = nullptr; bytes = 0; }
        if (n == 0) n = 16;
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) { p = nullptr; return fail(MF_ENOMEM, "cudaMalloc(%zu): %s", n, cudaGetErrorString(e)); }
        bytes = n;
        return 0;
    }
    template <typename T> int upload(const std::vector<T> &v, cudaStream_t s) {
        int rc = ensure(std::max<size_t>(16, v.size() * sizeof(T)));
        if (rc) return rc;
        if (!v.empty()) CU(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
        return 0;
    }
};

struct GraphExec {
    cudaGraphExec_t exec = nullptr;
    int launches[4] = {0, 0, 0, 0};  // ghost fill, stencil, coarse-fine interp, average-down kernels
    int nev = 0;                     // timing events recorded by the graph (0: untimed)
    std::vector<char> kinds;         // kinds[i]: phase between events i-1 and i (0 fill, 1 stencil, 2 other)
    ~GraphExec() { if (exec) cudaGraphExecDestroy(exec); }
};

// ------------------------------------------------------------------ the handle

// A work list numbered cell by cell: segment q (a run or a region) holds cells
// [start[q], start[q+1]); wfirst[w] is the segment holding cell 32 w.
struct CellList {
    std::vector<int> start, wfirst;
    int ncells = 0;
    DevBuf d_start, d_wfirst;
    void finish() {
        ncells = start.back();
        wfirst.assign((size_t)((ncells + 31) / 32), 0);
        size_t q = 0;
        for (size_t w = 0; w < wfirst.size(); ++w) {
            const int c = (int)(w * 32);
            while (start[q + 1] <= c) ++q;
            wfirst[w] = (int)q;
        }
    }
    int upload(cudaStream_t s) {
        int rc = d_start.upload(start, s);
        return rc ? rc : d_wfirst.upload(wfirst, s);
    }
};

// Coarse-fine interpolation plan of a fine level against one coarse layout: the runs of fine
// ghost cells no fine box covers, numbered cell by cell.
struct InterpPlan {
    const mf_t *crse = nullptr;
    int ratio = 0;
    std::vector<InterpRun> runs;
    CellList cells;
    DevBuf d_runs;
};

// Refluxing plan of a (fine, coarse) level pair: the coarse faces of the coarse-fine interface,
// their fine faces, the coarse cells to correct, and the FP64 flux registers.
struct RefluxPlan {
    const mf_t *crse = nullptr;
    int ratio = 0;
    std::vector<CFace> faces;
    std::vector<FFace> ff;
    std::vector<CCell> cells;
    DevBuf d_faces, d_ff, d_cells, d_regc, d_regf;
};

// The coarse level's ghost exchange inside the two-level advance, limited to the ghost cells
// that are read.  Per FillBoundary region of the coarse level: the bounding box of its cells that
// the interpolation reads (ip), that the interpolation or the coarse flux registers read (cf),
// and, for face regions, of the cells whose source lies within one cell of the fine-covered
// region (stale: the average-down and the flux correction rewrite those sources after the
// stencil's ghost push delivered them).  Boxes as {lo[3], n[3]} within the region, n[0] = 0
// for none.
struct AmrFill {
    const mf_t *fine = nullptr;
    int ratio = 0, R = 0;
    bool reflux = false;
    std::vector<std::array<int, 6>> ip, cf, stale;
    unsigned long long gen = ~0ull;  // the coarse build generation the task lists belong to
    std::vector<FbTask> t_first, t_next, t_post;
    DevBuf d_first, d_next, d_post;
};

// Average-down plan of a coarse level from one fine level: the coarse regions under the fine
// boxes, numbered cell by cell.
struct AvgPlan {
    const mf_t *fine = nullptr;
    int ratio = 0;
    bool vec = true;  // every fine offset and pitch a multiple of ratio: vector loads of children
    std::vector<AvgRegion> regs;
    CellList cells;
    DevBuf d_regs;
};

struct mf {
    Box domain;
    std::vector<Box> boxes;  // the FArrayBoxes: the boxes, or the regions of a regional level
    // Regional storage (Sec. 2, Fig. 2): the level's data live in regions, each a rectangle that
    // a group of its boxes covers exactly, and the boxes are logical tiles of the regions: they
    // keep defining the level's cells but no longer their own allocations or ghost cells.
    bool regional = false;
    std::vector<Box> lboxes;      // the boxes of a regional level, in the order given
    std::vector<int> lbox_region;  // the region holding each of them
    int ncomp = 1, ngrow = 0, dtype = F64, esize = 8;
    // layout
    std::vector<FabInfo> fabs;     // level slot 0
    std::vector<long long> fab_start;  // element offset of each FArrayBox's allocation
    size_t level_elems = 0;        // elements per time level (multiple of 256 bytes)
    // FillBoundary
    std::vector<FbEntry> fb;
    std::vector<FbTask> fbtasks;
    long long ghost_cells = 0;     // per component
    std::vector<int> fb_group;     // first entry of each destination box (size nbox+1)
    std::vector<int> fb_cbeg;      // cells before entry within its destination-box group
    std::vector<std::array<int, 6>> fb_corner;  // global lower corners: dst (may lie outside
                                                // the domain), then src
    std::vector<int> fb_kind;      // 2*d + (side > 0) for a face region along d, 6 for edges/corners
    std::vector<FbTask> fbtasks_adv;  // the fill inside mf_advance when the stencil pulls x halos
    // tiles
    int tile[3] = {0, 0, 0};
    bool tile_auto = true;
    // tile shapes per box-size class (tile_class): the y and z tile extents of the boxes of a
    // class, -1 for the level's (tile[1], tile[2]); a z override applies only where the level's
    // tile has a z extent (with a whole-box z extent the balanced schedule splits every box)
    int cty[kTileClasses] = {-1, -1, -1, -1, -1}, ctz[kTileClasses] = {-1, -1, -1, -1, -1};
    std::vector<Tile> tiles;
    int block[2] = {32, 8};
    // attach
    char *base = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;    // private stream for graph capture
    // a second capture stream and two events: a branch of the two-level advance's graph that runs
    // beside the coarse stencil (the first fine substep)
    cudaStream_t cap2 = nullptr;
    cudaEvent_t fork_ev[2] = {nullptr, nullptr};
    int cur = 0;
    bool attached = false;
    DevBuf d_fabs, d_fb, d_fbtasks, d_tiles, d_cbeg, d_partials, d_sumout;
    DevBuf d_rowpre;  // first valid row (y, z) of every FArrayBox in the reductions' row list
    // TMA-staged stencil: tensor maps of every FArrayBox over each time level, plane geometry
    DevBuf d_maps, d_tfab, d_err, d_smaps, d_strips, d_fbtasks_adv, d_push, d_fbtasks_res;
    // fixed-point steps (MF_FIXED_DIFF): three FixSet grid states that rotate over the steps
    DevBuf d_fix;
    std::vector<FbTask> fbtasks_res;  // the fill left once the stencil pushes face ghosts
    bool tma_push = false;
    bool push_pref = true;         // the autotuner's choice between the ghost push and the face fill
    bool tma_strips = false;  // x halos pulled from neighbour boxes (fill skips x faces)
    int tma_R = 0;            // tma_key of the radius and arithmetic the maps were built for (0 = none)
    bool tma_ok = false;      // current tile shape fits the TMA kernel
    int tma_cpt = 32, tma_slot = 0, tma_ns = 0;  // tma_cpt: CTA threads of the TMA stencil
    int tma_rows = 2;     // rows per consumer thread (autotuned; clipped to what the radius allows)
    int tma_gb = 16;      // bytes per row group of a consumer thread, 16 or 32 (autotuned)
    int tma_ns_pref = 0;  // ring slots (0: by radius; autotuned)
    int tma_main_slot = 0, tma_strip_rows = 0, tma_strip_bytes = 0, tma_strip_pitch = 0, tma_strip_w = 0;
    bool use_tma = true;
    // balanced schedule (tile z extent 0): CTA b of exactly tma_grid CTAs takes tiles
    // [cta_tiles[b], cta_tiles[b + 1])
    std::vector<int> cta_tiles;
    DevBuf d_cta;
    int tma_grid = 0;
    unsigned long long gen = 0;    // changes whenever state baked into a captured graph changes
    double *h_sum = nullptr;       // pinned
    size_t tile_capacity = 0;
    std::map<std::string, std::unique_ptr<GraphExec>> graphs;
    // phase timing: events recorded inside the captured graph around every launch
    bool timing = false;
    std::vector<cudaEvent_t> ev;   // 2*nsteps+1 of the last timed advance
    int ev_used = 0;
    std::vector<char> ev_kinds;    // phase of each interval of the last timed advance
    int launches[4] = {0, 0, 0, 0};  // kernel launches of the last advance (see GraphExec)
    std::vector<std::unique_ptr<InterpPlan>> interp;
    std::vector<std::unique_ptr<RefluxPlan>> reflux;
    std::vector<std::unique_ptr<AvgPlan>> avg;
    std::vector<std::unique_ptr<AmrFill>> amrfill;
    ~mf() {
        // work this handle queued may still run: let it finish before its graphs and device
        // lists go (an error here, e.g. after the context is gone, leaves nothing to wait for)
        if (attached) cudaStreamSynchronize(stream);
        graphs.clear();
        for (auto e : ev) cudaEventDestroy(e);
        if (cap) cudaStreamDestroy(cap);
        if (cap2) cudaStreamDestroy(cap2);
        for (auto e : fork_ev)
            if (e) cudaEventDestroy(e);
        if (h_sum) cudaFreeHost(h_sum);
    }
    // Runge-Kutta stage level (slot 2), caller-owned like the two time levels
    char *stage = nullptr;
    void *level_ptr(int which) const {
        return which == 2 ? (void *)stage : (void *)(base + (size_t)which * level_elems * esize);
    }
};

// ------------------------------------------------------------------ layout

static void build_layout(mf_t *m) {
    const int g = m->ngrow, S = m->esize;
    const long long align = 256 / S;       // FArrayBox start alignment in elements
    long long off = 0;
    m->fabs.clear();
    m->fab_start.clear();
    for (auto &b : m->boxes) {
        FabInfo f{};
        for (int d = 0; d < 3; ++d) { f.n[d] = b.len(d); f.lo[d] = b.lo[d]; }
        // rows lie back to back at a pitch of whole 32-byte sectors (dense DRAM pages, aligned
        // whole-row TMA loads); the left ghost cells are padded so that valid x = 0 starts a
        // 32-byte sector: a row of valid cells is whole sectors, read and written without
        // partial sectors
        const int AS = 32 / S;
        const int fpad = (AS - g % AS) % AS;
        f.px = (int)(((long long)fpad + f.n[0] + 2 * g + AS - 1) / AS * AS);
        const long long py = f.n[1] + 2 * g, nzg = f.n[2] + 2 * g;
        f.plane = (long long)f.px * py;
        f.cstride = f.plane * nzg;
        off = (off + align - 1) / align * align;
        m->fab_start.push_back(off);
        f.org = off + g * f.plane + (long long)g * f.px + fpad + g;
        f.level = 0;
        m->fabs.push_back(f);
        off += f.cstride * m->ncomp;
    }
    off = (off + align - 1) / align * align;
    m->level_elems = (size_t)off;
}

// Row element of valid x = 0 in every FArrayBox (the layout's left padding plus the ghosts).
static int valid_x_elem(const mf_t *m) {
    const int AS = 32 / m->esize, g = m->ngrow;
    return (g + AS - 1) / AS * AS;
}

static long long elem_at(const FabInfo &f, int i, int j, int k) {  // global (i,j,k), comp 0
    return f.org + (long long)(k - f.lo[2]) * f.plane + (long long)(j - f.lo[1]) * f.px + (i - f.lo[0]);
}

// ------------------------------------------------------------------ FillBoundary list

// FillBoundary tasks for the entries selected by `use`: CTA-sized pieces (256 threads x 4 cells).
// Appends the fill tasks of one FillBoundary region (or a clipped part of one).
static void append_fill_tasks(const mf_t *m, const FbEntry &en, std::vector<FbTask> &out) {
    const int kTask = 256;  // one warp of the fill kernel: 32 lanes x 8 cells (or vectors)
    const long long V = 16 / m->esize;  // elements per 16-byte vector
    const FabInfo &sf = m->fabs[en.sfab], &df = m->fabs[en.dfab];
    // rows that start and end on 16-byte boundaries on both sides copy as 16-byte vectors
    // (pitches, planes and component strides are whole 32-byte sectors by construction)
    const bool vec = en.n[0] % V == 0 && en.src % V == 0 && en.dst % V == 0;
    const long long u = vec ? V : 1;
    const int n0 = (int)(en.n[0] / u);
    const long long cells = (long long)n0 * en.n[1] * en.n[2] * m->ncomp;
    for (long long f = 0; f < cells; f += kTask) {
        FbTask t{};
        t.src = en.src / u;
        t.dst = en.dst / u;
        t.s_pl = (int)(sf.plane / u);
        t.d_pl = (int)(df.plane / u);
        t.s_cs = (int)(sf.cstride / u);
        t.d_cs = (int)(df.cstride / u);
        t.s_px = (int)(sf.px / u);
        t.d_px = (int)(df.px / u);
        t.n0 = n0;
        t.n1 = en.n[1];
        t.n2 = en.n[2];
        t.first = (int)f;
        t.count = (int)std::min<long long>(kTask, cells - f);
        t.level = en.level;
        t.f0 = make_fastdiv((uint32_t)n0);
        t.f1 = make_fastdiv((uint32_t)en.n[1]);
        t.f2 = make_fastdiv((uint32_t)en.n[2]);
        t.vec = vec ? 1 : 0;
        out.push_back(t);
    }
}

static void make_fill_tasks(const mf_t *m, const std::vector<char> &use, std::vector<FbTask> &out) {
    out.clear();
    for (int e = 0; e < (int)m->fb.size(); ++e)
        if (use[e]) append_fill_tasks(m, m->fb[e], out);
}

// The part [lo, lo + n) (offsets within the region) of FillBoundary region e.
static FbEntry clip_entry(const mf_t *m, int e, const int lo[3], const int n[3]) {
    FbEntry c = m->fb[e];
    const FabInfo &sf = m->fabs[c.sfab], &df = m->fabs[c.dfab];
    c.src += lo[2] * sf.plane + (long long)lo[1] * sf.px + lo[0];
    c.dst += lo[2] * df.plane + (long long)lo[1] * df.px + lo[0];
    for (int d = 0; d < 3; ++d) c.n[d] = n[d];
    return c;
}

static int build_fb(mf_t *m) {
    const int nb = (int)m->boxes.size(), g = m->ngrow;
    m->fb.clear();
    m->fbtasks.clear();
    m->fb_group.assign(nb + 1, 0);
    m->fb_cbeg.clear();
    m->fb_corner.clear();
    m->fb_kind.clear();
    m->ghost_cells = 0;
    if (g == 0) return 0;
    BinHash hash;
    hash.build(m->domain, m->boxes);
    std::vector<int> cand, stamp(nb, -1);
    int tag = 0;
    const int L[3] = {m->domain.len(0), m->domain.len(1), m->domain.len(2)};
    for (int b = 0; b < nb; ++b) {
        m->fb_group[b] = (int)m->fb.size();
        const Box gb = grow(m->boxes[b], g);
        int cells_in_group = 0;
        for (int sz = -1; sz <= 1; ++sz)
            for (int sy = -1; sy <= 1; ++sy)
                for (int sx = -1; sx <= 1; ++sx) {
                    const int s[3] = {sx * L[0], sy * L[1], sz * L[2]};
                    const int ms[3] = {-s[0], -s[1], -s[2]};
                    const Box q = shift(gb, ms);  // the grown box seen from the periodic image
                    hash.query(q, cand, stamp, ++tag);
                    std::sort(cand.begin(), cand.end());
                    for (int a : cand) {
                        if (a == b && sx == 0 && sy == 0 && sz == 0) continue;
                        const Box src0 = intersect(m->boxes[a], q);
                        if (src0.empty()) continue;
                        const Box dst0 = shift(src0, s);
                        // split by the 27 parts of the grown box: faces, edges, corners
                        const Box &B = m->boxes[b];
                        for (int pz = 0; pz < 3; ++pz)
                            for (int py = 0; py < 3; ++py)
                                for (int px = 0; px < 3; ++px) {
                                    const int part[3] = {px, py, pz};
                                    Box cut;
                                    int outside = 0, fdim = -1, fside = 0;
                                    for (int d = 0; d < 3; ++d) {
                                        const int lo = part[d] == 0 ? B.lo[d] - g : part[d] == 1 ? B.lo[d] : B.hi[d] + 1;
                                        const int hi = part[d] == 0 ? B.lo[d] - 1 : part[d] == 1 ? B.hi[d] : B.hi[d] + g;
                                        cut.lo[d] = lo;
                                        cut.hi[d] = hi;
                                        if (part[d] != 1) { ++outside; fdim = d; fside = part[d] == 2 ? 1 : 0; }
                                    }
                                    const Box dst = intersect(dst0, cut);
                                    if (dst.empty()) continue;
                                    const Box src = shift(dst, ms);
                                    FbEntry e{};
                                    for (int d = 0; d < 3; ++d) e.n[d] = src.len(d);
                                    e.sfab = a;
                                    e.dfab = b;
                                    e.level = 0;
                                    e.src = elem_at(m->fabs[a], src.lo[0], src.lo[1], src.lo[2]);
                                    e.dst = elem_at(m->fabs[b], dst.lo[0], dst.lo[1], dst.lo[2]);
                                    const long long cells = src.cells() * m->ncomp;
                                    if (cells > 0x7fffffffLL) return fail(MF_EINVAL, "ghost region too large");
                                    m->fb_cbeg.push_back(cells_in_group);
                                    m->fb_corner.push_back(
                                        {dst.lo[0], dst.lo[1], dst.lo[2], src.lo[0], src.lo[1], src.lo[2]});
                                    m->fb_kind.push_back(outside == 1 ? 2 * fdim + fside : 6);
                                    cells_in_group += (int)cells;
                                    m->ghost_cells += src.cells();
                                    m->fb.push_back(e);
                                }
                    }
                }
    }
    m->fb_group[nb] = (int)m->fb.size();
    std::vector<char> all(m->fb.size(), 1);
    make_fill_tasks(m, all, m->fbtasks);
    return 0;
}

// ------------------------------------------------------------------ tiles

// The box-size class of an FArrayBox for its tile shape: its y extent up to 8, 16, 32, 64 cells,
// or above.
static int tile_class(const FabInfo &f) {
    const int ny = f.n[1];
    return ny <= 8 ? 0 : ny <= 16 ? 1 : ny <= 32 ? 2 : ny <= 64 ? 3 : 4;
}

static void make_tiles(const mf_t *m, const int tile[3], std::vector<Tile> &out) {
    out.clear();
    for (int b = 0; b < (int)m->boxes.size(); ++b) {
        const FabInfo &f = m->fabs[b];
        const int k = tile_class(f);
        int sh[3] = {tile[0], m->cty[k] >= 0 ? m->cty[k] : tile[1], tile[2]};
        if (tile[2] > 0 && m->ctz[k] >= 0) sh[2] = m->ctz[k];
        int t[3];
        for (int d = 0; d < 3; ++d) t[d] = (sh[d] <= 0 || sh[d] > f.n[d]) ? f.n[d] : sh[d];
        for (int c = 0; c < m->ncomp; ++c)
            for (int z = 0; z < f.n[2]; z += t[2])
                for (int y = 0; y < f.n[1]; y += t[1])
                    for (int x = 0; x < f.n[0]; x += t[0]) {
                        Tile w;
                        w.fab = b;
                        w.comp = c;
                        w.x0 = (short)x; w.y0 = (short)y; w.z0 = (short)z;
                        w.tx = (short)std::min(t[0], f.n[0] - x);
                        w.ty = (short)std::min(t[1], f.n[1] - y);
                        w.tz = (short)std::min(t[2], f.n[2] - z);
                        out.push_back(w);
                    }
    }
}

// Candidate tile shapes for the autotuner (Sec. 3.2: the tile size can differ per loop).
static std::vector<std::array<int, 3>> tile_candidates(const mf_t *m) {
    int mx[3] = {1, 1, 1};
    for (auto &b : m->boxes) for (int d = 0; d < 3; ++d) mx[d] = std::max(mx[d], b.len(d));
    std::vector<std::array<int, 3>> c;
    const int xs[] = {0, 64, 32};
    const int ys[] = {4, 8, 16, 32, 0};
    const int zs[] = {8, 16, 32, 0};
    for (int x : xs) for (int y : ys) for (int z : zs) {
        std::array<int, 3> t = {x, y, z};
        // normalise: a size >= the largest box extent means "whole box"
        for (int d = 0; d < 3; ++d) if (t[d] >= mx[d]) t[d] = 0;
        if (std::find(c.begin(), c.end(), t) == c.end()) c.push_back(t);
    }
    return c;
}

// ------------------------------------------------------------------ creation

static int check_create(const int dlo[3], const int dhi[3], int ncomp, int ngrow, int dtype) {
    if (!dlo || !dhi) return fail(MF_EINVAL, "null domain");
    for (int d = 0; d < 3; ++d)
        if (dhi[d] < dlo[d]) return fail(MF_EINVAL, "empty domain along %d", d);
    if (ncomp < 1 || ncomp > kMaxComp) return fail(MF_EINVAL, "ncomp must be in [1, %d]", kMaxComp);
    if (ngrow < 0) return fail(MF_EINVAL, "ngrow must be >= 0");
    for (int d = 0; d < 3; ++d)
        if (ngrow >= dhi[d] - dlo[d] + 1) return fail(MF_EINVAL, "ngrow must be smaller than the domain");
    if (dtype != F64 && dtype != F32 && dtype != BF16) return fail(MF_EINVAL, "unknown dtype %d", dtype);
    return 0;
}

static int finish_create(mf_t *m) {
    build_layout(m);
    for (auto &f : m->fabs)  // offsets within one FArrayBox are 32-bit in the kernels
        if (f.cstride * m->ncomp >= (1LL << 31)) return fail(MF_EINVAL, "an FArrayBox of 2^31 or more elements");
    int rc = build_fb(m);
    if (rc) return rc;
    make_tiles(m, m->tile, m->tiles);
    return 0;
}

extern "C" int mf_create(mf_t **out, const int domain_lo[3], const int domain_hi[3], int max_grid_size, int ncomp,
                         int ngrow, int dtype) {
    if (!out) return fail(MF_EINVAL, "null out");
    *out = nullptr;
    int rc = check_create(domain_lo, domain_hi, ncomp, ngrow, dtype);
    if (rc) return rc;
    if (max_grid_size < 1) return fail(MF_EINVAL, "max_grid_size must be >= 1");
    std::unique_ptr<mf_t> m(new (std::nothrow) mf_t());
    if (!m) return fail(MF_ENOMEM, "host allocation");
    for (int d = 0; d < 3; ++d) { m->domain.lo[d] = domain_lo[d]; m->domain.hi[d] = domain_hi[d]; }
    int n[3];
    for (int d = 0; d < 3; ++d) n[d] = (m->domain.len(d) + max_grid_size - 1) / max_grid_size;
    if ((long long)n[0] * n[1] * n[2] > (1 << 24)) return fail(MF_EINVAL, "too many boxes");
    for (int bz = 0; bz < n[2]; ++bz)
        for (int by = 0; by < n[1]; ++by)
            for (int bx = 0; bx < n[0]; ++bx) {
                Box b;
                const int idx[3] = {bx, by, bz};
                for (int d = 0; d < 3; ++d) {
                    b.lo[d] = domain_lo[d] + idx[d] * max_grid_size;
                    b.hi[d] = std::min(b.lo[d] + max_grid_size - 1, domain_hi[d]);
                }
                m->boxes.push_back(b);
            }
    m->ncomp = ncomp;
    m->ngrow = ngrow;
    m->dtype = dtype;
    m->esize = dtype_size(dtype);
    for (auto &b : m->boxes)
        for (int d = 0; d < 3; ++d)
            if (b.len(d) > 32767) return fail(MF_EINVAL, "box side above 32767");
    rc = finish_create(m.get());
    if (rc) return rc;
    *out = m.release();
    return 0;
}

// Regions of a list of disjoint boxes (regional storage): rectangles, each covered exactly by
// the boxes it holds, with every side at most max_ext cells.  Guillotine recursion over the
// boxes' bounding box: a rectangle that its boxes cover and that fits becomes a region;
// otherwise (too large, or with holes) it is cut by the plane that crosses no box and lies
// closest to the middle of the longest side that has one, and each part (shrunk to its boxes'
// bounding box) is treated the same way.  Boxes that no such plane separates each become a
// region of their own.
// region_of[i]: the region of box i.
static void build_regions(const std::vector<Box> &bx, int max_ext, std::vector<Box> &regions,
                          std::vector<int> &region_of) {
    regions.clear();
    region_of.assign(bx.size(), -1);
    std::vector<int> all(bx.size());
    for (size_t i = 0; i < bx.size(); ++i) all[i] = (int)i;
    auto bbox = [&](const std::vector<int> &ids) {
        Box r = bx[ids[0]];
        for (int i : ids)
            for (int d = 0; d < 3; ++d) { r.lo[d] = std::min(r.lo[d], bx[i].lo[d]); r.hi[d] = std::max(r.hi[d], bx[i].hi[d]); }
        return r;
    };
    auto emit = [&](const Box &r, const std::vector<int> &ids) {
        for (int i : ids) region_of[i] = (int)regions.size();
        regions.push_back(r);
    };
    // explicit stack: (ids) per pending rectangle
    std::vector<std::vector<int>> stack;
    stack.push_back(std::move(all));
    while (!stack.empty()) {
        std::vector<int> ids = std::move(stack.back());
        stack.pop_back();
        const Box r = bbox(ids);
        long long vol = 0;
        for (int i : ids) vol += bx[i].cells();
        const bool covered = vol == r.cells();
        const bool fits = r.len(0) <= max_ext && r.len(1) <= max_ext && r.len(2) <= max_ext;
        if (covered && fits) {  // (a single box is covered by itself)
            emit(r, ids);
            continue;
        }
        // the cut: a plane x_d = p (between cells p - 1 and p) that no box crosses
        int best_d = -1, best_p = 0;
        int dims[3] = {0, 1, 2};
        std::sort(dims, dims + 3, [&](int a, int b) { return r.len(a) > r.len(b) || (r.len(a) == r.len(b) && a < b); });
        for (int d : dims) {
            std::vector<std::pair<int, int>> iv;  // crossed cut positions (lo, hi]
            iv.reserve(ids.size());
            for (int i : ids) iv.push_back({bx[i].lo[d], bx[i].hi[d]});
            std::sort(iv.begin(), iv.end());
            const double mid = r.lo[d] + r.len(d) * 0.5;
            int reach = iv[0].second;  // positions <= reach are crossed by a box seen so far
            double bestdist = 1e30;
            for (size_t k = 1; k < iv.size(); ++k) {
                const int p = iv[k].first;  // a box starts here: a cut if no earlier box crosses p
                if (p > reach && std::fabs(p - mid) < bestdist) {
                    bestdist = std::fabs(p - mid);
                    best_p = p;
                    best_d = d;
                }
                reach = std::max(reach, iv[k].second);
            }
            if (best_d >= 0) break;
        }
        if (best_d < 0) {
            for (int i : ids) emit(bx[i], {i});
            continue;
        }
        std::vector<int> a, b;
        for (int i : ids) (bx[i].hi[best_d] < best_p ? a : b).push_back(i);
        stack.push_back(std::move(b));
        stack.push_back(std::move(a));
    }
}

static int read_boxes(const int *boxes, int nboxes, const int domain_lo[3], const int domain_hi[3],
                      std::vector<Box> &out) {
    if (nboxes < 1 || !boxes) return fail(MF_EINVAL, "need at least one box");
    out.clear();
    for (int i = 0; i < nboxes; ++i) {
        Box b;
        for (int d = 0; d < 3; ++d) { b.lo[d] = boxes[6 * i + d]; b.hi[d] = boxes[6 * i + 3 + d]; }
        if (b.empty()) return fail(MF_EINVAL, "box %d is empty", i);
        for (int d = 0; d < 3; ++d) {
            if (b.lo[d] < domain_lo[d] || b.hi[d] > domain_hi[d]) return fail(MF_EINVAL, "box %d outside the domain", i);
            if (b.len(d) > 32767) return fail(MF_EINVAL, "box side above 32767");
        }
        out.push_back(b);
    }
    // overlap check through the bin hash
    Box dom;
    for (int d = 0; d < 3; ++d) { dom.lo[d] = domain_lo[d]; dom.hi[d] = domain_hi[d]; }
    BinHash hash;
    hash.build(dom, out);
    std::vector<int> cand, stamp(nboxes, -1);
    for (int i = 0; i < nboxes; ++i) {
        hash.query(out[i], cand, stamp, i);
        for (int a : cand)
            if (a != i && !intersect(out[a], out[i]).empty())
                return fail(MF_EINVAL, "boxes %d and %d overlap", std::min(a, i), std::max(a, i));
    }
    return 0;
}

static int create_from_boxes(mf_t **out, const int domain_lo[3], const int domain_hi[3], const int *boxes,
                             int nboxes, int ncomp, int ngrow, int dtype, int max_region) {
    if (!out) return fail(MF_EINVAL, "null out");
    *out = nullptr;
    int rc = check_create(domain_lo, domain_hi, ncomp, ngrow, dtype);
    if (rc) return rc;
    std::unique_ptr<mf_t> m(new (std::nothrow) mf_t());
    if (!m) return fail(MF_ENOMEM, "host allocation");
    for (int d = 0; d < 3; ++d) { m->domain.lo[d] = domain_lo[d]; m->domain.hi[d] = domain_hi[d]; }
    if ((rc = read_boxes(boxes, nboxes, domain_lo, domain_hi, m->boxes))) return rc;
    if (max_region > 0) {
        m->regional = true;
        m->lboxes = m->boxes;
        build_regions(m->lboxes, max_region, m->boxes, m->lbox_region);
    }
    m->ncomp = ncomp;
    m->ngrow = ngrow;
    m->dtype = dtype;
    m->esize = dtype_size(dtype);
    rc = finish_create(m.get());
    if (rc) return rc;
    *out = m.release();
    return 0;
}

extern "C" int mf_create_boxes(mf_t **out, const int domain_lo[3], const int domain_hi[3], const int *boxes,
                               int nboxes, int ncomp, int ngrow, int dtype) {
    return create_from_boxes(out, domain_lo, domain_hi, boxes, nboxes, ncomp, ngrow, dtype, 0);
}

extern "C" int mf_create_regional(mf_t **out, const int domain_lo[3], const int domain_hi[3], const int *boxes,
                                  int nboxes, int ncomp, int ngrow, int dtype, int max_region) {
    if (max_region < 1 || max_region > 240)
        return fail(MF_EINVAL, "max_region must be in [1, 240] (a region row, ghosts included, fits one TMA box)");
    return create_from_boxes(out, domain_lo, domain_hi, boxes, nboxes, ncomp, ngrow, dtype, max_region);
}

extern "C" int mf_box_regions(const int *boxes, int nboxes, int max_region, int *regions_out, int *region_of_out) {
    if (!boxes || nboxes < 1 || max_region < 1 || !region_of_out) return fail(MF_EINVAL, "bad argument");
    std::vector<Box> bx(nboxes), rg;
    std::vector<int> of;
    for (int i = 0; i < nboxes; ++i)
        for (int d = 0; d < 3; ++d) { bx[i].lo[d] = boxes[6 * i + d]; bx[i].hi[d] = boxes[6 * i + 3 + d]; }
    build_regions(bx, max_region, rg, of);
    for (int i = 0; i < nboxes; ++i) region_of_out[i] = of[i];
    if (regions_out)
        for (size_t r = 0; r < rg.size(); ++r)
            for (int d = 0; d < 3; ++d) { regions_out[6 * r + d] = rg[r].lo[d]; regions_out[6 * r + 3 + d] = rg[r].hi[d]; }
    return (int)rg.size();
}

extern "C" void mf_destroy(mf_t *m) { delete m; }

static const std::vector<Box> &user_boxes(const mf_t *m) { return m->regional ? m->lboxes : m->boxes; }

extern "C" int mf_nboxes(const mf_t *m) { return m ? (int)user_boxes(m).size() : fail(MF_EINVAL, "null handle"); }

extern "C" int mf_get_boxes(const mf_t *m, int *out) {
    if (!m || !out) return fail(MF_EINVAL, "null argument");
    const auto &bx = user_boxes(m);
    for (size_t i = 0; i < bx.size(); ++i)
        for (int d = 0; d < 3; ++d) { out[6 * i + d] = bx[i].lo[d]; out[6 * i + 3 + d] = bx[i].hi[d]; }
    return 0;
}

extern "C" int mf_nregions(const mf_t *m) { return m ? (int)m->boxes.size() : fail(MF_EINVAL, "null handle"); }

extern "C" int mf_get_regions(const mf_t *m, int *regions_out, int *region_of_out) {
    if (!m) return fail(MF_EINVAL, "null handle");
    if (regions_out)
        for (size_t i = 0; i < m->boxes.size(); ++i)
            for (int d = 0; d < 3; ++d) {
                regions_out[6 * i + d] = m->boxes[i].lo[d];
                regions_out[6 * i + 3 + d] = m->boxes[i].hi[d];
            }
    if (region_of_out)
        for (size_t i = 0; i < user_boxes(m).size(); ++i) region_of_out[i] = m->regional ? m->lbox_region[i] : (int)i;
    return 0;
}

extern "C" size_t mf_bytes(const mf_t *m) { return m ? 2 * m->level_elems * m->esize : 0; }

extern "C" long long mf_fb_regions(const mf_t *m, long long *ghost_cells_out) {
    if (!m) return fail(MF_EINVAL, "null handle");
    if (ghost_cells_out) *ghost_cells_out = m->ghost_cells;
    return (long long)m->fb.size();
}

extern "C" long long mf_get_fb_regions(const mf_t *m, int *out, long long max) {
    if (!m || !out) return fail(MF_EINVAL, "null argument");
    long long n = std::min<long long>(max, (long long)m->fb.size());
    for (long long i = 0; i < n; ++i) {
        const FbEntry &e = m->fb[i];
        int *o = out + 11 * i;
        o[0] = e.dfab;
        o[1] = e.sfab;
        for (int d = 0; d < 3; ++d) {
            o[2 + d] = m->fb_corner[i][d];
            o[5 + d] = m->fb_corner[i][3 + d];
            o[8 + d] = e.n[d];
        }
    }
    return n;
}

extern "C" const char *mf_last_error(void) { return g_err.c_str(); }

extern "C" int mf_current(const mf_t *m) { return m ? m->cur : fail(MF_EINVAL, "null handle"); }

extern "C" double mf_step_bytes(const mf_t *m, int R) {
    if (!m) return 0.0;
    double V = 0, Gf = 0;
    for (auto &b : m->boxes) {
        const double n0 = b.len(0), n1 = b.len(1), n2 = b.len(2);
        V += n0 * n1 * n2;
        Gf += 2.0 * R * (n0 * n1 + n1 * n2 + n0 * n2);
    }
    return (double)m->esize * m->ncomp * (2.0 * V + 2.0 * (double)m->ghost_cells + Gf);
}

// ------------------------------------------------------------------ attach

// Graphs bake in kernel parameters (buffer addresses, ring geometry, tile counts).  Every
// change of that state drops the handle's own graphs and takes a new generation number, which
// is part of every graph key -- also of the two-level graphs another handle keeps.
static std::atomic<unsigned long long> g_generation{0};
static void invalidate_graphs(mf_t *m) {
    m->graphs.clear();
    m->gen = ++g_generation;
}

extern "C" int mf_attach(mf_t *m, void *dev_ptr, size_t bytes, void *stream) {
    if (!m) return fail(MF_EINVAL, "null handle");
    if (!dev_ptr || ((uintptr_t)dev_ptr & 255)) return fail(MF_EALIGN, "device pointer must be 256-byte aligned");
    if (bytes < mf_bytes(m)) return fail(MF_EALIGN, "buffer of %zu bytes, need %zu", bytes, mf_bytes(m));
    invalidate_graphs(m);
    m->base = (char *)dev_ptr;
    m->bytes = bytes;
    m->stream = (cudaStream_t)stream;
    m->cur = 0;
    if (!m->cap) CU(cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking));
    if (!m->cap2) CU(cudaStreamCreateWithFlags(&m->cap2, cudaStreamNonBlocking));
    for (auto &e : m->fork_ev)
        if (!e) CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (!m->h_sum) CU(cudaMallocHost((void **)&m->h_sum, sizeof(double)));
    int rc;
    if ((rc = m->d_fabs.upload(m->fabs, m->stream))) return rc;
    if ((rc = m->d_fb.upload(m->fb, m->stream))) return rc;
    if ((rc = m->d_fbtasks.upload(m->fbtasks, m->stream))) return rc;
    if ((rc = m->d_cbeg.upload(m->fb_cbeg, m->stream))) return rc;
    {
        std::vector<long long> rowpre(m->fabs.size() + 1, 0);
        for (size_t b = 0; b < m->fabs.size(); ++b)
            rowpre[b + 1] = rowpre[b] + (long long)m->fabs[b].n[1] * m->fabs[b].n[2];
        if ((rc = m->d_rowpre.upload(rowpre, m->stream))) return rc;
    }
    // tile buffer large enough for every autotune candidate
    size_t cap = m->tiles.size();
    std::vector<Tile> tmp;
    for (auto &t : tile_candidates(m)) {
        make_tiles(m, t.data(), tmp);
        cap = std::max(cap, tmp.size());
    }
    m->tile_capacity = cap;
    if ((rc = m->d_tiles.ensure(cap * sizeof(Tile)))) return rc;
    CU(cudaMemcpyAsync(m->d_tiles.p, m->tiles.data(), m->tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice, m->stream));
    if ((rc = m->d_partials.ensure(512 * sizeof(double2)))) return rc;
    if ((rc = m->d_maps.ensure(3 * m->fabs.size() * sizeof(CUtensorMap)))) return rc;  // two levels + stage
    if ((rc = m->d_tfab.ensure(m->fabs.size() * sizeof(TmaFab)))) return rc;
    if ((rc = m->d_err.ensure(sizeof(int)))) return rc;
    CU(cudaMemsetAsync(m->d_err.p, 0, sizeof(int), m->stream));
    if ((rc = m->d_fix.ensure(3 * sizeof(FixSet)))) return rc;
    m->tma_R = 0;
    if ((rc = m->d_sumout.ensure(sizeof(double)))) return rc;
    CU(cudaStreamSynchronize(m->stream));  // host vectors may change after return
    m->attached = true;
    return 0;
}

static int need_attached(const mf_t *m) {
    if (!m) return fail(MF_EINVAL, "null handle");
    if (!m->attached) return fail(MF_ESTATE, "handle not attached");
    return 0;
}

static int check_device_error(mf_t *m) {
    if (!m->d_err.p) return 0;
    int e = 0;
    CU(cudaMemcpy(&e, m->d_err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        cudaMemsetAsync(m->d_err.p, 0, sizeof(int), m->stream);
        if (e & 1) return fail(MF_ECUDA, "a bounded wait inside a stencil kernel expired (device error word %d)", e);
        return fail(MF_ECUDA, "a non-finite value reached the fixed-point stencil (MF_FIXED_DIFF; device error word %d)", e);
    }
    return 0;
}

static int set_tiles(mf_t *m, const int t[3]) {
    for (int d = 0; d < 3; ++d) m->tile[d] = t[d];
    make_tiles(m, m->tile, m->tiles);
    if (m->attached) {
        if (m->tiles.size() > m->tile_capacity) {  // only from mf_set_tile, never while advancing
            int rc = m->d_tiles.ensure(m->tiles.size() * sizeof(Tile));
            if (rc) return rc;
            m->tile_capacity = m->tiles.size();
        }
        CU(cudaMemcpyAsync(m->d_tiles.p, m->tiles.data(), m->tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice,
                           m->stream));
        CU(cudaStreamSynchronize(m->stream));
        invalidate_graphs(m);
    }
    m->tma_R = 0;  // plane geometry follows the tile shape
    return 0;
}

extern "C" int mf_set_tile(mf_t *m, const int tile[3]) {
    if (!m) return fail(MF_EINVAL, "null handle");
    if (!tile) {
        m->tile_auto = true;
        return 0;
    }
    for (int d = 0; d < 3; ++d)
        if (tile[d] > 32767) return fail(MF_EINVAL, "tile size too large");
    m->tile_auto = false;
    m->push_pref = true;
    for (int k = 0; k < kTileClasses; ++k) m->cty[k] = m->ctz[k] = -1;
    int rc = set_tiles(m, tile);
    if (rc) return rc;
    m->tma_R = 0;
    return 0;
}

extern "C" int mf_set_class_tile(mf_t *m, int cls, int ty, int tz) {
    if (!m) return fail(MF_EINVAL, "null handle");
    if (cls < 0 || cls >= kTileClasses) return fail(MF_EINVAL, "class must be in [0, %d)", kTileClasses);
    if (ty < -1 || tz < -1 || ty > 32767 || tz > 32767) return fail(MF_EINVAL, "tile extents must be -1, 0 or positive");
    m->cty[cls] = ty;
    m->ctz[cls] = tz;
    m->tile_auto = false;
    return set_tiles(m, m->tile);
}

extern "C" int mf_get_class_tiles(const mf_t *m, int out[3 * kTileClasses]) {
    if (!m || !out) return fail(MF_EINVAL, "null argument");
    int cells[kTileClasses] = {0};
    for (auto &f : m->fabs) cells[tile_class(f)] = 1;
    for (int k = 0; k < kTileClasses; ++k) {
        out[3 * k] = cells[k];
        out[3 * k + 1] = m->cty[k];
        out[3 * k + 2] = m->ctz[k];
    }
    return 0;
}

extern "C" int mf_set_kernel(mf_t *m, int variant) {
    if (!m) return fail(MF_EINVAL, "null handle");
    if (variant != MF_KERNEL_TMA && variant != MF_KERNEL_GLOBAL) return fail(MF_EINVAL, "unknown kernel variant");
    m->use_tma = variant == MF_KERNEL_TMA;
    m->tma_R = 0;
    invalidate_graphs(m);
    return 0;
}

extern "C" int mf_get_tile(const mf_t *m, int tile[3]) {
    if (!m || !tile) return fail(MF_EINVAL, "null argument");
    for (int d = 0; d < 3; ++d) tile[d] = m->tile[d];
    return m->tile_auto ? 1 : 0;
}

// ------------------------------------------------------------------ host <-> device copies

static int dense_extent(const mf_t *m, int dn[3]) {
    for (int d = 0; d < 3; ++d) dn[d] = m->domain.len(d);
    return 0;
}

extern "C" int mf_copy_from_host(mf_t *m, const double *dense) {
    int rc = need_attached(m);
    if (rc) return rc;
    if (!dense) return fail(MF_EINVAL, "null dense");
    int dn[3];
    dense_extent(m, dn);
    const long long plane = (long long)dn[0] * dn[1];
    const long long cap = (long long)(m->level_elems * m->esize / sizeof(double));
    const long long zc = std::min<long long>(dn[2], cap / plane);
    if (zc < 1) return fail(MF_EINVAL, "a dense z-plane does not fit in one time level");
    double *stage = (double *)m->level_ptr(1 - m->cur);
    void *dst = m->level_ptr(m->cur);
    for (int c = 0; c < m->ncomp; ++c)
        for (long long z0 = 0; z0 < dn[2]; z0 += zc) {
            const long long z1 = std::min<long long>(dn[2], z0 + zc);
            CU(cudaMemcpyAsync(stage, dense + ((long long)c * dn[2] + z0) * plane, (z1 - z0) * plane * sizeof(double),
                               cudaMemcpyHostToDevice, m->stream));
            CU(launch_scatter_dense(m->dtype, dst, (const FabInfo *)m->d_fabs.p, (int)m->fabs.size(), stage,
                                    m->domain.lo, dn, m->domain.lo[2] + (int)z0, m->domain.lo[2] + (int)z1, c, 1,
                                    m->stream));
        }
    return 0;
}

extern "C" int mf_copy_to_host(mf_t *m, double *dense) {
    int rc = need_attached(m);
    if (rc) return rc;
    if (!dense) return fail(MF_EINVAL, "null dense");
    int dn[3];
    dense_extent(m, dn);
    const long long plane = (long long)dn[0] * dn[1];
    const long long cap = (long long)(m->level_elems * m->esize / sizeof(double));
    const long long zc = std::min<long long>(dn[2], cap / plane);
    if (zc < 1) return fail(MF_EINVAL, "a dense z-plane does not fit in one time level");
    double *stage = (double *)m->level_ptr(1 - m->cur);
    const void *src = m->level_ptr(m->cur);
    for (int c = 0; c < m->ncomp; ++c)
        for (long long z0 = 0; z0 < dn[2]; z0 += zc) {
            const long long z1 = std::min<long long>(dn[2], z0 + zc);
            CU(launch_gather_dense(m->dtype, src, (const FabInfo *)m->d_fabs.p, (int)m->fabs.size(), stage,
                                   m->domain.lo, dn, m->domain.lo[2] + (int)z0, m->domain.lo[2] + (int)z1, c, 1,
                                   m->stream));
            CU(cudaMemcpyAsync(dense + ((long long)c * dn[2] + z0) * plane, stage, (z1 - z0) * plane * sizeof(double),
                               cudaMemcpyDeviceToHost, m->stream));
        }
    CU(cudaStreamSynchronize(m->stream));
    return check_device_error(m);
}

// Host conversions for the FArrayBox debug copies.
static double bf16_to_double(uint16_t h) {
    uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}
static uint16_t double_to_bf16(double d) {
    // round to odd into float (24 bits >= 8 + 2), then round-to-nearest-even into bf16
    float f = (float)d;
    if (std::isfinite(f) && std::fabs((double)f) > std::fabs(d)) f = std::nextafter(f, 0.0f);
    uint32_t u;
    memcpy(&u, &f, 4);
    if (std::isfinite(d) && (double)f != d) u |= 1u;
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)((u >> 16) | ((u & 0xffff) ? 0x40 : 0));
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    return (uint16_t)(u >> 16);
}

// The window of box `box` (a logical box of a regional level) in its FArrayBox: the FArrayBox,
// the box's lower corner relative to the FArrayBox's valid corner, and the grown box's shape.
static int fab_window(const mf_t *m, int box, int *fab, int off[3], long long sh[3]) {
    if (box < 0 || box >= (int)user_boxes(m).size()) return fail(MF_EINVAL, "bad box");
    *fab = m->regional ? m->lbox_region[box] : box;
    const Box &b = user_boxes(m)[box], &r = m->boxes[*fab];
    for (int d = 0; d < 3; ++d) {
        off[d] = b.lo[d] - r.lo[d];
        sh[d] = b.len(d) + 2 * m->ngrow;
    }
    return 0;
}

extern "C" int mf_copy_fab_to_host(mf_t *m, int box, double *out) {
    int rc = need_attached(m);
    if (rc) return rc;
    int fab, off[3];
    long long sh[3];
    if (!out) return fail(MF_EINVAL, "null out");
    if ((rc = fab_window(m, box, &fab, off, sh))) return rc;
    const FabInfo &f = m->fabs[fab];
    const size_t n = (size_t)f.cstride * m->ncomp;
    std::vector<char> raw(n * m->esize);
    CU(cudaMemcpyAsync(raw.data(), (char *)m->level_ptr(m->cur) + (size_t)m->fab_start[fab] * m->esize,
                       raw.size(), cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    const long long org_local = f.org - m->fab_start[fab] + off[2] * f.plane + (long long)off[1] * f.px + off[0];
    const int g = m->ngrow;
    size_t q = 0;
    for (int c = 0; c < m->ncomp; ++c)
        for (long long z = 0; z < sh[2]; ++z)
            for (long long y = 0; y < sh[1]; ++y)
                for (long long x = 0; x < sh[0]; ++x) {
                    const long long at = org_local + c * f.cstride + (z - g) * f.plane + (y - g) * f.px + (x - g);
                    const char *p = raw.data() + at * m->esize;
                    double v;
                    if (m->dtype == F64) memcpy(&v, p, 8);
                    else if (m->dtype == F32) { float t; memcpy(&t, p, 4); v = t; }
                    else { uint16_t t; memcpy(&t, p, 2); v = bf16_to_double(t); }
                    out[q++] = v;
                }
    return 0;
}

extern "C" int mf_copy_fab_from_host(mf_t *m, int box, const double *in) {
    int rc = need_attached(m);
    if (rc) return rc;
    int fab, off[3];
    long long sh[3];
    if (!in) return fail(MF_EINVAL, "null in");
    if ((rc = fab_window(m, box, &fab, off, sh))) return rc;
    const FabInfo &f = m->fabs[fab];
    const size_t n = (size_t)f.cstride * m->ncomp;
    std::vector<char> raw(n * m->esize);
    char *dev = (char *)m->level_ptr(m->cur) + (size_t)m->fab_start[fab] * m->esize;
    CU(cudaMemcpyAsync(raw.data(), dev, raw.size(), cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    const long long org_local = f.org - m->fab_start[fab] + off[2] * f.plane + (long long)off[1] * f.px + off[0];
    const int g = m->ngrow;
    size_t q = 0;
    for (int c = 0; c < m->ncomp; ++c)
        for (long long z = 0; z < sh[2]; ++z)
            for (long long y = 0; y < sh[1]; ++y)
                for (long long x = 0; x < sh[0]; ++x) {
                    const long long at = org_local + c * f.cstride + (z - g) * f.plane + (y - g) * f.px + (x - g);
                    char *p = raw.data() + at * m->esize;
                    const double v = in[q++];
                    // in a region the box's ghost frame is other boxes' cells or the region's ghosts:
                    // only the box's own cells are written
                    if (m->regional && (x < g || y < g || z < g || x >= sh[0] - g || y >= sh[1] - g || z >= sh[2] - g))
                        continue;
                    if (m->dtype == F64) memcpy(p, &v, 8);
                    else if (m->dtype == F32) { float t = (float)v; memcpy(p, &t, 4); }
                    else { uint16_t t = double_to_bf16(v); memcpy(p, &t, 2); }
                }
    CU(cudaMemcpyAsync(dev, raw.data(), raw.size(), cudaMemcpyHostToDevice, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    return 0;
}

// ------------------------------------------------------------------ TMA tensor maps

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
    }
    return fn;
}

// The schedule the TMA build uses: the chosen rows and group bytes where the kernel variant
// (plain arithmetic, or fixed point -- bit 8 of the build key) has them, else one row and
// 16-byte groups.
static bool tma_has(const mf_t *m, int R, int rows, int gb) {
    return (m->tma_R & 8) ? tma_has_group_fix(R, rows, gb) : tma_has_group(m->dtype, R, rows, gb);
}
static int eff_rows(const mf_t *m, int R) {
    const int rows = std::min(m->tma_rows, tma_max_rows(R));
    return tma_has(m, R, rows, 16) ? rows : 1;
}
static int eff_gb(const mf_t *m, int R) { return tma_has(m, R, eff_rows(m, R), m->tma_gb) ? m->tma_gb : 16; }

// Plane geometry of every FArrayBox for the current tile shape and radius R; false when a
// box needs a plane wider than the TMA box limit (256 per dimension) or more cells per
// thread than the kernel keeps in registers.  A box whose two x faces are served by strips
// (served[2b], served[2b+1]) loads only its valid cells of each row, rounded up to 16 bytes;
// the others load the whole row, ghost columns and padding included.
static bool tma_geometry(mf_t *m, int R, bool fix, const std::vector<char> &served, std::vector<TmaFab> &tf,
                         int &slot_bytes, int &gpt) {
    const int S = m->esize, A = 16 / S, g = m->ngrow;
    tf.assign(m->fabs.size(), TmaFab{});
    int maxplane = 0, maxgroups = 0;
    const int VXg = eff_gb(m, R) / S;  // cells per group
    for (auto &t : m->tiles) {
        // the TMA kernel streams whole rows of every plane; a thread owns one group in ROWS
        // consecutive rows
        if (t.x0 != 0 || t.tx != m->fabs[t.fab].n[0]) return false;
        const int rows = eff_rows(m, R);
        maxgroups = std::max(maxgroups, (m->fabs[t.fab].n[0] + VXg - 1) / VXg * (((int)t.ty + rows - 1) / rows));
    }
    for (size_t b = 0; b < m->fabs.size(); ++b) {
        int ty = 1;
        for (auto &t : m->tiles)
            if (t.fab == (int)b && t.comp == 0) ty = std::max(ty, (int)t.ty);
        const int xvg = valid_x_elem(m);
        const bool narrow = !served.empty() && served[2 * b] && served[2 * b + 1];
        tf[b].bx = narrow ? (m->fabs[b].n[0] + A - 1) / A * A : m->fabs[b].px;
        tf[b].by = ty + 2 * R;
        tf[b].ngrow = g;
        tf[b].xs = narrow ? xvg : 0;
        tf[b].xv = xvg - tf[b].xs;
        if (tf[b].bx > 256 || tf[b].by > 256) return false;
        // slack rows after the plane: a thread of a tile's last, partial row set reads up to
        // rows - 1 rows past it (values that feed only unused results), and a 32-byte group
        // on a narrow row up to 16 bytes past the last row
        const int slack = std::max(eff_rows(m, R) - 1, eff_gb(m, R) > 16 ? 1 : 0);
        maxplane = std::max(maxplane, tf[b].bx * (tf[b].by + slack) * S);
    }
    // a producer warp plus one consumer thread per group, rounded up to a warp
    gpt = 32 + (maxgroups + 31) / 32 * 32;
    if (gpt > (fix ? tma_max_threads_fix(R, eff_rows(m, R), eff_gb(m, R)) : tma_max_threads(m->dtype, R))) return false;
    slot_bytes = (maxplane + 127) / 128 * 128;
    return true;
}

// x-halo strips: for a tile whose x halo leaves its box on the low (high) side, the box
// owning the column just outside that face over all the tile's rows and planes, when one box
// owns all of it.  The strip holds that box's R valid cells next to the face.
static void find_strips(mf_t *m, int R, std::vector<TileStrip> &st, std::vector<char> &served) {
    const int S = m->esize, A = 16 / S, g = m->ngrow;
    const int nb = (int)m->boxes.size();
    st.assign(m->tiles.size(), TileStrip{-1, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0});
    // served[2b + side]: every tile on that face pulls its halo from a neighbour
    served.assign(2 * (size_t)nb, 1);
    std::vector<char> touched(2 * (size_t)nb, 0);
    BinHash hash;
    hash.build(m->domain, m->boxes);
    std::vector<int> cand, stamp(nb, -1);
    int tag = 0;
    const int Lx = m->domain.len(0);
    for (size_t w = 0; w < m->tiles.size(); ++w) {
        const Tile &t = m->tiles[w];
        const Box &B = m->boxes[t.fab];
        for (int side = 0; side < 2; ++side) {
            // the tile's x halo leaves the box on this side
            const bool at_face = side == 0 ? t.x0 < R : t.x0 + t.tx + R > B.len(0);
            if (!at_face) continue;
            touched[2 * t.fab + side] = 1;
            const int X = side == 0 ? B.lo[0] - 1 : B.hi[0] + 1;
            const int wx = m->domain.lo[0] + (((X - m->domain.lo[0]) % Lx) + Lx) % Lx;
            Box q;
            q.lo[0] = q.hi[0] = wx;
            q.lo[1] = B.lo[1] + t.y0;
            q.hi[1] = q.lo[1] + t.ty - 1;
            q.lo[2] = B.lo[2] + t.z0;
            q.hi[2] = q.lo[2] + t.tz - 1;
            hash.query(q, cand, stamp, ++tag);
            int owner = -1;
            for (int a : cand) {
                const Box &Ab = m->boxes[a];
                bool in = true;
                for (int d = 0; d < 3; ++d) in = in && Ab.lo[d] <= q.lo[d] && q.hi[d] <= Ab.hi[d];
                if (in) { owner = a; break; }
            }
            const bool ok = owner >= 0 && m->boxes[owner].len(0) >= R;
            if (!ok) {
                served[2 * t.fab + side] = 0;
                continue;
            }
            const Box &Ab = m->boxes[owner];
            const int nA = Ab.len(0);
            // strip: XW elements of the owner's rows, starting 16-byte aligned at or before the R
            // cells next to the face (row element of cell x is xv + x)
            const int xvA = valid_x_elem(m);
            const int start = side == 0 ? (xvA + nA - R) / A * A : xvA;
            const int y = g + q.lo[1] - Ab.lo[1], z = g + q.lo[2] - Ab.lo[2];
            if (side == 0) {
                st[w].lfab = owner; st[w].lx = start; st[w].ly = y; st[w].lz = z;
                st[w].lidx0 = xvA + nA - start;
            } else {
                st[w].rfab = owner; st[w].rx = start; st[w].ry = y; st[w].rz = z;
                st[w].ridx0 = xvA - start;
            }
        }
    }
    // a tile whose column has one owner uses its strip whether or not the rest of the face
    // does; the fill copies only the parts of unserved faces that tiles without a strip read
    for (size_t i = 0; i < served.size(); ++i) served[i] = served[i] && touched[i];
}

// The x-face FillBoundary region e (kind 0 or 1) restricted to the rows and planes of the tiles
// of its destination box that read that x halo from ghost cells (no strip on that side).  The
// tiles of different components may be cut at different planes and a fill task copies every
// component, so the parts come from the tiles of all components (each distinct part once).
// tiles_of[b]: the indices of box b's tiles.
static void append_unserved_x(const mf_t *m, int e, const std::vector<TileStrip> &st,
                              const std::vector<std::vector<int>> &tiles_of, std::vector<FbTask> &out) {
    const FbEntry &en = m->fb[e];
    const int side = m->fb_kind[e];
    const auto &cr = m->fb_corner[e];
    const Box &B = m->boxes[en.dfab];
    std::vector<std::array<int, 4>> parts;
    for (int w : tiles_of[en.dfab]) {
        const Tile &t = m->tiles[w];
        if ((side == 0 ? st[w].lfab : st[w].rfab) >= 0) continue;
        const int ylo = std::max(cr[1], B.lo[1] + t.y0), yhi = std::min(cr[1] + en.n[1], B.lo[1] + t.y0 + t.ty);
        const int zlo = std::max(cr[2], B.lo[2] + t.z0), zhi = std::min(cr[2] + en.n[2], B.lo[2] + t.z0 + t.tz);
        if (ylo < yhi && zlo < zhi) parts.push_back({ylo, yhi, zlo, zhi});
    }
    std::sort(parts.begin(), parts.end());
    parts.erase(std::unique(parts.begin(), parts.end()), parts.end());
    for (const auto &q : parts) {
        const int lo[3] = {0, q[0] - cr[1], q[2] - cr[2]}, n[3] = {en.n[0], q[1] - q[0], q[3] - q[2]};
        append_fill_tasks(m, clip_entry(m, e, lo, n), out);
    }
}

// Balanced schedule for G CTAs: the tile shape's columns (its x and y extents, every plane of
// the box) in order, each plane weighted by its cells, cut into G runs of equal weight; CTA b
// takes the planes whose midpoints fall into run b, as one tile per column it touches.
static void balance_tiles(const mf_t *m, int G, std::vector<Tile> &out, std::vector<int> &first) {
    std::vector<Tile> cols;
    const int shape[3] = {m->tile[0], m->tile[1], 0};
    make_tiles(m, shape, cols);
    double total = 0;
    for (auto &c : cols) total += (double)c.tx * c.ty * c.tz;
    out.clear();
    first.assign((size_t)G + 1, 0);
    double acc = 0;
    int cur = 0;  // CTA of the last tile emitted
    auto owner = [&](double at) { return std::min(G - 1, (int)(at * G / total)); };
    for (auto &c : cols) {
        const double a = (double)c.tx * c.ty;
        for (int k = 0; k < c.tz;) {
            const int b = owner(acc + (k + 0.5) * a);
            int k1 = k + 1;
            while (k1 < c.tz && owner(acc + (k1 + 0.5) * a) == b) ++k1;
            while (cur < b) first[++cur] = (int)out.size();
            Tile t = c;
            t.z0 = (short)(c.z0 + k);
            t.tz = (short)(k1 - k);
            out.push_back(t);
            k = k1;
        }
        acc += a * c.tz;
    }
    while (cur < G) first[++cur] = (int)out.size();
}

// The TMA build (tensor maps, plane geometry, schedule, push and fill lists) depends on the
// radius and, through the CTA size and residency, on the kernel variant: plain arithmetic, or
// the fixed-point differences of FP64 storage.
static int tma_key(int R, bool fix) { return R + (fix ? 8 : 0); }

static int build_tma(mf_t *m, int R, bool fix = false) {
    invalidate_graphs(m);
    m->tma_ok = false;
    m->tma_strips = false;
    m->tma_push = false;
    m->tma_R = tma_key(R, fix);
    m->tma_grid = 0;
    m->cta_tiles.clear();
    if (!m->use_tma) return 0;
    const int S = m->esize, A = 16 / S;
    const int XW = (R + A - 1 + A - 1) / A * A;  // strip width: R cells from any 16-byte start
    int srows = 1;
    for (auto &t : m->tiles) srows = std::max(srows, (int)t.ty);
    std::vector<TmaFab> tf;
    int main_slot = 0, gpt = 0;
    {
        // faces served by strips for whole-box z extents stay served for any z split of them,
        // so they fix the plane geometry before the balanced schedule is made
        std::vector<TileStrip> st0;
        std::vector<char> served0;
        find_strips(m, R, st0, served0);
        if (!tma_geometry(m, R, fix, served0, tf, main_slot, gpt)) return 0;
    }
    const int strip_bytes = XW * srows * S;
    const int strip_pitch = (strip_bytes + 127) / 128 * 128;
    const int slot = main_slot + 2 * strip_pitch;
    int ns = m->tma_ns_pref ? m->tma_ns_pref : (R == 4 ? 16 : 8);  // ring slots (power of two)
    if (ns < 2 * R + 1) ns = R == 4 ? 16 : 8;
    // the ring shrinks towards 160 KB while it keeps 2R + 1 planes and some in flight; a CTA may
    // take up to 227 KB of shared memory, of which the kernel's static tables use below 8 KB
    const int ns_floor = R == 4 ? 16 : 8;
    while (ns > ns_floor && (long long)ns * slot + 128 > 160 * 1024) ns /= 2;
    if (ns < 2 * R + 1 || (long long)ns * slot + 128 > 227 * 1024 - 8192) return 0;
    if (m->tile[2] <= 0) {
        // whole-box z extent: split the columns over exactly one wave of CTAs
        const int per_sm = fix ? tma_ctas_per_sm_fix(R, eff_rows(m, R), eff_gb(m, R), gpt, ns * slot + 128)
                               : tma_ctas_per_sm(m->dtype, R, eff_rows(m, R), eff_gb(m, R), gpt, ns * slot + 128);
        if (per_sm < 1) return 0;
        const int G = per_sm * sm_count();
        balance_tiles(m, G, m->tiles, m->cta_tiles);
        if (m->tiles.size() > m->tile_capacity) {
            int rc = m->d_tiles.ensure(m->tiles.size() * sizeof(Tile));
            if (rc) return rc;
            m->tile_capacity = m->tiles.size();
        }
        CU(cudaMemcpyAsync(m->d_tiles.p, m->tiles.data(), m->tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice,
                           m->stream));
        int rc = m->d_cta.upload(m->cta_tiles, m->stream);
        if (rc) return rc;
        m->tma_grid = G;
    }
    std::vector<TileStrip> strips;
    std::vector<char> served;
    find_strips(m, R, strips, served);
    auto encode = tensor_map_encoder();
    if (!encode) return 0;
    const int nf = (int)m->fabs.size();
    std::vector<CUtensorMap> maps(3 * (size_t)nf), smaps(3 * (size_t)nf);  // levels 0, 1 and the stage level
    const CUtensorMapDataType dt = m->dtype == F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : m->dtype == F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                     : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    for (int which = 0; which < (m->stage ? 3 : 2); ++which)
        for (int b = 0; b < nf; ++b) {
            const FabInfo &f = m->fabs[b];
            const int g = m->ngrow;
            cuuint64_t dims[4] = {(cuuint64_t)f.px, (cuuint64_t)(f.n[1] + 2 * g), (cuuint64_t)(f.n[2] + 2 * g),
                                  (cuuint64_t)m->ncomp};
            cuuint64_t strides[3] = {(cuuint64_t)f.px * S, (cuuint64_t)f.plane * S, (cuuint64_t)f.cstride * S};
            cuuint32_t box[4] = {(cuuint32_t)tf[b].bx, (cuuint32_t)tf[b].by, 1, 1};
            cuuint32_t sbox[4] = {(cuuint32_t)XW, (cuuint32_t)srows, 1, 1};
            cuuint32_t estr[4] = {1, 1, 1, 1};
            void *gaddr = (char *)m->level_ptr(which) + (size_t)m->fab_start[b] * S;
            CUresult r = encode(&maps[(size_t)which * nf + b], dt, 4, gaddr, dims, strides, box, estr,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return fail(MF_ECUDA, "cuTensorMapEncodeTiled failed (%d) for box %d", (int)r, b);
            r = encode(&smaps[(size_t)which * nf + b], dt, 4, gaddr, dims, strides, sbox, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return fail(MF_ECUDA, "cuTensorMapEncodeTiled (strip) failed (%d)", (int)r);
        }
    // the fill inside the advance: faces only (the star stencil reads no edge or corner), and
    // of the x faces only the parts that tiles without a strip read
    std::vector<std::vector<int>> tiles_of(m->boxes.size());
    for (size_t w = 0; w < m->tiles.size(); ++w) tiles_of[m->tiles[w].fab].push_back((int)w);
    m->fbtasks_adv.clear();
    for (size_t e = 0; e < m->fb.size(); ++e) {
        const int k = m->fb_kind[e];
        if (k == 6 || (k < 2 && served[2 * (size_t)m->fb[e].dfab + k])) continue;
        if (k < 2) append_unserved_x(m, (int)e, strips, tiles_of, m->fbtasks_adv);
        else append_fill_tasks(m, m->fb[e], m->fbtasks_adv);
    }
    // ghost push: every y/z face region is written by the tiles that compute its source cells;
    // the fill of later steps copies only the x faces not served by strips and the regions of
    // tiles with more than kMaxPush pieces (such a tile pushes nothing)
    std::vector<PushPiece> pieces;
    std::vector<int> piece_entry;     // the FillBoundary region of each piece
    std::vector<char> unpushed(m->fb.size(), 0);
    {
        std::vector<std::vector<int>> by_src(m->boxes.size());
        for (size_t e = 0; e < m->fb.size(); ++e)
            if (m->fb_kind[e] >= 2 && m->fb_kind[e] < 6) by_src[m->fb[e].sfab].push_back((int)e);
        for (size_t w = 0; w < m->tiles.size(); ++w) {
            const Tile &t = m->tiles[w];
            const Box &B = m->boxes[t.fab];
            const int tlo[3] = {B.lo[0] + t.x0, B.lo[1] + t.y0, B.lo[2] + t.z0};
            const int thi[3] = {tlo[0] + t.tx - 1, tlo[1] + t.ty - 1, tlo[2] + t.tz - 1};
            strips[w].pfirst = (int)pieces.size();
            for (int e : by_src[t.fab]) {
                const FbEntry &en = m->fb[e];
                const auto &cr = m->fb_corner[e];
                int lo[3], hi[3];
                bool empty = false;
                for (int d = 0; d < 3; ++d) {
                    lo[d] = std::max(cr[3 + d], tlo[d]);
                    hi[d] = std::min(cr[3 + d] + en.n[d] - 1, thi[d]);
                    empty = empty || lo[d] > hi[d];
                }
                if (empty) continue;
                PushPiece pp{};
                pp.dfab = en.dfab;
                pp.x0 = lo[0] - tlo[0]; pp.y0 = lo[1] - tlo[1]; pp.z0 = lo[2] - tlo[2];
                pp.nx = hi[0] - lo[0] + 1; pp.ny = hi[1] - lo[1] + 1; pp.nz = hi[2] - lo[2] + 1;
                const int dx = cr[0] + (lo[0] - cr[3]);
                pp.dst = elem_at(m->fabs[en.dfab], dx, cr[1] + (lo[1] - cr[4]), cr[2] + (lo[2] - cr[5]));
                // the destination rows are laid out exactly like the tile's rows: whole 16-byte
                // groups (don't-care values in ghost / padding positions included) may be stored
                pp.full_row = pp.x0 == 0 && pp.nx == t.tx && dx == m->boxes[en.dfab].lo[0] &&
                              m->boxes[en.dfab].len(0) == t.tx;
                pieces.push_back(pp);
                piece_entry.push_back(e);
            }
            strips[w].pcount = (int)pieces.size() - strips[w].pfirst;
            if (strips[w].pcount > kMaxPush) {  // this tile pushes nothing; the fill copies its regions
                for (size_t i = strips[w].pfirst; i < pieces.size(); ++i) unpushed[piece_entry[i]] = 1;
                pieces.resize(strips[w].pfirst);
                piece_entry.resize(strips[w].pfirst);
                strips[w].pcount = 0;
            }
        }
        m->fbtasks_res.clear();
        for (size_t e = 0; e < m->fb.size(); ++e) {
            const int k = m->fb_kind[e];
            if (k < 2 && !served[2 * (size_t)m->fb[e].dfab + k]) append_unserved_x(m, (int)e, strips, tiles_of, m->fbtasks_res);
            else if (unpushed[e]) append_fill_tasks(m, m->fb[e], m->fbtasks_res);
        }
    }
    int rc;
    if ((rc = m->d_maps.upload(maps, m->stream))) return rc;
    if ((rc = m->d_smaps.upload(smaps, m->stream))) return rc;
    if ((rc = m->d_tfab.upload(tf, m->stream))) return rc;
    if ((rc = m->d_strips.upload(strips, m->stream))) return rc;
    if ((rc = m->d_fbtasks_adv.upload(m->fbtasks_adv, m->stream))) return rc;
    if ((rc = m->d_fbtasks_res.upload(m->fbtasks_res, m->stream))) return rc;
    if ((rc = m->d_push.upload(pieces, m->stream))) return rc;
    CU(cudaStreamSynchronize(m->stream));
    m->tma_cpt = gpt;
    m->tma_slot = slot;
    m->tma_ns = ns;
    m->tma_main_slot = main_slot;
    m->tma_strip_rows = srows;
    m->tma_strip_bytes = strip_bytes;
    m->tma_strip_pitch = strip_pitch;
    m->tma_strip_w = XW;
    m->tma_ok = true;
    m->tma_strips = true;
    m->tma_push = true;
    return 0;
}

// ------------------------------------------------------------------ phases

static LevelPtrs level_ptrs(const mf_t *m, int which) {
    LevelPtrs lv{};
    lv.base[0] = m->level_ptr(which);
    return lv;
}

static int enqueue_fill(mf_t *m, int which, cudaStream_t s) {
    CU(launch_fill(m->dtype, level_ptrs(m, which), (const FbTask *)m->d_fbtasks.p, (int)m->fbtasks.size(), 0, s));
    return 0;
}

// The stencil writes the y and z face ghosts of the level it produces (the ghost push), so later
// steps fill only the residual regions.
static bool use_push(const mf_t *m) { return m->use_tma && m->tma_ok && m->tma_push && m->push_pref; }

// The ghost exchange a time step needs: with the TMA stencil, only the face regions it reads
// from ghost cells (edges and corners are never read by a star stencil; x faces whose tiles
// take their halo from the neighbour box are skipped).
static size_t fill_step_tasks(const mf_t *m) {
    return (m->use_tma && m->tma_ok && m->tma_strips) ? m->fbtasks_adv.size() : m->fbtasks.size();
}

static int enqueue_fill_step(mf_t *m, int which, cudaStream_t s) {
    if (!(m->use_tma && m->tma_ok && m->tma_strips)) return enqueue_fill(m, which, s);
    CU(launch_fill(m->dtype, level_ptrs(m, which), (const FbTask *)m->d_fbtasks_adv.p, (int)m->fbtasks_adv.size(), 0,
                   s));
    return 0;
}

// One stencil launch: level `from` (ghosts filled) -> level `to` (default: the other time
// level).  With u0 >= 0 the launch is a Runge-Kutta stage and writes
// rk_a * (level u0) + rk_b * (forward-Euler value).
struct StageArgs {
    int to = -1, u0 = -1;
    double rk_a = 0.0, rk_b = 1.0;
};

static StencilParams stencil_params(const mf_t *m, int from, const double *lam, const StageArgs &sa = StageArgs{}) {
    StencilParams p{};
    p.src[0] = m->level_ptr(from);
    p.dst[0] = m->level_ptr(sa.to >= 0 ? sa.to : 1 - from);
    p.u0[0] = sa.u0 >= 0 ? m->level_ptr(sa.u0) : nullptr;
    p.rk_a = sa.rk_a;
    p.rk_b = sa.rk_b;
    p.ftab = (const FabInfo *)m->d_fabs.p;
    p.tiles = (const Tile *)m->d_tiles.p;
    p.ntiles = (int)m->tiles.size();
    for (int c = 0; c < m->ncomp; ++c) p.lam[0][c] = lam[c];
    return p;
}

// round(lam / den * 2^64) exactly (lam < 1): lam = m 2^(e - 53) with a 53-bit integer m.
static unsigned long long fix_q(double lam, int den) {
    int e = 0;
    const double f = std::frexp(lam, &e);
    const unsigned long long mant = (unsigned long long)std::ldexp(f, 53);
    const int sh = e + 11;  // lam 2^64 = mant 2^(e + 11)
    unsigned __int128 num = mant, dd = (unsigned __int128)den;
    if (sh >= 0) num <<= sh;
    else if (-sh < 100) dd <<= -sh;
    else return 0ull;
    return (unsigned long long)((num + dd / 2) / dd);
}

// fixstep >= 0: the fixed-point kernel (the level holds 64-bit fixed point), as step fixstep of an
// advance: it reads grid state fixstep % 3 (level `from`), writes state (fixstep + 1) % 3 (the
// level it produces) and clears state (fixstep + 2) % 3 for the step after it.
static int enqueue_stencil(mf_t *m, int from, int R, bool fp64diff, const double *lam, cudaStream_t s,
                           bool push = false, const StageArgs &sa = StageArgs{}, int fixstep = -1) {
    const bool fix = fixstep >= 0;
    if (m->use_tma && m->tma_R != tma_key(R, fix)) {
        int rc = build_tma(m, R, fix);
        if (rc) return rc;
    }
    if (fix && !(m->use_tma && m->tma_ok))
        return fail(MF_EINVAL, "MF_FIXED_DIFF runs on the TMA stencil, which this tile shape or kernel choice excludes");
    if (m->use_tma && m->tma_ok) {
        StencilTmaParams p{};
        p.maps = (const CUtensorMap *)m->d_maps.p + (size_t)from * m->fabs.size();
        p.tfab = (const TmaFab *)m->d_tfab.p;
        p.ftab = (const FabInfo *)m->d_fabs.p;
        p.tiles = (const Tile *)m->d_tiles.p;
        p.ntiles = (int)m->tiles.size();
        p.nstages = m->tma_ns;
        p.nstages_log2 = 0;
        while ((1 << p.nstages_log2) < m->tma_ns) ++p.nstages_log2;
        p.slot_bytes = m->tma_slot;
        p.dst[0] = m->level_ptr(sa.to >= 0 ? sa.to : 1 - from);
        p.u0[0] = sa.u0 >= 0 ? m->level_ptr(sa.u0) : nullptr;
        p.rk_a = sa.rk_a;
        p.rk_b = sa.rk_b;
        p.err = (int *)m->d_err.p;
        p.smaps = (const CUtensorMap *)m->d_smaps.p + (size_t)from * m->fabs.size();
        p.strips = (const TileStrip *)m->d_strips.p;
        p.strip_rows = m->tma_strip_rows;
        p.strip_off = m->tma_main_slot;
        p.strip_bytes = m->tma_strip_bytes;
        p.strip_pitch = m->tma_strip_pitch;
        p.strip_w = m->tma_strip_w;
        p.push = (push && m->tma_push) ? (const PushPiece *)m->d_push.p : nullptr;
        p.cta_tiles = m->tma_grid ? (const int *)m->d_cta.p : nullptr;
        for (int c = 0; c < m->ncomp; ++c) p.lam[0][c] = lam[c];
        if (fix) {
            FixSet *w = (FixSet *)m->d_fix.p;
            p.fix_in = w + fixstep % 3;
            p.fix_out = w + (fixstep + 1) % 3;
            p.fix_clear = w + (fixstep + 2) % 3;
            for (int c = 0; c < m->ncomp; ++c) p.fix_q[c] = fix_q(lam[c], fix_den(R));
            CU(launch_stencil_tma_fix(R, eff_rows(m, R), eff_gb(m, R), m->tma_cpt, p, m->tma_grid, s));
            return 0;
        }
        CU(launch_stencil_tma(m->dtype, R, fp64diff, eff_rows(m, R), eff_gb(m, R), m->tma_cpt, p, m->tma_grid, s));
        return 0;
    }
    StencilParams p = stencil_params(m, from, lam, sa);
    CU(launch_stencil(m->dtype, R, fp64diff, p, m->block[0], m->block[1], 0, s));
    return 0;
}

static int fab_maxz(const mf_t *m) {
    int maxz = 1;
    for (auto &f : m->fabs) maxz = std::max(maxz, f.n[2]);
    return maxz;
}

// Entering the fixed-point representation at the start of an advance: the three grid states
// cleared, the largest |u| of level `which` reduced, and the level's valid cells mapped in place
// to 64-bit fixed point on the first grid (state 0, which step 0 reads).  convert = false (the
// autotuner's timing launches) leaves the data and the cleared states as they are.
static int enqueue_fix_start(mf_t *m, int which, int R, cudaStream_t s, bool convert = true) {
    CU(cudaMemsetAsync(m->d_fix.p, 0, 3 * sizeof(FixSet), s));
    if (!convert) return 0;
    FixSet *w = (FixSet *)m->d_fix.p;
    const FabInfo *ft = (const FabInfo *)m->d_fabs.p;
    const int nf = (int)m->fabs.size(), mz = fab_maxz(m);
    CU(launch_fix_emax(m->level_ptr(which), ft, nf, m->ncomp, mz, w, s));
    CU(launch_fix_in(R, m->level_ptr(which), ft, nf, m->ncomp, mz, w, (int *)m->d_err.p, s));
    return 0;
}

// Leaving it after nsteps steps: level `which` back to FP64 from the grid of state nsteps % 3.
static int enqueue_fix_end(mf_t *m, int which, int nsteps, cudaStream_t s) {
    CU(launch_fix_out(m->level_ptr(which), (const FabInfo *)m->d_fabs.p, (int)m->fabs.size(), m->ncomp, fab_maxz(m),
                      (const FixSet *)m->d_fix.p + nsteps % 3, s));
    return 0;
}

extern "C" int mf_fill_boundary(mf_t *m) {
    int rc = need_attached(m);
    if (rc) return rc;
    return enqueue_fill(m, m->cur, m->stream);
}

static int check_stencil(const mf_t *m, const mf_stencil *st, double dt, double lam[kMaxComp], double dx_scale) {
    if (!st) return fail(MF_EINVAL, "null stencil");
    const int R = st->kind;
    if (R != 1 && R != 2 && R != 4) return fail(MF_EINVAL, "stencil kind must be 1, 2 or 4");
    if (m->ngrow < R) return fail(MF_EINVAL, "ngrow %d below the stencil radius %d", m->ngrow, R);
    if (!st->diffusivity) return fail(MF_EINVAL, "null diffusivity");
    if (!(dt > 0.0)) return fail(MF_EINVAL, "dt must be positive");
    const int N = m->domain.len(0);  // cubic cells of side dx = 1 / N_x
    // |sigma_R(pi)|: 4, 16/3, 2048/315
    const double smax = R == 1 ? 4.0 : R == 2 ? 16.0 / 3.0 : 2048.0 / 315.0;
    const double n2 = (double)N * (double)N * dx_scale;
    for (int c = 0; c < m->ncomp; ++c) {
        const double D = st->diffusivity[c];
        if (!(D > 0.0)) return fail(MF_EINVAL, "diffusivity[%d] must be positive", c);
        lam[c] = D * dt * n2;
        if (lam[c] * 3.0 * smax > 2.0 * (1.0 + 1e-12))
            return fail(MF_EUNSTABLE, "lam = %.6g exceeds the forward-Euler limit %.6g", lam[c], 2.0 / (3.0 * smax));
    }
    return 0;
}

// Autotune: time every candidate schedule -- tile shape, and for the TMA kernel rows per
// thread and ring depth -- on the live data (current -> other level, which is scratch at this
// point) and keep the fastest.  Synchronous; runs once per handle.
// ------------------------------------------------------------------ autotuner schedule cache
// The autotuner's choice per level geometry, kind of step and GPU, kept for the process and, when
// the environment variable MF_AUTOTUNE_CACHE names a file, read from and appended to that file
// (one line per choice: the key, then tile[3], rows, ring slots, group bytes, push, and the
// per-class y and z tile extents), so that a level seen before skips the timing runs.
struct TuneChoice {
    int tile[3], rows, ns, gb, push;
    int cty[kTileClasses], ctz[kTileClasses];
};

static std::mutex g_tune_mu;
static std::map<std::string, TuneChoice> g_tune;
static std::string g_tune_loaded;  // the file read into g_tune ("" = none)

static std::string tune_key(const mf_t *m, int R, bool fp64diff, bool fix) {
    unsigned long long h = 1469598103934665603ull;  // FNV-1a over the storage geometry
    auto mix = [&](long long v) {
        for (int i = 0; i < 8; ++i) {
            h ^= (unsigned long long)((v >> (8 * i)) & 0xff);
            h *= 1099511628211ull;
        }
    };
    mix((long long)m->boxes.size());
    for (auto &b : m->boxes)
        for (int d = 0; d < 3; ++d) { mix(b.lo[d]); mix(b.hi[d]); }
    for (int d = 0; d < 3; ++d) { mix(m->domain.lo[d]); mix(m->domain.hi[d]); }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    std::string name = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? prop.name : "gpu";
    for (auto &ch : name)
        if (ch == ' ' || ch == '\t') ch = '_';
    char buf[256];
    snprintf(buf, sizeof buf, "v1:%016llx:d%d:c%d:g%d:R%d:x%d:f%d:k%d:sm%d:%s", h, m->dtype, m->ncomp, m->ngrow, R,
             (int)fp64diff, (int)fix, (int)m->use_tma, sm_count(), name.c_str());
    return buf;
}

static void tune_load_locked() {
    const char *path = getenv("MF_AUTOTUNE_CACHE");
    if (!path || !*path || g_tune_loaded == path) return;
    g_tune_loaded = path;
    FILE *fp = fopen(path, "r");
    if (!fp) return;
    char line[1024];
    while (fgets(line, sizeof line, fp)) {
        char key[512];
        TuneChoice c;
        int n = 0;
        if (sscanf(line, "%511s %d %d %d %d %d %d %d%n", key, &c.tile[0], &c.tile[1], &c.tile[2], &c.rows, &c.ns,
                   &c.gb, &c.push, &n) != 8)
            continue;
        bool ok = true;
        const char *q = line + n;
        for (int k = 0; k < kTileClasses && ok; ++k) {
            int used = 0;
            ok = sscanf(q, "%d %d%n", &c.cty[k], &c.ctz[k], &used) == 2;
            q += used;
        }
        if (ok) g_tune[key] = c;  // later lines win
    }
    fclose(fp);
}

static bool tune_get(const std::string &key, TuneChoice &c) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(key);
    if (it == g_tune.end()) return false;
    c = it->second;
    return true;
}

static void tune_put(const std::string &key, const TuneChoice &c) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    g_tune[key] = c;
    const char *path = getenv("MF_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE *fp = fopen(path, "a");
    if (!fp) return;
    fprintf(fp, "%s %d %d %d %d %d %d %d", key.c_str(), c.tile[0], c.tile[1], c.tile[2], c.rows, c.ns, c.gb, c.push);
    for (int k = 0; k < kTileClasses; ++k) fprintf(fp, " %d %d", c.cty[k], c.ctz[k]);
    fprintf(fp, "\n");
    fclose(fp);
}

extern "C" int mf_autotune_cache_reset(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
    g_tune_loaded.clear();
    return 0;
}

static int autotune(mf_t *m, int R, bool fp64diff, const double *lam, bool fix = false) {
    const std::string key = tune_key(m, R, fp64diff, fix);
    {
        TuneChoice c;
        if (tune_get(key, c)) {
            for (int k = 0; k < kTileClasses; ++k) { m->cty[k] = c.cty[k]; m->ctz[k] = c.ctz[k]; }
            m->tma_rows = c.rows;
            m->tma_ns_pref = c.ns;
            m->tma_gb = c.gb;
            m->tile_auto = false;
            m->push_pref = c.push != 0;
            return set_tiles(m, c.tile);
        }
    }
    for (int k = 0; k < kTileClasses; ++k) m->cty[k] = m->ctz[k] = -1;
    auto tiles = tile_candidates(m);
    struct Cand { std::array<int, 3> t; int rows, ns, gb; };
    std::vector<Cand> cands;
    // fixed point: the timing launches read the FP64 data as if it were fixed point, from cleared
    // grid states (the time does not depend on the values)
    const int fixstep = fix ? 0 : -1;
    if (fix) {
        int rc = enqueue_fix_start(m, m->cur, R, m->stream, false);
        if (rc) return rc;
    }
    for (auto &t : tiles) {
        if (fix && !(m->use_tma && t[0] == 0)) continue;  // the fixed-point path is TMA only
        if (m->use_tma && t[0] == 0) {
            for (int rows = 1; rows <= tma_max_rows(R); ++rows)
                for (int gb : {16, 32})
                    if (fix ? tma_has_group_fix(R, rows, gb) : tma_has_group(m->dtype, R, rows, gb))
                        for (int ns : {4, 8, 16})
                            if (ns >= 2 * R + 1) cands.push_back({t, rows, ns, gb});
        } else {
            cands.push_back({t, 2, 0, 16});
        }
    }
    struct Events {  // destroyed on every return
        cudaEvent_t a = nullptr, b = nullptr;
        ~Events() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev;
    CU(cudaEventCreate(&ev.a));
    CU(cudaEventCreate(&ev.b));
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    // time one candidate: a warm-up launch (also encodes the tensor maps), then n launches,
    // with the ghost push on as in mf_advance (the other level is scratch here)
    auto time_cand = [&](const Cand &c, int n, float *ms) -> int {
        m->tma_rows = c.rows;
        m->tma_ns_pref = c.ns;
        m->tma_gb = c.gb;
        int rc = set_tiles(m, c.t.data());
        if (rc) return rc;
        if (fix) {  // a tile shape the TMA kernel cannot take is no candidate here
            if ((rc = build_tma(m, R, true))) return rc;
            if (!(m->use_tma && m->tma_ok)) {
                if (ms) *ms = 1e30f;
                return 0;
            }
        }
        if ((rc = enqueue_stencil(m, m->cur, R, fp64diff, lam, m->stream, true, StageArgs{}, fixstep))) return rc;
        if (!ms) return 0;
        CU(cudaEventRecord(e0, m->stream));
        for (int i = 0; i < n; ++i)
            if ((rc = enqueue_stencil(m, m->cur, R, fp64diff, lam, m->stream, true, StageArgs{}, fixstep))) return rc;
        CU(cudaEventRecord(e1, m->stream));
        CU(cudaEventSynchronize(e1));
        CU(cudaEventElapsedTime(ms, e0, e1));
        *ms /= (float)n;
        return 0;
    };
    // first pass: every candidate, 3 launches; second: the four fastest, 3 interleaved passes of
    // 6 launches each, keeping each candidate's best pass
    std::vector<std::pair<float, size_t>> r1;
    for (size_t i = 0; i < cands.size(); ++i) {
        float ms = 0;
        int rc = time_cand(cands[i], 3, &ms);
        if (rc) return rc;
        r1.push_back({ms, i});
    }
    std::sort(r1.begin(), r1.end());
    const size_t top = std::min<size_t>(4, r1.size());
    std::vector<float> r2(top, 1e30f);
    for (int pass = 0; pass < 3; ++pass)
        for (size_t j = 0; j < top; ++j) {
            float ms = 0;
            int rc = time_cand(cands[r1[j].second], 6, &ms);
            if (rc) return rc;
            r2[j] = std::min(r2[j], ms);
        }
    Cand bc = cands[r1[std::min_element(r2.begin(), r2.end()) - r2.begin()].second];
    m->tile_auto = false;
    m->push_pref = true;
    int rc = time_cand(bc, 1, nullptr);  // installs the schedule (and builds its lists)
    // Per box-size class (tile_class; Sec. 3.2: tile sizes per loop, here per box size within one
    // launch): other y (and, with a tile z extent, z) extents for the boxes of one class, the
    // other classes as chosen, kept where the level's launch gets faster by more than 2%.
    // Classes holding at least 5% of the cells, largest first, on levels with two or more.
    if (!rc && bc.t[0] == 0 && m->use_tma) {
        double cells[kTileClasses] = {0}, total = 0;
        int ymax[kTileClasses] = {0}, zmax[kTileClasses] = {0};
        for (auto &f : m->fabs) {
            const int k = tile_class(f);
            const double v = (double)f.n[0] * f.n[1] * f.n[2];
            cells[k] += v;
            total += v;
            ymax[k] = std::max(ymax[k], f.n[1]);
            zmax[k] = std::max(zmax[k], f.n[2]);
        }
        int order[kTileClasses], nc = 0;
        for (int k = 0; k < kTileClasses; ++k)
            if (cells[k] > 0) order[nc++] = k;
        std::sort(order, order + nc, [&](int a, int b) { return cells[a] > cells[b]; });
        auto best_of = [&](float *ms) -> int {
            float a = 0, b = 0;
            int r = time_cand(bc, 6, &a);
            if (!r) r = time_cand(bc, 6, &b);
            *ms = std::min(a, b);
            return r;
        };
        float cur = 0;
        if (nc >= 2 && !(rc = best_of(&cur))) {
            for (int oi = 0; oi < nc && !rc; ++oi) {
                const int k = order[oi];
                if (cells[k] < 0.05 * total) continue;
                const int ty0 = m->cty[k], tz0 = m->ctz[k];
                int bty = ty0, btz = tz0;
                float best = cur;
                // the class's candidates (a size at or above the class's largest extent is the
                // whole box), each once, the current shape excluded
                std::vector<std::pair<int, int>> cand;
                for (int ty : {4, 8, 16, 32, 0})
                    for (int tz : {8, 16, 32, 0}) {
                        const int y = ty >= ymax[k] ? 0 : ty;
                        const int z = bc.t[2] > 0 ? (tz >= zmax[k] ? 0 : tz) : -1;
                        const int y0 = ty0 >= 0 ? ty0 : (bc.t[1] >= ymax[k] ? 0 : bc.t[1]);
                        const int z0 = bc.t[2] > 0 ? (tz0 >= 0 ? tz0 : (bc.t[2] >= zmax[k] ? 0 : bc.t[2])) : -1;
                        if ((y == y0 && z == z0) || std::find(cand.begin(), cand.end(), std::make_pair(y, z)) != cand.end())
                            continue;
                        cand.push_back({y, z});
                    }
                for (auto &yz : cand) {
                    m->cty[k] = yz.first;
                    m->ctz[k] = yz.second;
                    float ms = 0;
                    if ((rc = best_of(&ms))) break;
                    if (ms < best * 0.98f) {
                        best = ms;
                        bty = yz.first;
                        btz = yz.second;
                    }
                }
                m->cty[k] = bty;
                m->ctz[k] = btz;
                cur = best;
            }
            if (!rc) rc = time_cand(bc, 1, nullptr);  // installs the per-class shapes
        }
    }
    // with that schedule, one step as the advance runs it: the ghost push and the residual fill,
    // or the face fill and the stencil alone, whichever is faster on this level
    if (!rc && m->use_tma && m->tma_ok && m->tma_push) {
        auto time_mode = [&](bool push, int n, float *ms) -> int {
            for (int i = -1; i < n; ++i) {
                if (i == 0) CU(cudaEventRecord(e0, m->stream));
                int r = 0;
                if (!push) r = enqueue_fill_step(m, m->cur, m->stream);
                else if (!m->fbtasks_res.empty())
                    CU(launch_fill(m->dtype, level_ptrs(m, m->cur), (const FbTask *)m->d_fbtasks_res.p,
                                   (int)m->fbtasks_res.size(), 0, m->stream));
                if (!r) r = enqueue_stencil(m, m->cur, R, fp64diff, lam, m->stream, push, StageArgs{}, fixstep);
                if (r) return r;
            }
            CU(cudaEventRecord(e1, m->stream));
            CU(cudaEventSynchronize(e1));
            CU(cudaEventElapsedTime(ms, e0, e1));
            return 0;
        };
        float tp = 1e30f, tf = 1e30f;
        for (int pass = 0; pass < 3 && !rc; ++pass) {
            float a = 0, b = 0;
            if (!(rc = time_mode(true, 6, &a)) && !(rc = time_mode(false, 6, &b))) {
                tp = std::min(tp, a);
                tf = std::min(tf, b);
            }
        }
        m->push_pref = tp <= tf;
    }
    if (!rc) {
        TuneChoice c;
        for (int d = 0; d < 3; ++d) c.tile[d] = m->tile[d];
        c.rows = bc.rows;
        c.ns = bc.ns;
        c.gb = bc.gb;
        c.push = m->push_pref ? 1 : 0;
        for (int k = 0; k < kTileClasses; ++k) { c.cty[k] = m->cty[k]; c.ctz[k] = m->ctz[k]; }
        tune_put(key, c);
    }
    return rc;
}

extern "C" int mf_set_schedule(mf_t *m, const int in[3]) {
    if (!m || !in) return fail(MF_EINVAL, "null argument");
    const int rows = in[0] ? in[0] : 2, ns = in[1], gb = in[2] ? in[2] : 16;
    if (rows < 1 || rows > 2) return fail(MF_EINVAL, "rows per thread must be 1 or 2");
    if (ns != 0 && (ns < 2 || ns > kMaxStages || (ns & (ns - 1)))) return fail(MF_EINVAL, "ring slots: a power of two <= %d", kMaxStages);
    if (gb != 16 && gb != 32) return fail(MF_EINVAL, "group bytes must be 16 or 32");
    m->tma_rows = rows;
    m->tma_ns_pref = ns;
    m->tma_gb = gb;
    m->tma_R = 0;  // rebuilt (and graphs dropped) at the next launch
    invalidate_graphs(m);
    return 0;
}

extern "C" int mf_get_schedule(const mf_t *m, int out[7]) {
    if (!m || !out) return fail(MF_EINVAL, "null argument");
    for (int d = 0; d < 3; ++d) out[d] = m->tile[d];
    const int R = m->tma_R ? (m->tma_R & 7) : 1;
    out[3] = eff_rows(m, R);
    out[4] = m->tma_ns;
    out[5] = (m->use_tma && m->tma_ok) ? MF_KERNEL_TMA : MF_KERNEL_GLOBAL;
    out[6] = eff_gb(m, R);
    return 0;
}

static std::string graph_key(const char *what, int R, bool fp64diff, const double *lam, int nc, int nsteps, int from) {
    std::string k = what;
    char buf[64];
    snprintf(buf, sizeof buf, "|R%d|d%d|n%d|f%d", R, (int)fp64diff, nsteps, from);
    k += buf;
    for (int c = 0; c < nc; ++c) {
        snprintf(buf, sizeof buf, "|%a", lam[c]);
        k += buf;
    }
    return k;
}

static int capture_begin(mf_t *m) {
    CU(cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal));
    return 0;
}

static int capture_end(mf_t *m, const std::string &key, int body_rc) {
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(m->cap, &graph);
    if (body_rc) { if (graph) cudaGraphDestroy(graph); return body_rc; }
    if (e != cudaSuccess) return fail(MF_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
    auto ge = std::make_unique<GraphExec>();
    e = cudaGraphInstantiate(&ge->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(MF_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    if (m->graphs.size() >= 16) m->graphs.erase(m->graphs.begin());
    m->graphs[key] = std::move(ge);
    return 0;
}

static int ensure_events(mf_t *m, int n) {
    while ((int)m->ev.size() < n) {
        cudaEvent_t e;
        CU(cudaEventCreate(&e));
        m->ev.push_back(e);
    }
    return 0;
}

static int record(mf_t *m, int i) {
    // an external record node: the event is recorded when the graph runs, and can be
    // synchronised on and timed afterwards
    CU(cudaEventRecordWithFlags(m->ev[i], m->cap, cudaEventRecordExternal));
    return 0;
}

// Launch bookkeeping while capturing an advance: counts the kernels of each kind and, when
// timing, records an event wherever the kind of work changes (so back-to-back stencil
// launches run without event nodes between them).
struct PhaseLog {
    mf_t *m;
    bool timing;
    int nev = 0;
    int open = -1;  // kind of the interval since the last event (-1: none yet)
    int launches[4] = {0, 0, 0, 0};
    std::vector<char> kinds;
    int start() {
        if (!timing) return 0;
        kinds.push_back(-1);
        return record(m, nev++);
    }
    // call before enqueueing a kernel of kind k (0 fill, 1 stencil, 2 interp, 3 average-down);
    // real = false: the launcher will find an empty list and launch nothing
    int before(int k, bool real = true) {
        if (!real) return 0;
        ++launches[k];
        const int phase = k < 2 ? k : 2;
        if (!timing || open == phase) { open = phase; return 0; }
        int rc = 0;
        if (open >= 0) {
            kinds.push_back((char)open);
            rc = record(m, nev++);
        }
        open = phase;
        return rc;
    }
    int finish() {
        if (!timing || open < 0) return 0;
        kinds.push_back((char)open);
        return record(m, nev++);
    }
    void store(GraphExec &g) const {
        for (int i = 0; i < 4; ++i) g.launches[i] = launches[i];
        g.nev = timing ? nev : 0;
        g.kinds = kinds;
    }
};

// The state mf_phase_ms and mf_launch_count report, from the graph just launched.
static void note_launch(mf_t *m, const GraphExec &g) {
    for (int i = 0; i < 4; ++i) m->launches[i] = g.launches[i];
    m->ev_used = g.nev;
    m->ev_kinds = g.kinds;
}

extern "C" int mf_launch_count(const mf_t *m, int out[4]) {
    if (!m || !out) return fail(MF_EINVAL, "null argument");
    for (int i = 0; i < 4; ++i) out[i] = m->launches[i];
    return 0;
}

extern "C" int mf_set_timing(mf_t *m, int on) {
    if (!m) return fail(MF_EINVAL, "null handle");
    m->timing = on != 0;
    return 0;
}

extern "C" int mf_phase_ms(mf_t *m, double out[2]) {
    if (!m || !out) return fail(MF_EINVAL, "null argument");
    out[0] = out[1] = 0.0;
    if (m->ev_used < 2) return fail(MF_ESTATE, "no timed advance recorded");
    CU(cudaEventSynchronize(m->ev[m->ev_used - 1]));
    for (int i = 1; i < m->ev_used; ++i) {
        float a = 0;
        CU(cudaEventElapsedTime(&a, m->ev[i - 1], m->ev[i]));
        if (m->ev_kinds[i] == 0) out[0] += a;
        if (m->ev_kinds[i] == 1) out[1] += a;
    }
    return 0;
}

static int advance_plain(mf_t *m, int R, const double *lam, int nsteps) {
    const int nb = (int)m->boxes.size();
    for (int s = 0; s < nsteps; ++s) {
        void *cur = m->level_ptr(m->cur), *nxt = m->level_ptr(1 - m->cur);
        for (int b = 0; b < nb; ++b) {
            const int e0 = m->fb_group[b], cnt = m->fb_group[b + 1] - e0;
            if (cnt == 0) continue;
            long long total = 0;
            for (int e = e0; e < e0 + cnt; ++e)
                total += (long long)m->fb[e].n[0] * m->fb[e].n[1] * m->fb[e].n[2] * m->ncomp;
            CU(launch_fill_plain(m->dtype, cur, (const FabInfo *)m->d_fabs.p, (const FbEntry *)m->d_fb.p + e0, cnt,
                                 total, (const int *)m->d_cbeg.p + e0, m->stream));
        }
        for (int b = 0; b < nb; ++b)
            for (int c = 0; c < m->ncomp; ++c)
                CU(launch_stencil_plain(m->dtype, R, cur, nxt, m->fabs[b], lam[c], c, m->stream));
        m->cur = 1 - m->cur;
    }
    return 0;
}

extern "C" int mf_advance(mf_t *m, const mf_stencil *st, double dt, int nsteps) {
    int rc = need_attached(m);
    if (rc) return rc;
    double lam[kMaxComp];
    if ((rc = check_stencil(m, st, dt, lam, 1.0))) return rc;
    if (nsteps < 0) return fail(MF_EINVAL, "nsteps must be >= 0");
    if (nsteps == 0) return 0;
    const int R = st->kind;
    const bool fp64diff = (st->flags & MF_FP64_DIFF) && m->dtype != F64;
    const bool fixed = (st->flags & MF_FIXED_DIFF) != 0;
    if (st->flags & MF_REFLUX) return fail(MF_EINVAL, "MF_REFLUX applies to mf_amr_advance only");
    if (fixed) {
        if (m->dtype != F64) return fail(MF_EINVAL, "MF_FIXED_DIFF applies to FP64 storage");
        if (st->flags & MF_PLAIN_PER_BOX) return fail(MF_EINVAL, "MF_FIXED_DIFF does not combine with MF_PLAIN_PER_BOX");
        if (!m->use_tma) return fail(MF_EINVAL, "MF_FIXED_DIFF runs on the TMA stencil (MF_KERNEL_TMA)");
    }
    if (st->flags & MF_PLAIN_PER_BOX) {
        if (fp64diff) return fail(MF_EINVAL, "MF_PLAIN_PER_BOX does not combine with MF_FP64_DIFF");
        return advance_plain(m, R, lam, nsteps);
    }
    if (m->tile_auto && (rc = autotune(m, R, fp64diff, lam, fixed))) return rc;
    if (m->use_tma && m->tma_R != tma_key(R, fixed) && (rc = build_tma(m, R, fixed))) return rc;  // never inside a capture
    if (fixed && !m->tma_ok) return fail(MF_EINVAL, "MF_FIXED_DIFF runs on the TMA stencil, which this tile shape excludes");
    char kb[48];
    snprintf(kb, sizeof kb, "%s|g%llu|x%d", m->timing ? "advT" : "adv", m->gen, (int)fixed);
    const std::string key = graph_key(kb, R, fp64diff, lam, m->ncomp, nsteps, m->cur);
    auto it = m->graphs.find(key);
    if (it == m->graphs.end()) {
        // an event wherever the kind of launch changes: at most two per step, the start, and the
        // fixed-point conversions before and after the steps
        if (m->timing && (rc = ensure_events(m, 2 * nsteps + 1 + (fixed ? 2 : 0)))) return rc;
        if ((rc = capture_begin(m))) return rc;
        int body = 0, from = m->cur;
        PhaseLog log{m, m->timing};
        body = log.start();
        // into the fixed-point representation (two passes over the level, counted with the fills)
        if (fixed && !body && !(body = log.before(0))) {
            body = enqueue_fix_start(m, from, R, m->cap);
            if (!body) body = log.before(0);
        }
        const bool push = use_push(m);
        for (int s = 0; s < nsteps && !body; ++s) {
            if (push && s > 0) {
                // the previous stencil launch pushed the face ghosts; fill what is left
                if (!m->fbtasks_res.empty() && !(body = log.before(0)))
                    body = launch_fill(m->dtype, level_ptrs(m, from), (const FbTask *)m->d_fbtasks_res.p,
                                       (int)m->fbtasks_res.size(), 0, m->cap) == cudaSuccess
                               ? 0
                               : fail(MF_ECUDA, "fill launch failed");
            } else if (!(body = log.before(0, fill_step_tasks(m) > 0))) {
                body = enqueue_fill_step(m, from, m->cap);
            }
            if (!body) body = log.before(1);
            if (!body) body = enqueue_stencil(m, from, R, fp64diff, lam, m->cap, push, StageArgs{}, fixed ? s : -1);
            from = 1 - from;
        }
        // back to FP64 (one pass, counted with the fills)
        if (fixed && !body && !(body = log.before(0))) body = enqueue_fix_end(m, from, nsteps, m->cap);
        if (!body) body = log.finish();
        if ((rc = capture_end(m, key, body))) return rc;
        it = m->graphs.find(key);
        log.store(*it->second);
    }
    note_launch(m, *it->second);
    CU(cudaGraphLaunch(it->second->exec, m->stream));
    if (nsteps & 1) m->cur = 1 - m->cur;
    return 0;
}

// ------------------------------------------------------------------ Runge-Kutta (Sec. 4.2)

extern "C" size_t mf_stage_bytes(const mf_t *m) { return m ? m->level_elems * m->esize : 0; }

extern "C" int mf_attach_stage(mf_t *m, void *dev_ptr, size_t bytes) {
    int rc = need_attached(m);
    if (rc) return rc;
    if (!dev_ptr || ((uintptr_t)dev_ptr & 255)) return fail(MF_EALIGN, "stage pointer must be 256-byte aligned");
    if (bytes < mf_stage_bytes(m)) return fail(MF_EALIGN, "stage buffer of %zu bytes, need %zu", bytes, mf_stage_bytes(m));
    m->stage = (char *)dev_ptr;
    m->tma_R = 0;  // the tensor maps of the stage level are encoded at the next launch
    invalidate_graphs(m);
    return 0;
}

// Stage weights of the three-stage SSP Runge-Kutta scheme (the reading of Sec. 4.2's third-order
// Runge-Kutta integration): stage k writes W[k][0] * u + W[k][1] * E(v_k), u the state at the
// start of the step, E one forward-Euler flux-form step.
static const double kRk3[3][2] = {{0.0, 1.0}, {0.75, 0.25}, {1.0 / 3.0, 2.0 / 3.0}};

extern "C" int mf_rk3_advance(mf_t *m, const mf_stencil *st, double dt, int nsteps) {
    int rc = need_attached(m);
    if (rc) return rc;
    if (!m->stage) return fail(MF_ESTATE, "no stage level attached (mf_attach_stage)");
    double lam[kMaxComp];
    if ((rc = check_stencil(m, st, dt, lam, 1.0))) return rc;
    if (nsteps < 0) return fail(MF_EINVAL, "nsteps must be >= 0");
    if (st->flags & (MF_PLAIN_PER_BOX | MF_REFLUX | MF_FIXED_DIFF))
        return fail(MF_EINVAL, "MF_PLAIN_PER_BOX, MF_REFLUX and MF_FIXED_DIFF do not apply to mf_rk3_advance");
    if (nsteps == 0) return 0;
    const int R = st->kind;
    const bool fp64diff = (st->flags & MF_FP64_DIFF) && m->dtype != F64;
    if (m->tile_auto && (rc = autotune(m, R, fp64diff, lam))) return rc;
    if (m->use_tma && m->tma_R != tma_key(R, false) && (rc = build_tma(m, R))) return rc;  // never inside a capture
    char kb[48];
    snprintf(kb, sizeof kb, "%s|g%llu", m->timing ? "rk3T" : "rk3", m->gen);
    const std::string key = graph_key(kb, R, fp64diff, lam, m->ncomp, nsteps, m->cur);
    auto it = m->graphs.find(key);
    if (it == m->graphs.end()) {
        if (m->timing && (rc = ensure_events(m, 6 * nsteps + 1))) return rc;
        if ((rc = capture_begin(m))) return rc;
        int body = 0, a = m->cur;
        PhaseLog log{m, m->timing};
        body = log.start();
        const bool push = use_push(m);
        // pushed[l]: the launch that last wrote level l also wrote its face ghosts
        bool pushed[3] = {false, false, false};
        for (int step = 0; step < nsteps && !body; ++step) {
            const int b = 1 - a;
            const int in[3] = {a, b, 2}, out[3] = {b, 2, b};  // u -> u1 (b) -> u2 (stage) -> new u (b)
            for (int k = 0; k < 3 && !body; ++k) {
                const int v = in[k];
                if (pushed[v]) {
                    if (!m->fbtasks_res.empty() && !(body = log.before(0)))
                        body = launch_fill(m->dtype, level_ptrs(m, v), (const FbTask *)m->d_fbtasks_res.p,
                                           (int)m->fbtasks_res.size(), 0, m->cap) == cudaSuccess
                                   ? 0
                                   : fail(MF_ECUDA, "fill launch failed");
                } else if (!(body = log.before(0, fill_step_tasks(m) > 0))) {
                    body = enqueue_fill_step(m, v, m->cap);
                }
                StageArgs sa;
                sa.to = out[k];
                if (k > 0) {
                    sa.u0 = a;
                    sa.rk_a = kRk3[k][0];
                    sa.rk_b = kRk3[k][1];
                }
                if (!body) body = log.before(1);
                if (!body) body = enqueue_stencil(m, v, R, fp64diff, lam, m->cap, push, sa);
                pushed[out[k]] = push;
            }
            a = b;
        }
        if (!body) body = log.finish();
        if ((rc = capture_end(m, key, body))) return rc;
        it = m->graphs.find(key);
        log.store(*it->second);
    }
    note_launch(m, *it->second);
    CU(cudaGraphLaunch(it->second->exec, m->stream));
    if (nsteps & 1) m->cur = 1 - m->cur;
    return 0;
}

// ------------------------------------------------------------------ reduction

extern "C" int mf_reduce(mf_t *m, int comp, int op, double *out) {
    int rc = need_attached(m);
    if (rc) return rc;
    if (comp < 0 || comp >= m->ncomp || !out) return fail(MF_EINVAL, "bad component or null out");
    if (op < MF_RED_SUM || op > MF_RED_NORM2) return fail(MF_EINVAL, "unknown reduction %d", op);
    const int grid = 304;  // fixed: the reduction tree, hence the bits, do not depend on the GPU
    CU(launch_reduce(m->dtype, op, m->level_ptr(m->cur), (const FabInfo *)m->d_fabs.p,
                     (const long long *)m->d_rowpre.p, (int)m->fabs.size(), comp, (double2 *)m->d_partials.p, grid,
                     (double *)m->d_sumout.p, m->stream));
    CU(cudaMemcpyAsync(m->h_sum, m->d_sumout.p, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    if ((rc = check_device_error(m))) return rc;
    *out = *m->h_sum;
    return 0;
}

extern "C" int mf_sum(mf_t *m, int comp, double *out) { return mf_reduce(m, comp, MF_RED_SUM, out); }

// ------------------------------------------------------------------ AMR

static int wrap_idx(int i, int lo, int len) {
    int r = (i - lo) % len;
    if (r < 0) r += len;
    return lo + r;
}

// The coarse-fine interface of a refined level: for every face of every fine box, each group of
// r x r fine faces whose outside coarse cell (periodic) lies in no fine box is one coarse face.
// Fine boxes must consist of whole coarse cells, and the coarse level must cover its domain.
static int build_reflux(const mf_t *fine, const mf_t *crse, int r, RefluxPlan &plan) {
    const Box &fd = fine->domain, &cd = crse->domain;
    int Lc[3];
    for (int d = 0; d < 3; ++d) {
        Lc[d] = cd.len(d);
        if (fd.lo[d] != r * cd.lo[d] || fd.len(d) != r * Lc[d]) return fail(MF_EINVAL, "fine domain is not the refined coarse domain");
    }
    std::vector<unsigned char> cov((size_t)Lc[0] * Lc[1] * Lc[2], 0);  // coarse cells under fine boxes
    for (auto &b : fine->boxes) {
        for (int d = 0; d < 3; ++d)
            if ((b.lo[d] - fd.lo[d]) % r || (b.hi[d] + 1 - fd.lo[d]) % r)
                return fail(MF_EINVAL, "refluxing needs fine boxes made of whole coarse cells");
        for (int z = floor_div(b.lo[2], r); z <= floor_div(b.hi[2], r); ++z)
            for (int y = floor_div(b.lo[1], r); y <= floor_div(b.hi[1], r); ++y)
                for (int x = floor_div(b.lo[0], r); x <= floor_div(b.hi[0], r); ++x)
                    cov[((size_t)(z - cd.lo[2]) * Lc[1] + (y - cd.lo[1])) * Lc[0] + (x - cd.lo[0])] = 1;
    }
    BinHash hash;
    hash.build(cd, crse->boxes);
    std::vector<int> cand, stamp(crse->boxes.size(), -1);
    int tag = 0;
    struct Tmp { long long c_elem; CFace f; };
    std::vector<Tmp> tmp;
    plan.ff.clear();
    for (size_t bf = 0; bf < fine->boxes.size(); ++bf) {
        const Box &B = fine->boxes[bf];
        const FabInfo &Ff = fine->fabs[bf];
        for (int d = 0; d < 3; ++d) {
            const int e0 = d == 0 ? 1 : 0, e1 = d == 2 ? 1 : 2;
            const long long fds = d == 0 ? 1 : d == 1 ? (long long)Ff.px : Ff.plane;
            for (int s = -1; s <= 1; s += 2) {
                const int in = s > 0 ? B.hi[d] : B.lo[d];
                const int outc = wrap_idx(((in + s) - fd.lo[d] + fd.len(d)) % fd.len(d) / r + cd.lo[d], cd.lo[d], Lc[d]);
                for (int b1 = B.lo[e1]; b1 <= B.hi[e1]; b1 += r)
                    for (int a0 = B.lo[e0]; a0 <= B.hi[e0]; a0 += r) {
                        int C[3];
                        C[d] = outc;
                        C[e0] = wrap_idx(floor_div(a0, r), cd.lo[e0], Lc[e0]);
                        C[e1] = wrap_idx(floor_div(b1, r), cd.lo[e1], Lc[e1]);
                        if (cov[((size_t)(C[2] - cd.lo[2]) * Lc[1] + (C[1] - cd.lo[1])) * Lc[0] + (C[0] - cd.lo[0])])
                            continue;  // the outside is another fine box
                        Box q;
                        for (int k = 0; k < 3; ++k) q.lo[k] = q.hi[k] = C[k];
                        hash.query(q, cand, stamp, ++tag);
                        int owner = -1;
                        for (int a : cand)
                            if (!intersect(crse->boxes[a], q).empty()) { owner = a; break; }
                        if (owner < 0) return fail(MF_EINVAL, "coarse level does not cover its domain");
                        const FabInfo &Fc = crse->fabs[owner];
                        Tmp t;
                        t.c_elem = elem_at(Fc, C[0], C[1], C[2]);
                        int Lw[3] = {C[0], C[1], C[2]};
                        if (-s < 0) Lw[d] -= 1;  // fine region on C's low side: the face's lower cell is C - e_d
                        t.f.c_low = elem_at(Fc, Lw[0], Lw[1], Lw[2]);
                        t.f.cstride = Fc.cstride;
                        t.f.dstride = d == 0 ? 1 : d == 1 ? (long long)Fc.px : Fc.plane;
                        t.f.sc = -s;
                        t.f.ffirst = (int)plan.ff.size();
                        for (int j1 = 0; j1 < r; ++j1)
                            for (int j0 = 0; j0 < r; ++j0) {
                                int P[3];
                                P[d] = s > 0 ? in : in - 1;  // lower cell of the fine face
                                P[e0] = a0 + j0;
                                P[e1] = b1 + j1;
                                FFace g;
                                g.f_low = elem_at(Ff, P[0], P[1], P[2]);
                                g.cstride = Ff.cstride;
                                g.dstride = fds;
                                plan.ff.push_back(g);
                            }
                        tmp.push_back(t);
                    }
            }
        }
    }
    // group the faces by coarse cell (fixed order: cell, then the order found)
    std::stable_sort(tmp.begin(), tmp.end(), [](const Tmp &a, const Tmp &b) { return a.c_elem < b.c_elem; });
    plan.faces.clear();
    plan.cells.clear();
    for (size_t i = 0; i < tmp.size(); ++i) {
        if (i == 0 || tmp[i].c_elem != tmp[i - 1].c_elem) {
            CCell c;
            c.c_elem = tmp[i].c_elem;
            c.cstride = tmp[i].f.cstride;
            c.efirst = (int)plan.faces.size();
            c.ecount = 0;
            plan.cells.push_back(c);
        }
        plan.faces.push_back(tmp[i].f);
        plan.cells.back().ecount++;
    }
    return 0;
}

static RefluxPlan *get_reflux(mf_t *fine, const mf_t *crse, int ratio, int *rc) {
    for (auto &p : fine->reflux)
        if (p->crse == crse && p->ratio == ratio) { *rc = 0; return p.get(); }
    auto p = std::make_unique<RefluxPlan>();
    p->crse = crse;
    p->ratio = ratio;
    if ((*rc = build_reflux(fine, crse, ratio, *p))) return nullptr;
    const size_t nreg = std::max<size_t>(1, p->faces.size() * (size_t)fine->ncomp) * sizeof(double);
    if ((*rc = p->d_faces.upload(p->faces, fine->stream))) return nullptr;
    if ((*rc = p->d_ff.upload(p->ff, fine->stream))) return nullptr;
    if ((*rc = p->d_cells.upload(p->cells, fine->stream))) return nullptr;
    if ((*rc = p->d_regc.ensure(nreg))) return nullptr;
    if ((*rc = p->d_regf.ensure(nreg))) return nullptr;
    if (cudaStreamSynchronize(fine->stream) != cudaSuccess) { *rc = fail(MF_ECUDA, "sync"); return nullptr; }
    fine->reflux.push_back(std::move(p));
    return fine->reflux.back().get();
}

static int build_interp(mf_t *fine, const mf_t *crse, int ratio, InterpPlan &plan) {
    for (int d = 0; d < 3; ++d)
        if (fine->domain.lo[d] != crse->domain.lo[d] * ratio || fine->domain.len(d) != crse->domain.len(d) * ratio)
            return fail(MF_EINVAL, "fine domain must be the coarse domain refined by %d", ratio);
    if (crse->ngrow < 1) return fail(MF_EINVAL, "coarse level needs ngrow >= 1");
    if (crse->ncomp != fine->ncomp || crse->dtype != fine->dtype)
        return fail(MF_EINVAL, "levels differ in ncomp or dtype");
    const int g = fine->ngrow;
    BinHash chash;
    chash.build(crse->domain, crse->boxes);
    std::vector<int> cand, stamp(crse->boxes.size(), -1);
    int tag = 0;
    auto crse_owner = [&](int i, int j, int k) -> int {
        Box q{{i, j, k}, {i, j, k}};
        chash.query(q, cand, stamp, ++tag);
        for (int a : cand) if (crse->boxes[a].contains(i, j, k)) return a;
        return -1;
    };
    plan.runs.clear();
    plan.cells.start.assign(1, 0);
    long long ncells = 0;
    for (int b = 0; b < (int)fine->boxes.size(); ++b) {
        const Box &B = fine->boxes[b];
        const Box gb = grow(B, g);
        const long long nx = gb.len(0), ny = gb.len(1), nz = gb.len(2);
        // todo: ghost cells that neither the box nor a fine-fine fill covers, not yet in a run
        std::vector<char> todo((size_t)(nx * ny * nz), 1);
        auto at = [&](int i, int j, int k) -> char & {
            return todo[(size_t)(((k - gb.lo[2]) * ny + (j - gb.lo[1])) * nx + (i - gb.lo[0]))];
        };
        for (int k = B.lo[2]; k <= B.hi[2]; ++k)
            for (int j = B.lo[1]; j <= B.hi[1]; ++j)
                for (int i = B.lo[0]; i <= B.hi[0]; ++i) at(i, j, k) = 0;
        const FabInfo &ff = fine->fabs[b];
        for (int e = fine->fb_group[b]; e < fine->fb_group[b + 1]; ++e) {
            const FbEntry &en = fine->fb[e];
            const int *c = fine->fb_corner[e].data();
            for (int z = 0; z < en.n[2]; ++z)
                for (int y = 0; y < en.n[1]; ++y)
                    for (int x = 0; x < en.n[0]; ++x) at(c[0] + x, c[1] + y, c[2] + z) = 0;
        }
        for (int k = gb.lo[2]; k <= gb.hi[2]; ++k)
            for (int j = gb.lo[1]; j <= gb.hi[1]; ++j)
                for (int i = gb.lo[0]; i <= gb.hi[0]; ++i) {
                    if (!at(i, j, k)) continue;
                    // a run along the direction the ghost slab extends in: x where the cell lies
                    // within the box's x range, else y, else z (corner cells: x)
                    const int p0[3] = {i, j, k};
                    bool in[3];
                    for (int d = 0; d < 3; ++d) in[d] = B.lo[d] <= p0[d] && p0[d] <= B.hi[d];
                    const int axis = in[0] ? 0 : in[1] ? 1 : in[2] ? 2 : 0;
                    // coarse owner and periodic shift of the cell floor(i/r)
                    int kc[3], wc[3];
                    for (int d = 0; d < 3; ++d) {
                        kc[d] = floor_div(p0[d], ratio);
                        wc[d] = wrap_idx(kc[d], crse->domain.lo[d], crse->domain.len(d));
                    }
                    const int a = crse_owner(wc[0], wc[1], wc[2]);
                    if (a < 0) return fail(MF_EINVAL, "coarse level does not cover its domain");
                    const FabInfo &cf = crse->fabs[a];
                    InterpRun run{};
                    run.I = i; run.J = j; run.K = k;
                    run.axis = axis;
                    run.fdst = elem_at(ff, i, j, k);
                    run.fstep = axis == 0 ? 1 : axis == 1 ? ff.px : (int)ff.plane;
                    run.fcs = (int)ff.cstride;
                    run.ccs = (int)cf.cstride;
                    run.cpx = cf.px;
                    run.cplane = (int)cf.plane;
                    run.cbase = cf.org - (long long)(kc[2] - wc[2] + cf.lo[2]) * cf.plane -
                                (long long)(kc[1] - wc[1] + cf.lo[1]) * cf.px - (kc[0] - wc[0] + cf.lo[0]);
                    int p[3] = {i, j, k}, len = 0;
                    while (p[axis] <= gb.hi[axis] && at(p[0], p[1], p[2])) {
                        const int kq = floor_div(p[axis], ratio);
                        const int wq = wrap_idx(kq, crse->domain.lo[axis], crse->domain.len(axis));
                        int w3[3] = {wc[0], wc[1], wc[2]};
                        w3[axis] = wq;
                        if (kq - wq != kc[axis] - wc[axis] || !crse->boxes[a].contains(w3[0], w3[1], w3[2])) break;
                        at(p[0], p[1], p[2]) = 0;
                        ++len;
                        ++p[axis];
                    }
                    ncells += len;
                    if (ncells > INT32_MAX - 64) return fail(MF_EINVAL, "too many ghost cells to interpolate");
                    plan.runs.push_back(run);
                    plan.cells.start.push_back((int)ncells);
                }
    }
    plan.cells.finish();
    return 0;
}

static InterpPlan *get_interp(mf_t *fine, const mf_t *crse, int ratio, int *rc) {
    for (auto &p : fine->interp)
        if (p->crse == crse && p->ratio == ratio) { *rc = 0; return p.get(); }
    auto p = std::make_unique<InterpPlan>();
    p->crse = crse;
    p->ratio = ratio;
    if ((*rc = build_interp(fine, crse, ratio, *p))) return nullptr;
    if ((*rc = p->d_runs.upload(p->runs, fine->stream))) return nullptr;
    if ((*rc = p->cells.upload(fine->stream))) return nullptr;
    if (cudaStreamSynchronize(fine->stream) != cudaSuccess) { *rc = fail(MF_ECUDA, "sync"); return nullptr; }
    fine->interp.push_back(std::move(p));
    return fine->interp.back().get();
}

static int build_avg(const mf_t *fine, mf_t *crse, int ratio, AvgPlan &plan) {
    for (int d = 0; d < 3; ++d)
        if (fine->domain.lo[d] != crse->domain.lo[d] * ratio || fine->domain.len(d) != crse->domain.len(d) * ratio)
            return fail(MF_EINVAL, "fine domain must be the coarse domain refined by %d", ratio);
    if (crse->ncomp != fine->ncomp || crse->dtype != fine->dtype)
        return fail(MF_EINVAL, "levels differ in ncomp or dtype");
    BinHash chash;
    chash.build(crse->domain, crse->boxes);
    std::vector<int> cand, stamp(crse->boxes.size(), -1);
    int tag = 0;
    plan.regs.clear();
    plan.cells.start.assign(1, 0);
    plan.vec = true;
    long long ncells = 0;
    for (int f = 0; f < (int)fine->boxes.size(); ++f) {
        const Box &B = fine->boxes[f];
        for (int d = 0; d < 3; ++d)
            if (B.lo[d] % ratio != 0 || (B.hi[d] + 1) % ratio != 0)
                return fail(MF_EINVAL, "fine box %d not aligned to the refinement ratio", f);
        const Box cb = coarsen(B, ratio);
        chash.query(cb, cand, stamp, ++tag);
        std::sort(cand.begin(), cand.end());
        for (int a : cand) {
            const Box r = intersect(cb, crse->boxes[a]);
            if (r.empty()) continue;
            const FabInfo &ff = fine->fabs[f], &cf = crse->fabs[a];
            AvgRegion g{};
            g.fsrc = elem_at(ff, r.lo[0] * ratio, r.lo[1] * ratio, r.lo[2] * ratio);
            g.cdst = elem_at(cf, r.lo[0], r.lo[1], r.lo[2]);
            g.fpx = ff.px;
            g.fplane = (int)ff.plane;
            g.fcs = (int)ff.cstride;
            g.cpx = cf.px;
            g.cplane = (int)cf.plane;
            g.ccs = (int)cf.cstride;
            for (int d = 0; d < 3; ++d) g.n[d] = r.len(d);
            if (g.fsrc % ratio || g.fpx % ratio || g.fplane % ratio || g.fcs % ratio) plan.vec = false;
            ncells += (long long)g.n[0] * g.n[1] * g.n[2];
            if (ncells > INT32_MAX - 64) return fail(MF_EINVAL, "too many coarse cells to average down");
            plan.regs.push_back(g);
            plan.cells.start.push_back((int)ncells);
        }
    }
    // the level allocation is 256-byte aligned: offsets that are multiples of ratio elements
    // give vector loads aligned to their size
    plan.cells.finish();
    return 0;
}

static AvgPlan *get_avg(const mf_t *fine, mf_t *crse, int ratio, int *rc) {
    for (auto &p : crse->avg)
        if (p->fine == fine && p->ratio == ratio) { *rc = 0; return p.get(); }
    auto p = std::make_unique<AvgPlan>();
    p->fine = fine;
    p->ratio = ratio;
    if ((*rc = build_avg(fine, crse, ratio, *p))) return nullptr;
    if ((*rc = p->d_regs.upload(p->regs, crse->stream))) return nullptr;
    if ((*rc = p->cells.upload(crse->stream))) return nullptr;
    if (cudaStreamSynchronize(crse->stream) != cudaSuccess) { *rc = fail(MF_ECUDA, "sync"); return nullptr; }
    crse->avg.push_back(std::move(p));
    return crse->avg.back().get();
}

// Bounding box, per FillBoundary region of m, of the destination cells whose element offset
// (component 0) is marked in bits.
static void mark_parts(const mf_t *m, const std::vector<uint64_t> &bits, std::vector<std::array<int, 6>> &out) {
    out.assign(m->fb.size(), std::array<int, 6>{0, 0, 0, 0, 0, 0});
    for (size_t e = 0; e < m->fb.size(); ++e) {
        const FbEntry &en = m->fb[e];
        const FabInfo &df = m->fabs[en.dfab];
        int lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {-1, -1, -1};
        for (int z = 0; z < en.n[2]; ++z)
            for (int y = 0; y < en.n[1]; ++y)
                for (int x = 0; x < en.n[0]; ++x) {
                    const long long el = en.dst + z * df.plane + (long long)y * df.px + x;
                    if (!((bits[(size_t)el >> 6] >> (el & 63)) & 1)) continue;
                    const int p[3] = {x, y, z};
                    for (int d = 0; d < 3; ++d) { lo[d] = std::min(lo[d], p[d]); hi[d] = std::max(hi[d], p[d]); }
                }
        if (hi[0] >= 0) out[e] = {lo[0], lo[1], lo[2], hi[0] - lo[0] + 1, hi[1] - lo[1] + 1, hi[2] - lo[2] + 1};
    }
}

static void append_parts(const mf_t *m, const std::vector<std::array<int, 6>> &parts, std::vector<FbTask> &out) {
    for (size_t e = 0; e < parts.size(); ++e)
        if (parts[e][3] > 0) append_fill_tasks(m, clip_entry(m, (int)e, parts[e].data(), parts[e].data() + 3), out);
}

static AmrFill *get_amr_fill(mf_t *crse, const mf_t *fine, int ratio, int R, const InterpPlan *ip,
                             const RefluxPlan *rp, int *rc) {
    AmrFill *af = nullptr;
    for (auto &p : crse->amrfill)
        if (p->fine == fine && p->ratio == ratio && p->R == R && p->reflux == (rp != nullptr)) af = p.get();
    if (!af) {
        auto p = std::make_unique<AmrFill>();
        p->fine = fine;
        p->ratio = ratio;
        p->R = R;
        p->reflux = rp != nullptr;
        // cells the interpolation reads: the 8 coarse points of every interpolated fine cell
        std::vector<uint64_t> bits((crse->level_elems + 63) / 64, 0);
        auto set = [&](long long el) { bits[(size_t)el >> 6] |= 1ull << (el & 63); };
        for (size_t q = 0; q < ip->runs.size(); ++q) {
            const InterpRun &run = ip->runs[q];
            for (int t = 0; t < ip->cells.start[q + 1] - ip->cells.start[q]; ++t) {
                int ix[3] = {run.I, run.J, run.K};
                ix[run.axis] += t;
                int k[3];
                for (int d = 0; d < 3; ++d) k[d] = floor_div(2 * ix[d] + 1 - ratio, 2 * ratio);
                const long long cb = run.cbase + (long long)k[2] * run.cplane + (long long)k[1] * run.cpx + k[0];
                for (int dz = 0; dz < 2; ++dz)
                    for (int dy = 0; dy < 2; ++dy)
                        for (int dx = 0; dx < 2; ++dx) set(cb + (long long)dz * run.cplane + dy * run.cpx + dx);
            }
        }
        mark_parts(crse, bits, p->ip);
        // ... and the cells of the coarse flux lines across the coarse-fine faces
        if (rp)
            for (const CFace &f : rp->faces)
                for (int k = -R + 1; k <= R; ++k) set(f.c_low + k * f.dstride);
        mark_parts(crse, bits, p->cf);
        // face regions whose source lies within one cell (26 directions, periodic) of a covered cell
        const Box &cd = crse->domain;
        const int L[3] = {cd.len(0), cd.len(1), cd.len(2)};
        std::vector<unsigned char> cov((size_t)L[0] * L[1] * L[2], 0), tmp;
        auto at = [&](int x, int y, int z) { return ((size_t)z * L[1] + y) * L[0] + x; };
        for (const Box &b : fine->boxes)
            for (int z = floor_div(b.lo[2], ratio); z <= floor_div(b.hi[2], ratio); ++z)
                for (int y = floor_div(b.lo[1], ratio); y <= floor_div(b.hi[1], ratio); ++y)
                    for (int x = floor_div(b.lo[0], ratio); x <= floor_div(b.hi[0], ratio); ++x)
                        cov[at(wrap_idx(x, cd.lo[0], L[0]) - cd.lo[0], wrap_idx(y, cd.lo[1], L[1]) - cd.lo[1],
                               wrap_idx(z, cd.lo[2], L[2]) - cd.lo[2])] = 1;
        for (int d = 0; d < 3; ++d) {  // dilate by one cell along each direction in turn
            tmp = cov;
            for (int z = 0; z < L[2]; ++z)
                for (int y = 0; y < L[1]; ++y)
                    for (int x = 0; x < L[0]; ++x) {
                        int p[3] = {x, y, z};
                        if (tmp[at(x, y, z)]) continue;
                        for (int sgn = -1; sgn <= 1; sgn += 2) {
                            int q[3] = {p[0], p[1], p[2]};
                            q[d] = (q[d] + sgn + L[d]) % L[d];
                            if (tmp[at(q[0], q[1], q[2])]) { cov[at(x, y, z)] = 1; break; }
                        }
                    }
        }
        p->stale.assign(crse->fb.size(), std::array<int, 6>{0, 0, 0, 0, 0, 0});
        for (size_t e = 0; e < crse->fb.size(); ++e) {
            const int kind = crse->fb_kind[e];
            if (kind < 2 || kind > 5) continue;  // the push writes the y and z face regions
            const FbEntry &en = crse->fb[e];
            const auto &cr = crse->fb_corner[e];
            int lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {-1, -1, -1};
            for (int z = 0; z < en.n[2]; ++z)
                for (int y = 0; y < en.n[1]; ++y)
                    for (int x = 0; x < en.n[0]; ++x) {
                        if (!cov[at(cr[3] + x - cd.lo[0], cr[4] + y - cd.lo[1], cr[5] + z - cd.lo[2])]) continue;
                        const int pp[3] = {x, y, z};
                        for (int d = 0; d < 3; ++d) { lo[d] = std::min(lo[d], pp[d]); hi[d] = std::max(hi[d], pp[d]); }
                    }
            if (hi[0] >= 0) p->stale[e] = {lo[0], lo[1], lo[2], hi[0] - lo[0] + 1, hi[1] - lo[1] + 1, hi[2] - lo[2] + 1};
        }
        crse->amrfill.push_back(std::move(p));
        af = crse->amrfill.back().get();
    }
    if (af->gen != crse->gen) {
        // first step: the step's face fill and the read cells; later steps with the ghost push:
        // the residual fill, the stale faces and the read cells; after the coarse stencil: the
        // cells the interpolation reads from the new coarse data
        const bool strips = crse->use_tma && crse->tma_ok && crse->tma_strips;
        const bool push = strips && use_push(crse);
        af->t_first = strips ? crse->fbtasks_adv : crse->fbtasks;
        if (strips) append_parts(crse, af->cf, af->t_first);
        af->t_next.clear();
        if (push) {
            af->t_next = crse->fbtasks_res;
            append_parts(crse, af->stale, af->t_next);
            append_parts(crse, af->cf, af->t_next);
        }
        af->t_post.clear();
        append_parts(crse, af->ip, af->t_post);
        if ((*rc = af->d_first.upload(af->t_first, crse->stream))) return nullptr;
        if ((*rc = af->d_next.upload(af->t_next, crse->stream))) return nullptr;
        if ((*rc = af->d_post.upload(af->t_post, crse->stream))) return nullptr;
        if (cudaStreamSynchronize(crse->stream) != cudaSuccess) { *rc = fail(MF_ECUDA, "sync"); return nullptr; }
        af->gen = crse->gen;
    }
    *rc = 0;
    return af;
}

static int enqueue_interp(mf_t *fine, int fwhich, const mf_t *cold, int cold_which, const mf_t *cnew, int cnew_which,
                          InterpPlan *plan, int ratio, double alpha, cudaStream_t s) {
    CU(launch_interp(fine->dtype, fine->level_ptr(fwhich), cold->level_ptr(cold_which), cnew->level_ptr(cnew_which),
                     (const InterpRun *)plan->d_runs.p, (const int *)plan->cells.d_start.p,
                     (const int *)plan->cells.d_wfirst.p, (int)plan->runs.size(), plan->cells.ncells, fine->ncomp,
                     ratio, alpha, s));
    return 0;
}

static int enqueue_avg(const mf_t *fine, int fwhich, mf_t *crse, int cwhich, AvgPlan *plan, int ratio,
                       cudaStream_t s) {
    CU(launch_avgdown(fine->dtype, fine->level_ptr(fwhich), crse->level_ptr(cwhich), (const AvgRegion *)plan->d_regs.p,
                      (const int *)plan->cells.d_start.p, (const int *)plan->cells.d_wfirst.p, (int)plan->regs.size(),
                      plan->cells.ncells, fine->ncomp, ratio, plan->vec, s));
    return 0;
}

extern "C" int mf_interp_cf(mf_t *fine, const mf_t *crse_old, const mf_t *crse_new, double alpha, int ratio) {
    int rc = need_attached(fine);
    if (rc) return rc;
    if ((rc = need_attached(crse_old)) || (rc = need_attached(crse_new))) return rc;
    if (ratio != 2 && ratio != 4) return fail(MF_EINVAL, "ratio must be 2 or 4");
    if (crse_old->boxes.size() != crse_new->boxes.size() || crse_old->level_elems != crse_new->level_elems)
        return fail(MF_EINVAL, "coarse handles must share one layout");
    InterpPlan *plan = get_interp(fine, crse_old, ratio, &rc);
    if (!plan) return rc;
    return enqueue_interp(fine, fine->cur, crse_old, crse_old->cur, crse_new, crse_new->cur, plan, ratio, alpha,
                          fine->stream);
}

extern "C" long long mf_interp_cells(const mf_t *fine, const mf_t *crse, int ratio, long long *runs_out) {
    if (!fine || !crse) return fail(MF_EINVAL, "null handle");
    if (ratio != 2 && ratio != 4) return fail(MF_EINVAL, "ratio must be 2 or 4");
    InterpPlan plan;  // host lists only: no device memory, no attach needed
    int rc = build_interp(const_cast<mf_t *>(fine), crse, ratio, plan);
    if (rc) return rc;
    if (runs_out) *runs_out = (long long)plan.runs.size();
    return plan.cells.ncells;
}

extern "C" long long mf_reflux_faces(const mf_t *fine, const mf_t *crse, int ratio, long long *cells_out) {
    if (!fine || !crse) return fail(MF_EINVAL, "null handle");
    if (ratio != 2 && ratio != 4) return fail(MF_EINVAL, "ratio must be 2 or 4");
    RefluxPlan plan;  // host lists only
    int rc = build_reflux(fine, crse, ratio, plan);
    if (rc) return rc;
    if (cells_out) *cells_out = (long long)plan.cells.size();
    return (long long)plan.faces.size();
}

extern "C" long long mf_avgdown_cells(const mf_t *fine, const mf_t *crse, int ratio, long long *regions_out) {
    if (!fine || !crse) return fail(MF_EINVAL, "null handle");
    if (ratio != 2 && ratio != 4) return fail(MF_EINVAL, "ratio must be 2 or 4");
    AvgPlan plan;  // host lists only
    int rc = build_avg(fine, const_cast<mf_t *>(crse), ratio, plan);
    if (rc) return rc;
    if (regions_out) *regions_out = (long long)plan.regs.size();
    return plan.cells.ncells;
}

extern "C" int mf_average_down(const mf_t *fine, mf_t *crse, int ratio) {
    int rc = need_attached(crse);
    if (rc) return rc;
    if ((rc = need_attached(fine))) return rc;
    if (ratio != 2 && ratio != 4) return fail(MF_EINVAL, "ratio must be 2 or 4");
    AvgPlan *plan = get_avg(fine, crse, ratio, &rc);
    if (!plan) return rc;
    return enqueue_avg(fine, fine->cur, crse, crse->cur, plan, ratio, crse->stream);
}

extern "C" int mf_amr_advance(mf_t *crse, mf_t *fine, const mf_stencil *st, double dt_crse, int ncrse_steps, int nsub,
                              int ratio) {
    int rc = need_attached(crse);
    if (rc) return rc;
    if ((rc = need_attached(fine))) return rc;
    if (ratio != 2 && ratio != 4) return fail(MF_EINVAL, "ratio must be 2 or 4");
    if (nsub < 1) return fail(MF_EINVAL, "nsub must be >= 1");
    if (ncrse_steps < 0) return fail(MF_EINVAL, "ncrse_steps must be >= 0");
    if (st && (st->flags & (MF_PLAIN_PER_BOX | MF_FIXED_DIFF)))
        return fail(MF_EINVAL, "MF_PLAIN_PER_BOX and MF_FIXED_DIFF are single-level only");
    double lam_c[kMaxComp], lam_f[kMaxComp];
    if ((rc = check_stencil(crse, st, dt_crse, lam_c, 1.0))) return rc;
    // fine: dx_f = dx_c / ratio, dt_f = dt_c / nsub; lam_f = D dt_f / dx_f^2 on the fine domain
    if ((rc = check_stencil(fine, st, dt_crse / nsub, lam_f, 1.0))) return rc;
    if (ncrse_steps == 0) return 0;
    const int R = st->kind;
    const bool fp64diff = (st->flags & MF_FP64_DIFF) && crse->dtype != F64;
    InterpPlan *ip = get_interp(fine, crse, ratio, &rc);
    if (!ip) return rc;
    AvgPlan *ap = get_avg(fine, crse, ratio, &rc);
    if (!ap) return rc;
    const bool do_reflux = (st->flags & MF_REFLUX) != 0;
    RefluxPlan *rp = nullptr;
    RefluxW wc{}, wf{};
    if (do_reflux) {
        if (fine->ncomp != crse->ncomp) return fail(MF_EINVAL, "levels differ in components");
        if (!(rp = get_reflux(fine, crse, ratio, &rc))) return rc;
        for (int c = 0; c < crse->ncomp; ++c) {
            wc.w[c] = lam_c[c];
            wf.w[c] = lam_f[c] / ((double)ratio * ratio * ratio);
        }
    }
    if (crse->tile_auto && (rc = autotune(crse, R, fp64diff, lam_c))) return rc;
    if (fine->tile_auto && (rc = autotune(fine, R, fp64diff, lam_f))) return rc;
    if (crse->use_tma && crse->tma_R != tma_key(R, false) && (rc = build_tma(crse, R))) return rc;
    if (fine->use_tma && fine->tma_R != tma_key(R, false) && (rc = build_tma(fine, R))) return rc;
    AmrFill *af = get_amr_fill(crse, fine, ratio, R, ip, rp, &rc);
    if (!af) return rc;
    const bool cpush = use_push(crse);
    const bool fpush = use_push(fine);
    // the coarse stream orders everything; the fine stream waits for nothing else (same
    // stream expected); capture the whole advance into one graph
    char buf[160];
    snprintf(buf, sizeof buf, "amr|%p|g%llu|g%llu|s%d|r%d|fc%d|x%d", (void *)fine, crse->gen, fine->gen, nsub, ratio,
             fine->cur, (int)do_reflux);
    const std::string key = graph_key(buf, R, fp64diff, lam_c, crse->ncomp, ncrse_steps, crse->cur);
    auto it = crse->graphs.find(key);
    if (it == crse->graphs.end()) {
        if ((rc = capture_begin(crse))) return rc;
        cudaStream_t s = crse->cap;
        int body = 0, c = crse->cur, f = fine->cur;
        PhaseLog log{crse, false};
        auto fill = [&](mf_t *m, int which, const DevBuf &t, size_t n) -> int {
            if (!n) return 0;
            int b = log.before(0);
            if (!b && launch_fill(m->dtype, level_ptrs(m, which), (const FbTask *)t.p, (int)n, 0, s) != cudaSuccess)
                b = fail(MF_ECUDA, "fill launch failed");
            return b;
        };
        // Independent work shares launches (launch_fill_interp, launch_fill_cflux,
        // launch_avg_reflux): per coarse step a coarse fill, the coarse stencil, the fill of the
        // new coarse level with the coarse face fluxes of the old one, then per substep the fine
        // fill with the interpolation, the fine face fluxes and the fine stencil, and last the
        // average-down with the flux correction.
        auto pair_kind = [](size_t a, size_t b, int ka, int kb) { return b ? kb : ka; };
        // The first fine substep reads only the old coarse level (its interpolation is at
        // alpha = 0), so in an untimed advance it runs as a graph branch beside the coarse stencil
        // and the new coarse level's fill; the branches join before the second substep.
        const bool branch = !log.timing && crse->cap2 && crse->fork_ev[0] && crse->fork_ev[1];
        auto ev_ok = [](cudaError_t e) { return e == cudaSuccess ? 0 : fail(MF_ECUDA, "graph branch: %s", cudaGetErrorString(e)); };
        for (int step = 0; step < ncrse_steps && !body; ++step) {
            // the coarse ghosts read in this step: the stencil's faces (or, with the ghost push,
            // what the push does not deliver or the last average-down and correction made
            // stale) and the cells the interpolation and the flux registers read
            const int nface = rp ? (int)rp->faces.size() : 0;
            if (step == 0 || !cpush) body = fill(crse, c, af->d_first, af->t_first.size());
            else body = fill(crse, c, af->d_next, af->t_next.size());
            auto coarse_part = [&]() -> int {
                int b = log.before(1);
                if (!b) b = enqueue_stencil(crse, c, R, fp64diff, lam_c, s, cpush);
                // the new level's ghosts that the interpolation reads, and the coarse face fluxes
                // at the interface from the old level (which the stencil only read)
                const size_t npost = af->t_post.size();
                if (!b && !(b = log.before(pair_kind(npost, (size_t)nface, 0, 2), npost + nface > 0)))
                    b = launch_fill_cflux(crse->dtype, R, level_ptrs(crse, 1 - c), (const FbTask *)af->d_post.p,
                                          (int)npost, crse->level_ptr(c), rp ? (const CFace *)rp->d_faces.p : nullptr,
                                          nface, crse->ncomp, wc, rp ? (double *)rp->d_regc.p : nullptr,
                                          s) == cudaSuccess
                            ? 0
                            : fail(MF_ECUDA, "coarse fill / flux register launch failed");
                return b;
            };
            auto sub_step = [&](int sub, cudaStream_t ss) -> int {
                // the fine level steps like a single level: a face fill first, then the push
                // and the residual fill; the interpolation writes the coarse-fine ghosts
                const bool face = (step == 0 && sub == 0) || !fpush;
                const bool strips = fine->use_tma && fine->tma_ok && fine->tma_strips;
                const DevBuf &ft = face ? (strips ? fine->d_fbtasks_adv : fine->d_fbtasks) : fine->d_fbtasks_res;
                const size_t nft = face ? fill_step_tasks(fine) : fine->fbtasks_res.size();
                const InterpArgs ia{fine->level_ptr(f), crse->level_ptr(c), crse->level_ptr(1 - c),
                                    (const InterpRun *)ip->d_runs.p, (const int *)ip->cells.d_start.p,
                                    (const int *)ip->cells.d_wfirst.p, (int)ip->runs.size(), ip->cells.ncells,
                                    fine->ncomp, ratio, (double)sub / (double)nsub};
                const size_t nip = ip->runs.empty() ? 0 : (size_t)ip->cells.ncells;
                int b = 0;
                if (!(b = log.before(pair_kind(nft, nip, 0, 2), nft + nip > 0)))
                    b = launch_fill_interp(fine->dtype, level_ptrs(fine, f), (const FbTask *)ft.p, (int)nft, ia,
                                           ss) == cudaSuccess
                            ? 0
                            : fail(MF_ECUDA, "fine fill / interpolation launch failed");
                if (!b && rp && !(b = log.before(2, nface > 0)))  // fine face fluxes, this substep
                    b = launch_cf_fine_flux(fine->dtype, R, fine->level_ptr(f), (const CFace *)rp->d_faces.p,
                                            (const FFace *)rp->d_ff.p, nface, ratio * ratio, fine->ncomp, wf,
                                            (double *)rp->d_regf.p, sub == 0, ss) == cudaSuccess
                            ? 0
                            : fail(MF_ECUDA, "flux register launch failed");
                if (!b && !(b = log.before(1))) b = enqueue_stencil(fine, f, R, fp64diff, lam_f, ss, fpush);
                f = 1 - f;
                return b;
            };
            if (!body && branch) {
                cudaStream_t s2 = crse->cap2;
                body = ev_ok(cudaEventRecord(crse->fork_ev[0], s));
                if (!body) body = ev_ok(cudaStreamWaitEvent(s2, crse->fork_ev[0], 0));
                if (!body) body = sub_step(0, s2);
                if (!body) body = coarse_part();
                if (!body) body = ev_ok(cudaEventRecord(crse->fork_ev[1], s2));
                if (!body) body = ev_ok(cudaStreamWaitEvent(s, crse->fork_ev[1], 0));
                for (int sub = 1; sub < nsub && !body; ++sub) body = sub_step(sub, s);
            } else if (!body) {
                body = coarse_part();
                for (int sub = 0; sub < nsub && !body; ++sub) body = sub_step(sub, s);
            }
            // the average-down writes the covered coarse cells, the flux correction the uncovered
            // ones next to the interface
            const AvgArgs aa{fine->level_ptr(f), crse->level_ptr(1 - c), (const AvgRegion *)ap->d_regs.p,
                             (const int *)ap->cells.d_start.p, (const int *)ap->cells.d_wfirst.p, (int)ap->regs.size(),
                             ap->regs.empty() ? 0 : ap->cells.ncells, fine->ncomp, ratio, ap->vec};
            const RefluxArgs ra{crse->level_ptr(1 - c), rp ? (const CCell *)rp->d_cells.p : nullptr,
                                rp ? (int)rp->cells.size() : 0, rp ? (const CFace *)rp->d_faces.p : nullptr,
                                crse->ncomp, rp ? (const double *)rp->d_regc.p : nullptr,
                                rp ? (const double *)rp->d_regf.p : nullptr};
            if (!body && !(body = log.before(3, aa.ncells + ra.ncell > 0)))
                body = launch_avg_reflux(crse->dtype, aa, ra, s) == cudaSuccess
                           ? 0
                           : fail(MF_ECUDA, "average-down / reflux launch failed");
            c = 1 - c;
        }
        if ((rc = capture_end(crse, key, body))) return rc;
        it = crse->graphs.find(key);
        log.store(*it->second);
    }
    note_launch(crse, *it->second);
    CU(cudaGraphLaunch(it->second->exec, crse->stream));
    if (ncrse_steps & 1) crse->cur = 1 - crse->cur;
    if ((ncrse_steps * nsub) & 1) fine->cur = 1 - fine->cur;
    return 0;
}
