// solver.cu -- batched FMSG solve (Sec. 2, Algorithms 1 and 2 of arXiv:1907.12334).
//
// Work decomposition.  Every grid (p,q) of every sample is an *item*: it is
// solved at stage L = (p-1)+(q-1) (the diagonals are processed in increasing
// order, Algorithm 2).  An item starts from the kappa-weighted cubic
// interpolation of its children's solutions and is iterated by mu-cycles of
// Algorithm 1 over its own hierarchy {(p',q'): p' <= p, q' <= q} until
// ||1 - A u||/||1|| <= eps.  Each cycle is a defect correction: the FP64
// residual r = 1 - A u is formed on the item's grid, one mu-cycle of
// Algorithm 1 (in FP32 for MSG_PREC_MIXED, FP64 otherwise) solves A e = r
// approximately from e = 0 on the item's scratch hierarchy, and u += e in FP64.
// For a linear cycle this is the same iteration as cycling on (u, 1).
//
// Launch structure of one cycle for all active items of a stage: diagonals
// d > cut of the items' hierarchies are visited by one launch per visit half
// (PRE: zero/smooth nu1/restrict; POST: prolong/smooth nu2) with one CTA per
// (item, grid) task; everything at or below the cut runs inside one launch
// (LOW) in which each warp executes the recursion of Algorithm 1 as a flat
// program in shared memory for a few items of one shape class in lockstep.
//
// Storage (all node-indexed with the boundary, see common.cuh):
//   u64          solution of every grid of every sample (FP64)
//   ax64, ay64   a/dx^2 at x-faces (i+1/2,j) and a/dy^2 at y-faces (i,j+1/2),
//                stored at node (i,j) (FP64; exact scaling by powers of two)
//   ax32, ay32   the same rounded to FP32 (mixed cycles only)
//   su, sbx, sby scratch of the active items' hierarchies: correction e and the
//                restrictions received from the x-parent and the y-parent.
#include <algorithm>
#include <type_traits>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "prof.cuh"

namespace msg {

// ---------------------------------------------------------------- tables --

struct SampleInfo {
    int P, Q;
    int64_t node_off;  // start of the sample's rectangle in u64 / coefficient arrays
    int64_t field_off; // start of the sample's field in Z
    int64_t q_off;     // start of the sample's P*Q outputs
};

// One launch covers a list of segments; segment i owns blocks
// [blk_start[i], blk_start[i] + count of its group) and each of those blocks
// is one sample of the group.
struct Segment {
    int g;              // shape group
    int pi, qi;         // item (top) grid
    int p, q;           // task grid (equal to the item grid for item-level lists)
    int64_t blk_start;  // first block of this segment in its launch
    int64_t count;      // blocks (samples) in this segment
    int64_t list_off;   // the segment's samples are slist[list_off .. list_off+count)
    int64_t scr_slot;   // offset of the item's hierarchy inside the sample's stage scratch
    int64_t stage_base; // item-level lists: index of (group, item) in the stage's flag array
};

struct Group {
    int P, Q;
    int start, count;       // range of the group's samples in perm[]
    int64_t scr_start;      // start of the group's stage scratch
    int64_t scr_per_sample; // stage scratch per sample of the group
};

struct DevCtx {
    const SampleInfo* samples;
    const int* gpos;    // position of each sample inside its group
    const int* slist;   // sample lists the segments index into
    const Group* groups;
    const Segment* segs;
    int nseg;
};

__device__ __forceinline__ int find_segment(const Segment* segs, int nseg, int64_t b)
{
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (segs[mid].blk_start <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct TaskRef {
    int s;          // sample
    const Segment* seg;
    int64_t scr;    // item hierarchy scratch base
    int64_t item;   // global item id (packed like Qout)
    int64_t sidx;   // index in the stage's flag array (item-level lists)
};

__device__ __forceinline__ TaskRef resolve_at(const DevCtx& cx, int64_t b)
{
    int si = find_segment(cx.segs, cx.nseg, b);
    const Segment* sg = &cx.segs[si];
    const Group& G = cx.groups[sg->g];
    TaskRef t;
    t.s = cx.slist[sg->list_off + (b - sg->blk_start)];
    t.seg = sg;
    const int gp = cx.gpos[t.s];
    t.scr = G.scr_start + (int64_t)gp * G.scr_per_sample + sg->scr_slot;
    const SampleInfo& S = cx.samples[t.s];
    t.item = S.q_off + (int64_t)(sg->pi - 1) * S.Q + (sg->qi - 1);
    t.sidx = sg->stage_base + gp;
    return t;
}

__device__ __forceinline__ TaskRef resolve(const DevCtx& cx) { return resolve_at(cx, blockIdx.x); }

// Task of this block in a 2-D launch: blockIdx.y is the segment, blockIdx.x the
// sample inside it (direct loads instead of a search; blocks past the
// segment's count have no task).
__device__ __forceinline__ bool resolve_2d(const DevCtx& cx, TaskRef& t)
{
    const Segment* sg = &cx.segs[blockIdx.y];
    if ((int64_t)blockIdx.x >= sg->count) return false;
    const Group& G = cx.groups[sg->g];
    t.s = cx.slist[sg->list_off + blockIdx.x];
    t.seg = sg;
    const int gp = cx.gpos[t.s];
    t.scr = G.scr_start + (int64_t)gp * G.scr_per_sample + sg->scr_slot;
    const SampleInfo& S = cx.samples[t.s];
    t.item = S.q_off + (int64_t)(sg->pi - 1) * S.Q + (sg->qi - 1);
    t.sidx = sg->stage_base + gp;
    return true;
}

// ------------------------------------------------------------ grid ops ----

// 1/x: in the FP32 cycles the hardware reciprocal approximation (at most 1 ulp
// from 1/x; the arguments, sums of a/h^2 > 0, are never subnormal), which is
// enough because those cycles only produce a correction and the FP64 residual
// decides convergence; exact division in FP64.
__host__ __device__ __forceinline__ float rcp_of(float x)
{
#ifdef __CUDA_ARCH__
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
#else
    return 1.0f / x;  // host builds (table checks) only
#endif
}
__host__ __device__ __forceinline__ double rcp_of(double x) { return 1.0 / x; }

template <class T>
struct GView {
    T* u;
    const T* bx;
    const T* by;
    int bmode;  // 0: b = bx, 1: b = by, 2: b = bx/2 + by/2
    const T* ax;
    const T* ay;
    int nx, ny;
};

template <class T>
__device__ __forceinline__ T b_at(const GView<T>& g, int c)
{
    if (g.bmode == 0) return g.bx[c];
    if (g.bmode == 1) return g.by[c];
    return T(0.5) * g.bx[c] + T(0.5) * g.by[c];
}

template <class T>
__device__ __forceinline__ T res_at(const GView<T>& g, int c, int W)
{
    T aw = g.ax[c - 1], ae = g.ax[c], as = g.ay[c - W], an = g.ay[c];
    T Au = (aw + ae + as + an) * g.u[c] - (aw * g.u[c - 1] + ae * g.u[c + 1]) - (as * g.u[c - W] + an * g.u[c + W]);
    return b_at(g, c) - Au;
}

// The thread group that runs one grid operation: a whole CTA.  `tid` and `n`
// index its threads; sync() orders its shared and global memory accesses.
struct CtaGroup {
    int tid, n;
    __device__ CtaGroup() : tid(threadIdx.x), n(blockDim.x) {}
    __device__ void sync() const { __syncthreads(); }
};

// CTA-wide: zero u on every node, boundary included.  Scratch is reused by
// hierarchies of other shapes from stage to stage, so a boundary node here may
// hold an interior value written by an earlier stage.
template <class T, class G>
__device__ void cta_zero(const G& grp, const GView<T>& g)
{
    const int n = (g.nx + 1) * (g.ny + 1);
    for (int k = grp.tid; k < n; k += grp.n) g.u[k] = T(0);
}

// CTA-wide red-black Gauss-Seidel sweeps (red = (i+j) even first).
template <class T, class G>
__device__ void cta_smooth(const G& grp, const GView<T>& g, int sweeps)
{
    // slot kk of row j of a colour is node i = first + 2 kk; nx/2 = 2^sh slots per row
    const int W = g.nx + 1, sh = __ffs(g.nx) - 2, n = (g.ny - 1) << sh;
    for (int sw = 0; sw < sweeps; ++sw)
        for (int colour = 0; colour < 2; ++colour) {
            for (int k = grp.tid; k < n; k += grp.n) {
                const int j = 1 + (k >> sh), kk = k & ((1 << sh) - 1);
                const int i = (((1 + j) & 1) == colour ? 1 : 2) + 2 * kk;
                if (i >= g.nx) continue;
                int c = j * W + i;
                T aw = g.ax[c - 1], ae = g.ax[c], as = g.ay[c - W], an = g.ay[c];
                T nb = (aw * g.u[c - 1] + ae * g.u[c + 1]) + (as * g.u[c - W] + an * g.u[c + W]);
                g.u[c] = (b_at(g, c) + nb) * rcp_of(aw + ae + as + an);
            }
            grp.sync();
        }
}

// Coarsest grid (1,1): one unknown, v = b / A (Algorithm 1, L = 0).
template <class T, class G>
__device__ void cta_coarsest(const G& grp, const GView<T>& g)
{
    if (grp.tid < 9) {  // all 3x3 nodes: boundary zeros (see cta_zero) and the unknown
        const int c = 1 * 3 + 1;
        g.u[grp.tid] = (grp.tid == c) ? b_at(g, c) / (g.ax[c - 1] + g.ax[c] + g.ay[c - 3] + g.ay[c]) : T(0);
    }
    grp.sync();
}

// Full-weighting restriction of the residual of g (Eq. (2.3)): R_x r into the
// x-child's bx (if cxb != nullptr), R_y r into the y-child's by.  The residual
// is formed once per interior node into shared memory `sr` (capacity `band`
// nodes, at least 3 rows) band by band: a band of B rows (B odd) starting at
// an odd row a holds rows a..a+B-1; it restricts its rows but the last in x
// (the last band all of them) and the coarse rows jc with 2jc-1 >= a and
// 2jc+1 <= a+B-1 in y; the next band starts at a+B-1.
template <class T, class G>
__device__ void cta_restrict(const G& grp, const GView<T>& g, T* cxb, T* cyb, T* sr, int band)
{
    const int W = g.nx + 1, sh = __ffs(g.nx) - 1, last = g.ny - 1;
    int B = band / W;
    if (B >= last) B = last;  // one band holds every interior row
    else B = (B - 1) | 1;     // odd, >= 3 (band >= 3 W)
    for (int a = 1; a <= last; a += max(B - 1, 1)) {
        const int e = min(a + B - 1, last);  // last row of the band
        const int nr = (e - a + 1) << sh;
        for (int k = grp.tid; k < nr; k += grp.n) {
            const int i = k & (g.nx - 1), j = a + (k >> sh);
            if (i == 0) continue;
            sr[(j - a) * W + i] = res_at(g, j * W + i, W);
        }
        grp.sync();
        if (cxb) {  // child (p-1,q): nx/2 = 2^shc cells, same rows (slot ic = 0 is the boundary)
            const int ncx = g.nx >> 1, Wc = ncx + 1, shc = sh - 1;
            const int ex = (e == last) ? e : e - 1, n = (ex - a + 1) << shc;
            for (int k = grp.tid; k < n; k += grp.n) {
                const int ic = k & (ncx - 1), j = a + (k >> shc);
                if (ic == 0) continue;
                const int r = (j - a) * W + 2 * ic;
                cxb[j * Wc + ic] = T(0.25) * (sr[r - 1] + T(2) * sr[r] + sr[r + 1]);
            }
        }
        if (cyb) {  // child (p,q-1): same columns, coarse row jc from fine rows 2jc-1..2jc+1
            const int j0 = (a + 1) >> 1, j1 = (e - 1) >> 1, n = max(j1 - j0 + 1, 0) << sh;
            for (int k = grp.tid; k < n; k += grp.n) {
                const int i = k & (g.nx - 1), jc = j0 + (k >> sh);
                if (i == 0) continue;
                const int r = (2 * jc - a) * W + i;
                cyb[jc * W + i] = T(0.25) * (sr[r - W] + T(2) * sr[r] + sr[r + W]);
            }
        }
        grp.sync();
        if (e == last) break;
    }
}

// Coarse-grid correction (Eq. (2.4) with linear P and the weights of Eq. (2.5)):
// u += omega * (kx Px e_x + ky Py e_y); one child only when q = 1 or p = 1.
template <class T, class G>
__device__ void cta_prolong(const G& grp, const GView<T>& g, const T* ucx, const T* ucy, T omega)
{
    const int W = g.nx + 1, sh = __ffs(g.nx) - 1, n = (g.ny - 1) << sh;
    for (int k = grp.tid; k < n; k += grp.n) {
        const int i = k & (g.nx - 1), j = 1 + (k >> sh);  // slot i = 0 is the boundary
        if (i == 0) continue;
        const int c = j * W + i;
        T vx = T(0), vy = T(0);
        if (ucx) {
            const int Wc = (g.nx >> 1) + 1, r = j * Wc + (i >> 1);
            vx = (i & 1) ? T(0.5) * (ucx[r] + ucx[r + 1]) : ucx[r];
        }
        if (ucy) {
            const int r = (j >> 1) * W + i;
            vy = (j & 1) ? T(0.5) * (ucy[r] + ucy[r + W]) : ucy[r];
        }
        T corr;
        if (ucx && ucy) {
            T cxv = g.ax[c - 1] + g.ax[c], cyv = g.ay[c - W] + g.ay[c];
            T x2 = cxv * cxv, y2 = cyv * cyv, s = rcp_of(x2 + y2);
            corr = (x2 * s) * vx + (y2 * s) * vy;
        } else {
            corr = ucx ? vx : vy;
        }
        g.u[c] += omega * corr;
    }
    grp.sync();
}

// ------------------------------------------------------- hierarchy views --

template <class T>
struct Hier {
    T* su;
    T* sbx;
    T* sby;
    const T* ax;  // sample's coefficient rectangle
    const T* ay;
    int Ps, Qs;   // sample's finest grid (coefficient layout)
    int pi, qi;   // item's top grid (scratch layout)
    int64_t scr;  // item scratch base
};

template <class T>
__device__ __forceinline__ GView<T> view_of(const Hier<T>& h, int p, int q)
{
    GView<T> g;
    int64_t so = h.scr + grid_offset(p, q, h.qi);
    int64_t co = grid_offset(p, q, h.Qs);
    g.u = h.su + so;
    g.bx = h.sbx + so;
    g.by = h.sby + so;
    bool hx = p < h.pi, hy = q < h.qi;  // parents inside the item's hierarchy
    g.bmode = (!hx && !hy) ? 0 : (hx && hy) ? 2 : (hx ? 0 : 1);
    g.ax = h.ax + co;
    g.ay = h.ay + co;
    g.nx = 1 << p;
    g.ny = 1 << q;
    return g;
}

// Visit halves of Algorithm 1 on one grid (p,q) of an item's hierarchy.
template <class T, class G>
__device__ void visit_pre(const G& grp, const Hier<T>& h, int p, int q, int zero_init, int nu1, T* sr, int band)
{
    GView<T> g = view_of(h, p, q);
    if (p == 1 && q == 1) { cta_coarsest(grp, g); return; }
    if (zero_init) { cta_zero(grp, g); grp.sync(); }
    cta_smooth(grp, g, nu1);
    T* cxb = (p > 1) ? h.sbx + h.scr + grid_offset(p - 1, q, h.qi) : nullptr;
    T* cyb = (q > 1) ? h.sby + h.scr + grid_offset(p, q - 1, h.qi) : nullptr;
    cta_restrict(grp, g, cxb, cyb, sr, band);
}

template <class T, class G>
__device__ void visit_post(const G& grp, const Hier<T>& h, int p, int q, int nu2, T omega)
{
    if (p == 1 && q == 1) return;
    GView<T> g = view_of(h, p, q);
    const T* ucx = (p > 1) ? h.su + h.scr + grid_offset(p - 1, q, h.qi) : nullptr;
    const T* ucy = (q > 1) ? h.su + h.scr + grid_offset(p, q - 1, h.qi) : nullptr;
    cta_prolong(grp, g, ucx, ucy, omega);
    cta_smooth(grp, g, nu2);
}

struct CycleParams {
    int mu, nu1, nu2;
    double omega;
};

// Grids of diagonal d of the hierarchy below (pi, qi).
__device__ __forceinline__ void diag_range(int d, int pi, int qi, int& plo, int& phi)
{
    plo = max(1, d + 2 - qi);
    phi = min(pi, d + 1);
}

// ----------------------------------------------------------------- kernels --

template <class T>
__device__ __forceinline__ Hier<T> hier_of(const DevCtx& cx, const TaskRef& t, T* su, T* sbx, T* sby, const T* ax,
                                           const T* ay)
{
    const SampleInfo& S = cx.samples[t.s];
    Hier<T> h;
    h.su = su; h.sbx = sbx; h.sby = sby;
    h.ax = ax + S.node_off; h.ay = ay + S.node_off;
    h.Ps = S.P; h.Qs = S.Q;
    h.pi = t.seg->pi; h.qi = t.seg->qi;
    h.scr = t.scr;
    return h;
}

template <class T>
__global__ void k_pre(DevCtx cx, T* su, T* sbx, T* sby, const T* ax, const T* ay, int zero_init, int nu1, int band)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];  // `band` residual nodes
    TaskRef t;
    if (!resolve_2d(cx, t)) return;
    Hier<T> h = hier_of(cx, t, su, sbx, sby, ax, ay);
    visit_pre(CtaGroup(), h, t.seg->p, t.seg->q, zero_init, nu1, (T*)smem_raw, band);
}

template <class T>
__global__ void k_post(DevCtx cx, T* su, T* sbx, T* sby, const T* ax, const T* ay, int nu2, double omega)
{
    TaskRef t;
    if (!resolve_2d(cx, t)) return;
    Hier<T> h = hier_of(cx, t, su, sbx, sby, ax, ay);
    visit_post(CtaGroup(), h, t.seg->p, t.seg->q, nu2, (T)omega);
}

// ------------------------------------------------------ convergence study --
//
// Residual history of plain cycles from a zero initial guess on each sample's
// finest grid, b = 1 (Sec. 2, numerical experiments): MSG cycles (Algorithm 1
// over the whole hierarchy, by the visit halves above), or multigrid with
// standard coarsening on the diagonal grids (P-k, Q-k) of the same hierarchy:
// full weighting (the tensor product of 1/4 [1 2 1]), bilinear interpolation,
// the same red-black smoother, coefficients and damping, and an exact solve
// of the first grid with a single interior line (p = 1 or q = 1).  The paper
// does not give its standard-coarsening operators; these are the textbook ones
// for vertex-centred grids.  One CTA per sample runs a host-built program of
// the cycle's operations, in FP64.

enum HistOp { H_PRE = 0, H_POST, H_STD_PRE, H_STD_POST, H_STD_LINE };

// nu1 sweeps, r = b - A u into the grid's by plane (free in this method), full
// weighting into the child's bx, child u = 0.
template <class T, class G>
__device__ void cta_std_pre(const G& grp, const Hier<T>& h, int p, int q, int nu1)
{
    GView<T> g = view_of(h, p, q);
    g.bmode = 0;
    cta_smooth(grp, g, nu1);
    const int W = g.nx + 1, n = (g.ny - 1) * W;
    T* r = h.sby + h.scr + grid_offset(p, q, h.qi);
    for (int k = grp.tid; k < n; k += grp.n) {
        const int c = W + k, i = c % W;
        if (i == 0 || i == g.nx) continue;
        r[c] = res_at(g, c, W);
    }
    grp.sync();
    const int ncx = g.nx >> 1, ncy = g.ny >> 1, Wc = ncx + 1;
    T* cb = h.sbx + h.scr + grid_offset(p - 1, q - 1, h.qi);
    T* cu = h.su + h.scr + grid_offset(p - 1, q - 1, h.qi);
    for (int k = grp.tid; k < Wc * (ncy + 1); k += grp.n) {
        const int jc = k / Wc, ic = k - jc * Wc;
        cu[k] = T(0);
        if (ic == 0 || ic == ncx || jc == 0 || jc == ncy) continue;
        const int c = 2 * jc * W + 2 * ic;
        const T edge = r[c - 1] + r[c + 1] + r[c - W] + r[c + W];
        const T corner = r[c - W - 1] + r[c - W + 1] + r[c + W - 1] + r[c + W + 1];
        cb[k] = (T(4) * r[c] + T(2) * edge + corner) / T(16);
    }
    grp.sync();
}

// u += omega * bilinear(child u), then nu2 sweeps.
template <class T, class G>
__device__ void cta_std_post(const G& grp, const Hier<T>& h, int p, int q, int nu2, T omega)
{
    GView<T> g = view_of(h, p, q);
    g.bmode = 0;
    const T* cu = h.su + h.scr + grid_offset(p - 1, q - 1, h.qi);
    const int W = g.nx + 1, Wc = (g.nx >> 1) + 1, n = (g.ny - 1) * W;
    for (int k = grp.tid; k < n; k += grp.n) {
        const int c = W + k, j = c / W, i = c - j * W;
        if (i == 0 || i == g.nx) continue;
        const int b0 = (j >> 1) * Wc + (i >> 1);
        T v;
        if (!(i & 1) && !(j & 1)) v = cu[b0];
        else if (!(j & 1)) v = T(0.5) * (cu[b0] + cu[b0 + 1]);
        else if (!(i & 1)) v = T(0.5) * (cu[b0] + cu[b0 + Wc]);
        else v = T(0.25) * (cu[b0] + cu[b0 + 1] + cu[b0 + Wc] + cu[b0 + Wc + 1]);
        g.u[c] += omega * v;
    }
    grp.sync();
    cta_smooth(grp, g, nu2);
}

// Exact solve on a grid with one interior line (Thomas algorithm, one thread;
// the by plane holds the elimination coefficients).
template <class T, class G>
__device__ void cta_std_line(const G& grp, const Hier<T>& h, int p, int q)
{
    GView<T> g = view_of(h, p, q);
    g.bmode = 0;
    T* e = h.sby + h.scr + grid_offset(p, q, h.qi);
    const int W = g.nx + 1, row = g.ny == 2, n = row ? g.nx - 1 : g.ny - 1;
    for (int k = grp.tid; k < W * (g.ny + 1); k += grp.n) g.u[k] = T(0);
    grp.sync();
    if (grp.tid == 0) {
        T cprev = T(0), dprev = T(0);
        for (int k = 0; k < n; ++k) {
            const int c = row ? W + k + 1 : (k + 1) * W + 1;
            const T aw = g.ax[c - 1], ae = g.ax[c], as = g.ay[c - W], an = g.ay[c];
            const T lo = row ? -aw : -as, up = row ? -ae : -an;
            const T d = (aw + ae + as + an) - (k > 0 ? lo * cprev : T(0));
            cprev = up / d;
            dprev = (g.bx[c] - (k > 0 ? lo * dprev : T(0))) / d;
            e[2 * k] = cprev;
            e[2 * k + 1] = dprev;
        }
        T next = T(0);
        for (int k = n - 1; k >= 0; --k) {
            const int c = row ? W + k + 1 : (k + 1) * W + 1;
            next = e[2 * k + 1] - e[2 * k] * next;
            g.u[c] = next;
        }
    }
    grp.sync();
}

// hist[s][k] = ||1 - A u_k||_h / ||1||_h on the sample's finest grid, k = 0..ncycles.
// prog: one cycle, op.x = kind | (p or diagonal) << 4 | q << 12, op.y = zero-init.
template <class T>
__global__ void k_cycle_history(DevCtx cx, T* su, T* sbx, T* sby, const T* ax, const T* ay, const int2* prog,
                                int nops, int ncycles, CycleParams cp, int band, double* hist)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];  // `band` residual nodes of the MSG restriction
    __shared__ double red[32];
    TaskRef t;
    if (!resolve_2d(cx, t)) return;
    const Hier<T> h = hier_of(cx, t, su, sbx, sby, ax, ay);
    const CtaGroup grp;
    const int P = h.pi, Q = h.qi;
    const GView<T> top = view_of(h, P, Q);  // no parents: b = bx
    const int W = top.nx + 1, n = W * (top.ny + 1);
    T* bx = h.sbx + h.scr + grid_offset(P, Q, Q);
    for (int k = grp.tid; k < n; k += grp.n) {
        const int j = k / W, i = k - j * W;
        top.u[k] = T(0);
        bx[k] = (i > 0 && i < top.nx && j > 0 && j < top.ny) ? T(1) : T(0);
    }
    grp.sync();
    double* hs = hist + (int64_t)t.s * (ncycles + 1);
    const double nb = sqrt((double)(top.nx - 1) * (top.ny - 1));
    for (int cyc = 0; cyc <= ncycles; ++cyc) {
        if (cyc > 0)
            for (int o = 0; o < nops; ++o) {
                const int2 op = prog[o];
                const int kind = op.x & 15, a = (op.x >> 4) & 255, b = (op.x >> 12) & 255;
                if (kind == H_PRE || kind == H_POST) {
                    for (int p = max(1, a + 2 - Q); p <= min(P, a + 1); ++p) {
                        if (kind == H_PRE) visit_pre(grp, h, p, a + 2 - p, op.y, cp.nu1, (T*)smem_raw, band);
                        else visit_post(grp, h, p, a + 2 - p, cp.nu2, (T)cp.omega);
                    }
                } else if (kind == H_STD_PRE) {
                    cta_std_pre(grp, h, a, b, cp.nu1);
                } else if (kind == H_STD_POST) {
                    cta_std_post(grp, h, a, b, cp.nu2, (T)cp.omega);
                } else {
                    cta_std_line(grp, h, a, b);
                }
            }
        double s = 0.0;
        for (int k = grp.tid; k < (top.ny - 1) * W; k += grp.n) {
            const int c = W + k, i = c % W;
            if (i == 0 || i == top.nx) continue;
            const double r = (double)res_at(top, c, W);
            s += r * r;
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((grp.tid & 31) == 0) red[grp.tid >> 5] = s;
        grp.sync();
        if (grp.tid == 0) {
            double tot = 0.0;
            for (int w = 0; w < (grp.n + 31) / 32; ++w) tot += red[w];
            hs[cyc] = sqrt(tot) / nb;
        }
        grp.sync();
    }
}

// --------------------------------------------- register-cached visits --
//
// Full launches of the global-memory visits above are bound by instruction
// issue, not by memory: the grid is served from L1 after its first touch, and
// every colour phase repeats the node's index arithmetic and reloads its four
// face coefficients and its right-hand side.  None of those change during a
// visit.  Here a thread keeps, for each of its nodes, the four coefficients,
// their sum and its reciprocal, and b in registers for the whole visit, and u
// sits in shared memory; a sweep then costs a node four shared loads, two
// fused multiply-adds, a multiply and a store.  Thread t owns colour slot
// t + m blockDim (m < NPT) of each colour.  The shared plane keeps the grid's
// rows (stride W = nx + 1) with the columns split by parity, even i in slots
// 0..nx/2 and odd i after them, so that the nodes of one colour in a row and
// each of their neighbours sit at consecutive addresses.  The arithmetic of a
// node is written with explicit fma, so every launch shape (threads, NPT)
// rounds alike.  Grids with more than 512 NPT nodes of a colour keep the
// global-memory visits.

constexpr int kRegThreadsMax = 512;  // threads per CTA of the register-cached visits

__device__ __forceinline__ int split_slot(int h, int i) { return (i & 1) ? h + (i >> 1) : (i >> 1); }

template <class T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src),
                 "n"((int)sizeof(T))
                 : "memory");
}

// Calls f(j, i) for every node of the grid, boundary included, consecutive
// threads on consecutive i (columns 0..nx-1 of all rows, then column nx).
template <class F>
__device__ __forceinline__ void for_each_node(int p, int ny, F f)
{
    const int nx = 1 << p, m = (ny + 1) << p, n = m + ny + 1;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        if (k < m) f(k >> p, k & (nx - 1));
        else f(k - m, nx);
    }
}

// Node of colour slot k (colour 0: red, (i+j) even): k = (j-1) nx/2 + kk with
// i = 2kk + 1 when i has the parity (j + colour) & 1 == 1, else i = 2kk + 2
// (kk = nx/2 - 1 is then the boundary and no node).  Returns false for no node.
__device__ __forceinline__ bool colour_node(int k, int colour, int p, int& i, int& j)
{
    const int sh = p - 1, half = 1 << sh;
    j = 1 + (k >> sh);
    const int kk = k & (half - 1), odd = (j + colour) & 1;
    i = odd ? 2 * kk + 1 : 2 * kk + 2;
    return odd || kk != half - 1;
}

// Rounding pinned: no contraction into or out of these.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// One visit half: PRE (pre = 1) = (zero,) nu red-black sweeps, residual and
// Eq. (2.3) restriction into the children's right-hand sides; POST = the
// Eq. (2.4)/(2.5) coarse-grid correction, then nu sweeps.  One CTA per (item,
// grid), NPT nodes of each colour per thread.
template <class T, int NPT>
__global__ void __launch_bounds__(kRegThreadsMax) k_visit_reg(DevCtx cx, T* su, T* sbx, T* sby, const T* ax,
                                                              const T* ay, int pre, int zero_init, int nu,
                                                              double omega_d)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TaskRef t;
    if (!resolve_2d(cx, t)) return;
    const Hier<T> h = hier_of(cx, t, su, sbx, sby, ax, ay);
    const int p = t.seg->p, q = t.seg->q;
    const GView<T> gv = view_of(h, p, q);
    const int nx = 1 << p, ny = 1 << q, W = nx + 1, hs = (nx >> 1) + 1, nslot = (ny - 1) << (p - 1);
    T* U = (T*)smem_raw;
    T* Rs = U + W * (ny + 1);  // PRE: the residual
    const bool zu = pre && zero_init;
    for_each_node(p, ny, [&](int j, int i) {
        T* d = U + j * W + split_slot(hs, i);
        if (zu) *d = T(0);
        else cp_async_elem(d, gv.u + j * W + i);
    });
    // the thread's nodes: slots, coefficients, diagonal, its reciprocal, b
    T aw[2][NPT], ae[2][NPT], as[2][NPT], an[2][NPT], dg[2][NPT], iv[2][NPT], bb[2][NPT];
    int ss[2][NPT], ww[2][NPT];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int m = 0; m < NPT; ++m) {
            const int k = threadIdx.x + m * blockDim.x;
            int i = 0, j = 0;
            ss[c][m] = -1;
            ww[c][m] = 0;
            aw[c][m] = ae[c][m] = as[c][m] = an[c][m] = dg[c][m] = iv[c][m] = bb[c][m] = T(0);
            if (k < nslot && colour_node(k, c, p, i, j)) {
                const int g = j * W + i;
                ss[c][m] = j * W + split_slot(hs, i);
                ww[c][m] = j * W + split_slot(hs, i - 1);
                aw[c][m] = gv.ax[g - 1];
                ae[c][m] = gv.ax[g];
                as[c][m] = gv.ay[g - W];
                an[c][m] = gv.ay[g];
                dg[c][m] = aw[c][m] + ae[c][m] + as[c][m] + an[c][m];
                iv[c][m] = rcp_of(dg[c][m]);
                bb[c][m] = b_at(gv, g);
            }
        }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (!pre) {  // coarse-grid correction from the children's corrections (global memory)
        const T omega = (T)omega_d;
        const T* ucx = (p > 1) ? h.su + h.scr + grid_offset(p - 1, q, h.qi) : nullptr;
        const T* ucy = (q > 1) ? h.su + h.scr + grid_offset(p, q - 1, h.qi) : nullptr;
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int m = 0; m < NPT; ++m) {
                int i, j;
                const int s = ss[c][m];
                if (s < 0) continue;
                colour_node(threadIdx.x + m * blockDim.x, c, p, i, j);
                T vx = T(0), vy = T(0);
                if (ucx) {
                    const int r = j * (hs) + (i >> 1);  // child row stride nx/2 + 1 = hs
                    vx = (i & 1) ? T(0.5) * (ucx[r] + ucx[r + 1]) : ucx[r];
                }
                if (ucy) {
                    const int r = (j >> 1) * W + i;
                    vy = (j & 1) ? T(0.5) * (ucy[r] + ucy[r + W]) : ucy[r];
                }
                T corr;
                if (ucx && ucy) {
                    const T cxv = aw[c][m] + ae[c][m], cyv = as[c][m] + an[c][m];
                    const T x2 = mul_rn(cxv, cxv), y2 = mul_rn(cyv, cyv), sc = rcp_of(x2 + y2);
                    corr = fma_rn(mul_rn(x2, sc), vx, mul_rn(mul_rn(y2, sc), vy));
                } else {
                    corr = ucx ? vx : vy;
                }
                U[s] = fma_rn(omega, corr, U[s]);
            }
        __syncthreads();
    }
    for (int sw = 0; sw < nu; ++sw)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
#pragma unroll
            for (int m = 0; m < NPT; ++m) {
                const int s = ss[c][m], w = ww[c][m];
                if (s < 0) continue;
                const T nb = fma_rn(aw[c][m], U[w], mul_rn(ae[c][m], U[w + 1])) +
                             fma_rn(as[c][m], U[s - W], mul_rn(an[c][m], U[s + W]));
                U[s] = (bb[c][m] + nb) * iv[c][m];
            }
            __syncthreads();
        }
    if (pre) {  // r = b - A u at every interior node
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int m = 0; m < NPT; ++m) {
                const int s = ss[c][m], w = ww[c][m];
                if (s < 0) continue;
                const T xw = fma_rn(aw[c][m], U[w], mul_rn(ae[c][m], U[w + 1]));
                const T xs = fma_rn(as[c][m], U[s - W], mul_rn(an[c][m], U[s + W]));
                Rs[s] = bb[c][m] - (fma_rn(dg[c][m], U[s], -xw) - xs);
            }
        __syncthreads();
    }
    for_each_node(p, ny, [&](int j, int i) { gv.u[j * W + i] = U[j * W + split_slot(hs, i)]; });
    if (!pre) return;
    if (p > 1) {  // x-child (p-1, q): R_x around fine column 2ic of every interior row
        T* cxb = h.sbx + h.scr + grid_offset(p - 1, q, h.qi);
        const int shc = p - 1, ncx = nx >> 1, Wc = ncx + 1, n = (ny - 1) << shc;  // ncx = 2^shc slots a row
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int ic = k & (ncx - 1), j = 1 + (k >> shc);
            if (ic == 0) continue;
            const int base = j * W;  // fine columns 2ic-1, 2ic, 2ic+1: slots hs+ic-1, ic, hs+ic
            cxb[j * Wc + ic] = T(0.25) * (Rs[base + hs + ic - 1] + T(2) * Rs[base + ic] + Rs[base + hs + ic]);
        }
    }
    if (q > 1) {  // y-child (p, q-1): R_y around fine row 2jc of every interior column
        T* cyb = h.sby + h.scr + grid_offset(p, q - 1, h.qi);
        const int n = ((ny >> 1) - 1) << p;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int i = k & (nx - 1), jc = 1 + (k >> p);
            if (i == 0) continue;
            const int s = 2 * jc * W + split_slot(hs, i);
            cyb[jc * W + i] = T(0.25) * (Rs[s - W] + T(2) * Rs[s] + Rs[s + W]);
        }
    }
}


// ---------------------------------------------- table-driven low diagonals --
//
// Diagonals d <= dl of an item's hierarchy are visited 2^(L-d) times per cycle
// (Algorithm 1 with mu = 2) but hold only a few hundred unknowns, so their cost
// is the latency of a long chain of small dependent phases; throughput comes
// from items in flight and from keeping lanes busy in the small phases.
//
// One warp runs KW items of the same shape class in lockstep: lane l works on
// item l / (32/KW) and on every (32/KW)-th table entry of the current phase, so
// a phase with a single node (the coarsest grid) still occupies KW lanes.  A
// lane only ever touches its own item's planes, so phases are separated by
// __syncwarp alone.  Each item's grids with p + q - 2 <= dl live in shared
// memory in five planes, all in a fixed layout of the full triangle below dl:
//   u   interior nodes of every grid, red ((i+j) even) then black, row by row,
//       after one slot (index 0) that stays zero and stands for every boundary
//       node, so that a stencil reads its neighbours through plain indices;
//   b   the same indexing as u;
//   fx  x-faces (i+1/2, j) of interior rows, row by row: the west and east faces
//       of node (i,j) are neighbours;
//   fy  y-faces (i, j+1/2) of interior columns, column by column: the south and
//       north faces of node (i,j) are neighbours;
//   r   the residual of the diagonal being restricted (row by row per grid).
// With the red-black order, consecutive entries of a smoothing phase touch
// consecutive u, b words, and the per-item stride (== 32/KW modulo 32 words)
// puts the KW items of a warp on disjoint banks.
//
// The mu-cycles run as a flat program of phases: the recursion of Algorithm 1
// unrolled on the host into (kind, diagonal) words and resolved per class of
// item, the clipped triangle (min(pi, dl+1), min(qi, dl+1), dl), into
// {kind, entries, first entry}.  An entry is four words of 16-bit indices
// into the planes.

constexpr int kLowMax = 5;  // highest diagonal the low kernel can take
constexpr int kLowGridsMax = (kLowMax + 1) * (kLowMax + 2) / 2;
constexpr int kLowClassesMax = 91;  // sum over dl = 0..kLowMax of (dl + 1)^2
constexpr int kLowWarpsMax = 16;    // warps per CTA of the low kernel

// phase kinds; a resolved program word is {kind | entries << 3, first entry}.
// LK_CALL2 stands for the mu recursive calls below diagonal 3, run in registers.
enum LowKind { LK_RED = 0, LK_BLACK, LK_RESID, LK_RESTRICT, LK_PROL, LK_CALL2, LK_NKIND };

// Class of the triangle below diagonal dl of an item (pic, qic in 1..dl+1).
__host__ __device__ __forceinline__ int low_class(int pic, int qic, int dl)
{
    return dl * (dl + 1) * (2 * dl + 1) / 6 + (pic - 1) * (dl + 1) + (qic - 1);
}

// Position of interior node (i, j) of a grid with ni = 2^p - 1 interior columns
// and nj interior rows in the red-black order of the u and b planes (relative
// to the grid's first slot).  Odd rows hold h + 1 red and h black nodes, even
// rows h red and h + 1 black, h = (ni - 1) / 2.
__host__ __device__ constexpr int low_rb(int ni, int nj, int i, int j)
{
    const int h = (ni - 1) >> 1;
    if (((i + j) & 1) == 0) return (j - 1) * h + (j >> 1) + ((i - 1) >> 1);
    return nj * h + ((nj + 1) >> 1) + (j - 1) * h + ((j - 1) >> 1) + ((i - 1) >> 1);
}

// Fixed plane layout of the full triangle below dl (independent of the class).
// Grids are ordered by diagonal, then p, so the layout of a lower dl is a
// prefix of each plane of the layout of a higher one.
struct LowGrid {
    int p, q;
    int gu;  // first slot of the grid in u and b
    int gx;  // first x-face in fx
    int gy;  // first y-face in fy
};
struct LowPlanes {
    int dl;
    int nu, nfx, nfy, nr;  // plane sizes (nu includes the zero slot)
    int ngrid;
    LowGrid g[kLowGridsMax];  // ordered by diagonal, then p
};

struct LowDesc {
    int dl, pic, qic;
    int prog, nops;                    // resolved program of the class (set per solve)
    int e0, e1;                        // the class's entries: table[e0 .. e1)
    int cnt[kLowMax + 1][LK_NKIND];    // entries of each (diagonal, kind)
    int off[kLowMax + 1][LK_NKIND];    // first table entry of the phase
};

// One warp's share of a launch: items first .. first + count - 1 of segment seg
// (count 0: an idle warp).  The warps of one CTA share the class cls.
struct LowTask {
    int seg, first, count, cls;
};

// Table entries (16-bit fields, low half first):
//   smooth / residual  x = c | uw   y = ue | us   z = un | xw   w = ys | r
//       node c with neighbours uw, ue, us, un (0 on the boundary), west face
//       xw (east xw + 1), south face ys (north ys + 1), residual slot r;
//   restrict           x = c | rx   y = ry | wy   z = has x-parent | has y-parent << 1
//       child node c; x-parent residual around rx (+-1), y-parent around ry (+-wy);
//   prolong            x = c | xw   y = ys | cx0  z = cx1 | cy0  w = cy1 | has x-child << 16 | has y-child << 17
//       fine node c; correction 1/2 (u[cx0] + u[cx1]) from the x-child (the two
//       coincide at even i), likewise from the y-child.

// Four entries of one phase at a time: no entry of a phase reads what another
// entry of the same phase writes, so all operands are gathered first (their
// shared-memory loads in flight together), then computed, then stored.
template <class T>
__host__ __device__ __forceinline__ void low_phase4(int kind, T* u, T* b, const T* fx, const T* fy, T* r,
                                                    const uint4 (&e)[4], T omega)
{
    if (kind <= LK_RESID) {
        // red-black Gauss-Seidel update of one colour, or the residual b - A u
        T aw[4], ae[4], as[4], an[4], uw[4], ue[4], us[4], un[4], bc[4], uc[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int xw = e[k].z >> 16, ys = e[k].w & 0xFFFF;
            aw[k] = fx[xw]; ae[k] = fx[xw + 1]; as[k] = fy[ys]; an[k] = fy[ys + 1];
            uw[k] = u[e[k].x >> 16]; ue[k] = u[e[k].y & 0xFFFF]; us[k] = u[e[k].y >> 16]; un[k] = u[e[k].z & 0xFFFF];
            bc[k] = b[e[k].x & 0xFFFF];
            uc[k] = kind == LK_RESID ? u[e[k].x & 0xFFFF] : T(0);
        }
        if (kind == LK_RESID) {
            T rv[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const T Au = (aw[k] + ae[k] + as[k] + an[k]) * uc[k] - (aw[k] * uw[k] + ae[k] * ue[k]) -
                             (as[k] * us[k] + an[k] * un[k]);
                rv[k] = bc[k] - Au;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) r[e[k].w >> 16] = rv[k];
        } else {
            T v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const T nb = (aw[k] * uw[k] + ae[k] * ue[k]) + (as[k] * us[k] + an[k] * un[k]);
                v[k] = (bc[k] + nb) * rcp_of(aw[k] + ae[k] + as[k] + an[k]);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) u[e[k].x & 0xFFFF] = v[k];
        }
    } else if (kind == LK_RESTRICT) {
        // Eq. (2.3) for one child node: b = R_x r of the x-parent and/or R_y r of the
        // y-parent, averaged when it has both; the child's correction restarts from 0
        // (the recursion's first visit of the child follows every restriction)
        T v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int rx = e[k].x >> 16, ry = e[k].y & 0xFFFF, wy = e[k].y >> 16;
            const bool hx = e[k].z & 1, hy = e[k].z & 2;
            // absent parents point at slot 0 with stride 0: the loads are valid and ignored
            const T x0 = r[hx ? rx - 1 : 0], x1 = r[rx], x2 = r[hx ? rx + 1 : 0];
            const T y0 = r[hy ? ry - wy : 0], y1 = r[ry], y2 = r[hy ? ry + wy : 0];
            const T vx = hx ? T(0.25) * (x0 + T(2) * x1 + x2) : T(0);
            const T vy = hy ? T(0.25) * (y0 + T(2) * y1 + y2) : T(0);
            v[k] = (hx && hy) ? T(0.5) * vx + T(0.5) * vy : (hx ? vx : vy);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            b[e[k].x & 0xFFFF] = v[k];
            u[e[k].x & 0xFFFF] = T(0);
        }
    } else {
        // Eq. (2.4) with linear P and the kappa weights of Eq. (2.5)
        T v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = e[k].x & 0xFFFF, xw = e[k].x >> 16, ys = e[k].y & 0xFFFF;
            const int cx0 = e[k].y >> 16, cx1 = e[k].z & 0xFFFF, cy0 = e[k].z >> 16, cy1 = e[k].w & 0xFFFF;
            const bool hx = (e[k].w >> 16) & 1, hy = (e[k].w >> 17) & 1;
            const T ux0 = u[cx0], ux1 = u[cx1], uy0 = u[cy0], uy1 = u[cy1], uc = u[c];
            const T f0 = fx[xw], f1 = fx[xw + 1], g0 = fy[ys], g1 = fy[ys + 1];
            const T vx = hx ? T(0.5) * (ux0 + ux1) : T(0), vy = hy ? T(0.5) * (uy0 + uy1) : T(0);
            T corr;
            if (hx && hy) {
                const T cxv = f0 + f1, cyv = g0 + g1;
                const T x2 = cxv * cxv, y2 = cyv * cyv, s = rcp_of(x2 + y2);
                corr = (x2 * s) * vx + (y2 * s) * vy;
            } else {
                corr = hx ? vx : vy;
            }
            v[k] = uc + omega * corr;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) u[e[k].x & 0xFFFF] = v[k];
    }
}

// One entry of a phase: the four-entry path with the entry repeated (the same
// value is written four times), so every node of every launch shape goes
// through one arithmetic definition.
template <class T>
__host__ __device__ __forceinline__ void low_phase(int kind, T* u, T* b, const T* fx, const T* fy, T* r, uint4 e,
                                                   T omega)
{
    const uint4 w[4] = {e, e, e, e};
    low_phase4(kind, u, b, fx, fy, r, w, omega);
}


// ------------------------------------------------ diagonals <= 2 in registers --
//
// Below diagonal 3 an item has at most six grids and 30 unknowns, and those
// levels hold most of the phases of a mu-cycle (each visit of diagonal 3 calls
// mu cycles on them).  One thread runs those calls for its item: u and b of the
// six grids live in registers (the code below is unrolled at compile time for
// each possible clipped shape (PIC, QIC) of the triangle, so every index is a
// constant), the coefficients are read from the item's face planes in shared
// memory (the six grids lead both face planes), and the arithmetic is that
// of the table phases, node for node.  Register slot k holds u-plane slot k + 1.
namespace r2 {
__host__ __device__ constexpr int grid(int p, int q)
{
    return (p == 1 && q == 1) ? 0 : (p == 1 && q == 2) ? 1 : (p == 2 && q == 1) ? 2 : (p == 1 && q == 3) ? 3
         : (p == 2 && q == 2) ? 4 : 5;
}
// the six grids in the layout's order (diagonal, then p) and their offsets in the
// planes: u/b slots of interior nodes, and x- and y-faces padded to 4 values
__host__ __device__ constexpr int gp(int g) { return g == 0 ? 1 : g == 1 ? 1 : g == 2 ? 2 : g == 3 ? 1 : g == 4 ? 2 : 3; }
__host__ __device__ constexpr int gq(int g) { return g == 0 ? 1 : g == 1 ? 2 : g == 2 ? 1 : g == 3 ? 3 : g == 4 ? 2 : 1; }
// (written out, not recursive, so that the compiler folds them into constant
// register indices; the host check compares them with the layout builder's)
__host__ __device__ constexpr int gu(int g) { return g == 0 ? 0 : g == 1 ? 1 : g == 2 ? 4 : g == 3 ? 7 : g == 4 ? 14 : 23; }
__host__ __device__ constexpr int gx(int g) { return g == 0 ? 0 : g == 1 ? 4 : g == 2 ? 12 : g == 3 ? 16 : g == 4 ? 32 : 44; }
__host__ __device__ constexpr int gy(int g) { return g == 0 ? 0 : g == 1 ? 4 : g == 2 ? 8 : g == 3 ? 16 : g == 4 ? 24 : 36; }
// register slot of interior node (i, j) of grid (p, q)
__host__ __device__ constexpr int at(int p, int q, int i, int j)
{
    return gu(grid(p, q)) + low_rb((1 << p) - 1, (1 << q) - 1, i, j);
}
constexpr int kN = 30;  // unknowns of the six grids
}  // namespace r2

template <class T, int PIC, int QIC>
struct Reg2 {
    // the coefficients stay in shared memory: every grid operation starts with a compiler
    // barrier, so they are re-read per operation (92 of them would not fit beside u, b)
    // while the loads inside one operation can still be issued together
    typedef const T* CP;
    __host__ __device__ static __forceinline__ void fence()
    {
#ifdef __CUDA_ARCH__
        asm volatile("" ::: "memory");
#endif
    }
    static constexpr bool has(int p, int q) { return p >= 1 && q >= 1 && p <= PIC && q <= QIC && p + q <= 4; }

    // u at node (i, j) of grid (p, q); boundary nodes read the zero slot's value
    template <int P, int Q>
    __host__ __device__ static __forceinline__ T get(const T* u, int i, int j)
    {
        // the index stays inside the array even for boundary nodes (whose value is 0), so that
        // the compiler can keep the unrolled array in registers
        const bool in = i > 0 && i < (1 << P) && j > 0 && j < (1 << Q);
        const T v = u[in ? r2::at(P, Q, i, j) : 0];
        return in ? v : T(0);
    }

    template <int P, int Q>
    __host__ __device__ static __forceinline__ void smooth(T* u, const T* b, CP fx, CP fy, int colour)
    {
        fence();
        constexpr int nx = 1 << P, ny = 1 << Q, g = r2::grid(P, Q);
#pragma unroll
        for (int j = 1; j < ny; ++j)
#pragma unroll
            for (int i = 1; i < nx; ++i) {
                if (((i + j) & 1) != colour) continue;
                const int xw = r2::gx(g) + (j - 1) * nx + (i - 1), ys = r2::gy(g) + (i - 1) * ny + (j - 1);
                const T aw = fx[xw], ae = fx[xw + 1], as = fy[ys], an = fy[ys + 1];
                const T nb = (aw * get<P, Q>(u, i - 1, j) + ae * get<P, Q>(u, i + 1, j)) +
                             (as * get<P, Q>(u, i, j - 1) + an * get<P, Q>(u, i, j + 1));
                const int c = r2::at(P, Q, i, j);
                u[c] = (b[c] + nb) * rcp_of(aw + ae + as + an);
            }
    }

    template <int P, int Q>
    __host__ __device__ static __forceinline__ T res(const T* u, const T* b, CP fx, CP fy, int i, int j)
    {
        constexpr int nx = 1 << P, ny = 1 << Q, g = r2::grid(P, Q);
        const int xw = r2::gx(g) + (j - 1) * nx + (i - 1), ys = r2::gy(g) + (i - 1) * ny + (j - 1);
        const T aw = fx[xw], ae = fx[xw + 1], as = fy[ys], an = fy[ys + 1];
        const T Au = (aw + ae + as + an) * get<P, Q>(u, i, j) - (aw * get<P, Q>(u, i - 1, j) + ae * get<P, Q>(u, i + 1, j)) -
                     (as * get<P, Q>(u, i, j - 1) + an * get<P, Q>(u, i, j + 1));
        return b[r2::at(P, Q, i, j)] - Au;
    }

    // Eq. (2.3) into child (P, Q) from its parents (P+1, Q) and (P, Q+1); the child's u restarts at 0
    template <int P, int Q>
    __host__ __device__ static __forceinline__ void restrict_to(T* u, T* b, CP fx, CP fy)
    {
        fence();
        constexpr bool hx = has(P + 1, Q), hy = has(P, Q + 1);
        constexpr int nx = 1 << P, ny = 1 << Q;
#pragma unroll
        for (int j = 1; j < ny; ++j)
#pragma unroll
            for (int i = 1; i < nx; ++i) {
                T vx = T(0), vy = T(0);
                if constexpr (hx)
                    vx = T(0.25) * (res<P + 1, Q>(u, b, fx, fy, 2 * i - 1, j) + T(2) * res<P + 1, Q>(u, b, fx, fy, 2 * i, j) +
                                    res<P + 1, Q>(u, b, fx, fy, 2 * i + 1, j));
                if constexpr (hy)
                    vy = T(0.25) * (res<P, Q + 1>(u, b, fx, fy, i, 2 * j - 1) + T(2) * res<P, Q + 1>(u, b, fx, fy, i, 2 * j) +
                                    res<P, Q + 1>(u, b, fx, fy, i, 2 * j + 1));
                const int c = r2::at(P, Q, i, j);
                b[c] = (hx && hy) ? T(0.5) * vx + T(0.5) * vy : (hx ? vx : vy);
                u[c] = T(0);
            }
    }

    // Eq. (2.4)/(2.5) into fine grid (P, Q) from its children (P-1, Q) and (P, Q-1)
    template <int P, int Q>
    __host__ __device__ static __forceinline__ void prolong(T* u, CP fx, CP fy, T omega)
    {
        fence();
        constexpr bool hx = P > 1, hy = Q > 1;
        constexpr int nx = 1 << P, ny = 1 << Q, g = r2::grid(P, Q);
#pragma unroll
        for (int j = 1; j < ny; ++j)
#pragma unroll
            for (int i = 1; i < nx; ++i) {
                T vx = T(0), vy = T(0);
                if constexpr (hx) vx = T(0.5) * (get<P - 1, Q>(u, i >> 1, j) + get<P - 1, Q>(u, (i + 1) >> 1, j));
                if constexpr (hy) vy = T(0.5) * (get<P, Q - 1>(u, i, j >> 1) + get<P, Q - 1>(u, i, (j + 1) >> 1));
                T corr;
                if constexpr (hx && hy) {
                    const int xw = r2::gx(g) + (j - 1) * nx + (i - 1), ys = r2::gy(g) + (i - 1) * ny + (j - 1);
                    const T cxv = fx[xw] + fx[xw + 1], cyv = fy[ys] + fy[ys + 1];
                    const T x2 = cxv * cxv, y2 = cyv * cyv, s = rcp_of(x2 + y2);
                    corr = (x2 * s) * vx + (y2 * s) * vy;
                } else {
                    corr = hx ? vx : vy;
                }
                u[r2::at(P, Q, i, j)] += omega * corr;  // the children's u are not written here
            }
    }

    __host__ __device__ static __forceinline__ void smooth_diag(int d, T* u, const T* b, CP fx, CP fy, int colour)
    {
        if (d == 2) {
            if constexpr (has(1, 3)) smooth<1, 3>(u, b, fx, fy, colour);
            if constexpr (has(2, 2)) smooth<2, 2>(u, b, fx, fy, colour);
            if constexpr (has(3, 1)) smooth<3, 1>(u, b, fx, fy, colour);
        } else {
            if constexpr (has(1, 2)) smooth<1, 2>(u, b, fx, fy, colour);
            if constexpr (has(2, 1)) smooth<2, 1>(u, b, fx, fy, colour);
        }
    }

    // mu-cycle of Algorithm 1 at diagonal 1 (one visit; diagonal 0 solved exactly once)
    __host__ __device__ static __forceinline__ void cycle1(T* u, T* b, CP fx, CP fy, int nu1, int nu2, T omega)
    {
        for (int s = 0; s < nu1; ++s) { smooth_diag(1, u, b, fx, fy, 0); smooth_diag(1, u, b, fx, fy, 1); }
        restrict_to<1, 1>(u, b, fx, fy);
        smooth<1, 1>(u, b, fx, fy, 0);
        if constexpr (has(1, 2)) prolong<1, 2>(u, fx, fy, omega);
        if constexpr (has(2, 1)) prolong<2, 1>(u, fx, fy, omega);
        for (int s = 0; s < nu2; ++s) { smooth_diag(1, u, b, fx, fy, 0); smooth_diag(1, u, b, fx, fy, 1); }
    }

    // mu-cycle of Algorithm 1 at diagonal 2
    __host__ __device__ static __forceinline__ void cycle2(T* u, T* b, CP fx, CP fy, int mu, int nu1, int nu2,
                                                           T omega)
    {
        for (int s = 0; s < nu1; ++s) { smooth_diag(2, u, b, fx, fy, 0); smooth_diag(2, u, b, fx, fy, 1); }
        if constexpr (has(1, 2)) restrict_to<1, 2>(u, b, fx, fy);
        if constexpr (has(2, 1)) restrict_to<2, 1>(u, b, fx, fy);
        for (int k = 0; k < mu; ++k) cycle1(u, b, fx, fy, nu1, nu2, omega);
        if constexpr (has(1, 3)) prolong<1, 3>(u, fx, fy, omega);
        if constexpr (has(2, 2)) prolong<2, 2>(u, fx, fy, omega);
        if constexpr (has(3, 1)) prolong<3, 1>(u, fx, fy, omega);
        for (int s = 0; s < nu2; ++s) { smooth_diag(2, u, b, fx, fy, 0); smooth_diag(2, u, b, fx, fy, 1); }
    }

    // the mu calls of a diagonal-3 visit: b of the diagonal-2 grids in, their u out (planes
    // indexed like the kernel's u and b planes, slot 0 the zero)
    __host__ __device__ static __forceinline__ void run(T* su, const T* sb, CP fx, CP fy, int mu, int nu1,
                                                        int nu2, T omega)
    {
        T u[r2::kN], b[r2::kN];
#pragma unroll
        for (int k = 0; k < r2::kN; ++k) {
            u[k] = T(0);
            b[k] = T(0);
        }
#pragma unroll
        for (int k = r2::gu(3); k < r2::kN; ++k) b[k] = sb[1 + k];
        for (int k = 0; k < mu; ++k) cycle2(u, b, fx, fy, mu, nu1, nu2, omega);
#pragma unroll
        for (int k = r2::gu(3); k < r2::kN; ++k) su[1 + k] = u[k];
    }
};

// Register path of one item for its class's clipped triangle below diagonal 3.
template <class T>
__host__ __device__ __forceinline__ void low_call2(int pic, int qic, T* u, const T* b, const T* fx, const T* fy, int mu,
                                                   int nu1, int nu2, T omega)
{
    pic = pic < 3 ? pic : 3;
    qic = qic < 3 ? qic : 3;
    switch (pic * 4 + qic) {
    case 1 * 4 + 3: Reg2<T, 1, 3>::run(u, b, fx, fy, mu, nu1, nu2, omega); break;
    case 2 * 4 + 2: Reg2<T, 2, 2>::run(u, b, fx, fy, mu, nu1, nu2, omega); break;
    case 2 * 4 + 3: Reg2<T, 2, 3>::run(u, b, fx, fy, mu, nu1, nu2, omega); break;
    case 3 * 4 + 1: Reg2<T, 3, 1>::run(u, b, fx, fy, mu, nu1, nu2, omega); break;
    case 3 * 4 + 2: Reg2<T, 3, 2>::run(u, b, fx, fy, mu, nu1, nu2, omega); break;
    case 3 * 4 + 3: Reg2<T, 3, 3>::run(u, b, fx, fy, mu, nu1, nu2, omega); break;
    default: break;  // no item has a smaller triangle below a diagonal-3 visit
    }
}

__device__ __forceinline__ TaskRef resolve_seg(const DevCtx& cx, int seg, int64_t local)
{
    const Segment* sg = &cx.segs[seg];
    const Group& G = cx.groups[sg->g];
    TaskRef t;
    t.s = cx.slist[sg->list_off + local];
    t.seg = sg;
    const int gp = cx.gpos[t.s];
    t.scr = G.scr_start + (int64_t)gp * G.scr_per_sample + sg->scr_slot;
    const SampleInfo& S = cx.samples[t.s];
    t.item = S.q_off + (int64_t)(sg->pi - 1) * S.Q + (sg->qi - 1);
    t.sidx = sg->stage_base + gp;
    return t;
}

// `calls` mu-cycles at diagonal lp.dl of each item, starting from zero.
// Reads the coefficients of the item's grids with d <= dl and the right-hand
// side of its diagonal-dl grids (combined from the parents' restrictions, or the
// item's own residual when dl is its top); writes back u of diagonal dl.
// All warps of a CTA run items of one class: the CTA first copies that class's
// resolved program (pcap words at most) and table entries (ecap at most) into
// shared memory, so the chain of phases touches no global memory.
template <class T, int KW>
__global__ void __launch_bounds__(32 * kLowWarpsMax) k_lowv(DevCtx cx, const LowTask* tasks, T* su, const T* sbx,
                                                           const T* sby, const T* img, int64_t istride, int ify,
                                                           const LowDesc* descs, const uint4* ent,
                                                           const uint2* rprog, LowPlanes lp, int stride, int pcap,
                                                           int ecap, int calls, CycleParams cp)
{
    const T omega = (T)cp.omega;
    constexpr int EW = 32 / KW;  // lanes per item
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint4* sent = (uint4*)smem_raw;
    uint2* sprog = (uint2*)(sent + ecap);
    T* planes = (T*)(sprog + pcap);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const LowDesc& D = descs[tasks[(size_t)blockIdx.x * wpb].cls];
    const int nops = D.nops, nent = D.e1 - D.e0;
    for (int k = threadIdx.x; k < nops; k += blockDim.x) sprog[k] = rprog[D.prog + k];
    for (int k = threadIdx.x; k < nent; k += blockDim.x) sent[k] = ent[D.e0 + k];
    __syncthreads();
    const LowTask tk = tasks[(size_t)blockIdx.x * wpb + warp];
    if (tk.count == 0) return;  // the whole warp; no CTA barrier follows
    const int k = lane / EW, el = lane % EW;
    const bool act = k < tk.count;
    T* u = planes + ((size_t)warp * KW + k) * stride;
    T* b = u + lp.nu;
    T* fx = b + lp.nu;
    T* fy = fx + lp.nfx;
    T* r = fy + lp.nfy;
    const int dl = lp.dl;
    if (act) {
        const TaskRef t = resolve_seg(cx, tk.seg, tk.first + k);
        const int pi = t.seg->pi, qi = t.seg->qi;
        // the face planes: 16-byte asynchronous copies of the prefixes of the sample's image
        {
            constexpr int V = 16 / sizeof(T);
            const T* im = img + (int64_t)t.s * istride;
            const uint32_t dfx = (uint32_t)__cvta_generic_to_shared(fx), dfy = (uint32_t)__cvta_generic_to_shared(fy);
            const bool aligned = ((dfx | dfy) & 15u) == 0 && (((uintptr_t)im | (uintptr_t)(im + ify)) & 15u) == 0;
            if (aligned) {
                for (int c = el; c < lp.nfx / V; c += EW)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dfx + 16 * c), "l"(im + c * V)
                                 : "memory");
                for (int c = el; c < lp.nfy / V; c += EW)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dfy + 16 * c), "l"(im + ify + c * V)
                                 : "memory");
                asm volatile("cp.async.commit_group;" ::: "memory");
            } else {  // not reached with the host's layout; plain copies keep every access legal
                for (int v = el; v < lp.nfx; v += EW) fx[v] = im[v];
                for (int v = el; v < lp.nfy; v += EW) fy[v] = im[ify + v];
            }
        }
        for (int v = el; v < lp.nu; v += EW) u[v] = T(0);
        for (int g = 0; g < lp.ngrid; ++g) {
            const LowGrid G = lp.g[g];
            const int p = G.p, q = G.q;
            if (p > D.pic || q > D.qic) continue;
            const int nx = 1 << p, ny = 1 << q, W = nx + 1;
            const int nxf = (ny - 1) << p;
            if (p + q - 2 == dl) {  // b at the interior nodes
                const int64_t so = t.scr + grid_offset(p, q, qi);
                const bool hx = p < pi, hy = q < qi;
                for (int v = el; v < nxf; v += EW) {
                    const int i = v & (nx - 1), j = 1 + (v >> p);
                    if (i == 0) continue;
                    const int64_t n = so + j * W + i;
                    T val;
                    if (hx && hy) val = T(0.5) * sbx[n] + T(0.5) * sby[n];
                    else if (hy) val = sby[n];
                    else val = sbx[n];  // x-parent only, or the item's own residual
                    b[G.gu + low_rb(nx - 1, ny - 1, i, j)] = val;
                }
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    __syncwarp();
    for (int call = 0; call < calls; ++call) {
        for (int o = 0; o < nops; ++o) {
            const uint2 op = sprog[o];
            const int kind = op.x & 7, cnt = (int)(op.x >> 3), off = (int)op.y;
            if (kind == LK_CALL2) {
                // FP32 only: the FP64 programs are built without this phase (the register path
                // would not fit beside the kernel's FP64 state)
                if constexpr (std::is_same<T, float>::value)
                    if (act && el == 0) low_call2(D.pic, D.qic, u, b, fx, fy, cp.mu, cp.nu1, cp.nu2, omega);
            } else if (act) {
                // entries of one phase are independent: four per lane in flight at a time
                // (a lane's last group repeats its first entry where it has fewer than four)
                for (int e = el; e < cnt; e += 4 * EW) {
                    uint4 w[4];
                    w[0] = sent[off + e];
                    w[1] = e + EW < cnt ? sent[off + e + EW] : w[0];
                    w[2] = e + 2 * EW < cnt ? sent[off + e + 2 * EW] : w[0];
                    w[3] = e + 3 * EW < cnt ? sent[off + e + 3 * EW] : w[0];
                    low_phase4(kind, u, b, fx, fy, r, w, omega);
                }
            }
            __syncwarp();
        }
    }
    if (act) {
        const TaskRef t = resolve_seg(cx, tk.seg, tk.first + k);
        const int qi = t.seg->qi;
        for (int g = 0; g < lp.ngrid; ++g) {
            const LowGrid G = lp.g[g];
            const int p = G.p, q = G.q;
            if (p + q - 2 != dl || p > D.pic || q > D.qic) continue;
            const int nx = 1 << p, ny = 1 << q, W = nx + 1, n = W * (ny + 1);
            T* dst = su + t.scr + grid_offset(p, q, qi);
            for (int v = el; v < n; v += EW) {
                const int j = v / W, i = v - j * W;
                const bool in = i > 0 && i < nx && j > 0 && j < ny;
                dst[v] = in ? u[G.gu + low_rb(nx - 1, ny - 1, i, j)] : T(0);
            }
        }
    }
}

// Coefficients on every grid (Sec. 2, direct discretisation on each grid).
// The finest grid takes a = exp(Z) at its face midpoints (field node
// (2i+1, 2j) for the x-face (i+1/2, j), (2i, 2j+1) for the y-face).  A coarser
// face covers sx = 2^(P-p) finest x-faces (sy finest y-faces): coef == 0 takes
// the series (harmonic) mean of their values along the flux direction,
// a = sx / sum_k exp(-Z_k); coef == 1 injects exp(Z) at the coarse face
// midpoint.  Stored scaled by 1/dx^2 and 1/dy^2 (exact: powers of two).
__global__ void k_coeffs(DevCtx cx, const double* Z, int coef, double* ax64, double* ay64, float* ax32, float* ay32)
{
    TaskRef t = resolve(cx);
    const SampleInfo& S = cx.samples[t.s];
    const int p = t.seg->p, q = t.seg->q, nx = 1 << p, ny = 1 << q, W = nx + 1;
    const int NFx = (1 << (S.P + 1)) + 1, sx = 1 << (S.P - p), sy = 1 << (S.Q - q);
    const double idx2 = (double)nx * nx, idy2 = (double)ny * ny;
    const double* Zs = Z + S.field_off;
    const int64_t off = S.node_off + grid_offset(p, q, S.Q);
    const int n = (nx + 1) * (ny + 1);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        int i = k % W, j = k / W;
        double vx = 0.0, vy = 0.0;
        if (i < nx) {
            const int64_t row = (int64_t)(2 * j * sy) * NFx;
            if (coef == 1 || sx == 1) {
                vx = exp(Zs[row + (2 * i + 1) * sx]);
            } else {
                double s = 0.0;
                for (int m = 0; m < sx; ++m) s += exp(-Zs[row + 2 * (i * sx + m) + 1]);
                vx = sx / s;
            }
            vx *= idx2;
        }
        if (j < ny) {
            if (coef == 1 || sy == 1) {
                vy = exp(Zs[(int64_t)((2 * j + 1) * sy) * NFx + 2 * i * sx]);
            } else {
                double s = 0.0;
                for (int m = 0; m < sy; ++m) s += exp(-Zs[(int64_t)(2 * (j * sy + m) + 1) * NFx + 2 * i * sx]);
                vy = sy / s;
            }
            vy *= idy2;
        }
        ax64[off + k] = vx;
        ay64[off + k] = vy;
        if (ax32) {
            ax32[off + k] = (float)vx;
            ay32[off + k] = (float)vy;
        }
    }
}

// Face image of each sample for the low-diagonal kernel: the x- and y-faces of
// its grids below diagonal kLowMax in the kernel's plane layout (x-faces from
// value 0, y-faces from value ify), built once per solve so that a launch copies
// them into shared memory in 16-byte pieces instead of gathering them.
template <class T>
__global__ void k_lowimg(const SampleInfo* samples, const T* ax, const T* ay, LowPlanes lp, T* img, int64_t istride,
                         int ify)
{
    const SampleInfo& S = samples[blockIdx.x];  // one block per sample
    T* im = img + (int64_t)blockIdx.x * istride;
    for (int g = 0; g < lp.ngrid; ++g) {
        const LowGrid G = lp.g[g];
        const int p = G.p, q = G.q;
        if (p > S.P || q > S.Q) continue;
        const int nx = 1 << p, ny = 1 << q, W = nx + 1;
        const int64_t co = S.node_off + grid_offset(p, q, S.Q);
        for (int v = threadIdx.x; v < ((ny - 1) << p); v += blockDim.x) {
            const int i = v & (nx - 1), j = 1 + (v >> p);
            im[G.gx + v] = ax[co + j * W + i];
        }
        for (int v = threadIdx.x; v < (ny << p); v += blockDim.x) {
            const int i = v & (nx - 1), j = v >> p;
            if (i == 0) continue;
            im[ify + G.gy + (i - 1) * ny + j] = ay[co + j * W + i];
        }
    }
}

// FMSG initial guess of an item (Algorithm 2): u = kappa_x Pc_x sol(p-1,q) +
// kappa_y Pc_y sol(p,q-1) with cubic Pc (odd-reflection boundary stencil);
// one child only on the q = 1 or p = 1 edge; u = 0 on G^(1,1).
__device__ __forceinline__ double cubic_at(const double* c, int stride, int m, int k)
{
    double cm1 = (k - 1 >= 0) ? c[(k - 1) * stride] : -c[stride];
    double c0 = c[k * stride];
    double c1 = c[(k + 1) * stride];
    double c2 = (k + 2 <= m) ? c[(k + 2) * stride] : -c[(m - 1) * stride];
    return (-cm1 + 9.0 * c0 + 9.0 * c1 - c2) / 16.0;
}

__global__ void k_interp(DevCtx cx, double* u64, const double* ax64, const double* ay64)
{
    TaskRef t = resolve(cx);
    const SampleInfo& S = cx.samples[t.s];
    const int p = t.seg->pi, q = t.seg->qi, nx = 1 << p, ny = 1 << q, W = nx + 1;
    double* u = u64 + S.node_off + grid_offset(p, q, S.Q);
    const double* ax = ax64 + S.node_off + grid_offset(p, q, S.Q);
    const double* ay = ay64 + S.node_off + grid_offset(p, q, S.Q);
    const double* ucx = (p > 1) ? u64 + S.node_off + grid_offset(p - 1, q, S.Q) : nullptr;
    const double* ucy = (q > 1) ? u64 + S.node_off + grid_offset(p, q - 1, S.Q) : nullptr;
    const int n = (nx - 1) * (ny - 1);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        int i = 1 + k % (nx - 1), j = 1 + k / (nx - 1);
        int c = j * W + i;
        if (!ucx && !ucy) { u[c] = 0.0; continue; }
        double vx = 0.0, vy = 0.0;
        if (ucx) {
            const int Wc = (nx >> 1) + 1;
            vx = (i & 1) ? cubic_at(ucx + j * Wc, 1, nx >> 1, i >> 1) : ucx[j * Wc + (i >> 1)];
        }
        if (ucy) vy = (j & 1) ? cubic_at(ucy + i, W, ny >> 1, j >> 1) : ucy[(j >> 1) * W + i];
        double corr;
        if (ucx && ucy) {
            double cxv = ax[c - 1] + ax[c], cyv = ay[c - W] + ay[c];
            double x2 = cxv * cxv, y2 = cyv * cyv;
            corr = (x2 / (x2 + y2)) * vx + (y2 / (x2 + y2)) * vy;
        } else {
            corr = ucx ? vx : vy;
        }
        u[c] = corr;
    }
}

// Block reduction of a double in a fixed order (result valid on thread 0).
__device__ double block_sum(double v)
{
    __shared__ double warp_part[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) warp_part[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        int nw = (blockDim.x + 31) >> 5;
        for (int k = 0; k < nw; ++k) s += warp_part[k];
    }
    return s;
}

// FP64 residual of the item's grid, convergence decision, and the right-hand
// side of the next correction cycle (written into the item's scratch).
template <class T>
__global__ void k_residual(DevCtx cx, const double* u64, const double* ax64, const double* ay64, T* sbx,
                           int max_cycles, double eps, int* nstep, int* sflag, int* cycles, double* relres,
                           int* status, int* counter)
{
    TaskRef t = resolve(cx);
    const SampleInfo& S = cx.samples[t.s];
    const int p = t.seg->pi, q = t.seg->qi, nx = 1 << p, ny = 1 << q, W = nx + 1;
    const int64_t off = S.node_off + grid_offset(p, q, S.Q);
    const double* u = u64 + off;
    const double* ax = ax64 + off;
    const double* ay = ay64 + off;
    T* rb = sbx + t.scr + grid_offset(p, q, q);
    const int n = (nx - 1) * (ny - 1);
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        int i = 1 + k % (nx - 1), j = 1 + k / (nx - 1);
        int c = j * W + i;
        double aw = ax[c - 1], ae = ax[c], as = ay[c - W], an = ay[c];
        double Au = (aw + ae + as + an) * u[c] - (aw * u[c - 1] + ae * u[c + 1]) - (as * u[c - W] + an * u[c + W]);
        double r = 1.0 - Au;
        acc += r * r;
        rb[c] = (T)r;
    }
    double ss = block_sum(acc);
    if (threadIdx.x == 0) {
        const int step = nstep[t.item];  // cycles done on this item so far
        double rr = sqrt(ss / (double)n);  // ||b|| with b = 1 on n interior nodes
        // diverged: worse than both the zero guess (1) and the item's initial guess, whose
        // relative residual is kept in relres until the item finishes
        int act;
        if (step == 0) { act = 1; relres[t.item] = rr; }  // at least one cycle
        else if (!(rr == rr) || isinf(rr)) { act = 0; atomicOr(&status[t.s], MSG_SAMPLE_NONFINITE); }
        else if (rr <= eps) act = 0;
        else if (step >= max_cycles || (rr > 1.0 && rr > relres[t.item])) {
            act = 0;
            atomicOr(&status[t.s], MSG_SAMPLE_NOT_CONVERGED);
        }
        else act = 1;
        sflag[t.sidx] = act;
        if (!act) {
            cycles[t.item] = step;
            relres[t.item] = rr;
        } else {
            nstep[t.item] = step + 1;
            atomicAdd(counter, 1);
        }
    }
}

template <class T>
__global__ void k_update(DevCtx cx, double* u64, const T* su)
{
    TaskRef t = resolve(cx);
    const SampleInfo& S = cx.samples[t.s];
    const int p = t.seg->pi, q = t.seg->qi, nx = 1 << p, ny = 1 << q, W = nx + 1;
    double* u = u64 + S.node_off + grid_offset(p, q, S.Q);
    const T* e = su + t.scr + grid_offset(p, q, q);
    const int n = (nx - 1) * (ny - 1);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        int i = 1 + k % (nx - 1), j = 1 + k / (nx - 1);
        int c = j * W + i;
        u[c] += (double)e[c];
    }
}

// QoI of the item's converged grid (Sec. 4).
__global__ void k_qoi(DevCtx cx, const double* u64, const double* Z, int qoi, double* Qout)
{
    TaskRef t = resolve(cx);
    const SampleInfo& S = cx.samples[t.s];
    const int p = t.seg->pi, q = t.seg->qi, nx = 1 << p, ny = 1 << q, W = nx + 1;
    const double* u = u64 + S.node_off + grid_offset(p, q, S.Q);
    const double dx = 1.0 / nx, dy = 1.0 / ny;
    double acc = 0.0;
    if (qoi == MSG_QOI_INTEGRAL) {
        const int n = (nx - 1) * (ny - 1);
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            int i = 1 + k % (nx - 1), j = 1 + k / (nx - 1);
            acc += u[j * W + i];
        }
        double s = block_sum(acc);
        if (threadIdx.x == 0) Qout[t.item] = dx * dy * s;
    } else if (qoi == MSG_QOI_POINT) {
        if (threadIdx.x == 0) Qout[t.item] = u[(ny / 2) * W + nx / 2];
    } else if (qoi == MSG_QOI_SUBDOMAIN) {
        if (p < 2 || q < 2) {
            if (threadIdx.x == 0) Qout[t.item] = nan("");
            return;
        }
        const int i0 = nx / 4, i1 = nx / 2, j0 = ny / 4, j1 = ny / 2, wi = i1 - i0 + 1;
        const int n = wi * (j1 - j0 + 1);
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            int i = i0 + k % wi, j = j0 + k / wi;
            double w = ((i == i0 || i == i1) ? 0.5 : 1.0) * ((j == j0 || j == j1) ? 0.5 : 1.0);
            acc += w * u[j * W + i];
        }
        double s = block_sum(acc);
        if (threadIdx.x == 0) Qout[t.item] = s * dx * dy / (0.25 * 0.25);
    } else {  // flux through x = 1
        const int NFx = (1 << (S.P + 1)) + 1, sy = 1 << (S.Q - q);
        const double* Zs = Z + S.field_off;
        for (int j = 1 + threadIdx.x; j < ny; j += blockDim.x) {
            double a = exp(Zs[(int64_t)(2 * j * sy) * NFx + (NFx - 1)]);
            acc += a * u[j * W + nx - 1] / dx;
        }
        double s = block_sum(acc);
        if (threadIdx.x == 0) Qout[t.item] = dy * s;
    }
}

// ------------------------------------------------------------------ plan --

namespace {

size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }
double pts(int p, int q) { return (double)((1 << p) - 1) * (double)((1 << q) - 1); }

// An item type of a stage: grid (pi, qi) of shape group g.
struct ItemType {
    int g, pi, qi;
    int64_t scr_slot;    // offset of its hierarchy in the sample's stage scratch
    int64_t stage_base;  // first flag index of this type in the stage's flag array
};

// ------------------------------------------------ low-diagonal host tables --

// Face counts are padded to whole 16-byte chunks (4 values) so that every plane
// and every grid's faces start 16-byte aligned: the face planes are copied into
// shared memory in 16-byte pieces.
static int low_pad4(int n) { return (n + 3) & ~3; }

// Fixed plane layout of the full triangle below dl.
static LowPlanes low_planes(int dl)
{
    LowPlanes L;
    std::memset(&L, 0, sizeof(L));
    L.dl = dl;
    L.nu = 1;  // slot 0: the zero that stands for boundary nodes
    for (int d = 0; d <= dl; ++d) {
        int nr = 0;
        for (int p = 1; p <= d + 1; ++p) {
            const int q = d + 2 - p, nx = 1 << p, ny = 1 << q;
            LowGrid& G = L.g[L.ngrid++];
            G.p = p;
            G.q = q;
            G.gu = L.nu;
            G.gx = L.nfx;
            G.gy = L.nfy;
            L.nu += (nx - 1) * (ny - 1);
            L.nfx += low_pad4(nx * (ny - 1));
            L.nfy += low_pad4((nx - 1) * ny);
            nr += (nx - 1) * (ny - 1);
        }
        L.nr = std::max(L.nr, nr);
    }
    L.nu = low_pad4(L.nu);
    return L;
}

// values of one item's planes (u, b, fx, fy, r)
static int low_values(const LowPlanes& L) { return 2 * L.nu + L.nfx + L.nfy + L.nr; }

// Shared-memory stride of one item: at least its values, and congruent to the
// lanes per item (32/kw) modulo the bank count so that the kw items of a warp
// sit on disjoint banks (4-byte banks; 16 bank pairs for 8-byte words).
static int low_stride(const LowPlanes& L, int kw, size_t es)
{
    const int ew = 32 / kw, m = es == 4 ? 32 : 16;
    const int v = low_values(L);
    return (v + m - 1) / m * m + (ew % m);
}

struct LowTables {
    std::vector<LowPlanes> planes;  // [dl]
    std::vector<LowDesc> desc;      // [class]
    std::vector<uint4> ent;
};

static void low_build_class(int pic, int qic, int dl, const LowPlanes& L, LowDesc& D, std::vector<uint4>& ent)
{
    std::memset(&D, 0, sizeof(D));
    D.dl = dl;
    D.pic = pic;
    D.qic = qic;
    D.e0 = (int)ent.size();
    auto exists = [&](int p, int q) { return p >= 1 && q >= 1 && p <= pic && q <= qic && p + q - 2 <= dl; };
    auto grid = [&](int p, int q) -> const LowGrid& {
        for (int k = 0; k < L.ngrid; ++k)
            if (L.g[k].p == p && L.g[k].q == q) return L.g[k];
        return L.g[0];  // not reached for grids of the triangle
    };
    // u/b slot of node (i, j) of grid (p, q); 0 on the boundary
    auto U = [&](int p, int q, int i, int j) -> uint32_t {
        const int nx = 1 << p, ny = 1 << q;
        if (i <= 0 || i >= nx || j <= 0 || j >= ny) return 0u;
        return (uint32_t)(grid(p, q).gu + low_rb(nx - 1, ny - 1, i, j));
    };
    // residual slot of interior node (i, j) of grid (p, q) on its diagonal (grids in p order)
    auto R = [&](int p, int q, int i, int j) -> uint32_t {
        int o = 0;
        for (int pp = 1; pp < p; ++pp) {
            const int qq = p + q - pp;
            if (exists(pp, qq)) o += ((1 << pp) - 1) * ((1 << qq) - 1);
        }
        return (uint32_t)(o + (j - 1) * ((1 << p) - 1) + (i - 1));
    };
    auto XW = [&](int p, int q, int i, int j) { return (uint32_t)(grid(p, q).gx + (j - 1) * (1 << p) + (i - 1)); };
    auto YS = [&](int p, int q, int i, int j) { return (uint32_t)(grid(p, q).gy + (i - 1) * (1 << q) + (j - 1)); };
    for (int d = 0; d <= dl; ++d) {
        // red then black entries of every grid of the diagonal, contiguous: the
        // residual phase runs over both lists at once
        for (int colour = 0; colour < 2; ++colour) {
            D.off[d][LK_RED + colour] = (int)ent.size();
            for (int p = 1; p <= d + 1; ++p) {
                const int q = d + 2 - p;
                if (!exists(p, q)) continue;
                const int nx = 1 << p, ny = 1 << q;
                for (int j = 1; j < ny; ++j)
                    for (int i = 1; i < nx; ++i)
                        if (((i + j) & 1) == colour)
                            ent.push_back(make_uint4(U(p, q, i, j) | U(p, q, i - 1, j) << 16,
                                                     U(p, q, i + 1, j) | U(p, q, i, j - 1) << 16,
                                                     U(p, q, i, j + 1) | XW(p, q, i, j) << 16,
                                                     YS(p, q, i, j) | R(p, q, i, j) << 16));
            }
            D.cnt[d][LK_RED + colour] = (int)ent.size() - D.off[d][LK_RED + colour];
        }
        D.off[d][LK_RESID] = D.off[d][LK_RED];
        D.cnt[d][LK_RESID] = D.cnt[d][LK_RED] + D.cnt[d][LK_BLACK];
        if (d == 0) continue;
        // Eq. (2.3), one entry per interior node (i, j) of each child (p, q) on
        // diagonal d-1: R_x from the x-parent (p+1, q) around its node (2i, j),
        // R_y from the y-parent (p, q+1) around its node (i, 2j)
        D.off[d][LK_RESTRICT] = (int)ent.size();
        for (int p = 1; p <= d; ++p) {
            const int q = d + 1 - p;
            if (!exists(p, q)) continue;
            const bool hx = exists(p + 1, q), hy = exists(p, q + 1);
            if (!hx && !hy) continue;  // only in classes no item has (pic + qic < dl + 2)
            const int nx = 1 << p, ny = 1 << q;
            for (int j = 1; j < ny; ++j)
                for (int i = 1; i < nx; ++i) {
                    const uint32_t rx = hx ? R(p + 1, q, 2 * i, j) : 0u, ry = hy ? R(p, q + 1, i, 2 * j) : 0u;
                    ent.push_back(make_uint4(U(p, q, i, j) | rx << 16, ry | (uint32_t)(nx - 1) << 16,
                                             (uint32_t)hx | (uint32_t)hy << 1, 0u));
                }
        }
        D.cnt[d][LK_RESTRICT] = (int)ent.size() - D.off[d][LK_RESTRICT];
        // Eq. (2.4)/(2.5): linear prolongation from each child, kappa-weighted
        D.off[d][LK_PROL] = (int)ent.size();
        for (int p = 1; p <= d + 1; ++p) {
            const int q = d + 2 - p;
            if (!exists(p, q)) continue;
            const int nx = 1 << p, ny = 1 << q;
            const bool hx = p > 1, hy = q > 1;
            for (int j = 1; j < ny; ++j)
                for (int i = 1; i < nx; ++i) {
                    const uint32_t cx0 = hx ? U(p - 1, q, i >> 1, j) : 0u, cx1 = hx ? U(p - 1, q, (i + 1) >> 1, j) : 0u;
                    const uint32_t cy0 = hy ? U(p, q - 1, i, j >> 1) : 0u, cy1 = hy ? U(p, q - 1, i, (j + 1) >> 1) : 0u;
                    ent.push_back(make_uint4(U(p, q, i, j) | XW(p, q, i, j) << 16, YS(p, q, i, j) | cx0 << 16,
                                             cx1 | cy0 << 16, cy1 | (uint32_t)hx << 16 | (uint32_t)hy << 17));
                }
        }
        D.cnt[d][LK_PROL] = (int)ent.size() - D.off[d][LK_PROL];
    }
    D.e1 = (int)ent.size();
}

static const LowTables& low_tables()
{
    static const LowTables tabs = [] {
        LowTables t;
        for (int dl = 0; dl <= kLowMax; ++dl) t.planes.push_back(low_planes(dl));
        t.desc.resize(kLowClassesMax);
        for (int dl = 0; dl <= kLowMax; ++dl)
            for (int pic = 1; pic <= dl + 1; ++pic)
                for (int qic = 1; qic <= dl + 1; ++qic)
                    low_build_class(pic, qic, dl, t.planes[dl], t.desc[low_class(pic, qic, dl)], t.ent);
        return t;
    }();
    return tabs;
}

// Algorithm 1 below diagonal dl as a flat program (the recursion unrolled): the
// visit of diagonal d smooths nu1 times, forms the residual and restricts it to
// diagonal d-1 (which also restarts the correction there from zero for the
// first of the mu visits), recurses mu times, prolongs and smooths nu2 times.
// Diagonal 0 is solved exactly (one unknown, u = b / A); its b does not change
// between the mu visits of one parent visit, so the repeats, which would write
// the same value, are left out.  The kernel starts every item from u = 0.
// With reg2, the mu calls below a diagonal-3 visit are one LK_CALL2 phase (the
// register path runs them for each item).
static void low_program_rec(int d, const msg_params& prm, bool reg2, std::vector<int>& prog)
{
    auto emit = [&](int kind, int dd) { prog.push_back(kind | dd << 3); };
    if (d == 0) { emit(LK_RED, 0); return; }
    for (int s = 0; s < prm.nu1; ++s) { emit(LK_RED, d); emit(LK_BLACK, d); }
    emit(LK_RESID, d);
    emit(LK_RESTRICT, d);
    if (reg2 && d == 3) emit(LK_CALL2, 2);
    else
        for (int k = 0; k < (d == 1 ? 1 : prm.mu); ++k) low_program_rec(d - 1, prm, reg2, prog);
    emit(LK_PROL, d);
    for (int s = 0; s < prm.nu2; ++s) { emit(LK_RED, d); emit(LK_BLACK, d); }
}

static std::vector<int> low_program(int dl, const msg_params& prm, bool reg2)
{
    std::vector<int> prog;
    low_program_rec(dl, prm, reg2, prog);
    return prog;
}

// Resolved programs of every class for these parameters: each (kind, diagonal)
// word becomes {kind | entries << 3, first entry relative to the class's e0};
// phases with no entries are dropped, and so is a residual phase whose
// restriction is empty.
static std::vector<uint2> low_resolve(const msg_params& prm, std::vector<LowDesc>& desc, bool reg2 = true)
{
    reg2 = reg2 && prm.precision == MSG_PREC_MIXED;  // the register path is built for FP32 cycles
    desc = low_tables().desc;
    std::vector<int> words[kLowMax + 1];
    for (int dl = 0; dl <= kLowMax; ++dl) words[dl] = low_program(dl, prm, reg2);
    std::vector<uint2> rp;
    for (LowDesc& D : desc) {
        D.prog = (int)rp.size();
        if (D.pic == 0) { D.nops = 0; continue; }
        for (int w : words[D.dl]) {
            const int kind = w & 7, d = w >> 3, cnt = D.cnt[d][kind];
            if (kind == LK_CALL2) {
                rp.push_back(make_uint2((uint32_t)LK_CALL2 | 1u << 3, 0u));
                continue;
            }
            if (cnt == 0) continue;
            if (kind == LK_RESID && D.cnt[d][LK_RESTRICT] == 0) continue;
            rp.push_back(make_uint2((uint32_t)kind | (uint32_t)cnt << 3, (uint32_t)(D.off[d][kind] - D.e0)));
        }
        D.nops = (int)rp.size() - D.prog;
    }
    return rp;
}

constexpr size_t kSmemMax = 227 * 1024;  // dynamic shared memory of one CTA
// Launch shape and cut of the low-diagonal kernel for these parameters.
struct LowShape {
    int cut;    // diagonals <= cut of a hierarchy run inside one k_lowv launch
    int items;  // items per warp (KW)
    int warps;  // warps per CTA
    int pcap[kLowMax + 1], ecap[kLowMax + 1];  // program words / entries of the largest class of each dl
    size_t smem[kLowMax + 1];                  // bytes per CTA of a launch at each dl
    double flops[kLowClassesMax];              // algorithmic FP operations of one mu-cycle of each class
};

// Algorithmic floating-point operations of one node entry of each phase kind
// (a reciprocal counts as one): smoothing 4 mul + 3 add for the neighbours, 3 add
// for the diagonal, rcp, add b, mul = 13; residual 4 + 3 + 3 + 1 mul + 2 sub +
// 1 sub = 14; restriction 2 x (2 add + 1 mul + 1 mul) + 3 = 11; prolongation
// 2 x (add + mul) + kappa (2 add, 2 mul, add, rcp, 2 mul) + 2 mul + add + fma = 16.
static double low_kind_flops(int kind)
{
    return kind <= LK_BLACK ? 13.0 : kind == LK_RESID ? 14.0 : kind == LK_RESTRICT ? 11.0 : 16.0;
}
static LowShape low_shape_at(const msg_params& prm, int cut, int items, int warps)
{
    const size_t es = prm.precision == MSG_PREC_MIXED ? sizeof(float) : sizeof(double);
    const LowTables& lt = low_tables();
    std::vector<LowDesc> desc;
    low_resolve(prm, desc);
    LowShape s;
    s.cut = cut;
    s.items = items;
    s.warps = warps;
    for (int dl = 0; dl <= kLowMax; ++dl) {
        s.pcap[dl] = s.ecap[dl] = 0;
        for (const LowDesc& D : desc)
            if (D.dl == dl) {
                s.pcap[dl] = std::max(s.pcap[dl], D.nops);
                s.ecap[dl] = std::max(s.ecap[dl], D.e1 - D.e0);
            }
        s.pcap[dl] = (s.pcap[dl] + 1) & ~1;  // whole 16-byte chunks: the planes after it start 16-byte aligned
        s.smem[dl] = sizeof(uint4) * s.ecap[dl] + sizeof(uint2) * s.pcap[dl] +
                     es * (size_t)low_stride(lt.planes[dl], items, es) * items * warps;
    }
    // work of one mu-cycle per class, counted on the all-table program (the register
    // path below diagonal 3 does the same node updates)
    std::vector<LowDesc> dt;
    const std::vector<uint2> rpt = low_resolve(prm, dt, false);
    for (int c = 0; c < kLowClassesMax; ++c) {
        double f = 0.0;
        for (int o = 0; o < dt[c].nops; ++o) {
            const uint2 w = rpt[dt[c].prog + o];
            f += (double)(w.x >> 3) * low_kind_flops((int)(w.x & 7));
        }
        s.flops[c] = f;
    }
    return s;
}
// Defaults (the fastest measured at 256 x 256): cut 4 with two items per warp
// and 16 warps per CTA for FP32 cycles (S = 4096), cut 4 with one item per warp
// and 8 warps for FP64 (S = 256: 16 samples/s against 9 with 16 warps, whose
// larger CTAs leave SMs idle on small batches).  With long programs (large mu or
// nu) the default cut drops until the CTA fits the shared memory.
static LowShape low_shape(const msg_params& prm)
{
    const bool mixed = prm.precision == MSG_PREC_MIXED;
    const int items = prm.tune_low_items ? prm.tune_low_items : (mixed ? 2 : 1);
    const int warps = prm.tune_low_warps ? prm.tune_low_warps : (mixed ? 16 : 8);
    if (prm.tune_low_cut) return low_shape_at(prm, prm.tune_low_cut, items, warps);
    for (int cut = 4; cut > 1; --cut) {
        LowShape s = low_shape_at(prm, cut, items, warps);
        if (s.smem[cut] <= 227 * 1024) return s;
    }
    return low_shape_at(prm, 1, items, warps);
}

struct Plan {
    int S = 0;
    std::vector<SampleInfo> samples;
    std::vector<int> perm;  // samples ordered by group
    std::vector<int> gpos;  // position of each sample inside its group
    std::vector<int> sgroup; // group of each sample
    std::vector<Group> groups;
    int Lmax = -1;
    std::vector<std::vector<Group>> stage_groups;   // [L]: groups with the stage's scratch layout
    std::vector<std::vector<ItemType>> stage_items; // [L]
    std::vector<int64_t> stage_nitems;              // [L]: flags (items) of the stage
    std::vector<Segment> all_segs;                  // one segment per grid type over all samples
    int64_t total_nodes = 0, total_field = 0, total_q = 0, scratch_nodes = 0;
    int64_t max_stage_items = 0, max_segs = 0;
};

int validate(const int32_t* PQ, int64_t S, const msg_params* prm)
{
    if (S < 0) { set_error("S < 0"); return MSG_ERR_INVALID; }
    if (S > (int64_t)1 << 30) { set_error("S too large"); return MSG_ERR_INVALID; }
    if (S > 0 && !PQ) { set_error("PQ is NULL"); return MSG_ERR_INVALID; }
    if (!prm) { set_error("params is NULL"); return MSG_ERR_INVALID; }
    if (prm->mu < 1 || prm->mu > 3 || prm->nu1 < 0 || prm->nu2 < 0 || prm->nu1 + prm->nu2 < 1 ||
        prm->nu1 > 64 || prm->nu2 > 64 || prm->max_cycles < 1 || !(prm->eps >= 0.0) || !(prm->omega > 0.0) || prm->omega > 2.0) {
        set_error("invalid solver parameters");
        return MSG_ERR_INVALID;
    }
    if (prm->precision != MSG_PREC_FP64 && prm->precision != MSG_PREC_MIXED) {
        set_error("precision must be MSG_PREC_FP64 or MSG_PREC_MIXED");
        return MSG_ERR_INVALID;
    }
    if (prm->qoi < 0 || prm->qoi > 3) { set_error("qoi out of range"); return MSG_ERR_INVALID; }
    if (prm->tune_block != 0 && (prm->tune_block < 32 || prm->tune_block > 1024 || prm->tune_block % 32)) {
        set_error("tune_block must be 0 or a multiple of 32 in [32, 1024]");
        return MSG_ERR_INVALID;
    }
    if (prm->tune_low_items != 0 && prm->tune_low_items != 1 && prm->tune_low_items != 2 &&
        prm->tune_low_items != 4 && prm->tune_low_items != 8) {
        set_error("tune_low_items must be 0, 1, 2, 4 or 8");
        return MSG_ERR_INVALID;
    }
    if (prm->tune_low_warps < 0 || prm->tune_low_warps > kLowWarpsMax) {
        set_error("tune_low_warps must be in [0, 16]");
        return MSG_ERR_INVALID;
    }
    if (prm->tune_low_cut < 0 || prm->tune_low_cut > kLowMax) {
        set_error("tune_low_cut must be in [0, 5]");
        return MSG_ERR_INVALID;
    }
    if (prm->tune_visit_smem < 0 || prm->tune_visit_smem > 227) {
        set_error("tune_visit_smem must be in [0, 227] (KB)");
        return MSG_ERR_INVALID;
    }
    const LowShape ls = low_shape(*prm);
    if (ls.smem[ls.cut] > kSmemMax) {
        set_error("tune_low_warps x tune_low_items items of the low-diagonal kernel do not fit the shared memory of one CTA");
        return MSG_ERR_INVALID;
    }
    if (prm->coef != MSG_COEF_SERIES && prm->coef != MSG_COEF_INJECT) {
        set_error("coef must be MSG_COEF_SERIES or MSG_COEF_INJECT");
        return MSG_ERR_INVALID;
    }
    for (int64_t i = 0; i < S; ++i) {
        if (PQ[2 * i] < 1 || PQ[2 * i] > 12 || PQ[2 * i + 1] < 1 || PQ[2 * i + 1] > 12) {
            set_error("grid exponents must satisfy 1 <= P, Q <= 12");
            return MSG_ERR_INVALID;
        }
    }
    return MSG_OK;
}

void build_plan(const int32_t* PQ, int64_t S, Plan& pl)
{
    pl.S = (int)S;
    pl.samples.resize(S);
    std::map<std::pair<int, int>, int> gid;
    std::vector<int> sample_group(S);
    for (int64_t i = 0; i < S; ++i) {
        SampleInfo& si = pl.samples[i];
        si.P = PQ[2 * i];
        si.Q = PQ[2 * i + 1];
        si.node_off = pl.total_nodes;
        si.field_off = pl.total_field;
        si.q_off = pl.total_q;
        pl.total_nodes += rect_nodes(si.P, si.Q);
        pl.total_field += field_nodes(si.P, si.Q);
        pl.total_q += (int64_t)si.P * si.Q;
        auto key = std::make_pair(si.P, si.Q);
        auto it = gid.find(key);
        if (it == gid.end()) {
            int g = (int)pl.groups.size();
            gid[key] = g;
            Group G{};
            G.P = si.P;
            G.Q = si.Q;
            pl.groups.push_back(G);
            sample_group[i] = g;
        } else {
            sample_group[i] = it->second;
        }
        pl.Lmax = std::max(pl.Lmax, si.P + si.Q - 2);
    }
    std::vector<int> cnt(pl.groups.size(), 0);
    for (int64_t i = 0; i < S; ++i) cnt[sample_group[i]]++;
    int acc = 0;
    for (size_t g = 0; g < pl.groups.size(); ++g) {
        pl.groups[g].start = acc;
        pl.groups[g].count = cnt[g];
        acc += cnt[g];
        cnt[g] = pl.groups[g].start;
    }
    pl.perm.resize(S);
    pl.gpos.resize(S);
    pl.sgroup = sample_group;
    for (int64_t i = 0; i < S; ++i) {
        int g = sample_group[i];
        pl.gpos[i] = cnt[g] - pl.groups[g].start;
        pl.perm[cnt[g]++] = (int)i;
    }
    int64_t blk = 0;
    for (size_t g = 0; g < pl.groups.size(); ++g)
        for (int p = 1; p <= pl.groups[g].P; ++p)
            for (int q = 1; q <= pl.groups[g].Q; ++q) {
                Segment sg{(int)g, p, q, p, q, blk, pl.groups[g].count, pl.groups[g].start, 0, 0};
                pl.all_segs.push_back(sg);
                blk += pl.groups[g].count;
            }
    pl.stage_groups.assign(pl.Lmax + 1, pl.groups);
    pl.stage_items.assign(pl.Lmax + 1, {});
    pl.stage_nitems.assign(pl.Lmax + 1, 0);
    for (int L = 0; L <= pl.Lmax; ++L) {
        std::vector<Group>& sg = pl.stage_groups[L];
        int64_t scr = 0, base = 0, nseg = 0;
        for (size_t g = 0; g < sg.size(); ++g) {
            int64_t per = 0;
            for (int p = 1; p <= sg[g].P; ++p) {
                int q = L + 2 - p;
                if (q < 1 || q > sg[g].Q) continue;
                pl.stage_items[L].push_back(ItemType{(int)g, p, q, per, base});
                per += rect_nodes(p, q);
                base += sg[g].count;
                nseg += (int64_t)p * q;  // tasks of all diagonals of this item's hierarchy
            }
            sg[g].scr_start = scr;
            sg[g].scr_per_sample = per;
            scr += per * sg[g].count;
        }
        pl.stage_nitems[L] = base;
        pl.scratch_nodes = std::max(pl.scratch_nodes, scr);
        pl.max_stage_items = std::max(pl.max_stage_items, base);
        pl.max_segs = std::max(pl.max_segs, nseg + (int64_t)pl.stage_items[L].size());
    }
}

struct WsLayout {
    size_t samples, perm, gpos, groups, allsegs;
    size_t nstep, cycles_i, relres_i;
    size_t u64, ax64, ay64, ax32, ay32;
    size_t low_desc, low_ent, low_prog;  // tables of the low-diagonal program
    size_t low_img;                      // per-sample face images of the low-diagonal kernel
    // per stage L: segment list, sample list, flags, counter, scratch (su, sbx, sby)
    std::vector<size_t> segs, tasks, slist, sflag, counter, su, sbx, sby;
    size_t total;
};

WsLayout layout_of(const Plan& pl, const msg_params& prm)
{
    const int precision = prm.precision;
    WsLayout w{};
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + std::max<size_t>(bytes, 1)); return o; };
    w.samples = take(sizeof(SampleInfo) * pl.S);
    w.perm = take(sizeof(int) * pl.S);
    w.gpos = take(sizeof(int) * pl.S);
    w.groups = take(sizeof(Group) * pl.groups.size() * (pl.Lmax + 2));
    w.allsegs = take(sizeof(Segment) * pl.all_segs.size());
    {
        std::vector<LowDesc> desc;
        w.low_desc = take(sizeof(LowDesc) * kLowClassesMax);
        w.low_ent = take(sizeof(uint4) * low_tables().ent.size());
        w.low_prog = take(sizeof(uint2) * low_resolve(prm, desc).size());
    }
    {
        const LowPlanes& lp = low_tables().planes[kLowMax];
        const size_t es_img = precision == MSG_PREC_MIXED ? sizeof(float) : sizeof(double);
        w.low_img = take(es_img * (size_t)pl.S * (lp.nfx + lp.nfy));
    }
    w.nstep = take(sizeof(int) * pl.total_q);
    w.cycles_i = take(sizeof(int) * pl.total_q);
    w.relres_i = take(sizeof(double) * pl.total_q);
    w.u64 = take(sizeof(double) * pl.total_nodes);
    w.ax64 = take(sizeof(double) * pl.total_nodes);
    w.ay64 = take(sizeof(double) * pl.total_nodes);
    const size_t es = precision == MSG_PREC_MIXED ? sizeof(float) : sizeof(double);
    if (precision == MSG_PREC_MIXED) {
        w.ax32 = take(sizeof(float) * pl.total_nodes);
        w.ay32 = take(sizeof(float) * pl.total_nodes);
    }
    for (int L = 0; L <= pl.Lmax; ++L) {
        int64_t nseg = 0, scr = 0;
        for (const ItemType& it : pl.stage_items[L]) nseg += 1 + (int64_t)it.pi * it.qi;
        for (const Group& g : pl.stage_groups[L]) scr += g.scr_per_sample * g.count;
        w.segs.push_back(take(sizeof(Segment) * nseg));
        w.tasks.push_back(take(sizeof(LowTask) * (pl.stage_nitems[L] + pl.stage_items[L].size() * kLowWarpsMax)));
        w.slist.push_back(take(sizeof(int) * pl.stage_nitems[L]));
        w.sflag.push_back(take(sizeof(int) * pl.stage_nitems[L]));
        w.counter.push_back(take(sizeof(int) * 4));
        w.su.push_back(take(es * scr));
        w.sbx.push_back(take(es * scr));
        w.sby.push_back(take(es * scr));
    }
    w.total = off + 256;
    return w;
}

constexpr int kThreads = 256;
constexpr int kVisitThreads = 128;       // threads per CTA of the PRE/POST visit kernels (default)
constexpr int kBandNodes = 4096;         // residual band of the restriction in shared memory (nodes)
// Register-cached visits: default shared-memory limit per CTA (KB).  1 KB keeps every
// visit in global memory: at 256 x 256 the register-cached visits measured no faster on
// diagonals 5..7 and slower on 8..10 (fewer resident CTAs at their register count).
constexpr int kVisitSmemKB = 1;


// Host staging for the per-step lists (pinned so the uploads are asynchronous).
struct Pinned {
    void* p = nullptr;
    ~Pinned() { if (p) cudaFreeHost(p); }
    int alloc(size_t b)
    {
        if (cudaMallocHost(&p, std::max<size_t>(b, 64)) != cudaSuccess) { p = nullptr; return MSG_ERR_CUDA; }
        return MSG_OK;
    }
};

// Hand-over of samples between the stage workers.
struct StageQueues {
    std::mutex mu;
    std::condition_variable cv;
    std::vector<std::vector<int>> ready;  // [L]: samples whose stage L may start
    std::vector<char> done;               // [L]: stage L worker finished
    bool abort = false;
};

}  // namespace

// ------------------------------------------------------------- entry point --

// Everything one stage worker needs (shared, read-only during the solve).
template <class T>
struct SolveCtx {
    const Plan& pl;
    const WsLayout& wl;
    char* ws;
    const msg_params& prm;
    const double* Z;
    int32_t* stat;
    DevCtx base;
    const Group* dgroups;
    double* u64;
    const double* ax64;
    const double* ay64;
    const T* ax;
    const T* ay;
    int* nstep;
    int* cyc;
    double* rel;
    CycleParams cp;
    int block;      // threads per CTA of the PRE/POST visit kernels
    size_t visit_smem;  // shared memory up to which a visit runs on a shared copy of its grid
    LowShape low;   // cut and launch shape of the low-diagonal kernel
    const LowDesc* low_desc;
    const uint4* low_ent;
    const uint2* low_prog;  // resolved programs of all classes
};

// Stage L of FMSG for the samples handed over by stage L-1: cubic
// interpolation when a sample enters, then defect-correction cycles of every
// item until it meets eps (or stops), each step on this stage's own stream.
// A sample moves on to stage L+1 as soon as all its stage-L items are done.
template <class T>
static int stage_worker(const SolveCtx<T>& C, int L, StageQueues& Qs, cudaStream_t st)
{
    const Plan& pl = C.pl;
    const WsLayout& wl = C.wl;
    const std::vector<ItemType>& its = pl.stage_items[L];
    const std::vector<Group>& hsg = pl.stage_groups[L];
    const size_t ng = pl.groups.size();
    const Group* sg = C.dgroups + ng * (1 + L);
    T* su = (T*)(C.ws + wl.su[L]);
    T* sbx = (T*)(C.ws + wl.sbx[L]);
    T* sby = (T*)(C.ws + wl.sby[L]);
    int* sflag = (int*)(C.ws + wl.sflag[L]);
    int* slist = (int*)(C.ws + wl.slist[L]);
    int* counter = (int*)(C.ws + wl.counter[L]);
    Segment* dsegs = (Segment*)(C.ws + wl.segs[L]);
    LowTask* dtasks = (LowTask*)(C.ws + wl.tasks[L]);
    const int cut = C.low.cut;
    const double es = sizeof(T);

    // item types of each group at this stage, and per-sample countdown of open items
    std::vector<std::vector<int>> types_of(ng);
    for (size_t k = 0; k < its.size(); ++k) types_of[its[k].g].push_back((int)k);
    std::vector<int> open(pl.S, 0);

    int64_t nseg_max = 0;
    for (const ItemType& it : its) nseg_max += 1 + (int64_t)it.pi * it.qi;
    Pinned pin;
    const size_t flag_bytes = sizeof(int) * std::max<int64_t>(pl.stage_nitems[L], 1);
    const size_t seg_bytes = sizeof(Segment) * std::max<int64_t>(nseg_max, 1);
    const size_t task_bytes = sizeof(LowTask) * (pl.stage_nitems[L] + its.size() * C.low.warps + 1);
    if (pin.alloc(64 + 2 * flag_bytes + seg_bytes + task_bytes) != MSG_OK) {
        set_error("cudaMallocHost failed");
        return MSG_ERR_CUDA;
    }
    int* h_counter = (int*)pin.p;
    int* h_flags = (int*)((char*)pin.p + 64);
    int* h_list = (int*)((char*)pin.p + 64 + flag_bytes);
    Segment* h_segs = (Segment*)((char*)pin.p + 64 + 2 * flag_bytes);
    LowTask* h_tasks = (LowTask*)((char*)pin.p + 64 + 2 * flag_bytes + seg_bytes);
    int ntasks = 0;

    std::vector<std::vector<int>> active(its.size()), fresh(its.size());
    size_t item_nseg = 0;
    std::vector<size_t> dseg0(L + 1, 0), dnseg(L + 1, 0);
    std::vector<double> dpre(L + 1, 0), dpost(L + 1, 0);
    int64_t nitems = 0;
    double item_pts = 0, low_bytes = 0, low_flops = 0;
    // Upload per-item sample lists and segments for `lists` (item level first,
    // then one list per diagonal above the warp cut when with_diag).
    auto build_lists = [&](const std::vector<std::vector<int>>& lists, bool with_diag) -> int {
        std::vector<int64_t> loff(its.size());
        int64_t nl = 0;
        item_pts = 0;
        for (size_t k = 0; k < its.size(); ++k) {
            loff[k] = nl;
            for (int s : lists[k]) h_list[nl++] = s;
            item_pts += (double)lists[k].size() * pts(its[k].pi, its[k].qi);
        }
        nitems = nl;
        size_t ns = 0;
        int64_t b = 0;
        for (size_t k = 0; k < its.size(); ++k) {
            if (lists[k].empty()) continue;
            const ItemType& it = its[k];
            h_segs[ns++] = Segment{it.g, it.pi, it.qi, it.pi, it.qi, b, (int64_t)lists[k].size(), loff[k], it.scr_slot,
                                   it.stage_base};
            b += (int64_t)lists[k].size();
        }
        item_nseg = ns;
        if (with_diag) {
            const int dl = std::min(L, cut);
            // warp tasks of the low-diagonal kernel: up to KW items of one segment (one class) each
            // (the warps of a CTA take tasks of one segment: idle warps pad each segment's last CTA)
            ntasks = 0;
            low_flops = 0;
            for (size_t k = 0; k < ns; ++k) {
                const Segment& sgk = h_segs[k];
                const int cls = low_class(std::min(sgk.pi, dl + 1), std::min(sgk.qi, dl + 1), dl);
                low_flops += (double)sgk.count * C.low.flops[cls];
                for (int64_t f = 0; f < sgk.count; f += C.low.items)
                    h_tasks[ntasks++] = LowTask{(int)k, (int)f, (int)std::min<int64_t>(C.low.items, sgk.count - f), cls};
                while (ntasks % C.low.warps) h_tasks[ntasks++] = LowTask{(int)k, 0, 0, cls};
            }
            low_bytes = 0;
            for (size_t k = 0; k < its.size(); ++k)
                for (int pp = 1; pp <= its[k].pi; ++pp)
                    for (int qq = 1; qq <= its[k].qi; ++qq) {
                        const int dd = pp + qq - 2;
                        if (dd > dl) continue;
                        const double n = (double)lists[k].size() * pts(pp, qq);
                        low_bytes += n * 2;
                        if (dd == dl) low_bytes += n * ((pp < its[k].pi && qq < its[k].qi) ? 3 : 2);
                    }
            low_bytes *= es;
            for (int d = cut + 1; d <= L; ++d) {
                dseg0[d] = ns;
                b = 0;
                dpre[d] = dpost[d] = 0;
                for (size_t k = 0; k < its.size(); ++k) {
                    if (lists[k].empty()) continue;
                    const ItemType& it = its[k];
                    for (int pp = std::max(1, d + 2 - it.qi); pp <= std::min(it.pi, d + 1); ++pp) {
                        const int qq = d + 2 - pp;
                        h_segs[ns++] = Segment{it.g, it.pi, it.qi, pp, qq, b, (int64_t)lists[k].size(), loff[k],
                                               it.scr_slot, it.stage_base};
                        b += (int64_t)lists[k].size();
                        const double n = (double)lists[k].size() * pts(pp, qq);
                        const double bw = (pp < it.pi && qq < it.qi) ? 2.0 : 1.0;
                        const double ch = (pp > 1 ? 0.5 : 0.0) + (qq > 1 ? 0.5 : 0.0);
                        dpre[d] += n * (bw + 2 + 1 + ch);
                        dpost[d] += n * (ch + bw + 2 + 2);
                    }
                }
                dnseg[d] = ns - dseg0[d];
            }
        }
        MSG_CUDA_TRY(cudaMemcpyAsync(slist, h_list, sizeof(int) * std::max<int64_t>(nl, 1), cudaMemcpyHostToDevice, st));
        MSG_CUDA_TRY(cudaMemcpyAsync(dsegs, h_segs, sizeof(Segment) * std::max<size_t>(ns, 1), cudaMemcpyHostToDevice,
                                     st));
        if (with_diag && ntasks > 0)
            MSG_CUDA_TRY(cudaMemcpyAsync(dtasks, h_tasks, sizeof(LowTask) * ntasks, cudaMemcpyHostToDevice, st));
        return MSG_OK;
    };
    auto ctx_of = [&](size_t seg0, size_t n) {
        DevCtx c = C.base;
        c.slist = slist;
        c.groups = sg;
        c.segs = dsegs + seg0;
        c.nseg = (int)n;
        return c;
    };
    auto finish = [&](int rc) {
        std::lock_guard<std::mutex> lk(Qs.mu);
        Qs.done[L] = 1;
        if (rc != MSG_OK) Qs.abort = true;
        Qs.cv.notify_all();
        return rc;
    };
    int64_t open_items = 0;
    // optional per-stage statistics on stderr (MSG_STAGE_STATS=1)
    static const bool stats = getenv("MSG_STAGE_STATS") != nullptr;
    int64_t n_steps = 0, n_item_cycles = 0, n_admitted = 0;
    const auto t_start = std::chrono::steady_clock::now();
    double t_first = -1.0;
    struct StatsOut {
        bool on; int L; int64_t *st, *ic, *ad; double* tf; std::chrono::steady_clock::time_point t0;
        ~StatsOut()
        {
            if (!on) return;
            double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            fprintf(stderr, "[stage %2d] admitted %lld steps %lld item-cycles %lld first-admit %.1f ms done %.1f ms\n", L,
                    (long long)*ad, (long long)*st, (long long)*ic, *tf, ms);
        }
    } stats_out{stats, L, &n_steps, &n_item_cycles, &n_admitted, &t_first, t_start};
    for (;;) {
        // ---- admit the samples stage L-1 has finished
        std::vector<int> admitted;
        {
            std::unique_lock<std::mutex> lk(Qs.mu);
            // MSG_SERIAL_STAGES=1 (diagnostics): stage L starts only once stage L-1 is finished
            static const bool serial = getenv("MSG_SERIAL_STAGES") != nullptr;
            if (serial && L > 0) Qs.cv.wait(lk, [&] { return Qs.abort || Qs.done[L - 1]; });
            if (open_items == 0)
                Qs.cv.wait(lk, [&] { return Qs.abort || !Qs.ready[L].empty() || (L == 0 || Qs.done[L - 1]); });
            if (Qs.abort) return finish(MSG_OK);
            admitted.swap(Qs.ready[L]);
            if (admitted.empty() && open_items == 0 && (L == 0 || Qs.done[L - 1])) break;
        }
        // the previous step's uploads read the pinned staging that is rewritten below
        if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("stage stream failed"); return finish(MSG_ERR_CUDA); }
        if (!admitted.empty()) {
            n_admitted += (int64_t)admitted.size();
            if (t_first < 0)
                t_first = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
            for (auto& f : fresh) f.clear();
            std::vector<int> pass_on;
            for (int s : admitted) {
                const int g = pl.sgroup[s];
                if (types_of[g].empty()) { pass_on.push_back(s); continue; }  // no grid of this sample at stage L
                open[s] = (int)types_of[g].size();
                open_items += open[s];
                for (int k : types_of[g]) fresh[k].push_back(s);
            }
            if (!pass_on.empty() && L < pl.Lmax) {
                std::lock_guard<std::mutex> lk(Qs.mu);
                for (int s : pass_on) Qs.ready[L + 1].push_back(s);
                Qs.cv.notify_all();
            }
            int rc = build_lists(fresh, false);
            if (rc != MSG_OK) return finish(rc);
            if (nitems > 0) {
                prof_begin(K_INTERP, st);
                k_interp<<<(unsigned)nitems, kThreads, 0, st>>>(ctx_of(0, item_nseg), C.u64, C.ax64, C.ay64);
                prof_end(K_INTERP, st, item_pts * (8.0 + 16.0 + 8.0), 0.0);
                if (cudaGetLastError() != cudaSuccess) { set_error("k_interp launch"); return finish(MSG_ERR_CUDA); }
            }
            for (size_t k = 0; k < its.size(); ++k) active[k].insert(active[k].end(), fresh[k].begin(), fresh[k].end());
            if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("stage stream failed"); return finish(MSG_ERR_CUDA); }
        }
        if (open_items == 0) continue;
        // ---- residual, convergence decision
        int rc = build_lists(active, false);
        if (rc != MSG_OK) return finish(rc);
        if (cudaMemsetAsync(counter, 0, sizeof(int), st) != cudaSuccess) return finish(MSG_ERR_CUDA);
        prof_begin(K_RESIDUAL, st);
        k_residual<T><<<(unsigned)nitems, kThreads, 0, st>>>(ctx_of(0, item_nseg), C.u64, C.ax64, C.ay64, sbx,
                                                             C.prm.max_cycles, C.prm.eps, C.nstep, sflag, C.cyc,
                                                             C.rel, C.stat, counter);
        prof_end(K_RESIDUAL, st, item_pts * (24.0 + es), 0.0);
        if (cudaGetLastError() != cudaSuccess) { set_error("k_residual launch"); return finish(MSG_ERR_CUDA); }
        if (cudaMemcpyAsync(h_counter, counter, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(h_flags, sflag, sizeof(int) * pl.stage_nitems[L], cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("stage step synchronisation failed");
            return finish(MSG_ERR_CUDA);
        }
        // ---- retire finished items; samples whose stage-L items are all done move on
        std::vector<int> completed;
        for (size_t k = 0; k < its.size(); ++k) {
            std::vector<int>& a = active[k];
            size_t w = 0;
            for (size_t r = 0; r < a.size(); ++r) {
                const int s = a[r];
                if (h_flags[its[k].stage_base + pl.gpos[s]]) { a[w++] = s; continue; }
                --open_items;
                if (--open[s] == 0) completed.push_back(s);
            }
            a.resize(w);
        }
        if (!completed.empty() && L < pl.Lmax) {
            std::lock_guard<std::mutex> lk(Qs.mu);
            for (int s : completed) Qs.ready[L + 1].push_back(s);
            Qs.cv.notify_all();
        }
        if (*h_counter == 0) continue;
        ++n_steps;
        n_item_cycles += *h_counter;
        // ---- one mu-cycle (Algorithm 1) of every active item
        rc = build_lists(active, true);
        if (rc != MSG_OK) return finish(rc);
        DevCtx ic = ctx_of(0, item_nseg);
        bool launch_err = false;
        auto launch_low = [&](int d, int calls) {
            if (ntasks == 0) return;
            const LowPlanes& lp = low_tables().planes[d];
            const int wpb = C.low.warps;
            const unsigned nb = (unsigned)(ntasks / wpb);  // tasks are padded to whole CTAs
            const int stride = low_stride(lp, C.low.items, sizeof(T));
            const size_t smem = C.low.smem[d];
            const int pc = C.low.pcap[d], ec = C.low.ecap[d];
            const CycleParams om = C.cp;
            const LowPlanes& lpm = low_tables().planes[kLowMax];
            const T* img = (const T*)(C.ws + wl.low_img);
            const int64_t istr = lpm.nfx + lpm.nfy;
            const int ify = lpm.nfx;
            prof_begin(K_LOW, st);
            switch (C.low.items) {
            case 1: k_lowv<T, 1><<<nb, 32 * wpb, smem, st>>>(ic, dtasks, su, sbx, sby, img, istr, ify, C.low_desc, C.low_ent,
                                                            C.low_prog, lp, stride, pc, ec, calls, om); break;
            case 2: k_lowv<T, 2><<<nb, 32 * wpb, smem, st>>>(ic, dtasks, su, sbx, sby, img, istr, ify, C.low_desc, C.low_ent,
                                                            C.low_prog, lp, stride, pc, ec, calls, om); break;
            case 4: k_lowv<T, 4><<<nb, 32 * wpb, smem, st>>>(ic, dtasks, su, sbx, sby, img, istr, ify, C.low_desc, C.low_ent,
                                                            C.low_prog, lp, stride, pc, ec, calls, om); break;
            default: k_lowv<T, 8><<<nb, 32 * wpb, smem, st>>>(ic, dtasks, su, sbx, sby, img, istr, ify, C.low_desc, C.low_ent,
                                                             C.low_prog, lp, stride, pc, ec, calls, om); break;
            }
            prof_end(K_LOW, st, low_bytes, low_flops * calls, d);
            launch_err |= cudaGetLastError() != cudaSuccess;
        };
        auto launch_half = [&](int d, int pre, int zi) {
            if (dnseg[d] == 0) return;
            DevCtx c = ctx_of(dseg0[d], dnseg[d]);
            prof_begin(pre ? K_PRE : K_POST, st);
            int64_t maxc = 0;
            for (size_t k = dseg0[d]; k < dseg0[d] + dnseg[d]; ++k) maxc = std::max<int64_t>(maxc, h_segs[k].count);
            const dim3 g2((unsigned)maxc, (unsigned)dnseg[d]);  // x: sample in segment, y: segment
            // threads per CTA: every grid of diagonal d has 2^(d+2) cells, 2^(d+1) points per
            // colour; small grids get no idle warps, the big ones (d >= 10) twice the block
            const int vb = d >= 10 ? std::min(2 * C.block, 1024) : std::min(C.block, std::max(32, 1 << (d + 1)));
            // register-cached visit when every grid of the launch has at most
            // kRegThreadsMax x NPT nodes of a colour and its shared planes (u; PRE also r)
            // fit the limit; else the global-memory visit
            const int nu = pre ? C.prm.nu1 : C.prm.nu2;
            int64_t nodes = 0, nslot = 0;
            for (size_t k = dseg0[d]; k < dseg0[d] + dnseg[d]; ++k) {
                const int sp = h_segs[k].p, sq = h_segs[k].q;
                nodes = std::max<int64_t>(nodes, (int64_t)((1 << sp) + 1) * ((1 << sq) + 1));
                nslot = std::max<int64_t>(nslot, (int64_t)((1 << sq) - 1) << (sp - 1));
            }
            const int nptmax = sizeof(T) == 4 ? 4 : 2;  // FP64 nodes take twice the registers
            int npt = 1;
            while (npt < nptmax && (nslot + npt - 1) / npt > C.block) npt *= 2;
            const int vr = (int)std::max<int64_t>(32, ((nslot + npt - 1) / npt + 31) / 32 * 32);
            const size_t rsm = (pre ? 2 : 1) * (size_t)nodes * sizeof(T);
            if (vr <= kRegThreadsMax && rsm <= C.visit_smem) {
                const double om = C.prm.omega;
                if (npt == 1) k_visit_reg<T, 1><<<g2, vr, rsm, st>>>(c, su, sbx, sby, C.ax, C.ay, pre, zi, nu, om);
                else if (npt == 2) k_visit_reg<T, 2><<<g2, vr, rsm, st>>>(c, su, sbx, sby, C.ax, C.ay, pre, zi, nu, om);
                else if constexpr (sizeof(T) == 4)
                    k_visit_reg<T, 4><<<g2, vr, rsm, st>>>(c, su, sbx, sby, C.ax, C.ay, pre, zi, nu, om);
            } else if (pre) {
                // residual band of the restriction: the whole grid when it has at most
                // kBandNodes nodes, else bands of at least 3 rows
                int band = 0;
                for (size_t k = dseg0[d]; k < dseg0[d] + dnseg[d]; ++k) {
                    const int W = (1 << h_segs[k].p) + 1, n = W * ((1 << h_segs[k].q) + 1);
                    band = std::max(band, std::min(n, std::max(kBandNodes, 3 * W)));
                }
                k_pre<T><<<g2, vb, sizeof(T) * band, st>>>(c, su, sbx, sby, C.ax, C.ay, zi, C.prm.nu1, band);
            } else {
                k_post<T><<<g2, vb, 0, st>>>(c, su, sbx, sby, C.ax, C.ay, C.prm.nu2, C.prm.omega);
            }
            prof_end(pre ? K_PRE : K_POST, st, (pre ? dpre[d] : dpost[d]) * es, 0.0, d);
            launch_err |= cudaGetLastError() != cudaSuccess;
        };
        if (L <= cut) {
            launch_low(L, 1);
        } else {
            struct Frame { int d, k, zi, phase; };
            std::vector<Frame> stack;
            stack.push_back({L, 0, 1, 0});
            while (!stack.empty()) {
                Frame& f = stack.back();
                if (f.phase == 0) {
                    launch_half(f.d, 1, f.zi);
                    f.phase = 1;
                    if (f.d - 1 <= cut) {
                        launch_low(f.d - 1, C.prm.mu);
                        f.phase = 2;
                    }
                    continue;
                }
                if (f.phase == 1) {
                    if (f.k < C.prm.mu) {
                        const int zi = (f.k == 0);
                        f.k += 1;
                        stack.push_back({f.d - 1, 0, zi, 0});
                        continue;
                    }
                    f.phase = 2;
                }
                launch_half(f.d, 0, 0);
                stack.pop_back();
            }
        }
        if (launch_err) { set_error("kernel launch failed in the cycle schedule"); return finish(MSG_ERR_CUDA); }
        prof_begin(K_UPDATE, st);
        k_update<T><<<(unsigned)nitems, kThreads, 0, st>>>(ic, C.u64, su);
        prof_end(K_UPDATE, st, item_pts * (16.0 + es), 0.0);
        if (cudaGetLastError() != cudaSuccess) { set_error("k_update launch"); return finish(MSG_ERR_CUDA); }
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return finish(MSG_ERR_CUDA);
    return finish(MSG_OK);
}

template <class T>
static int run_solve(const Plan& pl, const WsLayout& wl, char* ws, const msg_params& prm, const double* Z,
                     double* Qout, int32_t* stat, int32_t* cycles_out, double* relres_out, cudaStream_t st)
{
    const bool mixed = prm.precision == MSG_PREC_MIXED;
    std::vector<Group> gtab;  // [0]: groups, [1+L]: stage L groups
    gtab.insert(gtab.end(), pl.groups.begin(), pl.groups.end());
    for (int L = 0; L <= pl.Lmax; ++L) gtab.insert(gtab.end(), pl.stage_groups[L].begin(), pl.stage_groups[L].end());
    MSG_CUDA_TRY(cudaMemcpyAsync(ws + wl.samples, pl.samples.data(), sizeof(SampleInfo) * pl.S, cudaMemcpyHostToDevice, st));
    MSG_CUDA_TRY(cudaMemcpyAsync(ws + wl.perm, pl.perm.data(), sizeof(int) * pl.S, cudaMemcpyHostToDevice, st));
    MSG_CUDA_TRY(cudaMemcpyAsync(ws + wl.gpos, pl.gpos.data(), sizeof(int) * pl.S, cudaMemcpyHostToDevice, st));
    MSG_CUDA_TRY(cudaMemcpyAsync(ws + wl.groups, gtab.data(), sizeof(Group) * gtab.size(), cudaMemcpyHostToDevice, st));
    MSG_CUDA_TRY(cudaMemcpyAsync(ws + wl.allsegs, pl.all_segs.data(), sizeof(Segment) * pl.all_segs.size(),
                                 cudaMemcpyHostToDevice, st));
    SolveCtx<T> C{pl, wl, ws, prm, Z, stat, DevCtx{}, (const Group*)(ws + wl.groups), (double*)(ws + wl.u64),
                  (const double*)(ws + wl.ax64), (const double*)(ws + wl.ay64), nullptr, nullptr,
                  (int*)(ws + wl.nstep), (int*)(ws + wl.cycles_i), (double*)(ws + wl.relres_i),
                  CycleParams{prm.mu, prm.nu1, prm.nu2, prm.omega}, prm.tune_block ? prm.tune_block : kVisitThreads,
                  (size_t)(prm.tune_visit_smem ? prm.tune_visit_smem : kVisitSmemKB) * 1024, low_shape(prm), (const LowDesc*)(ws + wl.low_desc), (const uint4*)(ws + wl.low_ent),
                  (const uint2*)(ws + wl.low_prog)};
    float* ax32 = mixed ? (float*)(ws + wl.ax32) : nullptr;
    float* ay32 = mixed ? (float*)(ws + wl.ay32) : nullptr;
    C.ax = mixed ? (const T*)ax32 : (const T*)(ws + wl.ax64);
    C.ay = mixed ? (const T*)ay32 : (const T*)(ws + wl.ay64);
    C.base.samples = (const SampleInfo*)(ws + wl.samples);
    C.base.gpos = (const int*)(ws + wl.gpos);

    MSG_CUDA_TRY(cudaMemsetAsync(stat, 0, sizeof(int32_t) * pl.S, st));
    MSG_CUDA_TRY(cudaMemsetAsync(C.u64, 0, sizeof(double) * pl.total_nodes, st));
    MSG_CUDA_TRY(cudaMemsetAsync(C.nstep, 0, sizeof(int) * pl.total_q, st));
    {
        DevCtx c = C.base;
        c.slist = (const int*)(ws + wl.perm);
        c.groups = C.dgroups;
        c.segs = (const Segment*)(ws + wl.allsegs);
        c.nseg = (int)pl.all_segs.size();
        const int64_t nb = pl.all_segs.empty() ? 0 : pl.all_segs.back().blk_start + pl.all_segs.back().count;
        double nodes = 0;
        for (const Segment& s : pl.all_segs) nodes += (double)s.count * ((1 << s.p) + 1) * ((1 << s.q) + 1);
        prof_begin(K_COEFFS, st);
        k_coeffs<<<(unsigned)nb, kThreads, 0, st>>>(c, Z, prm.coef, (double*)(ws + wl.ax64), (double*)(ws + wl.ay64),
                                                   ax32, ay32);
        prof_end(K_COEFFS, st, nodes * (16.0 + 16.0 + (mixed ? 8.0 : 0.0)), 0.0);
        MSG_CHECK_LAUNCH();
        const LowPlanes& lp = low_tables().planes[kLowMax];
        prof_begin(K_COEFFS, st);
        k_lowimg<T><<<(unsigned)pl.S, kThreads, 0, st>>>(C.base.samples, C.ax, C.ay, lp, (T*)(ws + wl.low_img),
                                                          (int64_t)(lp.nfx + lp.nfy), lp.nfx);
        prof_end(K_COEFFS, st, (double)pl.S * (lp.nfx + lp.nfy) * 2.0 * sizeof(T), 0.0);
        MSG_CHECK_LAUNCH();
    }
    {
        // tables of the low-diagonal program: class descriptors, node entries, programs
        const LowTables& lt = low_tables();
        std::vector<LowDesc> desc;
        const std::vector<uint2> rp = low_resolve(prm, desc);
        MSG_CUDA_TRY(cudaMemcpyAsync(ws + wl.low_desc, desc.data(), sizeof(LowDesc) * desc.size(),
                                     cudaMemcpyHostToDevice, st));
        MSG_CUDA_TRY(cudaMemcpyAsync(ws + wl.low_ent, lt.ent.data(), sizeof(uint4) * lt.ent.size(),
                                     cudaMemcpyHostToDevice, st));
        MSG_CUDA_TRY(cudaMemcpyAsync(ws + wl.low_prog, rp.data(), sizeof(uint2) * rp.size(),
                                     cudaMemcpyHostToDevice, st));
        // the sources are host vectors: finish the copies before they go out of scope
        MSG_CUDA_TRY(cudaStreamSynchronize(st));
    }
    // the residual band: 3 rows of a 2^12-cell-wide grid at most
    MSG_CUDA_TRY(cudaFuncSetAttribute(k_pre<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(T) * std::max(kBandNodes, 3 * ((1 << 12) + 1)))));
    MSG_CUDA_TRY(cudaFuncSetAttribute(k_visit_reg<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    MSG_CUDA_TRY(cudaFuncSetAttribute(k_visit_reg<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    if constexpr (sizeof(T) == 4)
        MSG_CUDA_TRY(cudaFuncSetAttribute(k_visit_reg<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)kSmemMax));
    MSG_CUDA_TRY(cudaFuncSetAttribute(k_lowv<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    MSG_CUDA_TRY(cudaFuncSetAttribute(k_lowv<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    MSG_CUDA_TRY(cudaFuncSetAttribute(k_lowv<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    MSG_CUDA_TRY(cudaFuncSetAttribute(k_lowv<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    MSG_CUDA_TRY(cudaStreamSynchronize(st));

    // ---- one worker (host thread + stream) per stage
    const int nst = pl.Lmax + 1;
    StageQueues Qs;
    Qs.ready.assign(nst, {});
    Qs.done.assign(nst, 0);
    Qs.ready[0] = pl.perm;
    std::vector<cudaStream_t> streams(nst, nullptr);
    for (int L = 0; L < nst; ++L) MSG_CUDA_TRY(cudaStreamCreateWithFlags(&streams[L], cudaStreamNonBlocking));
    std::vector<int> rcs(nst, MSG_OK);
    std::vector<std::string> errs(nst);
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::vector<std::thread> th;
        for (int L = 0; L < nst; ++L)
            th.emplace_back([&, L] {
                cudaSetDevice(dev);
                rcs[L] = stage_worker<T>(C, L, Qs, streams[L]);
                if (rcs[L] != MSG_OK) errs[L] = msg_last_error();
            });
        for (auto& t : th) t.join();
    }
    for (int L = 0; L < nst; ++L) cudaStreamDestroy(streams[L]);
    for (int L = 0; L < nst; ++L)
        if (rcs[L] != MSG_OK) { set_error("stage " + std::to_string(L) + ": " + errs[L]); return rcs[L]; }

    // ---- QoI of every grid
    {
        DevCtx c = C.base;
        c.slist = (const int*)(ws + wl.perm);
        c.groups = C.dgroups;
        c.segs = (const Segment*)(ws + wl.allsegs);
        c.nseg = (int)pl.all_segs.size();
        const int64_t nb = pl.all_segs.empty() ? 0 : pl.all_segs.back().blk_start + pl.all_segs.back().count;
        prof_begin(K_QOI, st);
        k_qoi<<<(unsigned)nb, kThreads, 0, st>>>(c, C.u64, Z, prm.qoi, Qout);
        prof_end(K_QOI, st, (double)pl.total_nodes * 8.0, 0.0);
        MSG_CHECK_LAUNCH();
    }
    if (cycles_out) MSG_CUDA_TRY(cudaMemcpyAsync(cycles_out, C.cyc, sizeof(int) * pl.total_q, cudaMemcpyDeviceToDevice, st));
    if (relres_out) MSG_CUDA_TRY(cudaMemcpyAsync(relres_out, C.rel, sizeof(double) * pl.total_q, cudaMemcpyDeviceToDevice, st));
    MSG_CUDA_TRY(cudaStreamSynchronize(st));
    return MSG_OK;
}

// ------------------------------------------------- convergence study (host) --
namespace {

void hist_prog_msg(int s, int zi, int mu, std::vector<int2>& prog)
{
    prog.push_back(make_int2(H_PRE | s << 4, zi));
    if (s == 0) return;
    for (int k = 0; k < mu; ++k) hist_prog_msg(s - 1, k == 0, mu, prog);
    prog.push_back(make_int2(H_POST | s << 4, 0));
}

void hist_prog_std(int p, int q, int mu, std::vector<int2>& prog)
{
    if (p == 1 || q == 1) {
        prog.push_back(make_int2(H_STD_LINE | p << 4 | q << 12, 0));
        return;
    }
    prog.push_back(make_int2(H_STD_PRE | p << 4 | q << 12, 0));
    for (int k = 0; k < mu; ++k) hist_prog_std(p - 1, q - 1, mu, prog);
    prog.push_back(make_int2(H_STD_POST | p << 4 | q << 12, 0));
}

std::vector<int2> hist_prog(int P, int Q, int method, int mu)
{
    std::vector<int2> prog;
    if (method == 0) hist_prog_msg(P + Q - 2, 0, mu, prog);  // the top keeps its iterate
    else hist_prog_std(P, Q, mu, prog);
    return prog;
}

struct HistLayout {
    size_t samples, gpos, slist, groups, segs, prog, ax, ay, su, sbx, sby, total;
};

HistLayout hist_layout(int P, int Q, int64_t S, size_t nprog)
{
    HistLayout w;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off += (b + 255) / 256 * 256; return o; };
    const size_t R = (size_t)rect_nodes(P, Q) * (size_t)S;
    w.samples = take(sizeof(SampleInfo) * S);
    w.gpos = take(sizeof(int) * S);
    w.slist = take(sizeof(int) * S);
    w.groups = take(sizeof(Group));
    w.segs = take(sizeof(Segment) * (P * Q + 1));
    w.prog = take(sizeof(int2) * nprog);
    w.ax = take(sizeof(double) * R);
    w.ay = take(sizeof(double) * R);
    w.su = take(sizeof(double) * R);
    w.sbx = take(sizeof(double) * R);
    w.sby = take(sizeof(double) * R);
    w.total = off;
    return w;
}

int hist_check(int P, int Q, int64_t S, const msg_params* prm, int method, int ncycles)
{
    const int32_t pq[2] = {P, Q};
    int rc = validate(pq, 1, prm);
    if (rc != MSG_OK) return rc;
    if (P > 10 || Q > 10) { set_error("history: P, Q <= 10"); return MSG_ERR_INVALID; }
    if (S < 0) { set_error("S < 0"); return MSG_ERR_INVALID; }
    if (method != MSG_HIST_MSG && method != MSG_HIST_STANDARD) { set_error("method must be MSG_HIST_MSG or MSG_HIST_STANDARD"); return MSG_ERR_INVALID; }
    if (ncycles < 1 || ncycles > 1000) { set_error("ncycles must be in [1, 1000]"); return MSG_ERR_INVALID; }
    return MSG_OK;
}

}  // namespace

}  // namespace msg

using namespace msg;

extern "C" size_t msg_workspace_bytes(const int32_t* PQ, int64_t S, const msg_params* prm)
{
    clear_error();
    if (validate(PQ, S, prm) != MSG_OK) return 0;
    Plan pl;
    build_plan(PQ, S, pl);
    // the per-sample status array is kept inside the workspace when the caller passes none
    return layout_of(pl, *prm).total + align_up(sizeof(int32_t) * std::max<int64_t>(S, 1));
}

extern "C" int32_t msg_solve_batch(const int32_t* PQ, int64_t S, const msg_params* prm, const double* Z, double* Qout,
                                   int32_t* status, int32_t* cycles, double* relres, void* workspace, size_t ws_bytes,
                                   void* stream)
{
    clear_error();
    int rc = validate(PQ, S, prm);
    if (rc != MSG_OK) return rc;
    if (S == 0) return MSG_OK;
    if (!Z || !Qout || !workspace) { set_error("Z, Qout and workspace must be non-NULL"); return MSG_ERR_INVALID; }
    Plan pl;
    build_plan(PQ, S, pl);
    WsLayout wl = layout_of(pl, *prm);
    const size_t need = wl.total + align_up(sizeof(int32_t) * S);
    if (ws_bytes < need) {
        set_error("workspace too small: need " + std::to_string(need) + " bytes");
        return MSG_ERR_WORKSPACE;
    }
    char* ws = (char*)(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    int32_t* stat = status ? status : (int32_t*)(ws + wl.total);
    cudaStream_t st = (cudaStream_t)stream;
    if (prm->precision == MSG_PREC_MIXED) return run_solve<float>(pl, wl, ws, *prm, Z, Qout, stat, cycles, relres, st);
    return run_solve<double>(pl, wl, ws, *prm, Z, Qout, stat, cycles, relres, st);
}

extern "C" int32_t msg_solution(const int32_t* PQ, int64_t S, const msg_params* prm, const void* workspace,
                                size_t ws_bytes, double* u_out, void* stream)
{
    clear_error();
    int rc = validate(PQ, S, prm);
    if (rc != MSG_OK) return rc;
    if (S == 0) return MSG_OK;
    if (!workspace || !u_out) { set_error("workspace and u_out must be non-NULL"); return MSG_ERR_INVALID; }
    Plan pl;
    build_plan(PQ, S, pl);
    WsLayout wl = layout_of(pl, *prm);
    if (ws_bytes < wl.total + align_up(sizeof(int32_t) * S)) {
        set_error("workspace smaller than msg_workspace_bytes for this batch");
        return MSG_ERR_WORKSPACE;
    }
    const char* ws = (const char*)(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    MSG_CUDA_TRY(cudaMemcpyAsync(u_out, ws + wl.u64, sizeof(double) * pl.total_nodes, cudaMemcpyDeviceToDevice,
                                 (cudaStream_t)stream));
    return MSG_OK;
}

extern "C" int64_t msg_solution_values(const int32_t* PQ, int64_t S)
{
    clear_error();
    if (S < 0 || (S > 0 && !PQ)) { set_error("bad PQ / S"); return -1; }
    int64_t n = 0;
    for (int64_t i = 0; i < S; ++i) {
        if (PQ[2 * i] < 1 || PQ[2 * i] > 12 || PQ[2 * i + 1] < 1 || PQ[2 * i + 1] > 12) {
            set_error("grid exponents must satisfy 1 <= P, Q <= 12");
            return -1;
        }
        n += rect_nodes(PQ[2 * i], PQ[2 * i + 1]);
    }
    return n;
}

extern "C" size_t msg_history_workspace_bytes(int32_t P, int32_t Q, int64_t S, const msg_params* prm, int32_t method)
{
    clear_error();
    if (hist_check(P, Q, S, prm, method, 1) != MSG_OK) return 0;
    return hist_layout(P, Q, S, hist_prog(P, Q, method, prm->mu).size()).total;
}

extern "C" int32_t msg_cycle_history(int32_t P, int32_t Q, int64_t S, const msg_params* prm, int32_t method,
                                     const double* Z, int32_t ncycles, double* hist, void* workspace, size_t ws_bytes,
                                     void* stream)
{
    clear_error();
    int rc = hist_check(P, Q, S, prm, method, ncycles);
    if (rc != MSG_OK) return rc;
    if (S == 0) return MSG_OK;
    if (!Z || !hist || !workspace) { set_error("Z, hist or workspace is NULL"); return MSG_ERR_INVALID; }
    if ((uintptr_t)workspace % 256) { set_error("workspace must be 256-byte aligned"); return MSG_ERR_INVALID; }
    const std::vector<int2> prog = hist_prog(P, Q, method, prm->mu);
    const HistLayout w = hist_layout(P, Q, S, prog.size());
    if (ws_bytes < w.total) {
        set_error("workspace too small: need " + std::to_string(w.total) + " bytes");
        return MSG_ERR_WORKSPACE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    const int64_t R = rect_nodes(P, Q), nf = field_nodes(P, Q);
    // one group, one sample list; segments: every grid (coefficients), then the top item (cycles)
    std::vector<SampleInfo> samples(S);
    std::vector<int> ids(S);
    for (int64_t s = 0; s < S; ++s) {
        samples[s] = SampleInfo{P, Q, s * R, s * nf, 0};
        ids[s] = (int)s;
    }
    const Group grp{P, Q, 0, (int)S, 0, R};
    std::vector<Segment> segs;
    for (int p = 1; p <= P; ++p)
        for (int q = 1; q <= Q; ++q)
            segs.push_back(Segment{0, P, Q, p, q, (int64_t)segs.size() * S, S, 0, 0, 0});
    segs.push_back(Segment{0, P, Q, P, Q, 0, S, 0, 0, 0});
    MSG_CUDA_TRY(cudaMemcpyAsync(ws + w.samples, samples.data(), sizeof(SampleInfo) * S, cudaMemcpyHostToDevice, st));
    MSG_CUDA_TRY(cudaMemcpyAsync(ws + w.gpos, ids.data(), sizeof(int) * S, cudaMemcpyHostToDevice, st));
    MSG_CUDA_TRY(cudaMemcpyAsync(ws + w.slist, ids.data(), sizeof(int) * S, cudaMemcpyHostToDevice, st));
    MSG_CUDA_TRY(cudaMemcpyAsync(ws + w.groups, &grp, sizeof(Group), cudaMemcpyHostToDevice, st));
    MSG_CUDA_TRY(cudaMemcpyAsync(ws + w.segs, segs.data(), sizeof(Segment) * segs.size(), cudaMemcpyHostToDevice, st));
    MSG_CUDA_TRY(cudaMemcpyAsync(ws + w.prog, prog.data(), sizeof(int2) * prog.size(), cudaMemcpyHostToDevice, st));
    DevCtx cx;
    cx.samples = (const SampleInfo*)(ws + w.samples);
    cx.gpos = (const int*)(ws + w.gpos);
    cx.slist = (const int*)(ws + w.slist);
    cx.groups = (const Group*)(ws + w.groups);
    cx.segs = (const Segment*)(ws + w.segs);
    cx.nseg = P * Q;
    double* ax = (double*)(ws + w.ax);
    double* ay = (double*)(ws + w.ay);
    prof_begin(K_COEFFS, st);
    k_coeffs<<<(unsigned)(P * Q * S), kThreads, 0, st>>>(cx, Z, prm->coef, ax, ay, nullptr, nullptr);
    prof_end(K_COEFFS, st, (double)S * R * 32.0, 0.0);
    MSG_CHECK_LAUNCH();
    DevCtx ch = cx;
    ch.segs = cx.segs + P * Q;
    ch.nseg = 1;
    const int band = std::max(kBandNodes, 3 * ((1 << P) + 1));
    const CycleParams cp{prm->mu, prm->nu1, prm->nu2, prm->omega};
    prof_begin(K_PRE, st);
    k_cycle_history<double><<<dim3((unsigned)S, 1), 256, sizeof(double) * band, st>>>(
        ch, (double*)(ws + w.su), (double*)(ws + w.sbx), (double*)(ws + w.sby), ax, ay,
        (const int2*)(ws + w.prog), (int)prog.size(), ncycles, cp, band, hist);
    prof_end(K_PRE, st, 0.0, 0.0);
    MSG_CHECK_LAUNCH();
    // the host tables above are read by the copies: finish before they go out of scope
    MSG_CUDA_TRY(cudaStreamSynchronize(st));
    return MSG_OK;
}
