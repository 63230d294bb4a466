// Host runtime of the discrete-PML library: the C ABI of include/pml.h.
//
// Responsibilities: validate arguments, build the damping profiles (edge-centred,
// Sec. 1.1.2) and the integer layout tables, carve the device workspace, encode the
// TMA tensor maps, and enqueue the step kernels on the caller's stream.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "common.cuh"
#include "pml.h"

using namespace pml;

namespace {

constexpr int kMaxSources = 1024;
constexpr int kMaxReceivers = 16384;
constexpr size_t kAlign = 256;
constexpr int64_t kDefaultCheckEvery = 1000;   // steps between finiteness scans of U and V

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

thread_local std::string g_create_error;

struct Plan {
    int nd = 0, esz = 0, nf = 0;
    int64_t T[3] = {1, 1, 1};
    Geom g{};
    size_t fields[2][8] = {};
    size_t adj[2][8] = {};
    size_t mid[8] = {};          // two-step blocks (2D FP32): first-step values of the widened frame
    bool tb2 = false;
    size_t lvl[2][8] = {};       // 3D level passes: two scratch states
    size_t ltiles[2][4] = {};    // 3D level passes: tiles of each level, forward / transposed
    size_t max_ltiles = 0;
    size_t slab_tiles[2] = {};   // 3D slab tiles (FP32), forward / transposed
    size_t max_slab = 0;
    size_t sig[3] = {};
    size_t tiles = 0, tiles_adj = 0, max_tiles = 0, tiles_l1 = 0, tiles_l2 = 0, tiles_l1_adj = 0, tiles_l2_adj = 0;
    size_t partials = 0, normout = 0, err = 0, queue = 0;
    size_t src_off = 0, src_xyz = 0, src_amp = 0, grad = 0, rec_off = 0, src_level = 0, rec_xyz = 0, rec_level = 0;
    size_t total = 0;
};

Geom make_geom(int nd, const int64_t T[3], bool wall = false)
{
    Geom g{};
    g.ndim = nd;
    g.wall = wall ? 1 : 0;
    for (int a = 0; a < 3; ++a) g.T[a] = a < nd ? T[a] : 1;
    for (int a = 0; a < 3; ++a) g.wrap[a] = wall ? 0 : g.T[a];
    g.P = round_up(g.T[0] + 2 * G, 32);
    g.R = g.T[1] + 2 * G;
    g.PS = g.P * g.R;
    g.planes = nd == 3 ? g.T[2] + 2 * G : 1;
    g.elems = g.PS * g.planes;
    g.origin = G + G * g.P + (nd == 3 ? G * g.PS : 0);
    return g;
}

// Upper bound of the number of layer tiles of one frame decomposition.
size_t tile_bound(int nd, int prec, const int64_t T[3])
{
    if (nd == 2)
        return size_t(3) * size_t(T[0] / layer2d_tile_cols(prec) + 3) * size_t(T[1] / 6 + 2);   // runs >= 6 rows
    const int TX = prec == 32 ? kLayer3TXf : kLayer3TXd, TY = prec == 32 ? kLayer3TYf : kLayer3TYd;
    return size_t(5) * size_t(T[0] / TX + 2) * size_t(T[1] / TY + 2) * size_t(T[2] / kLayer3LZ + 2);
}

bool make_plan(const pml_grid *grid, int w, int prec, int flags, Plan *p, std::string *why)
{
    if (!grid) { *why = "grid is NULL"; return false; }
    if (grid->ndim != 2 && grid->ndim != 3) { *why = "ndim must be 2 or 3"; return false; }
    if (w < 0) { *why = "pml_width must be >= 0"; return false; }
    if (prec != 32 && prec != 64) { *why = "precision must be 32 or 64"; return false; }
    p->nd = grid->ndim;
    p->esz = prec == 32 ? 4 : 8;
    p->nf = 2 + 2 * p->nd;
    for (int a = 0; a < p->nd; ++a) {
        if (grid->n[a] < 1) { *why = "every axis needs at least one interior vertex"; return false; }
        p->T[a] = grid->n[a] + 2 * int64_t(w);
        if (p->T[a] < 2 * G) { *why = "every axis needs n + 2w >= 8 vertices"; return false; }
        if (p->T[a] > (int64_t(1) << 30)) { *why = "axis too long"; return false; }
    }
    p->g = make_geom(p->nd, p->T, (flags & PML_FLAG_WALL) != 0);
    size_t off = 0;
    const size_t fb = align_up(size_t(p->g.elems) * p->esz, kAlign);
    for (int s = 0; s < 2; ++s)
        for (int f = 0; f < p->nf; ++f) { p->fields[s][f] = off; off += fb; }
    if (flags & PML_FLAG_ADJOINT)
        for (int s = 0; s < 2; ++s)
            for (int f = 0; f < p->nf; ++f) { p->adj[s][f] = off; off += fb; }
    p->tb2 = p->nd == 2 && interior2d_tb2_variants(prec) > 0;
    if (p->tb2)
        for (int f = 0; f < p->nf; ++f) { p->mid[f] = off; off += fb; }
    if (p->nd == 3)
        for (int s = 0; s < 2; ++s)
            for (int f = 0; f < p->nf; ++f) { p->lvl[s][f] = off; off += fb; }
    for (int a = 0; a < p->nd; ++a) { p->sig[a] = off; off += align_up(size_t(p->T[a]) * p->esz, kAlign); }
    p->max_tiles = tile_bound(p->nd, prec, p->T);
    p->tiles = off; off += align_up(p->max_tiles * sizeof(LayerTile), kAlign);
    p->tiles_adj = off; off += align_up(p->max_tiles * sizeof(LayerTile), kAlign);
    if (p->tb2) {
        p->tiles_l1 = off; off += align_up(p->max_tiles * sizeof(LayerTile), kAlign);
        p->tiles_l2 = off; off += align_up(p->max_tiles * sizeof(LayerTile), kAlign);
        if (flags & PML_FLAG_ADJOINT) {
            p->tiles_l1_adj = off; off += align_up(p->max_tiles * sizeof(LayerTile), kAlign);
            p->tiles_l2_adj = off; off += align_up(p->max_tiles * sizeof(LayerTile), kAlign);
        }
    }
    if (p->nd == 3 && prec == 32) {
        // slab tiles: at least 21 x 8 outputs per tile in (x, y) (after the alignment of the
        // region's first column), z items of at least a quarter of kSlabItemZ planes or a
        // whole run of the frame; a few runs of constant class per axis
        p->max_slab = size_t(4) * size_t(p->T[0] / 21 + 12) * size_t(p->T[1] / 8 + 12) *
                      size_t(p->T[2] / (kSlabItemZ / 4) + 12);
        for (int d = 0; d < ((flags & PML_FLAG_ADJOINT) ? 2 : 1); ++d) {
            p->slab_tiles[d] = off;
            off += align_up(p->max_slab * sizeof(LayerTile), kAlign);
        }
    }
    if (p->nd == 3) {
        p->max_ltiles = size_t(3) * size_t(p->T[0] / kLevel3TX + 2) * size_t(p->T[1] / kLevel3TY + 2) *
                        size_t(p->T[2] / kLevel3TZ + 3);
        for (int d = 0; d < ((flags & PML_FLAG_ADJOINT) ? 2 : 1); ++d)
            for (int k = 0; k < 4; ++k) {
                p->ltiles[d][k] = off;
                off += align_up(p->max_ltiles * sizeof(LayerTile), kAlign);
            }
    }
    p->partials = off; off += align_up(size_t(kNormBlocks) * kNormVals * sizeof(double), kAlign);
    p->normout = off; off += kAlign;
    p->err = off; off += kAlign;
    p->queue = off; off += kAlign;
    p->src_off = off; off += align_up(kMaxSources * sizeof(int64_t), kAlign);
    p->src_xyz = off; off += align_up(kMaxSources * 3 * sizeof(int32_t), kAlign);
    p->src_amp = off; off += align_up(kMaxSources * sizeof(double), kAlign);
    p->grad = off; off += align_up(kMaxSources * sizeof(double), kAlign);
    p->rec_off = off; off += align_up(kMaxReceivers * sizeof(int64_t), kAlign);
    p->src_level = off; off += align_up(kMaxSources * sizeof(int32_t), kAlign);
    p->rec_xyz = off; off += align_up(kMaxReceivers * 3 * sizeof(int32_t), kAlign);
    p->rec_level = off; off += align_up(kMaxReceivers * sizeof(int32_t), kAlign);
    p->total = off;
    return true;
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

}  // namespace

struct pml_ctx {
    Plan plan;
    int nd = 0, prec = 0, esz = 0, nf = 0, flags = 0, w = 0;
    int64_t N[3] = {1, 1, 1}, T[3] = {1, 1, 1};
    double h = 1, dt = 0.5;
    std::vector<double> sig[3];
    std::vector<uint8_t> phi[3], psi[3], inner[3];
    Range ir[3], ir_adj[3];
    Geom g{};
    cudaStream_t st = nullptr;
    bool own_ws = false;
    char *ws = nullptr;
    void *fld[2][8] = {}, *adj[2][8] = {};
    int cur = 0, acur = 0;
    void *dsig[3] = {};
    LayerTile *dtiles = nullptr, *dtiles_adj = nullptr;
    int ntiles = 0, ntiles_adj = 0;
    int class_off[9] = {}, class_off_adj[9] = {};
    double *dpart = nullptr, *dnorm = nullptr, *dgrad = nullptr;
    DeviceError *derr = nullptr;
    int *dqueue = nullptr;              // work counters: interior fwd 0/1, adj 2/3; 2D layer fwd 4/5, adj 6/7,
                                        // second layer pass of a two-step block 8/9 (transposed 10/11)
    int64_t launches_fwd = 0, launches_adj = 0, launches_layer_fwd = 0, launches_layer_adj = 0, launches_layer2 = 0,
            launches_layer2_adj = 0;
    int ns = 0, nr = 0;
    int64_t *dsrc_off = nullptr, *drec_off = nullptr;
    int32_t *dsrc_xyz = nullptr, *dsrc_level = nullptr, *drec_xyz = nullptr, *drec_level = nullptr;
    int src_levels = 0, rec_levels = 0;
    double *dsrc_amp = nullptr;
    double f_peak = 0, t_delay = 0;
    void *trace = nullptr;
    int64_t trace_cap = 0, trace_k = 0;
    int64_t step = 0, astep = 0;
    bool adj_ready = false;
    CUtensorMap tm_int[2][2], tm_lay[2][8], tm_int_adj[2][2], tm_lay_adj[2][8];
    int grid_int = 0, grid_int_adj = 0, sm_count = 0;
    int ivar = 0;                       // kernel variant: 2D interior shape (one step per pass); 3D frame
                                        // kernel (0 tile kernel, 1 level passes, 2 slab tiles)
    // temporal blocking depth 2 (2D FP32): forward steps without sources or receiver rows
    // advance two at a time (layer pass 1 on the frame widened by 6 into mid, layer pass 2
    // on the frame widened by 2, two-step interior kernel on the run shrunk by 2)
    int tb = 1, tbvar = 0, grid_tb = 0, grid_tb_adj = 0;
    void *mid[8] = {};
    CUtensorMap tm_mid[8], tm_tb[2][2], tm_tb_adj[2][2];
    LayerTile *dtiles_l1 = nullptr, *dtiles_l2 = nullptr, *dtiles_l1_adj = nullptr, *dtiles_l2_adj = nullptr;
    int ntiles_l1 = 0, ntiles_l2 = 0, ntiles_l1_adj = 0, ntiles_l2_adj = 0;
    Range ir_tb[3], ir_tb_adj[3];
    // 3D: variant 1 advances the layer frame by level passes (frame3d.cu) instead of the
    // z-streaming tile kernel: scratch states and each level's tiles (forward / transposed)
    void *lvl[2][8] = {};
    LayerTile *dlt[2][4] = {};
    int nlt[2][4] = {};
    // 3D FP32: variant 2 advances the layer frame by slab tiles (slab3d.cuh): tiles and
    // class offsets (forward / transposed) and the tensor maps of each class's box,
    // [forward / transposed][input parity][class * 8 + field]
    LayerTile *dslab[2] = {};
    int nslab[2] = {};
    int slab_off[2][9] = {};
    CUtensorMap tm_slab[2][2][64];
    // failure detection: limit of every bounded device wait (0: the default 2 s) and the
    // interval in steps of the finiteness scan of U and V (0: off)
    uint64_t wait_ns = 0;
    int64_t check_every = kDefaultCheckEvery;
    // kernel timing (pml_profile_enable)
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;   // pairs
    // pml_set_initial clears the fields its copies do not fill on a side stream, so that the
    // clearing overlaps the host-to-device copies (created at the first call; none: serial)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool side_tried = false;
    std::vector<int> prof_kind;
    size_t prof_n = 0;
    std::string err;
};

namespace {

pml_status fail(pml_ctx *c, pml_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_create_error = buf;
    return s;
}

pml_status cuda_fail(pml_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, PML_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define PML_CU(c, call, what)                                      \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail((c), e_, (what));  \
    } while (0)

// depth of edge e in the layer: 0 on the physical edges and on both interface edges
int64_t edge_depth(int64_t e, int64_t N, int64_t w)
{
    const int64_t a = w, b = w + N - 1;
    int64_t d = 0;
    if (a - 1 - e > d) d = a - 1 - e;
    if (e - b > d) d = e - b;
    return d;
}

pml_status build_sigma(pml_ctx *c, const pml_sigma_profile *pr)
{
    if (!pr) return fail(c, PML_EINVAL, "profile is NULL");
    if (!(pr->sigma_max >= 0.0) || !std::isfinite(pr->sigma_max))
        return fail(c, PML_EINVAL, "sigma_max must be finite and >= 0");
    for (int a = 0; a < c->nd; ++a) {
        const int64_t T = c->T[a], N = c->N[a], w = c->w;
        std::vector<double> &s = c->sig[a];
        s.assign(size_t(T), 0.0);
        if ((pr->kind == PML_SIGMA_RANDOM || pr->kind == PML_SIGMA_USER) && !pr->user[a])
            return fail(c, PML_EINVAL, "profile kind %d needs user[%d]", pr->kind, a);
        for (int64_t e = 0; e < T; ++e) {
            const int64_t d = edge_depth(e, N, w);
            double v = 0.0;
            switch (pr->kind) {
            case PML_SIGMA_CONSTANT: v = d > 0 ? pr->sigma_max : 0.0; break;
            case PML_SIGMA_POWER:
                if (!(pr->order > 0.0)) return fail(c, PML_EINVAL, "power profile needs order > 0");
                v = d > 0 ? pr->sigma_max * std::pow(double(d) / double(w), pr->order) : 0.0;
                break;
            case PML_SIGMA_RANDOM: {
                const double u = pr->user[a][e];
                if (!(u >= 0.0 && u <= 1.0)) return fail(c, PML_EINVAL, "random draws must lie in [0,1]");
                v = d > 0 ? pr->sigma_max * u : 0.0;
                break;
            }
            case PML_SIGMA_USER:
                v = pr->user[a][e];
                if (!std::isfinite(v) || v < 0.0) return fail(c, PML_EINVAL, "user sigma must be finite and >= 0");
                if (d == 0 && v != 0.0)
                    return fail(c, PML_EINVAL, "user sigma must vanish on the physical edges (axis %d, edge %lld)", a,
                                (long long)e);
                break;
            default: return fail(c, PML_EINVAL, "unknown profile kind %d", pr->kind);
            }
            s[size_t(e)] = v;
        }
        if (c->flags & PML_FLAG_WALL) s[size_t(T - 1)] = 0.0;   // a wall leaves no edge T-1 -> 0
    }
    return PML_OK;
}

// Supports of Phi / Psi and the layer-free run around the centre vertex.  `reach` is the
// set of edge offsets that must carry zero damping: {-2..1} for the forward step and
// {-3..2} for the transposed step.
Range layer_free_run(const std::vector<double> &s, int64_t centre, int lo_off, int hi_off)
{
    const int64_t T = int64_t(s.size());
    auto ok = [&](int64_t i) {
        for (int k = lo_off; k <= hi_off; ++k)
            if (s[size_t(((i + k) % T + T) % T)] != 0.0) return false;
        return true;
    };
    bool all = true;
    for (int64_t e = 0; e < T; ++e)
        if (s[size_t(e)] != 0.0) { all = false; break; }
    if (all) return {0, T - 1};
    if (!ok(centre)) return {1, 0};
    int64_t lo = centre, hi = centre;
    while (lo - 1 >= 0 && ok(lo - 1)) --lo;
    while (hi + 1 <= T - 1 && ok(hi + 1)) ++hi;
    return {lo, hi};
}

// The run shrunk by k vertices at both ends; a run that is the whole periodic axis (no
// layer on it) has no ends and stays whole.
Range shrink_run(const Range &r, int64_t T, int64_t k)
{
    if (r.lo == 0 && r.hi == T - 1) return r;
    return {r.lo + k, r.hi - k};
}

void build_layout(pml_ctx *c)
{
    for (int a = 0; a < c->nd; ++a) {
        const int64_t T = c->T[a];
        const std::vector<double> &s = c->sig[a];
        c->phi[a].assign(size_t(T), 0);
        c->psi[a].assign(size_t(T), 0);
        c->inner[a].assign(size_t(T), 0);
        for (int64_t i = 0; i < T; ++i) {
            c->phi[a][size_t(i)] = s[size_t(i)] != 0.0;
            c->psi[a][size_t(i)] = s[size_t((i - 1 + T) % T)] != 0.0;
        }
        const int64_t centre = c->w + c->N[a] / 2;
        c->ir[a] = layer_free_run(s, centre, -2, 1);
        c->ir_adj[a] = layer_free_run(s, centre, -3, 2);
        if (c->flags & PML_FLAG_WALL)   // the closed form needs real vertices on both sides
            for (Range *r : {&c->ir[a], &c->ir_adj[a]}) {
                r->lo = std::max<int64_t>(r->lo, 1);
                r->hi = std::min<int64_t>(r->hi, T - 2);
            }
        for (int64_t i = c->ir[a].lo; i <= c->ir[a].hi; ++i) c->inner[a][size_t(i)] = 1;
    }
    for (int a = c->nd; a < 3; ++a) c->ir[a] = c->ir_adj[a] = {0, 0};
}

bool range_empty(const Range &r) { return r.lo > r.hi; }

bool axis_active(const pml_ctx *c, int a, int64_t lo, int64_t hi)
{
    const int64_t T = c->T[a];
    for (int64_t i = lo; i < hi; ++i) {
        const size_t k = size_t(((i % T) + T) % T);
        if (c->phi[a][k] || c->psi[a][k]) return true;
    }
    return false;
}

struct Rect {
    int64_t lo[3], hi[3];
};

// Frame = box minus the layer-free box ir[0] x ir[1] (x ir[2]), as disjoint rectangles.
std::vector<Rect> frame_rects(const pml_ctx *c, const Range *ir)
{
    std::vector<Rect> out;
    Rect full;
    for (int a = 0; a < 3; ++a) { full.lo[a] = 0; full.hi[a] = a < c->nd ? c->T[a] - 1 : 0; }
    bool empty = false;
    for (int a = 0; a < c->nd; ++a) empty = empty || ir[a].lo > ir[a].hi;
    if (empty) { out.push_back(full); return out; }
    // peel axis by axis: slabs of axis a outside ir[a], restricted to ir of the earlier axes.
    // In 3D the two z slabs form one band across the periodic seam (the z-streaming layer
    // kernel loads plane by plane and wraps z itself), so it is one rectangle with an
    // unwrapped z range ir.hi+1 .. T + ir.lo - 1.
    Rect rest = full;
    for (int a = c->nd - 1; a >= 0; --a) {
        const bool lo_gap = ir[a].lo > 0, hi_gap = ir[a].hi < c->T[a] - 1;
        if (a == 2 && !c->g.wall && (lo_gap || hi_gap)) {
            Rect r = rest; r.lo[a] = ir[a].hi + 1; r.hi[a] = c->T[a] + ir[a].lo - 1; out.push_back(r);
        } else {
            if (lo_gap) { Rect r = rest; r.lo[a] = 0; r.hi[a] = ir[a].lo - 1; out.push_back(r); }
            if (hi_gap) { Rect r = rest; r.lo[a] = ir[a].hi + 1; r.hi[a] = c->T[a] - 1; out.push_back(r); }
        }
        rest.lo[a] = ir[a].lo;
        rest.hi[a] = ir[a].hi;
    }
    return out;
}

// Activity of axis a per coordinate: aux fields of that axis are active within 4 vertices.
// Along an inactive stretch the layer kernels need a halo of 2 instead of 4.
std::vector<uint8_t> axis_activity(const pml_ctx *c, int a)
{
    std::vector<uint8_t> act(size_t(c->T[a]), 0);
    if (a < c->nd)
        for (int64_t i = 0; i < c->T[a]; ++i) act[size_t(i)] = axis_active(c, a, i - 4, i + 5) ? 1 : 0;
    return act;
}

struct ActRun {
    int64_t lo, hi;
    bool on;
};

// Maximal runs of constant activity over the coordinates lo..hi (unwrapped: coordinate i
// reads act[i mod T]).
std::vector<ActRun> activity_runs(const std::vector<uint8_t> &act, int64_t lo, int64_t hi)
{
    const int64_t T = int64_t(act.size());
    auto on = [&](int64_t i) { return act[size_t(((i % T) + T) % T)] != 0; };
    std::vector<ActRun> r;
    for (int64_t i = lo; i <= hi;) {
        const bool o = on(i);
        int64_t j = i;
        while (j + 1 <= hi && on(j + 1) == o) ++j;
        r.push_back({i, j, o});
        i = j + 1;
    }
    return r;
}

// Layer tiles of the frame, sorted by flags (bit a: aux fields of axis a reach the tile's
// footprint) so that each class runs with its own field count.
//  2D: strips of 32 columns streamed down the rows by one warp, laid over the stretches
//      of constant activity along x (see axis_activity): 24 outputs with a halo of 4 where
//      x is active, 28 with a halo of 2 where it is not (an active-x strip may run on into
//      inactive columns).  The rows outside ir[1] form one band across the periodic seam
//      of y (unwrapped rows ir[1].hi + 1 .. T1 + ir[1].lo - 1), cut into near-equal runs of
//      at most band_rows rows over the full width; the columns outside ir[0] (rows ir[1])
//      are cut into runs of at most slab_rows rows; strips active along both axes take
//      2/5 of those lengths.  With a wall there is no seam: two bands.
//  3D: (x, y) column tiles streamed over z segments of at most kLayer3LZ planes (zlo..zhi,
//      unwrapped).
std::vector<LayerTile> build_tiles(const pml_ctx *c, const Range *ir, int class_off[9],
                                   int64_t band_rows = kLayer2BandRows, int64_t slab_rows = kLayer2SlabRows)
{
    std::vector<LayerTile> t;
    if (c->nd == 2) {
        // strips of 32 columns: 24 outputs along a damped x (halo 4), 28 along an undamped
        // one (halo 2); the first column of a strip's box is a multiple of 4 (TMA alignment)
        const int COLS = layer2d_box_cols(c->prec);
        const std::vector<uint8_t> act0 = axis_activity(c, 0), act1 = axis_activity(c, 1);
        // Row runs of one class: a short inactive run next to an active one joins it (an
        // item over active rows is exact anywhere; a few inactive rows of their own would
        // cost a whole item's start-up for little output).
        auto row_runs = [&](int64_t ylo, int64_t yhi) {
            std::vector<ActRun> r = activity_runs(act1, ylo, yhi), m;
            for (size_t i = 0; i < r.size(); ++i) {
                ActRun q = r[i];
                const bool next_on = (i > 0 && r[i - 1].on) || (i + 1 < r.size() && r[i + 1].on);
                if (!q.on && next_on && q.hi - q.lo + 1 < kLayer2MinOffRows) q.on = true;
                if (!m.empty() && m.back().on == q.on) m.back().hi = q.hi;
                else m.push_back(q);
            }
            return m;
        };
        // Strips over the columns xlo..xhi, greedily from the left: an inactive-class strip
        // (28 outputs) where the inactive run from its first column reaches at least as far
        // as an active-class strip (24 outputs) would; otherwise an active-class strip, which
        // may run on into inactive columns (exact there too).
        struct Strip {
            int64_t x0, lo, hi;
            bool on;
        };
        auto strips = [&](int64_t xlo, int64_t xhi) {
            std::vector<Strip> s;
            const std::vector<ActRun> runs = activity_runs(act0, xlo, xhi);
            size_t k = 0;
            for (int64_t x = xlo; x <= xhi;) {
                while (runs[k].hi < x) ++k;
                const int64_t x0on = x - ((((x - 4) % 4) + 4) % 4);
                const int64_t endon = std::min<int64_t>(x0on + (COLS - 8) - 1, xhi);
                Strip st{x0on, x, endon, true};
                if (!runs[k].on) {
                    const int64_t x0off = x - ((((x - 2) % 4) + 4) % 4);
                    const int64_t endoff = std::min<int64_t>(x0off + (COLS - 4) - 1, runs[k].hi);
                    if (endoff >= endon) st = Strip{x0off, x, endoff, false};
                }
                s.push_back(st);
                x = st.hi + 1;
            }
            return s;
        };
        auto add = [&](int64_t xlo, int64_t xhi, int64_t ylo, int64_t yhi, int64_t maxrows) {
            if (xhi < xlo || yhi < ylo) return;
            const std::vector<Strip> sx = strips(xlo, xhi);
            for (const ActRun &ry : row_runs(ylo, yhi)) {
                const int64_t H = ry.hi - ry.lo + 1;
                // strips active along both axes (the corners: six fields and both damping
                // terms, about 1.5 times the work per row) get proportionally shorter runs,
                // so that they do not outlast the other items of a launch
                for (int corner = 0; corner < 2; ++corner) {
                    const int64_t mr = corner ? std::max<int64_t>(8, maxrows * 2 / 5) : maxrows;
                    const int64_t nseg = (H + mr - 1) / mr;
                    int64_t y0 = ry.lo;
                    for (int64_t sgi = 0; sgi < nseg; ++sgi) {
                        const int64_t len = H / nseg + (sgi < H % nseg ? 1 : 0);
                        for (const Strip &st : sx) {
                            if ((st.on && ry.on) != (corner != 0)) continue;
                            LayerTile L{};
                            L.x0 = int32_t(st.x0); L.y0 = int32_t(y0); L.z0 = 0;
                            L.xlo = int32_t(st.lo); L.xhi = int32_t(st.hi);
                            L.ylo = int32_t(y0); L.yhi = int32_t(y0 + len - 1);
                            L.flags = (st.on ? 1 : 0) | (ry.on ? 2 : 0);
                            t.push_back(L);
                        }
                        y0 += len;
                    }
                }
            }
        };
        const int64_t T0 = c->T[0], T1 = c->T[1];
        if (range_empty(ir[0]) || range_empty(ir[1])) {
            add(0, T0 - 1, 0, T1 - 1, band_rows);
        } else if (c->g.wall) {   // no seam to cross: two bands
            if (ir[1].lo > 0) add(0, T0 - 1, 0, ir[1].lo - 1, band_rows);
            if (ir[1].hi < T1 - 1) add(0, T0 - 1, ir[1].hi + 1, T1 - 1, band_rows);
            if (ir[0].lo > 0) add(0, ir[0].lo - 1, ir[1].lo, ir[1].hi, slab_rows);
            if (ir[0].hi < T0 - 1) add(ir[0].hi + 1, T0 - 1, ir[1].lo, ir[1].hi, slab_rows);
        } else {
            const int64_t band = T1 - (ir[1].hi - ir[1].lo + 1);
            if (band > 0) add(0, T0 - 1, ir[1].hi + 1, ir[1].hi + band, band_rows);
            if (ir[0].lo > 0) add(0, ir[0].lo - 1, ir[1].lo, ir[1].hi, slab_rows);
            if (ir[0].hi < T0 - 1) add(ir[0].hi + 1, T0 - 1, ir[1].lo, ir[1].hi, slab_rows);
        }
    } else {
        const int TX = layer3d_tile_x(c->prec), TY = layer3d_tile_y(c->prec), TZ = kLayer3LZ;
        for (const Rect &r : frame_rects(c, ir)) {
            for (int64_t z0 = r.lo[2]; z0 <= r.hi[2]; z0 += TZ)
                for (int64_t y0 = r.lo[1]; y0 <= r.hi[1]; y0 += TY)
                    for (int64_t x0 = r.lo[0] & ~int64_t(3); x0 <= r.hi[0]; x0 += TX) {
                        LayerTile L{};
                        L.x0 = int32_t(x0); L.y0 = int32_t(y0); L.z0 = int32_t(z0);
                        L.xlo = int32_t(r.lo[0]); L.xhi = int32_t(r.hi[0]);
                        L.ylo = int32_t(r.lo[1]); L.yhi = int32_t(r.hi[1]);
                        L.zlo = int32_t(z0); L.zhi = int32_t(std::min<int64_t>(z0 + TZ - 1, r.hi[2]));
                        int fl = 0;
                        if (axis_active(c, 0, x0 - 4, x0 + TX + 4)) fl |= 1;
                        if (axis_active(c, 1, y0 - 4, y0 + TY + 4)) fl |= 2;
                        if (axis_active(c, 2, L.zlo - 4, L.zhi + 5)) fl |= 4;
                        L.flags = fl;
                        t.push_back(L);
                    }
        }
    }
    std::stable_sort(t.begin(), t.end(), [](const LayerTile &a, const LayerTile &b) { return a.flags < b.flags; });
    for (int m = 0; m <= 8; ++m) class_off[m] = 0;
    for (const LayerTile &L : t) class_off[L.flags + 1]++;
    for (int m = 0; m < 8; ++m) class_off[m + 1] += class_off[m];
    return t;
}

// 2D frame tiles: on small grids, where the default runs give fewer items than half the
// warps of a full layer launch, proportionally shorter runs (down to 8 band / 6 slab rows):
// a warp streams its item's rows one after another, so there the launch lasts as long as
// its longest item.  (Below that point longer items win: a layer item has a start-up cost.)
std::vector<LayerTile> build_tiles_2d(const pml_ctx *c, const Range *ir, int class_off[9],
                                      int64_t band0 = kLayer2BandRows, int64_t slab0 = kLayer2SlabRows)
{
    std::vector<LayerTile> t = build_tiles(c, ir, class_off, band0, slab0);
    const size_t target = size_t(8) * size_t(std::max(c->sm_count, 1));
    if (c->nd != 2 || t.empty() || t.size() >= target) return t;
    const double f = double(t.size()) / double(target);
    return build_tiles(c, ir, class_off, std::max<int64_t>(8, int64_t(band0 * f)), std::max<int64_t>(6, int64_t(slab0 * f)));
}

// Slab tiles of the 3D frame of `ir` (FP32 variant 2).  Along each axis a coordinate is
// active when aux fields of that axis are active within 4 vertices of it; each frame
// rectangle is cut into boxes of constant class (the set of active axes), and each box
// into tiles of its class's shape: regions of rx x ry columns whose first column is a
// multiple of 4 (TMA alignment), outputs inset by hx, hy, z items of at most kSlabItemZ
// output planes (z unwrapped across the periodic seam, as in frame_rects).
std::vector<LayerTile> build_slab_tiles(const pml_ctx *c, const Range *ir, int class_off[9])
{
    std::vector<LayerTile> t;
    const std::vector<uint8_t> act[3] = {axis_activity(c, 0), axis_activity(c, 1), axis_activity(c, 2)};
    auto runs = [&](int a, int64_t lo, int64_t hi) { return activity_runs(act[a], lo, hi); };
    auto floor4 = [](int64_t v) { return v >= 0 ? v / 4 * 4 : -((-v + 3) / 4 * 4); };
    for (const Rect &r : frame_rects(c, ir)) {
        for (const ActRun &rz : runs(2, r.lo[2], r.hi[2]))
            for (const ActRun &ry : runs(1, r.lo[1], r.hi[1]))
                for (const ActRun &rx : runs(0, r.lo[0], r.hi[0])) {
                    const int mask = (rx.on ? 1 : 0) | (ry.on ? 2 : 0) | (rz.on ? 4 : 0);
                    int RX, RY, HX, HY;
                    slab3d_shape(mask, &RX, &RY, &HX, &HY);
                    const int64_t nz = rz.hi - rz.lo + 1, nzi = (nz + kSlabItemZ - 1) / kSlabItemZ;
                    int64_t z0 = rz.lo;
                    for (int64_t zi = 0; zi < nzi; ++zi) {
                        const int64_t len = nz / nzi + (zi < nz % nzi ? 1 : 0);
                        for (int64_t ylo = ry.lo; ylo <= ry.hi;) {
                            const int64_t ry0 = ylo - HY, yhi = std::min<int64_t>(ry0 + RY - 1 - HY, ry.hi);
                            for (int64_t xlo = rx.lo; xlo <= rx.hi;) {
                                const int64_t rx0 = floor4(xlo - HX), xhi = std::min<int64_t>(rx0 + RX - 1 - HX, rx.hi);
                                LayerTile L{};
                                L.x0 = int32_t(rx0); L.y0 = int32_t(ry0); L.z0 = int32_t(z0);
                                L.xlo = int32_t(xlo); L.xhi = int32_t(xhi);
                                L.ylo = int32_t(ylo); L.yhi = int32_t(yhi);
                                L.zlo = int32_t(z0); L.zhi = int32_t(z0 + len - 1);
                                L.flags = mask;
                                t.push_back(L);
                                xlo = xhi + 1;
                            }
                            ylo = yhi + 1;
                        }
                        z0 += len;
                    }
                }
    }
    std::stable_sort(t.begin(), t.end(), [](const LayerTile &a, const LayerTile &b) { return a.flags < b.flags; });
    for (int m = 0; m <= 8; ++m) class_off[m] = 0;
    for (const LayerTile &L : t) class_off[L.flags + 1]++;
    for (int m = 0; m < 8; ++m) class_off[m + 1] += class_off[m];
    return t;
}

// Tiles of the 3D level passes over the frame of `ir`: kLevel3TX x kLevel3TY columns by
// kLevel3TZ planes (z unwrapped across the periodic seam, as in frame_rects), with the set of
// axes whose aux fields reach the tile and its one-vertex neighbourhood.
std::vector<LayerTile> level_tiles(const pml_ctx *c, const Range *ir)
{
    std::vector<LayerTile> t;
    for (const Rect &r : frame_rects(c, ir))
        for (int64_t z0 = r.lo[2]; z0 <= r.hi[2]; z0 += kLevel3TZ)
            for (int64_t y0 = r.lo[1]; y0 <= r.hi[1]; y0 += kLevel3TY)
                for (int64_t x0 = r.lo[0] & ~int64_t(kLevel3TX - 1); x0 <= r.hi[0]; x0 += kLevel3TX) {
                    LayerTile L{};
                    L.x0 = int32_t(x0); L.y0 = int32_t(y0); L.z0 = int32_t(z0);
                    L.xlo = int32_t(std::max<int64_t>(x0, r.lo[0]));
                    L.xhi = int32_t(std::min<int64_t>(x0 + kLevel3TX - 1, r.hi[0]));
                    L.ylo = int32_t(y0);
                    L.yhi = int32_t(std::min<int64_t>(y0 + kLevel3TY - 1, r.hi[1]));
                    L.zlo = int32_t(z0);
                    L.zhi = int32_t(std::min<int64_t>(z0 + kLevel3TZ - 1, r.hi[2]));
                    int fl = 0;
                    if (axis_active(c, 0, L.xlo - 2, L.xhi + 3)) fl |= 1;
                    if (axis_active(c, 1, L.ylo - 2, L.yhi + 3)) fl |= 2;
                    if (axis_active(c, 2, L.zlo - 2, L.zhi + 3)) fl |= 4;
                    L.flags = fl;
                    t.push_back(L);
                }
    return t;
}

pml_status encode_map(pml_ctx *c, CUtensorMap *m, void *base, const uint32_t *box)
{
    if (!g_encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return fail(c, PML_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const Geom &g = c->g;
    const cuuint32_t rank = c->nd == 2 ? 2 : 3;
    cuuint64_t dims[3] = {cuuint64_t(g.P), cuuint64_t(g.R), cuuint64_t(g.planes)};
    cuuint64_t strides[2] = {cuuint64_t(g.P) * c->esz, cuuint64_t(g.PS) * c->esz};
    cuuint32_t bx[3] = {box[0], box[1], box[2]};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = g_encode(m, c->esz == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, rank,
                          base, dims, strides, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(c, PML_ECUDA, "cuTensorMapEncodeTiled failed (%d)", int(r));
    return PML_OK;
}

pml_status check_device_error(pml_ctx *c)
{
    DeviceError h{};
    PML_CU(c, cudaMemcpyAsync(&h, c->derr, sizeof h, cudaMemcpyDeviceToHost, c->st), "read error flag");
    PML_CU(c, cudaStreamSynchronize(c->st), "stream synchronize");
    if (h.code == 1) return fail(c, PML_ETIMEOUT, "a bounded device wait gave up (site %d)", h.where);
    if (h.code == 2)
        return fail(c, PML_ENONFINITE, "the state holds a non-finite value (field %s, scan after step %lld)",
                    h.where == 0 ? "U" : "V", h.step);
    if (h.code != 0) return fail(c, PML_ECUDA, "unknown device error code %d", h.code);
    return PML_OK;
}

cudaMemcpyKind kind_of(bool to_dev, bool from_dev)
{
    if (to_dev && from_dev) return cudaMemcpyDeviceToDevice;
    if (to_dev) return cudaMemcpyHostToDevice;
    if (from_dev) return cudaMemcpyDeviceToHost;
    return cudaMemcpyHostToHost;
}

// dense T-grid <-> padded field (interior of the ghost ring)
pml_status copy_dense(pml_ctx *c, void *padded, const void *dense, bool dense_on_dev, bool to_padded)
{
    const Geom &g = c->g;
    cudaMemcpy3DParms p{};
    char *pbase = static_cast<char *>(padded) + size_t(g.origin) * c->esz;
    cudaPitchedPtr pp = make_cudaPitchedPtr(pbase, size_t(g.P) * c->esz, size_t(g.T[0]), size_t(g.R));
    cudaPitchedPtr dp = make_cudaPitchedPtr(const_cast<void *>(dense), size_t(g.T[0]) * c->esz, size_t(g.T[0]),
                                            size_t(g.T[1]));
    p.extent = make_cudaExtent(size_t(g.T[0]) * c->esz, size_t(g.T[1]), size_t(g.T[2]));
    if (to_padded) { p.srcPtr = dp; p.dstPtr = pp; p.kind = kind_of(true, dense_on_dev); }
    else { p.srcPtr = pp; p.dstPtr = dp; p.kind = kind_of(dense_on_dev, true); }
    PML_CU(c, cudaMemcpy3DAsync(&p, c->st), "cudaMemcpy3DAsync");
    return PML_OK;
}

void step_coef(const pml_ctx *c, bool adjoint, StepCoef *k)
{
    const double dt = c->dt, h2 = c->h * c->h, h4 = h2 * h2;
    const double d1 = dt, d2 = dt * dt / 2.0, d3 = dt * dt * dt / 6.0, d4 = dt * dt * dt * dt / 24.0;
    if (!adjoint) {
        k->d = {d1, d2 / h2, d3 / h2, d4 / h4, 0.0, 0.0, d1 / h2, d2 / h2, d3 / h4, d4 / h4};
    } else {
        k->d = {0.0, d2 / h2, d1 / h2, d4 / h4, d3 / h4, d1, d3 / h2, d2 / h2, 0.0, d4 / h4};
    }
    const StepCoefT<double> &e = k->d;
    k->f = {float(e.a1), float(e.a2), float(e.a3), float(e.a4), float(e.a5),
            float(e.b1), float(e.b2), float(e.b3), float(e.b4), float(e.b5)};
}

LayerConst layer_const(const pml_ctx *c)
{
    LayerConst k;
    k.d = {1.0 / c->h, 1.0 / (c->h * c->h), 0.5 / c->h, c->dt / 4.0, c->dt / 3.0, c->dt / 2.0, c->dt};
    k.f = {float(k.d.ih), float(k.d.ih2), float(k.d.i2h), float(k.d.c4), float(k.d.c3), float(k.d.c2), float(k.d.c1)};
    return k;
}

PointArgs point_args(const pml_ctx *c)
{
    PointArgs a{};
    a.g = c->g;
    a.ns = c->ns;
    a.src_off = c->dsrc_off;
    a.src_xyz = c->dsrc_xyz;
    a.src_amp = c->dsrc_amp;
    a.f_peak = c->f_peak;
    a.t_delay = c->t_delay;
    a.nr = c->nr;
    a.rec_off = c->drec_off;
    a.src_level = c->dsrc_level;
    a.src_levels = c->src_levels;
    a.rec_xyz = c->drec_xyz;
    a.rec_level = c->drec_level;
    a.rec_levels = c->rec_levels;
    a.dt = c->dt;
    a.h = c->h;
    return a;
}

// Event pair around one kernel launch when profiling is on; returns the pair index.
long prof_begin(pml_ctx *c, int kind)
{
    if (!c->prof_on) return -1;
    if (c->prof_n == c->prof_kind.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) return -1;
        if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return -1; }
        c->prof_ev.push_back(a);
        c->prof_ev.push_back(b);
        c->prof_kind.push_back(kind);
    }
    const size_t i = c->prof_n++;
    c->prof_kind[i] = kind;
    cudaEventRecord(c->prof_ev[2 * i], c->st);
    return long(i);
}

void prof_end(pml_ctx *c, long i)
{
    if (i >= 0) cudaEventRecord(c->prof_ev[2 * size_t(i) + 1], c->st);
}

// NVTX range over one library call (header-only NVTX: without an attached tool the push
// and pop cost a branch each).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Finiteness scan of the given state's U and V when the step counter went from `before`
// to `after` across a multiple of the scan interval.
pml_status maybe_check_finite(pml_ctx *c, void *const *state, int64_t before, int64_t after)
{
    const int64_t k = c->check_every;
    if (k <= 0 || before == after) return PML_OK;
    auto fl = [k](int64_t v) { return v >= 0 ? v / k : -((-v + k - 1) / k); };
    if (fl(before) == fl(after)) return PML_OK;
    const long pi = prof_begin(c, 2);
    const cudaError_t e = launch_check_finite(c->prec, state[0], state[1], c->g, c->derr, after, c->st);
    prof_end(c, pi);
    if (e != cudaSuccess) return cuda_fail(c, e, "finiteness scan");
    return PML_OK;
}

// Row chunks {x0, x1, y, z} (at most kStageChunkMax vertices) of C_r: the vertices within r
// stencil steps of those the damping-gradient contraction reads (along each axis a, the
// coordinates e and e + 1 of every edge e with sigma_a[e] != 0).  The stencil is a cross,
// so C_r is the union over the axes of those slabs widened by r along their own axis
// (periodic distance, or plain distance with walls).
void gradient_segments(const pml_ctx *c, int r, std::vector<int4> *out)
{
    std::vector<uint8_t> m[3];
    for (int a = 0; a < 3; ++a) {
        const int64_t T = c->T[a];
        m[a].assign(size_t(T), 0);
        if (a >= c->nd) continue;
        std::vector<uint8_t> base(size_t(T), 0);
        for (int64_t e = 0; e < T; ++e)
            if (c->sig[a][size_t(e)] != 0.0) {
                base[size_t(e)] = 1;
                base[size_t((e + 1) % T)] = 1;
            }
        for (int64_t i = 0; i < T; ++i) {
            if (!base[size_t(i)]) continue;
            for (int64_t d = -r; d <= r; ++d) {
                int64_t j = i + d;
                if (c->g.wall) {
                    if (j < 0 || j >= T) continue;
                } else {
                    j = ((j % T) + T) % T;
                }
                m[a][size_t(j)] = 1;
            }
        }
    }
    out->clear();
    const int64_t T0 = c->T[0], T1 = c->T[1], T2 = c->nd == 3 ? c->T[2] : 1;
    for (int64_t z = 0; z < T2; ++z)
        for (int64_t y = 0; y < T1; ++y) {
            auto push = [&](int64_t x0, int64_t x1) {   // chunks of at most kStageChunkMax vertices
                for (int64_t a0 = x0; a0 <= x1; a0 += kStageChunkMax)
                    out->push_back(make_int4(int(a0), int(std::min<int64_t>(a0 + kStageChunkMax - 1, x1)), int(y), int(z)));
            };
            if (m[1][size_t(y)] || (c->nd == 3 && m[2][size_t(z)])) {
                push(0, T0 - 1);
                continue;
            }
            for (int64_t x = 0; x < T0;) {
                if (!m[0][size_t(x)]) { ++x; continue; }
                int64_t x1 = x;
                while (x1 + 1 < T0 && m[0][size_t(x1 + 1)]) ++x1;
                push(x, x1);
                x = x1 + 1;
            }
        }
}

// Steps between checkpoints of the damping gradient: `interval`, or ceil(sqrt(n)) for 0.
int64_t checkpoint_interval(int64_t n, int64_t interval)
{
    int64_t K = interval;
    if (K <= 0) {
        K = int64_t(std::ceil(std::sqrt(double(n))));
        while (K * K < n) ++K;
    }
    return K > n ? n : K;
}

pml_status clear_device_error(pml_ctx *c)
{
    PML_CU(c, cudaMemsetAsync(c->derr, 0, sizeof(DeviceError), c->st), "clear error flag");
    return PML_OK;
}

// One step (forward or transposed) from buffers `in` to buffers `out`.
pml_status enqueue_step(pml_ctx *c, bool adjoint, int p)
{
    const int q = 1 - p;
    void **out = adjoint ? c->adj[q] : c->fld[q];
    const Range *ir = adjoint ? c->ir_adj : c->ir;
    StepCoef k;
    step_coef(c, adjoint, &k);
    const CUtensorMap *ti = adjoint ? c->tm_int_adj[p] : c->tm_int[p];
    const CUtensorMap *tl = adjoint ? c->tm_lay_adj[p] : c->tm_lay[p];
    cudaError_t e;
    if (c->nd == 2) {
        Layer2DArgs l{};
        l.g = c->g; l.k = layer_const(c);
        l.sig[0] = c->dsig[0]; l.sig[1] = c->dsig[1];
        l.tiles = adjoint ? c->dtiles_adj : c->dtiles;
        l.ntiles = adjoint ? c->ntiles_adj : c->ntiles;
        l.err = c->derr;
        l.wait_ns = c->wait_ns;
        int64_t &ll = adjoint ? c->launches_layer_adj : c->launches_layer_fwd;
        l.queue = c->dqueue + (adjoint ? 6 : 4);
        l.parity = int(ll & 1);
        if (l.ntiles > 0) ++ll;
        long pi = prof_begin(c, 1);
        e = launch_layer2d(c->prec, adjoint, tl, out, l, layer2d_grid(c->prec, l.ntiles, c->sm_count), c->st);
        prof_end(c, pi);
        if (e != cudaSuccess) return cuda_fail(c, e, "layer 2D kernel");
        Interior2DArgs a{};
        a.g = c->g; a.xr = ir[0]; a.yr = ir[1]; a.c = k; a.err = c->derr; a.wait_ns = c->wait_ns;
        // small grids: shorter work items (down to 16 rows) so that every warp of the launch
        // gets one (a warp streams its item's rows one after another)
        if (!range_empty(ir[0]) && !range_empty(ir[1])) {
            const int64_t nrows = ir[1].hi - ir[1].lo + 1;
            const int64_t nstrips = (ir[0].hi - (ir[0].lo & ~int64_t(3))) / 120 + 1;
            const int64_t warps = int64_t(adjoint ? c->grid_int_adj : c->grid_int) * 4;
            const int64_t items = nstrips * ((nrows + 63) / 64);
            if (items < warps) a.rows = int(std::max<int64_t>(16, (nrows * nstrips + warps - 1) / warps));
        }
        int64_t &nl = adjoint ? c->launches_adj : c->launches_fwd;
        a.queue = c->dqueue + (adjoint ? 2 : 0);
        a.parity = int(nl & 1);
        // overlap with the layer kernel only when no event sits between the two launches
        pi = prof_begin(c, 0);
        e = launch_interior2d(c->prec, adjoint, c->ivar, &ti[0], &ti[1], out[0], out[1], a,
                              adjoint ? c->grid_int_adj : c->grid_int, c->st, l.ntiles > 0 && !c->prof_on);
        prof_end(c, pi);
        if (e != cudaSuccess) return cuda_fail(c, e, "interior 2D kernel");
        if (!range_empty(ir[0]) && !range_empty(ir[1])) ++nl;
    } else {
        // layer classes first (chained), then the interior kernel overlapping them; all
        // read only the step's input and write disjoint outputs
        bool layer_launched;
        if (c->ivar == 1) {   // level passes: z4, z3, z2 into the scratch states, then y'
            void **in = adjoint ? c->adj[p] : c->fld[p];
            const int d = adjoint ? 1 : 0;
            Level3Args L{};
            L.g = c->g; L.k = layer_const(c);
            for (int a2 = 0; a2 < 3; ++a2) L.sig[a2] = c->dsig[a2];
            for (int f = 0; f < 8; ++f) L.base[f] = in[f];
            layer_launched = false;
            for (int k = 0; k < 4; ++k) {
                for (int f = 0; f < 8; ++f) {
                    L.in[f] = k == 0 ? in[f] : c->lvl[(k - 1) & 1][f];
                    L.out[f] = k == 3 ? out[f] : c->lvl[k & 1][f];
                }
                L.tiles = c->dlt[d][k];
                L.ntiles = c->nlt[d][k];
                L.level = 4 - k;
                long pi = prof_begin(c, 1);
                e = launch_level3d(c->prec, adjoint, L, c->st);
                prof_end(c, pi);
                if (e != cudaSuccess) return cuda_fail(c, e, "level pass 3D kernel");
                layer_launched = layer_launched || L.ntiles > 0;
            }
        } else if (c->ivar == 2) {   // slab tiles (FP32)
            const int d = adjoint ? 1 : 0;
            Layer3DArgs l{};
            l.g = c->g; l.k = layer_const(c);
            for (int a2 = 0; a2 < 3; ++a2) l.sig[a2] = c->dsig[a2];
            l.tiles = c->dslab[d];
            l.ntiles = c->nslab[d];
            for (int m = 0; m < 9; ++m) l.class_off[m] = c->slab_off[d][m];
            l.err = c->derr;
            l.wait_ns = c->wait_ns;
            long pi = prof_begin(c, 1);
            e = launch_slab3d(adjoint, c->tm_slab[d][p], out, l, c->st);
            prof_end(c, pi);
            if (e != cudaSuccess) {
                char what[256];
                std::snprintf(what, sizeof what, "slab 3D kernel (%s)", slab3d_describe(adjoint, c->g.wall != 0).c_str());
                return cuda_fail(c, e, what);
            }
            layer_launched = l.ntiles > 0;
        } else {
            Layer3DArgs l{};
            l.g = c->g; l.k = layer_const(c);
            for (int a2 = 0; a2 < 3; ++a2) l.sig[a2] = c->dsig[a2];
            l.tiles = adjoint ? c->dtiles_adj : c->dtiles;
            l.ntiles = adjoint ? c->ntiles_adj : c->ntiles;
            for (int m = 0; m < 9; ++m) l.class_off[m] = adjoint ? c->class_off_adj[m] : c->class_off[m];
            l.err = c->derr;
            l.wait_ns = c->wait_ns;
            long pi = prof_begin(c, 1);
            e = launch_layer3d(c->prec, adjoint, tl, out, l, c->st);
            prof_end(c, pi);
            if (e != cudaSuccess) return cuda_fail(c, e, "layer 3D kernel");
            layer_launched = l.ntiles > 0;
        }
        Interior3DArgs a{};
        a.g = c->g; a.xr = ir[0]; a.yr = ir[1]; a.zr = ir[2]; a.c = k; a.err = c->derr; a.wait_ns = c->wait_ns;
        int64_t &nl = adjoint ? c->launches_adj : c->launches_fwd;
        a.queue = c->dqueue + (adjoint ? 2 : 0);
        a.parity = int(nl & 1);
        if (!range_empty(ir[0]) && !range_empty(ir[1]) && !range_empty(ir[2])) ++nl;
        const long pi = prof_begin(c, 0);
        e = launch_interior3d(c->prec, adjoint, &ti[0], &ti[1], out[0], out[1], a,
                              adjoint ? c->grid_int_adj : c->grid_int, layer_launched && !c->prof_on, c->st);
        prof_end(c, pi);
        if (e != cudaSuccess) return cuda_fail(c, e, "interior 3D kernel");
    }
    return PML_OK;
}

// Two forward steps from buffers `p` to buffers `1 - p` (temporal blocking depth 2, 2D):
//   layer pass 1: step n+1 on the frame of the run shrunk by 6, fld[p] -> mid;
//   layer pass 2: step n+2 on the frame of the run shrunk by 2, mid -> fld[1-p]; launched
//                 early, it waits for pass 1 before reading;
//   interior:     steps n+1, n+2 in one pass on the run shrunk by 2, fld[p] -> fld[1-p];
//                 launched while pass 2 runs, it completes only after pass 2.
pml_status enqueue_double_step(pml_ctx *c, bool adjoint, int p)
{
    const int q = 1 - p;
    StepCoef k;
    step_coef(c, adjoint, &k);
    void **out = adjoint ? c->adj[q] : c->fld[q];
    Layer2DArgs l{};
    l.g = c->g; l.k = layer_const(c);
    l.sig[0] = c->dsig[0]; l.sig[1] = c->dsig[1];
    l.err = c->derr;
    l.wait_ns = c->wait_ns;
    l.tiles = adjoint ? c->dtiles_l1_adj : c->dtiles_l1;
    l.ntiles = adjoint ? c->ntiles_l1_adj : c->ntiles_l1;
    int64_t &ll = adjoint ? c->launches_layer_adj : c->launches_layer_fwd;
    l.queue = c->dqueue + (adjoint ? 6 : 4);
    l.parity = int(ll & 1);
    if (l.ntiles > 0) ++ll;
    long pi = prof_begin(c, 1);
    cudaError_t e = launch_layer2d(c->prec, adjoint, adjoint ? c->tm_lay_adj[p] : c->tm_lay[p], c->mid, l,
                                   layer2d_grid(c->prec, l.ntiles, c->sm_count), c->st);
    prof_end(c, pi);
    if (e != cudaSuccess) return cuda_fail(c, e, "layer 2D kernel (pass 1)");
    const bool pass1 = l.ntiles > 0;
    l.tiles = adjoint ? c->dtiles_l2_adj : c->dtiles_l2;
    l.ntiles = adjoint ? c->ntiles_l2_adj : c->ntiles_l2;
    int64_t &l2 = adjoint ? c->launches_layer2_adj : c->launches_layer2;
    l.queue = c->dqueue + (adjoint ? 10 : 8);
    l.parity = int(l2 & 1);
    if (l.ntiles > 0) ++l2;
    pi = prof_begin(c, 1);
    e = launch_layer2d(c->prec, adjoint, c->tm_mid, out, l, layer2d_grid(c->prec, l.ntiles, c->sm_count), c->st,
                       pass1 && !c->prof_on);
    prof_end(c, pi);
    if (e != cudaSuccess) return cuda_fail(c, e, "layer 2D kernel (pass 2)");
    Interior2DArgs a{};
    const Range *irt = adjoint ? c->ir_tb_adj : c->ir_tb;
    a.g = c->g; a.xr = irt[0]; a.yr = irt[1]; a.c = k; a.err = c->derr; a.wait_ns = c->wait_ns;
    int64_t &nl = adjoint ? c->launches_adj : c->launches_fwd;
    a.queue = c->dqueue + (adjoint ? 2 : 0);
    a.parity = int(nl & 1);
    const CUtensorMap *tt = adjoint ? c->tm_tb_adj[p] : c->tm_tb[p];
    pi = prof_begin(c, 0);
    e = launch_interior2d_tb2(c->prec, adjoint, c->tbvar, &tt[0], &tt[1], out[0], out[1], a,
                              adjoint ? c->grid_tb_adj : c->grid_tb, c->st, (pass1 || l.ntiles > 0) && !c->prof_on);
    prof_end(c, pi);
    if (e != cudaSuccess) return cuda_fail(c, e, "interior 2D kernel (two steps)");
    if (!range_empty(a.xr) && !range_empty(a.yr)) ++nl;
    return PML_OK;
}

// 2D: the interior kernel's shapes; 3D: 0 the z-streaming layer tile kernel, 1 level passes,
// 2 (FP32) slab tiles
int one_step_variants(const pml_ctx *c) { return c->nd == 2 ? interior2d_variants(c->prec) : (c->prec == 32 ? 3 : 2); }
int two_step_variants(const pml_ctx *c) { return c->plan.tb2 ? interior2d_tb2_variants(c->prec) : 0; }

// Grid sizes of the interior kernels for the current variant: all resident CTAs.
pml_status interior_grids(pml_ctx *c)
{
    const bool adj = (c->flags & PML_FLAG_ADJOINT) != 0;
    int bps = c->nd == 2 ? interior2d_max_blocks_per_sm(c->prec, false, c->ivar) : interior3d_max_blocks_per_sm(c->prec, false);
    int bpa = adj ? (c->nd == 2 ? interior2d_max_blocks_per_sm(c->prec, true, c->ivar) : interior3d_max_blocks_per_sm(c->prec, true))
                  : 0;
    if (bps <= 0 || (adj && bpa <= 0))
        return fail(c, PML_ECUDA, "interior kernel cannot be resident (shared memory / registers)");
    c->grid_int = bps * c->sm_count;
    c->grid_int_adj = bpa * c->sm_count;
    if (c->plan.tb2) {
        const int bt = interior2d_tb2_max_blocks_per_sm(c->prec, false, c->tbvar);
        const int bta = adj ? interior2d_tb2_max_blocks_per_sm(c->prec, true, c->tbvar) : 1;
        if (bt <= 0 || bta <= 0)
            return fail(c, PML_ECUDA, "two-step interior kernel cannot be resident (shared memory / registers)");
        c->grid_tb = bt * c->sm_count;
        c->grid_tb_adj = bta * c->sm_count;
    }
    return PML_OK;
}

// Tensor maps of the two-step interior kernel (U, V of both ping-pong halves) for its
// current variant's box.
pml_status encode_tb_maps(pml_ctx *c)
{
    if (!c->plan.tb2) return PML_OK;
    uint32_t box[3] = {uint32_t(interior2d_tb2_box_cols(c->prec, c->tbvar)),
                       uint32_t(interior2d_tb2_box_rows(c->prec, c->tbvar)), 1};
    pml_status s;
    for (int p = 0; p < 2; ++p)
        for (int f = 0; f < 2; ++f) {
            if ((s = encode_map(c, &c->tm_tb[p][f], c->fld[p][f], box)) != PML_OK) return s;
            if ((c->flags & PML_FLAG_ADJOINT) && (s = encode_map(c, &c->tm_tb_adj[p][f], c->adj[p][f], box)) != PML_OK)
                return s;
        }
    return PML_OK;
}

// Tensor maps of the 2D interior kernel for the current variant's box.
pml_status encode_interior_maps(pml_ctx *c)
{
    if (c->nd != 2) return PML_OK;
    uint32_t box[3] = {uint32_t(interior2d_box_cols(c->prec, c->ivar)), uint32_t(interior2d_box_rows(c->prec, c->ivar)), 1};
    pml_status s;
    for (int p = 0; p < 2; ++p)
        for (int f = 0; f < 2; ++f) {
            if ((s = encode_map(c, &c->tm_int[p][f], c->fld[p][f], box)) != PML_OK) return s;
            if ((c->flags & PML_FLAG_ADJOINT) && (s = encode_map(c, &c->tm_int_adj[p][f], c->adj[p][f], box)) != PML_OK)
                return s;
        }
    return PML_OK;
}

}  // namespace

namespace pml {
// error text of context-free calls (read back by pml_last_error(NULL))
void set_global_error(const char *msg) { g_create_error = msg; }
}  // namespace pml

extern "C" {

const char *pml_status_string(pml_status s)
{
    switch (s) {
    case PML_OK: return "ok";
    case PML_EINVAL: return "invalid argument";
    case PML_ENOMEM: return "out of memory";
    case PML_ECUDA: return "CUDA error";
    case PML_ESTATE: return "invalid state";
    case PML_EUNSTABLE: return "time step beyond the RK4 stability limit";
    case PML_ENONFINITE: return "non-finite value";
    case PML_ETIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

const char *pml_last_error(const pml_ctx *c) { return c ? c->err.c_str() : g_create_error.c_str(); }

pml_status pml_workspace_bytes(const pml_grid *grid, int pml_width, int precision, int flags, size_t *bytes)
{
    Plan p;
    std::string why;
    if (!bytes) return fail(nullptr, PML_EINVAL, "bytes is NULL");
    if (!make_plan(grid, pml_width, precision, flags, &p, &why)) return fail(nullptr, PML_EINVAL, "%s", why.c_str());
    *bytes = p.total;
    return PML_OK;
}

pml_status pml_plan_layer_items(const pml_grid *grid, int pml_width, const pml_sigma_profile *profile,
                                int precision, int flags, int sm_count, int which, int32_t *out, int64_t cap,
                                int64_t *count)
{
    if (!count) return fail(nullptr, PML_EINVAL, "count is NULL");
    *count = 0;
    Plan plan;
    std::string why;
    if (!make_plan(grid, pml_width, precision, flags, &plan, &why)) return fail(nullptr, PML_EINVAL, "%s", why.c_str());
    if (sm_count < 1) return fail(nullptr, PML_EINVAL, "sm_count must be >= 1");
    if (which < 0 || which > 4) return fail(nullptr, PML_EINVAL, "which must be 0..4");
    if ((which == 1 || which == 2 || which == 4) && !(plan.nd == 2 && precision == 32))
        return fail(nullptr, PML_EINVAL, "item sets 1, 2 and 4 belong to 2D FP32 boxes");
    if (which == 3 && !(plan.nd == 3 && precision == 32))
        return fail(nullptr, PML_EINVAL, "item set 3 belongs to 3D FP32 boxes");
    if (which == 0 && plan.nd != 2) return fail(nullptr, PML_EINVAL, "item set 0 belongs to 2D boxes");
    if (cap < 0 || (cap > 0 && !out)) return fail(nullptr, PML_EINVAL, "out is NULL or cap < 0");
    // a host-side context: the damping, its supports and the layer-free runs, no device state
    std::unique_ptr<pml_ctx> c(new pml_ctx());
    c->plan = plan;
    c->nd = plan.nd; c->prec = precision; c->esz = plan.esz; c->nf = plan.nf; c->flags = flags;
    c->w = pml_width; c->g = plan.g; c->sm_count = sm_count;
    for (int a = 0; a < 3; ++a) { c->N[a] = a < c->nd ? grid->n[a] : 1; c->T[a] = plan.T[a]; }
    pml_status s = build_sigma(c.get(), profile);
    if (s != PML_OK) return s;
    build_layout(c.get());
    int co[9];
    std::vector<LayerTile> t;
    Range r[3];
    switch (which) {
    case 0: {
        const int64_t slab1 = c->g.wall ? kLayer2SlabRowsWall : kLayer2SlabRows;
        t = build_tiles_2d(c.get(), c->ir, co, kLayer2BandRows, slab1);
        break;
    }
    case 1:
    case 2:
        for (int a = 0; a < 3; ++a) r[a] = shrink_run(c->ir[a], c->T[a], which == 1 ? 6 : 2);
        t = build_tiles_2d(c.get(), r, co, kLayer2BandRowsTB, c->g.wall ? kLayer2SlabRowsWall : kLayer2SlabRowsTB);
        break;
    case 3: t = build_slab_tiles(c.get(), c->ir, co); break;
    default: t = build_tiles(c.get(), c->ir, co, kLayer2BandRowsBatch, kLayer2SlabRowsBatch); break;
    }
    *count = int64_t(t.size());
    for (int64_t i = 0; i < cap && i < *count; ++i) {
        const LayerTile &L = t[size_t(i)];
        const int32_t v[10] = {L.x0, L.y0, L.z0, L.xlo, L.xhi, L.ylo, L.yhi, L.zlo, L.zhi, L.flags};
        for (int k = 0; k < 10; ++k) out[10 * i + k] = v[k];
    }
    return PML_OK;
}

pml_status pml_create(const pml_grid *grid, double h, double dt, int pml_width, const pml_sigma_profile *profile,
                      int precision, void *cuda_stream, void *workspace, size_t workspace_bytes, int flags,
                      pml_ctx **out)
{
    if (!out) return fail(nullptr, PML_EINVAL, "out is NULL");
    *out = nullptr;
    Plan plan;
    std::string why;
    if (!make_plan(grid, pml_width, precision, flags, &plan, &why)) return fail(nullptr, PML_EINVAL, "%s", why.c_str());
    if (!(h > 0.0) || !std::isfinite(h)) return fail(nullptr, PML_EINVAL, "h must be finite and > 0");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(nullptr, PML_EINVAL, "dt must be finite and > 0");
    // RK4 is stable on the imaginary axis up to |z| = 2 sqrt(2); the discrete Laplacian's
    // largest frequency is 2 sqrt(d) / h, hence dt <= sqrt(2/d) h.
    if (dt > std::sqrt(2.0 / grid->ndim) * h * (1.0 + 1e-12))
        return fail(nullptr, PML_EUNSTABLE, "dt = %g exceeds sqrt(2/%d) h = %g", dt, grid->ndim,
                    std::sqrt(2.0 / grid->ndim) * h);
    if (workspace && workspace_bytes < plan.total)
        return fail(nullptr, PML_ENOMEM, "workspace has %zu bytes, %zu needed", workspace_bytes, plan.total);
    if (workspace && (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0)
        return fail(nullptr, PML_EINVAL, "workspace must be 256-byte aligned");

    pml_ctx *c = new pml_ctx();
    c->plan = plan;
    c->nd = plan.nd; c->prec = precision; c->esz = plan.esz; c->nf = plan.nf; c->flags = flags;
    c->w = pml_width; c->h = h; c->dt = dt; c->g = plan.g;
    for (int a = 0; a < 3; ++a) { c->N[a] = a < c->nd ? grid->n[a] : 1; c->T[a] = plan.T[a]; }
    c->st = static_cast<cudaStream_t>(cuda_stream);

    auto bail = [&](pml_status s) {
        g_create_error = c->err;
        if (c->own_ws && c->ws) cudaFree(c->ws);
        delete c;
        return s;
    };
    pml_status s = build_sigma(c, profile);
    if (s != PML_OK) return bail(s);
    build_layout(c);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        fail(c, PML_ECUDA, "no CUDA device");
        return bail(PML_ECUDA);
    }
    if (workspace) {
        c->ws = static_cast<char *>(workspace);
    } else {
        cudaError_t e = cudaMalloc(&c->ws, plan.total);
        if (e != cudaSuccess) {
            c->ws = nullptr;
            fail(c, PML_ENOMEM, "cudaMalloc(%zu): %s", plan.total, cudaGetErrorString(e));
            return bail(PML_ENOMEM);
        }
        c->own_ws = true;
    }
    for (int p = 0; p < 2; ++p)
        for (int f = 0; f < c->nf; ++f) {
            c->fld[p][f] = c->ws + plan.fields[p][f];
            if (flags & PML_FLAG_ADJOINT) c->adj[p][f] = c->ws + plan.adj[p][f];
        }
    if (plan.tb2) {
        for (int f = 0; f < c->nf; ++f) c->mid[f] = c->ws + plan.mid[f];
        c->dtiles_l1 = reinterpret_cast<LayerTile *>(c->ws + plan.tiles_l1);
        c->dtiles_l2 = reinterpret_cast<LayerTile *>(c->ws + plan.tiles_l2);
        if (flags & PML_FLAG_ADJOINT) {
            c->dtiles_l1_adj = reinterpret_cast<LayerTile *>(c->ws + plan.tiles_l1_adj);
            c->dtiles_l2_adj = reinterpret_cast<LayerTile *>(c->ws + plan.tiles_l2_adj);
        }
    }
    if (c->nd == 3)
        for (int s2 = 0; s2 < 2; ++s2)
            for (int f = 0; f < c->nf; ++f) c->lvl[s2][f] = c->ws + plan.lvl[s2][f];
    for (int a = 0; a < c->nd; ++a) c->dsig[a] = c->ws + plan.sig[a];
    c->dtiles = reinterpret_cast<LayerTile *>(c->ws + plan.tiles);
    c->dtiles_adj = reinterpret_cast<LayerTile *>(c->ws + plan.tiles_adj);
    c->dpart = reinterpret_cast<double *>(c->ws + plan.partials);
    c->dnorm = reinterpret_cast<double *>(c->ws + plan.normout);
    c->derr = reinterpret_cast<DeviceError *>(c->ws + plan.err);
    c->dqueue = reinterpret_cast<int *>(c->ws + plan.queue);
    c->dsrc_off = reinterpret_cast<int64_t *>(c->ws + plan.src_off);
    c->dsrc_xyz = reinterpret_cast<int32_t *>(c->ws + plan.src_xyz);
    c->dsrc_amp = reinterpret_cast<double *>(c->ws + plan.src_amp);
    c->dgrad = reinterpret_cast<double *>(c->ws + plan.grad);
    c->drec_off = reinterpret_cast<int64_t *>(c->ws + plan.rec_off);
    c->dsrc_level = reinterpret_cast<int32_t *>(c->ws + plan.src_level);
    c->drec_xyz = reinterpret_cast<int32_t *>(c->ws + plan.rec_xyz);
    c->drec_level = reinterpret_cast<int32_t *>(c->ws + plan.rec_level);

    // state = 0 everywhere (both ping-pong halves, adjoint too)
    {
        cudaError_t e = cudaMemsetAsync(c->ws, 0, plan.sig[0], c->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->derr, 0, sizeof(DeviceError), c->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->dqueue, 0, 16 * sizeof(int), c->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->dgrad, 0, kMaxSources * sizeof(double), c->st);
        if (e != cudaSuccess) { cuda_fail(c, e, "clear workspace"); return bail(PML_ECUDA); }
    }
    // damping in the state precision
    for (int a = 0; a < c->nd; ++a) {
        std::vector<char> buf(size_t(c->T[a]) * c->esz);
        for (int64_t i = 0; i < c->T[a]; ++i) {
            if (c->esz == 4) reinterpret_cast<float *>(buf.data())[i] = float(c->sig[a][size_t(i)]);
            else reinterpret_cast<double *>(buf.data())[i] = c->sig[a][size_t(i)];
        }
        cudaError_t e = cudaMemcpy(c->dsig[a], buf.data(), buf.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cuda_fail(c, e, "upload sigma"); return bail(PML_ECUDA); }
    }
    // layer tiles
    {
        const int64_t slab1 = c->g.wall ? kLayer2SlabRowsWall : kLayer2SlabRows;
        std::vector<LayerTile> tf = build_tiles_2d(c, c->ir, c->class_off, kLayer2BandRows, slab1),
                               ta = build_tiles_2d(c, c->ir_adj, c->class_off_adj, kLayer2BandRows, slab1);
        if (tf.size() > plan.max_tiles || ta.size() > plan.max_tiles) {
            fail(c, PML_ENOMEM, "layer tile table exceeds its bound");
            return bail(PML_ENOMEM);
        }
        c->ntiles = int(tf.size());
        c->ntiles_adj = int(ta.size());
        cudaError_t e = cudaSuccess;
        if (!tf.empty()) e = cudaMemcpy(c->dtiles, tf.data(), tf.size() * sizeof(LayerTile), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !ta.empty() && (flags & PML_FLAG_ADJOINT))
            e = cudaMemcpy(c->dtiles_adj, ta.data(), ta.size() * sizeof(LayerTile), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cuda_fail(c, e, "upload tiles"); return bail(PML_ECUDA); }
    }
    // 3D level passes: level 4 - k on the frame of the run shrunk by 3 - k
    if (c->nd == 3) {
        for (int d = 0; d < ((flags & PML_FLAG_ADJOINT) ? 2 : 1); ++d)
            for (int k = 0; k < 4; ++k) {
                Range rr[3];
                for (int a = 0; a < 3; ++a) rr[a] = shrink_run(d ? c->ir_adj[a] : c->ir[a], c->T[a], 3 - k);
                std::vector<LayerTile> lt = level_tiles(c, rr);
                if (lt.size() > plan.max_ltiles) {
                    fail(c, PML_ENOMEM, "level tile table exceeds its bound");
                    return bail(PML_ENOMEM);
                }
                c->dlt[d][k] = reinterpret_cast<LayerTile *>(c->ws + plan.ltiles[d][k]);
                c->nlt[d][k] = int(lt.size());
                cudaError_t e = lt.empty() ? cudaSuccess
                                           : cudaMemcpy(c->dlt[d][k], lt.data(), lt.size() * sizeof(LayerTile),
                                                        cudaMemcpyHostToDevice);
                if (e != cudaSuccess) { cuda_fail(c, e, "upload level tiles"); return bail(PML_ECUDA); }
            }
    }
    // 3D FP32 slab tiles (variant 2)
    if (c->nd == 3 && c->prec == 32) {
        for (int d = 0; d < ((flags & PML_FLAG_ADJOINT) ? 2 : 1); ++d) {
            std::vector<LayerTile> st = build_slab_tiles(c, d ? c->ir_adj : c->ir, c->slab_off[d]);
            if (st.size() > plan.max_slab) {
                fail(c, PML_ENOMEM, "slab tile table exceeds its bound");
                return bail(PML_ENOMEM);
            }
            c->dslab[d] = reinterpret_cast<LayerTile *>(c->ws + plan.slab_tiles[d]);
            c->nslab[d] = int(st.size());
            cudaError_t e = st.empty() ? cudaSuccess
                                       : cudaMemcpy(c->dslab[d], st.data(), st.size() * sizeof(LayerTile),
                                                    cudaMemcpyHostToDevice);
            if (e != cudaSuccess) { cuda_fail(c, e, "upload slab tiles"); return bail(PML_ECUDA); }
        }
    }
    // two-step blocks: the second pass writes the frame of the run shrunk by 2, from first-
    // step values the first pass writes on the frame of the run shrunk by 6 (4 more: the
    // reach of one layer step)
    if (plan.tb2) {
        Range r6[3], r2[3];
        for (int a = 0; a < 3; ++a) {
            r6[a] = shrink_run(c->ir[a], c->T[a], 6);
            r2[a] = c->ir_tb[a] = shrink_run(c->ir[a], c->T[a], 2);
        }
        // shorter items than the one-step frame's: these passes run alone or beside the
        // interior kernel, so a pass lasts as long as its longest item; about one short item
        // per warp of a full launch
        int dummy[9];
        const int64_t slab2 = c->g.wall ? kLayer2SlabRowsWall : kLayer2SlabRowsTB;
        std::vector<LayerTile> t1 = build_tiles_2d(c, r6, dummy, kLayer2BandRowsTB, slab2),
                               t2 = build_tiles_2d(c, r2, dummy, kLayer2BandRowsTB, slab2);
        if (t1.size() > plan.max_tiles || t2.size() > plan.max_tiles) {
            fail(c, PML_ENOMEM, "layer tile table exceeds its bound");
            return bail(PML_ENOMEM);
        }
        c->ntiles_l1 = int(t1.size());
        c->ntiles_l2 = int(t2.size());
        cudaError_t e = cudaSuccess;
        if (!t1.empty()) e = cudaMemcpy(c->dtiles_l1, t1.data(), t1.size() * sizeof(LayerTile), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !t2.empty())
            e = cudaMemcpy(c->dtiles_l2, t2.data(), t2.size() * sizeof(LayerTile), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cuda_fail(c, e, "upload tiles"); return bail(PML_ECUDA); }
        if (flags & PML_FLAG_ADJOINT) {   // the same for the transposed step's frames
            for (int a = 0; a < 3; ++a) {
                r6[a] = shrink_run(c->ir_adj[a], c->T[a], 6);
                r2[a] = c->ir_tb_adj[a] = shrink_run(c->ir_adj[a], c->T[a], 2);
            }
            std::vector<LayerTile> a1 = build_tiles_2d(c, r6, dummy, kLayer2BandRowsTB, slab2),
                                   a2 = build_tiles_2d(c, r2, dummy, kLayer2BandRowsTB, slab2);
            if (a1.size() > plan.max_tiles || a2.size() > plan.max_tiles) {
                fail(c, PML_ENOMEM, "layer tile table exceeds its bound");
                return bail(PML_ENOMEM);
            }
            c->ntiles_l1_adj = int(a1.size());
            c->ntiles_l2_adj = int(a2.size());
            if (!a1.empty()) e = cudaMemcpy(c->dtiles_l1_adj, a1.data(), a1.size() * sizeof(LayerTile), cudaMemcpyHostToDevice);
            if (e == cudaSuccess && !a2.empty())
                e = cudaMemcpy(c->dtiles_l2_adj, a2.data(), a2.size() * sizeof(LayerTile), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) { cuda_fail(c, e, "upload tiles"); return bail(PML_ECUDA); }
        }
    }
    // tensor maps
    {
        uint32_t box_int[3], box_lay[3];
        if (c->nd == 2) {
            box_int[0] = uint32_t(interior2d_box_cols(precision, c->ivar));
            box_int[1] = uint32_t(interior2d_box_rows(precision, c->ivar)); box_int[2] = 1;
            box_lay[0] = uint32_t(layer2d_box_cols(precision)); box_lay[1] = uint32_t(layer2d_box_rows());
            box_lay[2] = 1;   // one warp's strip
        } else {
            box_int[0] = uint32_t(interior3d_box_cols(precision)); box_int[1] = uint32_t(interior3d_tile_y(precision) + 4); box_int[2] = uint32_t(interior3d_box_rows(precision));
            box_lay[0] = uint32_t(layer3d_tile_x(precision) + 8); box_lay[1] = uint32_t(layer3d_tile_y(precision) + 8);
            box_lay[2] = 1;
        }
        for (int p = 0; p < 2; ++p) {
            for (int f = 0; f < 2; ++f) {
                if ((s = encode_map(c, &c->tm_int[p][f], c->fld[p][f], box_int)) != PML_OK) return bail(s);
                if ((flags & PML_FLAG_ADJOINT) &&
                    (s = encode_map(c, &c->tm_int_adj[p][f], c->adj[p][f], box_int)) != PML_OK)
                    return bail(s);
            }
            for (int f = 0; f < c->nf; ++f) {
                if ((s = encode_map(c, &c->tm_lay[p][f], c->fld[p][f], box_lay)) != PML_OK) return bail(s);
                if ((flags & PML_FLAG_ADJOINT) &&
                    (s = encode_map(c, &c->tm_lay_adj[p][f], c->adj[p][f], box_lay)) != PML_OK)
                    return bail(s);
            }
            for (int f = c->nf; f < 8; ++f) { c->tm_lay[p][f] = c->tm_lay[p][0]; c->tm_lay_adj[p][f] = c->tm_lay_adj[p][0]; }
        }
        if (c->nd == 3 && c->prec == 32)   // slab tiles: one box shape per class
            for (int m = 0; m < 8; ++m) {
                int RX, RY, HX, HY;
                slab3d_shape(m, &RX, &RY, &HX, &HY);
                const uint32_t box_s[3] = {uint32_t(RX), uint32_t(RY), 1};
                for (int d = 0; d < ((flags & PML_FLAG_ADJOINT) ? 2 : 1); ++d)
                    for (int p = 0; p < 2; ++p)
                        for (int f = 0; f < 8; ++f)
                            if ((s = encode_map(c, &c->tm_slab[d][p][m * 8 + f], (d ? c->adj : c->fld)[p][f < c->nf ? f : 0],
                                                box_s)) != PML_OK)
                                return bail(s);
            }
        if (plan.tb2) {
            for (int f = 0; f < c->nf; ++f)
                if ((s = encode_map(c, &c->tm_mid[f], c->mid[f], box_lay)) != PML_OK) return bail(s);
            for (int f = c->nf; f < 8; ++f) c->tm_mid[f] = c->tm_mid[0];
            if ((s = encode_tb_maps(c)) != PML_OK) return bail(s);
        }
    }
    if (c->nd == 3 && c->prec == 32) c->ivar = 2;   // slab tiles: the fastest 3D frame variant
    if ((s = interior_grids(c)) != PML_OK) return bail(s);
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) { cuda_fail(c, e, "create"); return bail(PML_ECUDA); }
    *out = c;
    return PML_OK;
}

pml_status pml_set_variant(pml_ctx *c, int variant)
{
    if (!c) return fail(nullptr, PML_EINVAL, "ctx is NULL");
    const int n1 = one_step_variants(c), n = n1 + two_step_variants(c);
    if (variant < 0 || variant >= n) return fail(c, PML_EINVAL, "variant %d not in [0, %d)", variant, n);
    PML_CU(c, cudaStreamSynchronize(c->st), "stream synchronize");
    const int old_ivar = c->ivar, old_tb = c->tb, old_tbvar = c->tbvar;
    if (variant < n1) {
        c->ivar = variant;
        c->tb = 1;
    } else {   // the one-step variant stays as it is: it serves single steps and the adjoint
        c->tb = 2;
        c->tbvar = variant - n1;
    }
    pml_status s = encode_interior_maps(c);
    if (s == PML_OK) s = encode_tb_maps(c);
    if (s == PML_OK) s = interior_grids(c);
    if (s != PML_OK) {
        c->ivar = old_ivar;
        c->tb = old_tb;
        c->tbvar = old_tbvar;
        encode_interior_maps(c);
        encode_tb_maps(c);
        interior_grids(c);
    }
    return s;
}

pml_status pml_get_variant(const pml_ctx *c, int *variant, int *count)
{
    if (!c) return fail(nullptr, PML_EINVAL, "ctx is NULL");
    if (variant) *variant = c->tb == 2 ? one_step_variants(c) + c->tbvar : c->ivar;
    if (count) *count = one_step_variants(c) + two_step_variants(c);
    return PML_OK;
}

pml_status pml_get_time_block(const pml_ctx *c, int *depth)
{
    if (!c) return fail(nullptr, PML_EINVAL, "ctx is NULL");
    if (!depth) return fail(const_cast<pml_ctx *>(c), PML_EINVAL, "depth is NULL");
    *depth = c->tb;
    return PML_OK;
}

pml_status pml_autotune(pml_ctx *c, int steps, double *times_ms, int *chosen)
{
    const NvtxRange nvtx_range("pml_autotune");
    if (!c) return fail(nullptr, PML_EINVAL, "ctx is NULL");
    if (steps < 1) return fail(c, PML_EINVAL, "steps must be >= 1");
    const int n1 = one_step_variants(c), n = n1 + two_step_variants(c);
    cudaEvent_t e0, e1;
    PML_CU(c, cudaEventCreate(&e0), "event");
    PML_CU(c, cudaEventCreate(&e1), "event");
    int best = c->tb == 2 ? n1 + c->tbvar : c->ivar, best1 = c->ivar;
    double best_ms = 1e300, best1_ms = 1e300;
    pml_status st = PML_OK;
    const int ns = c->ns, nr = c->nr;
    c->ns = 0;   // time the step alone: no sources, no receiver rows consumed
    c->nr = 0;
    for (int v = 0; v < n && st == PML_OK; ++v) {
        if ((st = pml_set_variant(c, v)) != PML_OK) break;
        if ((st = pml_step(c, 2)) != PML_OK) break;      // warm-up
        cudaEventRecord(e0, c->st);
        if ((st = pml_step(c, steps)) != PML_OK) break;
        cudaEventRecord(e1, c->st);
        if (cudaEventSynchronize(e1) != cudaSuccess) { st = fail(c, PML_ECUDA, "autotune sync"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = double(ms) / steps;
        if (times_ms) times_ms[v] = per;
        if (per < best_ms) { best_ms = per; best = v; }
        if (v < n1 && per < best1_ms) { best1_ms = per; best1 = v; }
        if (v == n1 - 1 && (st = pml_set_variant(c, best1)) != PML_OK) break;   // kept for single steps
    }
    c->ns = ns;
    c->nr = nr;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PML_OK) return st;
    if (chosen) *chosen = best;
    return pml_set_variant(c, best);
}

pml_status pml_profile_enable(pml_ctx *c, int enable)
{
    if (!c) return fail(nullptr, PML_EINVAL, "ctx is NULL");
    c->prof_on = enable != 0;
    return PML_OK;
}

pml_status pml_profile_read(pml_ctx *c, double ms[3], int64_t launches[3])
{
    if (!c || !ms || !launches) return fail(c, PML_EINVAL, "NULL argument");
    PML_CU(c, cudaStreamSynchronize(c->st), "stream synchronize");
    for (int k = 0; k < 3; ++k) { ms[k] = 0.0; launches[k] = 0; }
    for (size_t i = 0; i < c->prof_n; ++i) {
        float t = 0.f;
        PML_CU(c, cudaEventElapsedTime(&t, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]), "event time");
        ms[c->prof_kind[i]] += double(t);
        launches[c->prof_kind[i]] += 1;
    }
    c->prof_n = 0;
    return PML_OK;
}

void pml_destroy(pml_ctx *c)
{
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);
    else cudaDeviceSynchronize();
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    if (c->own_ws && c->ws) cudaFree(c->ws);
    delete c;
}

pml_status pml_set_initial(pml_ctx *c, const void *u0, const void *v0, int on_device)
{
    if (!c) return fail(nullptr, PML_EINVAL, "ctx is NULL");
    const size_t fb = align_up(size_t(c->g.elems) * c->esz, kAlign);
    // The copies below fill every value of U (V) of the new state when given and the box is
    // periodic (the ghost ring is then filled from the copy); everything else of both
    // ping-pong states is cleared, on a side stream that runs beside the copies.
    const bool fill_u = u0 && !c->g.wall, fill_v = v0 && !c->g.wall;
    if ((fill_u || fill_v) && !c->side_tried) {
        c->side_tried = true;
        if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
            (void)cudaGetLastError();
            if (c->side) cudaStreamDestroy(c->side);
            if (c->ev_fork) cudaEventDestroy(c->ev_fork);
            if (c->ev_join) cudaEventDestroy(c->ev_join);
            c->side = nullptr;
            c->ev_fork = c->ev_join = nullptr;
        }
    }
    const bool forked = (fill_u || fill_v) && c->side;
    if (forked) {   // the side stream starts after all work already queued on the context's stream
        PML_CU(c, cudaEventRecord(c->ev_fork, c->st), "fork");
        PML_CU(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0), "fork");
    }
    cudaStream_t zs = forked ? c->side : c->st;
    char *s0 = static_cast<char *>(c->fld[0][0]);   // the two states' fields, nf each, contiguous
    if (fill_u && fill_v) {
        PML_CU(c, cudaMemsetAsync(s0 + 2 * fb, 0, fb * size_t(2 * c->nf - 2), zs), "clear state");
    } else if (fill_u) {
        PML_CU(c, cudaMemsetAsync(s0 + fb, 0, fb * size_t(2 * c->nf - 1), zs), "clear state");
    } else if (fill_v) {
        PML_CU(c, cudaMemsetAsync(s0, 0, fb, zs), "clear state");
        PML_CU(c, cudaMemsetAsync(s0 + 2 * fb, 0, fb * size_t(2 * c->nf - 2), zs), "clear state");
    } else {
        PML_CU(c, cudaMemsetAsync(s0, 0, fb * size_t(2 * c->nf), c->st), "clear state");
    }
    c->cur = 0;
    if (u0) {
        pml_status s = copy_dense(c, c->fld[0][0], u0, on_device != 0, true);
        if (s != PML_OK) return s;
    }
    if (v0) {
        pml_status s = copy_dense(c, c->fld[0][1], v0, on_device != 0, true);
        if (s != PML_OK) return s;
    }
    if (forked) {   // the context's stream goes on once the clearing is done
        PML_CU(c, cudaEventRecord(c->ev_join, c->side), "join");
        PML_CU(c, cudaStreamWaitEvent(c->st, c->ev_join, 0), "join");
    }
    if (!c->g.wall) {   // with a wall the ghost ring stays zero
        PML_CU(c, launch_fill_ghosts(c->prec, c->fld[0][0], c->g, c->st), "ghost fill");
        PML_CU(c, launch_fill_ghosts(c->prec, c->fld[0][1], c->g, c->st), "ghost fill");
    }
    c->step = 0;
    c->trace_k = 0;
    return clear_device_error(c);   // a new state: earlier device errors no longer apply
}

pml_status pml_set_sources(pml_ctx *c, int ns, const int64_t *coords, const double *amp, double f_peak,
                           double t_delay)
{
    if (!c) return fail(nullptr, PML_EINVAL, "ctx is NULL");
    if (ns < 0 || ns > kMaxSources) return fail(c, PML_EINVAL, "0 <= ns <= %d", kMaxSources);
    if (ns > 0 && (!coords || !amp)) return fail(c, PML_EINVAL, "coords/amp are NULL");
    if (!std::isfinite(f_peak) || !std::isfinite(t_delay)) return fail(c, PML_EINVAL, "non-finite wavelet parameters");
    std::vector<int64_t> off(static_cast<size_t>(ns));
    std::vector<int32_t> xyz(size_t(3 * ns), 0);
    for (int s = 0; s < ns; ++s) {
        if (!std::isfinite(amp[s])) return fail(c, PML_ENONFINITE, "source amplitude %d is not finite", s);
        int64_t o = 0;
        const int64_t st[3] = {1, c->g.P, c->g.PS};
        for (int a = 0; a < c->nd; ++a) {
            const int64_t x = coords[s * c->nd + a];
            if (x < c->ir[a].lo || x > c->ir[a].hi)
                return fail(c, PML_EINVAL, "source %d: coordinate %lld of axis %d is outside the layer-free run [%lld, %lld]",
                            s, (long long)x, a, (long long)c->ir[a].lo, (long long)c->ir[a].hi);
            xyz[size_t(3 * s + a)] = int32_t(x);
            o += x * st[a];
        }
        off[size_t(s)] = o;
    }
    // levels: sources whose stencils (vertex and its 2d neighbours) meet add in index order
    std::vector<int32_t> lvl(static_cast<size_t>(ns), 0);
    int nlev = ns > 0 ? 1 : 0;
    for (int s = 0; s < ns; ++s) {
        for (int t = 0; t < s; ++t) {
            int64_t d = 0;
            for (int a = 0; a < c->nd; ++a) {
                const int64_t e = std::llabs(int64_t(xyz[size_t(3 * s + a)]) - xyz[size_t(3 * t + a)]);
                d += std::min<int64_t>(e, c->T[a] - e);
            }
            if (d <= 2) lvl[size_t(s)] = std::max(lvl[size_t(s)], lvl[size_t(t)] + 1);
        }
        nlev = std::max(nlev, lvl[size_t(s)] + 1);
    }
    if (ns > 0) {
        PML_CU(c, cudaMemcpy(c->dsrc_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice), "sources");
        PML_CU(c, cudaMemcpy(c->dsrc_xyz, xyz.data(), xyz.size() * sizeof(int32_t), cudaMemcpyHostToDevice), "sources");
        PML_CU(c, cudaMemcpy(c->dsrc_level, lvl.data(), lvl.size() * sizeof(int32_t), cudaMemcpyHostToDevice), "sources");
        PML_CU(c, cudaMemcpy(c->dsrc_amp, amp, size_t(ns) * sizeof(double), cudaMemcpyHostToDevice), "sources");
    }
    c->ns = ns;
    c->src_levels = nlev;
    c->f_peak = f_peak;
    c->t_delay = t_delay;
    return PML_OK;
}

pml_status pml_set_receivers(pml_ctx *c, int nr, const int64_t *coords, void *trace_buf, int64_t capacity)
{
    if (!c) return fail(nullptr, PML_EINVAL, "ctx is NULL");
    if (nr < 0 || nr > kMaxReceivers) return fail(c, PML_EINVAL, "0 <= nr <= %d", kMaxReceivers);
    if (nr > 0 && (!coords || !trace_buf || capacity < 0)) return fail(c, PML_EINVAL, "receiver arguments");
    std::vector<int64_t> off(static_cast<size_t>(nr));
    std::vector<int32_t> xyz(size_t(3 * nr), 0), lvl(static_cast<size_t>(nr), 0);
    const int64_t st[3] = {1, c->g.P, c->g.PS};
    int nlev = nr > 0 ? 1 : 0;
    for (int r = 0; r < nr; ++r) {
        int64_t o = 0;
        for (int a = 0; a < c->nd; ++a) {
            const int64_t x = coords[r * c->nd + a];
            if (x < 0 || x >= c->T[a]) return fail(c, PML_EINVAL, "receiver %d outside the box", r);
            o += x * st[a];
            xyz[size_t(3 * r + a)] = int32_t(x);
        }
        off[size_t(r)] = o;
        for (int q = 0; q < r; ++q)   // receivers at one vertex inject in index order
            if (off[size_t(q)] == o) lvl[size_t(r)] = std::max(lvl[size_t(r)], lvl[size_t(q)] + 1);
        nlev = std::max(nlev, lvl[size_t(r)] + 1);
    }
    if (nr > 0) {
        PML_CU(c, cudaMemcpy(c->drec_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice), "receivers");
        PML_CU(c, cudaMemcpy(c->drec_xyz, xyz.data(), xyz.size() * sizeof(int32_t), cudaMemcpyHostToDevice), "receivers");
        PML_CU(c, cudaMemcpy(c->drec_level, lvl.data(), lvl.size() * sizeof(int32_t), cudaMemcpyHostToDevice), "receivers");
    }
    c->rec_levels = nlev;
    c->nr = nr;
    c->trace = trace_buf;
    c->trace_cap = capacity;
    c->trace_k = 0;
    return PML_OK;
}

pml_status pml_step(pml_ctx *c, int64_t n)
{
    const NvtxRange nvtx_range("pml_step");
    if (!c) return fail(nullptr, PML_EINVAL, "ctx is NULL");
    if (n < 0) return fail(c, PML_EINVAL, "n must be >= 0");
    const PointArgs pa = point_args(c);
    const int64_t step0 = c->step;
    for (int64_t k = 0; k < n; ++k) {
        const int p = c->cur, q = 1 - p;
        // two steps per pass where nothing has to happen between the two
        if (c->tb == 2 && n - k >= 2 && c->ns == 0 && !(c->nr > 0 && c->trace_k < c->trace_cap)) {
            pml_status s = enqueue_double_step(c, false, p);
            if (s != PML_OK) return s;
            c->cur = q;
            c->step += 2;
            ++k;
            continue;
        }
        pml_status s = enqueue_step(c, false, p);
        if (s != PML_OK) return s;
        void *row = nullptr;
        if (c->nr > 0 && c->trace_k < c->trace_cap)
            row = static_cast<char *>(c->trace) + size_t(c->trace_k) * size_t(c->nr) * c->esz;
        if (c->ns > 0 || row) {
            long pi = prof_begin(c, 2);
            cudaError_t e = launch_post_step(c->prec, c->fld[q][0], c->fld[q][1], pa, c->step, row, c->st);
            prof_end(c, pi);
            if (e != cudaSuccess) return cuda_fail(c, e, "post-step kernel");
        }
        if (row) c->trace_k++;
        c->cur = q;
        c->step++;
    }
    return maybe_check_finite(c, c->fld[c->cur], step0, c->step);
}

pml_status pml_read_field(pml_ctx *c, int field, void *dst, int on_device)
{
    if (!c) return fail(nullptr, PML_EINVAL, "ctx is NULL");
    if (field < 0 || field >= c->nf || !dst) return fail(c, PML_EINVAL, "bad field %d or NULL dst", field);
    pml_status s = copy_dense(c, c->fld[c->cur][field], dst, on_device != 0, false);
    if (s != PML_OK) return s;
    if (!on_device) return check_device_error(c);
    return PML_OK;
}

pml_status pml_norms(pml_ctx *c, const double *ref, double out[5])
{
    if (!c) return fail(nullptr, PML_EINVAL, "ctx is NULL");
    if (!out) return fail(c, PML_EINVAL, "out is NULL");
    int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int a = 0; a < c->nd; ++a) { lo[a] = c->w; hi[a] = c->w + c->N[a] - 1; }
    PML_CU(c, launch_norms(c->prec, c->fld[c->cur][0], c->fld[c->cur][1], c->g, lo, hi, c->h, ref, c->dpart,
                           kNormBlocks, c->dnorm, c->st), "norms kernel");
    PML_CU(c, cudaMemcpyAsync(out, c->dnorm, kNormVals * sizeof(double), cudaMemcpyDeviceToHost, c->st), "norms copy");
    return check_device_error(c);
}

pml_status pml_get_step(const pml_ctx *c, int64_t *step)
{
    if (!c || !step) return fail(nullptr, PML_EINVAL, "NULL argument");
    *step = c->step;
    return PML_OK;
}

pml_status pml_sync(pml_ctx *c)
{
    if (!c) return fail(nullptr, PML_EINVAL, "ctx is NULL");
    return check_device_error(c);
}

pml_status pml_set_wait_limit(pml_ctx *c, uint64_t ns)
{
    if (!c) return fail(nullptr, PML_EINVAL, "ctx is NULL");
    c->wait_ns = ns;
    return PML_OK;
}

pml_status pml_set_check_interval(pml_ctx *c, int64_t steps)
{
    if (!c) return fail(nullptr, PML_EINVAL, "ctx is NULL");
    if (steps < 0) return fail(c, PML_EINVAL, "steps must be >= 0");
    c->check_every = steps;
    return PML_OK;
}

pml_status pml_query_layout(const pml_ctx *c, int axis, uint8_t *phi_active, uint8_t *psi_active, uint8_t *interior)
{
    if (!c) return fail(nullptr, PML_EINVAL, "ctx is NULL");
    if (axis < 0 || axis >= c->nd) return fail(const_cast<pml_ctx *>(c), PML_EINVAL, "bad axis");
    const size_t T = size_t(c->T[axis]);
    if (phi_active) std::memcpy(phi_active, c->phi[axis].data(), T);
    if (psi_active) std::memcpy(psi_active, c->psi[axis].data(), T);
    if (interior) std::memcpy(interior, c->inner[axis].data(), T);
    return PML_OK;
}

pml_status pml_query_sigma(const pml_ctx *c, int axis, double *sigma)
{
    if (!c || !sigma) return fail(nullptr, PML_EINVAL, "NULL argument");
    if (axis < 0 || axis >= c->nd) return fail(const_cast<pml_ctx *>(c), PML_EINVAL, "bad axis");
    std::memcpy(sigma, c->sig[axis].data(), c->sig[axis].size() * sizeof(double));
    return PML_OK;
}

pml_status pml_adjoint_reset(pml_ctx *c)
{
    if (!c) return fail(nullptr, PML_EINVAL, "ctx is NULL");
    if (!(c->flags & PML_FLAG_ADJOINT)) return fail(c, PML_ESTATE, "context was created without PML_FLAG_ADJOINT");
    const size_t fb = align_up(size_t(c->g.elems) * c->esz, kAlign);
    PML_CU(c, cudaMemsetAsync(c->adj[0][0], 0, fb * size_t(2 * c->nf), c->st), "clear adjoint");
    PML_CU(c, cudaMemsetAsync(c->dgrad, 0, kMaxSources * sizeof(double), c->st), "clear gradient");
    c->acur = 0;
    c->astep = c->step;
    c->adj_ready = true;
    return PML_OK;
}

pml_status pml_adjoint_step(pml_ctx *c, int64_t n, const void *residual, void *grad_u, double *grad_amp)
{
    const NvtxRange nvtx_range("pml_adjoint_step");
    if (!c) return fail(nullptr, PML_EINVAL, "ctx is NULL");
    if (!c->adj_ready) return fail(c, PML_ESTATE, "call pml_adjoint_reset first");
    if (n < 0) return fail(c, PML_EINVAL, "n must be >= 0");
    const PointArgs pa = point_args(c);
    const int64_t astep0 = c->astep;
    for (int64_t k = 0; k < n; ++k) {
        const int p = c->acur;
        const int64_t m = c->astep;
        // two transposed steps per pass where nothing is injected or accumulated between them
        if (c->tb == 2 && n - k >= 2 && c->ns == 0 && !(residual && c->nr > 0)) {
            pml_status s = enqueue_double_step(c, true, p);
            if (s != PML_OK) return s;
            c->acur = 1 - p;
            c->astep = m - 2;
            ++k;
            continue;
        }
        const void *row = (residual && c->nr > 0)
                              ? static_cast<const char *>(residual) + size_t(k) * size_t(c->nr) * c->esz
                              : nullptr;
        if (row || c->ns > 0)
            PML_CU(c, launch_adjoint_points(c->prec, c->adj[p][0], c->adj[p][1], pa, m, row,
                                            c->ns > 0 ? c->dgrad : nullptr, c->st), "adjoint point kernel");
        pml_status s = enqueue_step(c, true, p);
        if (s != PML_OK) return s;
        c->acur = 1 - p;
        c->astep = m - 1;
    }
    {
        pml_status s = maybe_check_finite(c, c->adj[c->acur], astep0, c->astep);
        if (s != PML_OK) return s;
    }
    if (grad_u) {
        pml_status s = copy_dense(c, c->adj[c->acur][0], grad_u, true, false);
        if (s != PML_OK) return s;
    }
    if (grad_amp && c->ns > 0) {
        PML_CU(c, cudaMemcpyAsync(grad_amp, c->dgrad, size_t(c->ns) * sizeof(double), cudaMemcpyDeviceToHost, c->st),
               "gradient copy");
        return check_device_error(c);
    }
    return PML_OK;
}

pml_status pml_sigma_gradient_bytes(const pml_ctx *c, int64_t n, int64_t interval, size_t *bytes)
{
    if (!c || !bytes) return fail(nullptr, PML_EINVAL, "NULL argument");
    if (n < 1) return fail(const_cast<pml_ctx *>(c), PML_EINVAL, "n must be >= 1");
    const size_t fb = align_up(size_t(c->g.elems) * c->esz, kAlign);
    const size_t sb = fb * size_t(c->nf);
    const int64_t K = checkpoint_interval(n, interval);
    const int64_t nck = (n + K - 1) / K;
    int64_t tot = 0;
    for (int a = 0; a < c->nd; ++a) tot += c->T[a];
    size_t off = sb * size_t(nck) + sb + sb * size_t(K) + sb * 6;
    off += align_up(size_t(n) * size_t(c->nr > 0 ? c->nr : 1) * c->esz, kAlign);
    off += align_up(size_t(tot) * sizeof(double), kAlign) + kAlign;
    for (int r = 0; r < 3; ++r) {
        std::vector<int4> sg;
        gradient_segments(c, r, &sg);
        off += align_up(std::max<size_t>(sg.size(), 1) * sizeof(int4), kAlign);
    }
    *bytes = off;
    return PML_OK;
}

pml_status pml_sigma_gradient(pml_ctx *c, int64_t n, const void *target, const void *residual, int64_t interval,
                              double *grad_sigma, double *misfit, double *grad_amp)
{
    const NvtxRange nvtx_range("pml_sigma_gradient");
    if (!c) return fail(nullptr, PML_EINVAL, "ctx is NULL");
    if (!(c->flags & PML_FLAG_ADJOINT)) return fail(c, PML_ESTATE, "context was created without PML_FLAG_ADJOINT");
    if (n < 1) return fail(c, PML_EINVAL, "n must be >= 1");
    if (!grad_sigma || !misfit) return fail(c, PML_EINVAL, "grad_sigma and misfit are required");
    if (c->nr > 0 && !target == !residual)
        return fail(c, PML_EINVAL, "give exactly one of target and residual when receivers are set");
    if (c->nr > 0 && c->trace_cap - c->trace_k < n)
        return fail(c, PML_EINVAL, "the receiver buffer has %lld free rows, %lld needed",
                    (long long)(c->trace_cap - c->trace_k), (long long)n);
    const int nf = c->nf;
    const size_t fb = align_up(size_t(c->g.elems) * c->esz, kAlign);
    const size_t sb = fb * size_t(nf);   // one state (the fields of one ping-pong half are contiguous)
    const int64_t K = checkpoint_interval(n, interval);
    const int64_t nck = (n + K - 1) / K;
    int64_t tot = 0;
    for (int a = 0; a < c->nd; ++a) tot += c->T[a];
    size_t off = 0;
    const size_t o_ck = off; off += sb * size_t(nck);
    const size_t o_end = off; off += sb;
    const size_t o_seg = off; off += sb * size_t(K);
    const size_t o_stage = off; off += sb * 6;
    const size_t o_res = off; off += align_up(size_t(n) * size_t(c->nr > 0 ? c->nr : 1) * c->esz, kAlign);
    const size_t o_acc = off; off += align_up(size_t(tot) * sizeof(double), kAlign);
    const size_t o_mis = off; off += kAlign;
    // row segments of C_0, C_1, C_2 (the vertices the contraction reads, widened by 0, 1, 2
    // stencil steps): the stages are formed there only
    std::vector<int4> segs[3];
    for (int r = 0; r < 3; ++r) gradient_segments(c, r, &segs[r]);
    size_t o_seg_tab[3];
    for (int r = 0; r < 3; ++r) {
        o_seg_tab[r] = off;
        off += align_up(std::max<size_t>(segs[r].size(), 1) * sizeof(int4), kAlign);
    }
    char *mem = nullptr;
    cudaError_t ce = cudaMalloc(&mem, off);
    if (ce != cudaSuccess) return fail(c, PML_ENOMEM, "cudaMalloc(%zu) for checkpoints: %s", off, cudaGetErrorString(ce));
    struct Free {
        char *p;
        ~Free() { if (p) cudaFree(p); }
    } guard{mem};
    auto state_at = [&](size_t base, void *out[8]) {
        for (int f = 0; f < nf; ++f) out[f] = mem + base + size_t(f) * fb;
    };
    void *Y2[8], *Y3[8], *Y4[8], *KB3[8], *KB2[8], *KB1[8];
    state_at(o_stage + 0 * sb, Y2);
    state_at(o_stage + 1 * sb, Y3);
    state_at(o_stage + 2 * sb, Y4);
    state_at(o_stage + 3 * sb, KB3);
    state_at(o_stage + 4 * sb, KB2);
    state_at(o_stage + 5 * sb, KB1);
    PML_CU(c, cudaMemsetAsync(mem + o_stage, 0, sb * 6, c->st), "clear stage buffers");
    double *dacc = reinterpret_cast<double *>(mem + o_acc), *dmis = reinterpret_cast<double *>(mem + o_mis);
    const int4 *dseg[3];
    for (int r = 0; r < 3; ++r) {
        dseg[r] = reinterpret_cast<const int4 *>(mem + o_seg_tab[r]);
        if (!segs[r].empty())
            PML_CU(c, cudaMemcpyAsync(mem + o_seg_tab[r], segs[r].data(), segs[r].size() * sizeof(int4),
                                      cudaMemcpyHostToDevice, c->st), "segment table");
    }
    PML_CU(c, cudaMemsetAsync(dacc, 0, size_t(tot) * sizeof(double), c->st), "clear gradient");
    PML_CU(c, cudaMemsetAsync(dmis, 0, sizeof(double), c->st), "clear misfit");

    // forward run with a checkpoint every K steps
    const int64_t s0 = c->step, tk0 = c->trace_k;
    nvtxRangePushA("forward with checkpoints");
    for (int64_t k = 0; k < n; ++k) {
        if (k % K == 0)
            PML_CU(c, cudaMemcpyAsync(mem + o_ck + size_t(k / K) * sb, c->fld[c->cur][0], sb, cudaMemcpyDeviceToDevice,
                                      c->st), "checkpoint");
        pml_status s = pml_step(c, 1);
        if (s != PML_OK) { nvtxRangePop(); return s; }
    }
    nvtxRangePop();
    PML_CU(c, cudaMemcpyAsync(mem + o_end, c->fld[c->cur][0], sb, cudaMemcpyDeviceToDevice, c->st), "final state");
    if (c->nr > 0 && target)
        PML_CU(c, launch_residual(c->prec, static_cast<const char *>(c->trace) + size_t(tk0) * size_t(c->nr) * c->esz,
                                  target, mem + o_res, n * c->nr, dmis, c->st), "residual kernel");
    else if (c->nr > 0)
        PML_CU(c, cudaMemcpyAsync(mem + o_res, residual, size_t(n) * size_t(c->nr) * c->esz, cudaMemcpyDeviceToDevice,
                                  c->st), "residual copy");

    // backwards, one segment of at most K steps at a time
    pml_status s = pml_adjoint_reset(c);
    if (s != PML_OK) return s;
    const SigmaPtrs sp = {{c->dsig[0], c->dsig[1], c->dsig[2]}};
    const PointArgs pa = point_args(c);
    const int nr_saved = c->nr;
    const double dt = c->dt;
    for (int64_t seg = nck - 1; seg >= 0; --seg) {
        const NvtxRange seg_range("segment: recompute, adjoint, contraction");
        const int64_t sa = seg * K, se = std::min<int64_t>(n, sa + K);
        PML_CU(c, cudaMemcpyAsync(c->fld[c->cur][0], mem + o_ck + size_t(seg) * sb, sb, cudaMemcpyDeviceToDevice,
                                  c->st), "restore checkpoint");
        c->step = s0 + sa;
        c->nr = 0;   // recomputation records no traces
        for (int64_t j = sa; j < se; ++j) {
            PML_CU(c, cudaMemcpyAsync(mem + o_seg + size_t(j - sa) * sb, c->fld[c->cur][0], sb,
                                      cudaMemcpyDeviceToDevice, c->st), "segment state");
            if (j + 1 < se && (s = pml_step(c, 1)) != PML_OK) { c->nr = nr_saved; return s; }
        }
        c->nr = nr_saved;
        for (int64_t m = se; m > sa; --m) {   // adjoint clock s0 + m: the step m-1 -> m
            const int p = c->acur;
            const void *row = nr_saved > 0 ? mem + o_res + size_t(m - 1) * size_t(nr_saved) * c->esz : nullptr;
            if (row || c->ns > 0)
                PML_CU(c, launch_adjoint_points(c->prec, c->adj[p][0], c->adj[p][1], pa, c->astep, row,
                                                c->ns > 0 ? c->dgrad : nullptr, c->st), "adjoint point kernel");
            void *Y1[8];
            state_at(o_seg + size_t(m - 1 - sa) * sb, Y1);
            void *const *yb = c->adj[p];
            void *const *ybv = yb;
            const int n0 = int(segs[0].size()), n1 = int(segs[1].size()), n2 = int(segs[2].size());
            // forward stage inputs: Y2 = Y1 + dt/2 A Y1 (on C_2), Y3 = Y1 + dt/2 A Y2 (C_1),
            // Y4 = Y1 + dt A Y3 (C_0)
            PML_CU(c, launch_stage(c->prec, false, Y1, Y1, Y2, nf, c->g, sp, c->h, 1.0, 0.5 * dt, dseg[2], n2, c->st), "stage");
            PML_CU(c, launch_stage(c->prec, false, Y2, Y1, Y3, nf, c->g, sp, c->h, 1.0, 0.5 * dt, dseg[1], n1, c->st), "stage");
            PML_CU(c, launch_stage(c->prec, false, Y3, Y1, Y4, nf, c->g, sp, c->h, 1.0, dt, dseg[0], n0, c->st), "stage");
            // stage cotangents of the reverse stage graph driven by ybar (kbar4 = dt/6 ybar):
            // kbar3 = dt/3 ybar + dt A^T kbar4 (C_2), kbar2 = dt/3 ybar + dt/2 A^T kbar3 (C_1),
            // kbar1 = dt/6 ybar + dt/2 A^T kbar2 (C_0)
            PML_CU(c, launch_stage(c->prec, true, yb, yb, KB3, nf, c->g, sp, c->h, dt / 3.0, dt * dt / 6.0, dseg[2], n2,
                                   c->st), "cotangent");
            PML_CU(c, launch_stage(c->prec, true, KB3, yb, KB2, nf, c->g, sp, c->h, dt / 3.0, 0.5 * dt, dseg[1], n1,
                                   c->st), "cotangent");
            PML_CU(c, launch_stage(c->prec, true, KB2, yb, KB1, nf, c->g, sp, c->h, dt / 6.0, 0.5 * dt, dseg[0], n0,
                                   c->st), "cotangent");
            // each cotangent contracted with its stage input, all four in one launch
            void *const *kbs[4] = {ybv, KB3, KB2, KB1};
            void *const *ys[4] = {Y4, Y3, Y2, Y1};
            const double scl[4] = {dt / 6.0, 1.0, 1.0, 1.0};
            PML_CU(c, launch_contract4(c->prec, kbs, ys, scl, nf, c->g, sp, c->h, dacc, c->st), "contraction");
            // the adjoint step itself
            if ((s = enqueue_step(c, true, p)) != PML_OK) return s;
            c->acur = 1 - p;
            c->astep = c->astep - 1;
        }
    }
    PML_CU(c, cudaMemcpyAsync(c->fld[c->cur][0], mem + o_end, sb, cudaMemcpyDeviceToDevice, c->st), "final state");
    c->step = s0 + n;
    PML_CU(c, cudaMemcpyAsync(grad_sigma, dacc, size_t(tot) * sizeof(double), cudaMemcpyDeviceToHost, c->st),
           "gradient copy");
    PML_CU(c, cudaMemcpyAsync(misfit, dmis, sizeof(double), cudaMemcpyDeviceToHost, c->st), "misfit copy");
    if (grad_amp && c->ns > 0)
        PML_CU(c, cudaMemcpyAsync(grad_amp, c->dgrad, size_t(c->ns) * sizeof(double), cudaMemcpyDeviceToHost, c->st),
               "gradient copy");
    return check_device_error(c);   // synchronises before the scratch is freed
}

pml_status pml_adjoint_read_field(pml_ctx *c, int field, void *dst, int on_device)
{
    if (!c) return fail(nullptr, PML_EINVAL, "ctx is NULL");
    if (!c->adj_ready) return fail(c, PML_ESTATE, "call pml_adjoint_reset first");
    if (field < 0 || field >= c->nf || !dst) return fail(c, PML_EINVAL, "bad field %d or NULL dst", field);
    pml_status s = copy_dense(c, c->adj[c->acur][field], dst, on_device != 0, false);
    if (s != PML_OK) return s;
    if (!on_device) return check_device_error(c);
    return PML_OK;
}

pml_status pml_state_bytes(const pml_ctx *c, size_t *bytes)
{
    if (!c || !bytes) return fail(nullptr, PML_EINVAL, "NULL argument");
    *bytes = 64 + size_t(c->nf) * size_t(c->g.elems) * c->esz;
    return PML_OK;
}

pml_status pml_save_state(pml_ctx *c, void *dst, int on_device)
{
    if (!c || !dst) return fail(c, PML_EINVAL, "NULL argument");
    int64_t hdr[8] = {0x504d4c53, c->step, c->nf, c->g.elems, c->esz, 0, 0, 0};
    char *d = static_cast<char *>(dst);
    const cudaMemcpyKind kh = on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    PML_CU(c, cudaMemcpyAsync(d, hdr, sizeof hdr, kh, c->st), "save header");
    const size_t fb = size_t(c->g.elems) * c->esz;
    for (int f = 0; f < c->nf; ++f)
        PML_CU(c, cudaMemcpyAsync(d + 64 + f * fb, c->fld[c->cur][f], fb,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st),
               "save field");
    return check_device_error(c);
}

pml_status pml_load_state(pml_ctx *c, const void *src, int on_device)
{
    if (!c || !src) return fail(c, PML_EINVAL, "NULL argument");
    int64_t hdr[8];
    PML_CU(c, cudaMemcpyAsync(hdr, src, sizeof hdr, on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, c->st),
           "load header");
    PML_CU(c, cudaStreamSynchronize(c->st), "load header");
    if (hdr[0] != 0x504d4c53 || hdr[2] != c->nf || hdr[3] != c->g.elems || hdr[4] != c->esz)
        return fail(c, PML_EINVAL, "checkpoint does not match this context");
    const char *sp = static_cast<const char *>(src);
    const size_t fb = size_t(c->g.elems) * c->esz;
    for (int f = 0; f < c->nf; ++f)
        PML_CU(c, cudaMemcpyAsync(c->fld[0][f], sp + 64 + f * fb, fb,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st),
               "load field");
    c->cur = 0;
    c->step = hdr[1];
    pml_status s = clear_device_error(c);   // a new state: earlier device errors no longer apply
    if (s != PML_OK) return s;
    return check_device_error(c);
}

}  // extern "C"

// ------------------------------------------------------------------------------------
// Batched stepping of many independent 2D contexts: one layer launch and one interior
// launch per step for the whole batch, runs of kBatchGraphSteps steps replayed from a
// CUDA graph captured once per kernel variant.
// ------------------------------------------------------------------------------------
namespace {
constexpr int kBatchGraphSteps = 32;   // even: a replay starts and ends at input parity 0
}

struct pml_batch {
    std::vector<pml_ctx *> ctx;
    int prec = 0, var = 0, sm_count = 0;
    cudaStream_t st = nullptr;    // the contexts' stream (work and graph replays)
    cudaStream_t cap = nullptr;   // private stream the graph is captured on
    char *mem = nullptr;
    GridDesc2 *ddesc = nullptr;
    int *ditem_off = nullptr, *dtile_grid = nullptr, *dqueue = nullptr;
    LayerTile *dtiles = nullptr;
    int n_items = 0, ntiles = 0, grid_int = 0;
    int64_t launches = 0;         // interior launches so far; its parity is the queue's
    // two steps per pass (FP32 batches whose contexts all have the two-step buffers):
    // `var` stays the one-step shape (odd steps), `var2` is the two-step shape when tb == 2
    bool tb_ok = false;
    int tb = 1, var2 = 0;
    int *ditem_off2 = nullptr, *dtile_grid1 = nullptr, *dtile_grid2 = nullptr;
    LayerTile *dtiles1 = nullptr, *dtiles2 = nullptr;
    int n_items2 = 0, ntiles1 = 0, ntiles2 = 0, grid_tb = 0;
    int64_t launches2 = 0;        // second layer passes so far; their counter parity
    cudaGraphExec_t exec = nullptr;
    bool pdl = true;              // interior launches overlap the layer launch
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_kind;
    size_t prof_n = 0;
};

namespace {

pml_status bfail(pml_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_create_error = buf;
    return s;
}

#define PML_BCU(call, what)                                                                 \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return bfail(PML_ECUDA, "%s: %s", (what), cudaGetErrorString(e_)); \
    } while (0)

// Device tables of the current variant: one descriptor per grid and the first interior
// work item of each grid.  The caller has synchronised the stream.
pml_status batch_upload(pml_batch *b)
{
    const int ng = int(b->ctx.size());
    const uint32_t box[3] = {uint32_t(batch2d_box_cols(b->prec, b->var)), uint32_t(batch2d_box_rows(b->prec, b->var)), 1};
    const int rows = batch2d_item_rows(b->prec, b->var), cols = batch2d_strip_cols(b->prec, b->var);
    std::vector<GridDesc2> desc(static_cast<size_t>(ng));
    std::vector<int> off(static_cast<size_t>(ng) + 1, 0), off2(static_cast<size_t>(ng) + 1, 0);
    int64_t items = 0, items2 = 0;
    for (int i = 0; i < ng; ++i) {
        pml_ctx *c = b->ctx[size_t(i)];
        GridDesc2 &d = desc[size_t(i)];
        std::memset(static_cast<void *>(&d), 0, sizeof d);
        for (int p = 0; p < 2; ++p) {
            for (int f = 0; f < 2; ++f)
                if (encode_map(c, &d.tm_int[p][f], c->fld[p][f], box) != PML_OK)
                    return bfail(PML_ECUDA, "grid %d: %s", i, c->err.c_str());
            for (int f = 0; f < 6; ++f) {
                d.tm_lay[p][f] = c->tm_lay[p][f];
                d.out[p][f] = c->fld[1 - p][f];
            }
        }
        d.in.g = c->g;
        d.in.xr = c->ir[0];
        d.in.yr = c->ir[1];
        step_coef(c, false, &d.in.c);
        d.in.err = c->derr;
        d.in.wait_ns = c->wait_ns;
        d.lay.g = c->g;
        d.lay.k = layer_const(c);
        d.lay.sig[0] = c->dsig[0];
        d.lay.sig[1] = c->dsig[1];
        d.lay.err = c->derr;
        d.lay.wait_ns = c->wait_ns;
        if (b->tb_ok) {
            const uint32_t box2[3] = {uint32_t(batch2d_tb2_box_cols(b->prec, b->var2)),
                                      uint32_t(batch2d_tb2_box_rows(b->prec, b->var2)), 1};
            for (int p = 0; p < 2; ++p)
                for (int f = 0; f < 2; ++f)
                    if (encode_map(c, &d.tm_tb[p][f], c->fld[p][f], box2) != PML_OK)
                        return bfail(PML_ECUDA, "grid %d: %s", i, c->err.c_str());
            for (int f = 0; f < 6; ++f) {
                d.tm_mid[f] = c->tm_mid[f];
                d.mid[f] = c->mid[f];
            }
            d.in2 = d.in;
            d.in2.xr = c->ir_tb[0];
            d.in2.yr = c->ir_tb[1];
            int64_t n2 = 0;
            if (!range_empty(c->ir_tb[0]) && !range_empty(c->ir_tb[1])) {
                const int rows2 = batch2d_tb2_item_rows(b->prec, b->var2), cols2 = batch2d_tb2_strip_cols(b->prec, b->var2);
                d.rblocks2 = int((c->ir_tb[1].hi - c->ir_tb[1].lo + 1 + rows2 - 1) / rows2);
                d.nstrips2 = int((c->ir_tb[0].hi - (c->ir_tb[0].lo & ~int64_t(3))) / cols2 + 1);
                n2 = int64_t(d.rblocks2) * d.nstrips2;
            }
            off2[size_t(i)] = int(items2);
            items2 += n2;
            if (items2 > (int64_t(1) << 30)) return bfail(PML_EINVAL, "batch has too many interior work items");
        }
        int64_t n = 0;
        if (!range_empty(c->ir[0]) && !range_empty(c->ir[1])) {
            d.rblocks = int((c->ir[1].hi - c->ir[1].lo + 1 + rows - 1) / rows);
            d.nstrips = int((c->ir[0].hi - (c->ir[0].lo & ~int64_t(3))) / cols + 1);
            n = int64_t(d.rblocks) * d.nstrips;
        }
        off[size_t(i)] = int(items);
        items += n;
        if (items > (int64_t(1) << 30)) return bfail(PML_EINVAL, "batch has too many interior work items");
    }
    off[size_t(ng)] = int(items);
    off2[size_t(ng)] = int(items2);
    b->n_items = int(items);
    b->n_items2 = int(items2);
    PML_BCU(cudaMemcpy(b->ddesc, desc.data(), desc.size() * sizeof(GridDesc2), cudaMemcpyHostToDevice), "upload batch descriptors");
    PML_BCU(cudaMemcpy(b->ditem_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice), "upload batch offsets");
    if (b->tb_ok) {
        PML_BCU(cudaMemcpy(b->ditem_off2, off2.data(), off2.size() * sizeof(int), cudaMemcpyHostToDevice),
                "upload batch offsets");
        const int bt = batch2d_tb2_blocks_per_sm(b->prec, b->var2);
        if (bt <= 0) return bfail(PML_ECUDA, "batched two-step interior kernel cannot be resident");
        b->grid_tb = bt * b->sm_count;
    }
    // (also sets the kernels' shared-memory limits, which must not happen during capture)
    const int bps = batch2d_interior_blocks_per_sm(b->prec, b->var);
    if (bps <= 0 || batch2d_interior_blocks_per_sm(b->prec, 0) <= 0)
        return bfail(PML_ECUDA, "batched interior kernel cannot be resident");
    b->grid_int = bps * b->sm_count;
    return PML_OK;
}

long bprof_begin(pml_batch *b, int kind, cudaStream_t st)
{
    if (!b->prof_on) return -1;
    if (b->prof_n == b->prof_kind.size()) {
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess) return -1;
        if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return -1; }
        b->prof_ev.push_back(e0);
        b->prof_ev.push_back(e1);
        b->prof_kind.push_back(kind);
    }
    const size_t i = b->prof_n++;
    b->prof_kind[i] = kind;
    cudaEventRecord(b->prof_ev[2 * i], st);
    return long(i);
}

void bprof_end(pml_batch *b, long i, cudaStream_t st)
{
    if (i >= 0) cudaEventRecord(b->prof_ev[2 * size_t(i) + 1], st);
}

// One step of every grid from input parity p (which is also the queue parity).
pml_status batch_enqueue(pml_batch *b, int p, cudaStream_t st, bool timed)
{
    Batch2DArgs a{};
    a.desc = b->ddesc;
    a.item_off = b->ditem_off;
    a.tiles = b->dtiles;
    a.tile_grid = b->dtile_grid;
    a.ngrid = int(b->ctx.size());
    a.n_items = b->n_items;
    a.ntiles = b->ntiles;
    a.queue = b->dqueue;
    a.parity = p;
    long pi = timed ? bprof_begin(b, 1, st) : -1;
    cudaError_t e = launch_batch2d_layer(b->prec, a, layer2d_grid(b->prec, b->ntiles, b->sm_count), b->ctx[0]->g.wall != 0, st);
    bprof_end(b, pi, st);
    if (e != cudaSuccess) return bfail(PML_ECUDA, "batched layer kernel: %s", cudaGetErrorString(e));
    pi = timed ? bprof_begin(b, 0, st) : -1;
    e = launch_batch2d_interior(b->prec, b->var, a, b->grid_int, st, b->pdl && b->ntiles > 0 && !timed);
    bprof_end(b, pi, st);
    if (e != cudaSuccess) return bfail(PML_ECUDA, "batched interior kernel: %s", cudaGetErrorString(e));
    return PML_OK;
}

// Two steps of every grid from input parity p: layer pass 1 (fields -> mid), layer pass 2
// (mid -> fields; launched early, waits for pass 1; counters of parity qp), two-step interior.
pml_status batch_enqueue_pair(pml_batch *b, int p, int qp, cudaStream_t st, bool timed)
{
    Batch2DArgs a{};
    a.desc = b->ddesc;
    a.ngrid = int(b->ctx.size());
    a.queue = b->dqueue;
    a.parity = p;
    a.qparity = qp;
    const bool wall = b->ctx[0]->g.wall != 0;
    a.tiles = b->dtiles1;
    a.tile_grid = b->dtile_grid1;
    a.ntiles = b->ntiles1;
    a.pass = 1;
    long pi = timed ? bprof_begin(b, 1, st) : -1;
    cudaError_t e = launch_batch2d_layer(b->prec, a, layer2d_grid(b->prec, a.ntiles, b->sm_count), wall, st, false);
    bprof_end(b, pi, st);
    if (e != cudaSuccess) return bfail(PML_ECUDA, "batched layer kernel (pass 1): %s", cudaGetErrorString(e));
    a.tiles = b->dtiles2;
    a.tile_grid = b->dtile_grid2;
    a.ntiles = b->ntiles2;
    a.pass = 2;
    pi = timed ? bprof_begin(b, 1, st) : -1;
    e = launch_batch2d_layer(b->prec, a, layer2d_grid(b->prec, a.ntiles, b->sm_count), wall, st,
                             b->pdl && !timed && b->ntiles1 > 0);
    bprof_end(b, pi, st);
    if (e != cudaSuccess) return bfail(PML_ECUDA, "batched layer kernel (pass 2): %s", cudaGetErrorString(e));
    a.pass = 0;
    a.item_off = b->ditem_off2;
    a.n_items = b->n_items2;
    pi = timed ? bprof_begin(b, 0, st) : -1;
    e = launch_batch2d_tb2(b->prec, b->var2, a, b->grid_tb, st, b->pdl && !timed && (b->ntiles1 + b->ntiles2) > 0);
    bprof_end(b, pi, st);
    if (e != cudaSuccess) return bfail(PML_ECUDA, "batched two-step interior kernel: %s", cudaGetErrorString(e));
    return PML_OK;
}

void batch_drop_graph(pml_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

// Capture kBatchGraphSteps steps from input parity 0 on the private stream.  If the
// driver refuses the programmatic (overlapping) edges in a graph, capture plain ones.
pml_status batch_capture(pml_batch *b)
{
    batch_drop_graph(b);
    for (int attempt = 0; attempt < 2; ++attempt) {
        cudaGraph_t g = nullptr;
        PML_BCU(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin graph capture");
        pml_status s = PML_OK;
        if (b->tb == 2)   // pairs from counter parity 0 (the caller aligns the second-pass counters)
            for (int k = 0; k < kBatchGraphSteps / 2 && s == PML_OK; ++k) s = batch_enqueue_pair(b, k & 1, k & 1, b->cap, false);
        else
            for (int k = 0; k < kBatchGraphSteps && s == PML_OK; ++k) s = batch_enqueue(b, k & 1, b->cap, false);
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (s == PML_OK && e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (s == PML_OK && e == cudaSuccess) return PML_OK;
        cudaGetLastError();
        b->exec = nullptr;
        if (!b->pdl) return s != PML_OK ? s : bfail(PML_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        b->pdl = false;
    }
    return bfail(PML_ECUDA, "graph capture failed");
}

}  // namespace

extern "C" {

pml_status pml_batch_create(int count, pml_ctx *const *ctxs, pml_batch **out)
{
    if (!out) return bfail(PML_EINVAL, "pml_batch_create: out is NULL");
    *out = nullptr;
    if (count < 1 || !ctxs) return bfail(PML_EINVAL, "pml_batch_create: need count >= 1 contexts");
    for (int i = 0; i < count; ++i) {
        const pml_ctx *c = ctxs[i];
        if (!c) return bfail(PML_EINVAL, "pml_batch_create: context %d is NULL", i);
        if (c->nd != 2) return bfail(PML_EINVAL, "pml_batch_create: context %d is not 2D", i);
        if (c->prec != ctxs[0]->prec) return bfail(PML_EINVAL, "pml_batch_create: contexts mix precisions");
        if (c->st != ctxs[0]->st) return bfail(PML_EINVAL, "pml_batch_create: contexts use different streams");
        if (c->g.wall != ctxs[0]->g.wall) return bfail(PML_EINVAL, "pml_batch_create: contexts mix walls and periodic boxes");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) return bfail(PML_EINVAL, "pml_batch_create: context %d appears twice", i);
    }
    pml_batch *b = new pml_batch();
    b->ctx.assign(ctxs, ctxs + count);
    b->prec = ctxs[0]->prec;
    b->st = ctxs[0]->st;
    b->sm_count = ctxs[0]->sm_count;
    auto bail = [&](pml_status s) {
        const std::string msg = g_create_error;
        pml_batch_destroy(b);
        g_create_error = msg;
        return s;
    };
    // layer tiles of all grids (the forward lists every context built at creation)
    std::vector<LayerTile> tiles;
    std::vector<int> tile_grid;
    for (int i = 0; i < count; ++i) {
        int co[9];
        std::vector<LayerTile> t =
            build_tiles(b->ctx[size_t(i)], b->ctx[size_t(i)]->ir, co, kLayer2BandRowsBatch, kLayer2SlabRowsBatch);
        tiles.insert(tiles.end(), t.begin(), t.end());
        tile_grid.insert(tile_grid.end(), t.size(), i);
    }
    // one class after another across all grids (warps that run the same class share code)
    auto by_class = [](std::vector<LayerTile> &tl, std::vector<int> &tg) {
        std::vector<size_t> order(tl.size());
        for (size_t k = 0; k < order.size(); ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return tl[a].flags < tl[b].flags; });
        std::vector<LayerTile> t2(tl.size());
        std::vector<int> g2(tl.size());
        for (size_t k = 0; k < order.size(); ++k) {
            t2[k] = tl[order[k]];
            g2[k] = tg[order[k]];
        }
        tl.swap(t2);
        tg.swap(g2);
    };
    by_class(tiles, tile_grid);
    // frames of the two layer passes of a two-step block (FP32 contexts with the buffers)
    b->tb_ok = batch2d_tb2_variants(b->prec) > 0;
    for (int i = 0; i < count; ++i) b->tb_ok = b->tb_ok && b->ctx[size_t(i)]->plan.tb2;
    std::vector<LayerTile> tiles1, tiles2;
    std::vector<int> grid1, grid2;
    if (b->tb_ok) {
        for (int i = 0; i < count; ++i) {
            pml_ctx *c = b->ctx[size_t(i)];
            Range r6[3];
            for (int a = 0; a < 3; ++a) r6[a] = shrink_run(c->ir[a], c->T[a], 6);
            int co[9];
            std::vector<LayerTile> t1 = build_tiles(c, r6, co, kLayer2BandRowsBatch, kLayer2SlabRowsBatch),
                                   t2 = build_tiles(c, c->ir_tb, co, kLayer2BandRowsBatch, kLayer2SlabRowsBatch);
            tiles1.insert(tiles1.end(), t1.begin(), t1.end());
            grid1.insert(grid1.end(), t1.size(), i);
            tiles2.insert(tiles2.end(), t2.begin(), t2.end());
            grid2.insert(grid2.end(), t2.size(), i);
        }
        by_class(tiles1, grid1);
        by_class(tiles2, grid2);
    }
    if (tiles.size() > size_t(1) << 30 || tiles1.size() > size_t(1) << 30 || tiles2.size() > size_t(1) << 30)
        return bail(bfail(PML_EINVAL, "batch has too many layer tiles"));
    b->ntiles = int(tiles.size());
    b->ntiles1 = int(tiles1.size());
    b->ntiles2 = int(tiles2.size());
    size_t off = 0;
    const size_t o_desc = off; off += align_up(size_t(count) * sizeof(GridDesc2), kAlign);
    const size_t o_item = off; off += align_up((size_t(count) + 1) * sizeof(int), kAlign);
    const size_t o_tile = off; off += align_up(std::max<size_t>(tiles.size(), 1) * sizeof(LayerTile), kAlign);
    const size_t o_tg = off; off += align_up(std::max<size_t>(tiles.size(), 1) * sizeof(int), kAlign);
    const size_t o_q = off; off += kAlign;
    const size_t o_item2 = off; off += align_up((size_t(count) + 1) * sizeof(int), kAlign);
    const size_t o_tile1 = off; off += align_up(std::max<size_t>(tiles1.size(), 1) * sizeof(LayerTile), kAlign);
    const size_t o_tg1 = off; off += align_up(std::max<size_t>(tiles1.size(), 1) * sizeof(int), kAlign);
    const size_t o_tile2 = off; off += align_up(std::max<size_t>(tiles2.size(), 1) * sizeof(LayerTile), kAlign);
    const size_t o_tg2 = off; off += align_up(std::max<size_t>(tiles2.size(), 1) * sizeof(int), kAlign);
    cudaError_t e = cudaMalloc(&b->mem, off);
    if (e != cudaSuccess) { b->mem = nullptr; return bail(bfail(PML_ENOMEM, "cudaMalloc(%zu): %s", off, cudaGetErrorString(e))); }
    b->ddesc = reinterpret_cast<GridDesc2 *>(b->mem + o_desc);
    b->ditem_off = reinterpret_cast<int *>(b->mem + o_item);
    b->dtiles = reinterpret_cast<LayerTile *>(b->mem + o_tile);
    b->dtile_grid = reinterpret_cast<int *>(b->mem + o_tg);
    b->dqueue = reinterpret_cast<int *>(b->mem + o_q);
    b->ditem_off2 = reinterpret_cast<int *>(b->mem + o_item2);
    b->dtiles1 = reinterpret_cast<LayerTile *>(b->mem + o_tile1);
    b->dtile_grid1 = reinterpret_cast<int *>(b->mem + o_tg1);
    b->dtiles2 = reinterpret_cast<LayerTile *>(b->mem + o_tile2);
    b->dtile_grid2 = reinterpret_cast<int *>(b->mem + o_tg2);
    if ((e = cudaStreamSynchronize(b->st)) != cudaSuccess) return bail(bfail(PML_ECUDA, "stream synchronize: %s", cudaGetErrorString(e)));
    if (!tiles.empty()) {
        e = cudaMemcpy(b->dtiles, tiles.data(), tiles.size() * sizeof(LayerTile), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->dtile_grid, tile_grid.data(), tile_grid.size() * sizeof(int), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && !tiles1.empty()) {
        e = cudaMemcpy(b->dtiles1, tiles1.data(), tiles1.size() * sizeof(LayerTile), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->dtile_grid1, grid1.data(), grid1.size() * sizeof(int), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && !tiles2.empty()) {
        e = cudaMemcpy(b->dtiles2, tiles2.data(), tiles2.size() * sizeof(LayerTile), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->dtile_grid2, grid2.data(), grid2.size() * sizeof(int), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemset(b->dqueue, 0, 8 * sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(bfail(PML_ECUDA, "batch tables: %s", cudaGetErrorString(e)));
    pml_status s = batch_upload(b);
    if (s != PML_OK) return bail(s);
    *out = b;
    return PML_OK;
}

pml_status pml_batch_step(pml_batch *b, int64_t n)
{
    const NvtxRange nvtx_range("pml_batch_step");
    if (!b) return bfail(PML_EINVAL, "pml_batch_step: batch is NULL");
    if (n < 0) return bfail(PML_EINVAL, "pml_batch_step: n must be >= 0");
    const int p0 = b->ctx[0]->cur;
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        const pml_ctx *c = b->ctx[i];
        if (c->cur != p0)
            return bfail(PML_ESTATE, "pml_batch_step: contexts 0 and %zu are at different step parities", i);
        if (c->ns > 0 || c->nr > 0)
            return bfail(PML_ESTATE, "pml_batch_step: context %zu has sources or receivers (step it with pml_step)", i);
    }
    if (n == 0) return PML_OK;
    int p = p0;
    if ((b->launches & 1) != p) {   // realign the queue parity with the field parity
        PML_BCU(cudaMemsetAsync(b->dqueue, 0, 4 * sizeof(int), b->st), "reset batch queues");
        b->launches = p;
    }
    int64_t left = n;
    while (left > 0) {
        if (b->tb == 2 && left >= 2) {   // two steps per pass
            if (p == 0 && left >= kBatchGraphSteps && !b->prof_on) {
                if (b->launches2 & 1) {   // the graph's second passes start on counter parity 0
                    PML_BCU(cudaMemsetAsync(b->dqueue + 4, 0, 2 * sizeof(int), b->st), "reset batch queues");
                    b->launches2 = 0;
                }
                if (!b->exec) {
                    pml_status s = batch_capture(b);
                    if (s != PML_OK) return s;
                }
                PML_BCU(cudaGraphLaunch(b->exec, b->st), "graph launch");
                left -= kBatchGraphSteps;
                b->launches += kBatchGraphSteps / 2;
                b->launches2 += kBatchGraphSteps / 2;
                continue;
            }
            pml_status s = batch_enqueue_pair(b, p, int(b->launches2 & 1), b->st, b->prof_on);
            if (s != PML_OK) return s;
            p ^= 1;
            left -= 2;
            ++b->launches;
            ++b->launches2;
            continue;
        }
        if (b->tb == 1 && p == 0 && left >= kBatchGraphSteps && !b->prof_on) {
            if (!b->exec) {
                pml_status s = batch_capture(b);
                if (s != PML_OK) return s;
            }
            PML_BCU(cudaGraphLaunch(b->exec, b->st), "graph launch");
            left -= kBatchGraphSteps;
            b->launches += kBatchGraphSteps;
            continue;
        }
        pml_status s = batch_enqueue(b, p, b->st, b->prof_on);
        if (s != PML_OK) return s;
        p ^= 1;
        --left;
        ++b->launches;
    }
    for (pml_ctx *c : b->ctx) {
        c->cur = p;
        c->step += n;
    }
    return PML_OK;
}

pml_status pml_batch_get_variant(const pml_batch *b, int *variant, int *count)
{
    if (!b) return bfail(PML_EINVAL, "pml_batch_get_variant: batch is NULL");
    const int n1 = batch2d_variants(b->prec);
    if (variant) *variant = b->tb == 2 ? n1 + b->var2 : b->var;
    if (count) *count = n1 + (b->tb_ok ? batch2d_tb2_variants(b->prec) : 0);
    return PML_OK;
}

pml_status pml_batch_get_time_block(const pml_batch *b, int *depth)
{
    if (!b || !depth) return bfail(PML_EINVAL, "pml_batch_get_time_block: NULL argument");
    *depth = b->tb;
    return PML_OK;
}

pml_status pml_batch_set_variant(pml_batch *b, int variant)
{
    if (!b) return bfail(PML_EINVAL, "pml_batch_set_variant: batch is NULL");
    const int n1 = batch2d_variants(b->prec), n = n1 + (b->tb_ok ? batch2d_tb2_variants(b->prec) : 0);
    if (variant < 0 || variant >= n) return bfail(PML_EINVAL, "pml_batch_set_variant: variant %d not in [0, %d)", variant, n);
    PML_BCU(cudaStreamSynchronize(b->st), "stream synchronize");
    batch_drop_graph(b);
    const int old = b->var, old_tb = b->tb, old2 = b->var2;
    if (variant < n1) {
        b->var = variant;
        b->tb = 1;
    } else {   // the one-step shape stays: it serves odd steps
        b->var2 = variant - n1;
        b->tb = 2;
    }
    pml_status s = batch_upload(b);
    if (s != PML_OK) {
        b->var = old;
        b->tb = old_tb;
        b->var2 = old2;
        batch_upload(b);
    }
    return s;
}

pml_status pml_batch_autotune(pml_batch *b, int steps, double *times_ms, int *chosen)
{
    if (!b) return bfail(PML_EINVAL, "pml_batch_autotune: batch is NULL");
    if (steps < 1) return bfail(PML_EINVAL, "pml_batch_autotune: steps must be >= 1");
    const int n1 = batch2d_variants(b->prec), n = n1 + (b->tb_ok ? batch2d_tb2_variants(b->prec) : 0);
    cudaEvent_t e0, e1;
    PML_BCU(cudaEventCreate(&e0), "event");
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return bfail(PML_ECUDA, "event"); }
    int best = b->tb == 2 ? n1 + b->var2 : b->var, best1 = b->var;
    double best_ms = 1e300, best1_ms = 1e300;
    pml_status s = PML_OK;
    for (int v = 0; v < n && s == PML_OK; ++v) {
        if ((s = pml_batch_set_variant(b, v)) != PML_OK) break;
        if ((s = pml_batch_step(b, 2)) != PML_OK) break;   // warm-up (and graph capture below)
        cudaEventRecord(e0, b->st);
        if ((s = pml_batch_step(b, steps)) != PML_OK) break;
        cudaEventRecord(e1, b->st);
        if (cudaEventSynchronize(e1) != cudaSuccess) { s = bfail(PML_ECUDA, "autotune synchronize"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = double(ms) / steps;
        if (times_ms) times_ms[v] = per;
        if (per < best_ms) { best_ms = per; best = v; }
        if (v < n1 && per < best1_ms) { best1_ms = per; best1 = v; }
        if (v == n1 - 1 && (s = pml_batch_set_variant(b, best1)) != PML_OK) break;   // kept for odd steps
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != PML_OK) return s;
    if (chosen) *chosen = best;
    return pml_batch_set_variant(b, best);
}

pml_status pml_batch_profile_enable(pml_batch *b, int enable)
{
    if (!b) return bfail(PML_EINVAL, "pml_batch_profile_enable: batch is NULL");
    b->prof_on = enable != 0;
    return PML_OK;
}

pml_status pml_batch_profile_read(pml_batch *b, double ms[2], int64_t launches[2])
{
    if (!b || !ms || !launches) return bfail(PML_EINVAL, "pml_batch_profile_read: NULL argument");
    PML_BCU(cudaStreamSynchronize(b->st), "stream synchronize");
    for (int k = 0; k < 2; ++k) { ms[k] = 0.0; launches[k] = 0; }
    for (size_t i = 0; i < b->prof_n; ++i) {
        float t = 0.f;
        PML_BCU(cudaEventElapsedTime(&t, b->prof_ev[2 * i], b->prof_ev[2 * i + 1]), "event time");
        ms[b->prof_kind[i]] += double(t);
        launches[b->prof_kind[i]] += 1;
    }
    b->prof_n = 0;
    return PML_OK;
}

pml_status pml_batch_info(const pml_batch *b, int64_t info[4])
{
    if (!b || !info) return bfail(PML_EINVAL, "pml_batch_info: NULL argument");
    info[0] = int64_t(b->ctx.size());
    info[1] = b->tb == 2 ? b->n_items2 : b->n_items;
    info[2] = b->tb == 2 ? b->ntiles1 + b->ntiles2 : b->ntiles;
    info[3] = b->tb == 2 ? b->grid_tb : b->grid_int;
    return PML_OK;
}

void pml_batch_destroy(pml_batch *b)
{
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    else cudaDeviceSynchronize();
    batch_drop_graph(b);
    for (cudaEvent_t e : b->prof_ev) cudaEventDestroy(e);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->mem) cudaFree(b->mem);
    delete b;
}

}  // extern "C"

