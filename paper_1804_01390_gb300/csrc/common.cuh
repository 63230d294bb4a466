// Internal declarations shared by the runtime and the kernels of the discrete-PML
// library (sm_103a).  Nothing here is part of the public ABI (include/pml.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace pml {

// Ghost ring width of every padded field array.  The layer kernels read a halo of 4
// vertices (one per RK4 stage), the interior kernels a halo of 2; the ghost ring holds
// periodic copies so that every tile load is a plain rectangular TMA box.
constexpr int G = 4;

// Padded storage of one field: logical vertex (x, y, z), x in [-G, T0+G) etc., lives at
// origin + x + y * P + z * PS.
struct Geom {
    int ndim;
    int wall;          // 0: periodic box (ghost ring = periodic images); 1: reflecting wall
                       // beyond both ends of every axis (ghost ring held at zero)
    int64_t T[3];      // vertices per axis (T[2] = 1 in 2D)
    int64_t wrap[3];   // offset of a vertex's ghost image: T[a] (periodic) or 0 (wall: the
                       // image store lands on the vertex itself and the ghosts stay zero)
    int64_t P;         // row pitch in elements (multiple of 32)
    int64_t R;         // rows per plane incl. ghosts: T[1] + 2G
    int64_t PS;        // plane stride = P * R
    int64_t planes;    // T[2] + 2G (3D) or 1 (2D)
    int64_t elems;     // elements per field array
    int64_t origin;    // element offset of logical (0, 0, 0)
};

// Inclusive output range of the layer-free ("interior") kernels per axis.
struct Range {
    int64_t lo, hi;    // lo > hi: empty
};

// Coefficients of one RK4 step written as the Taylor polynomial
// P(dt A) = I + dt A + (dt A)^2/2 + (dt A)^3/6 + (dt A)^4/24 restricted to the layer-free
// region, where A = [[0, I], [L, 0]] on (U, V) and L = D / h^2 (D the unscaled
// 5-/7-point difference).  Expanding the powers of A:
//   U' = U + a1 V + a2 DU + a3 DV + a4 D^2U + a5 D^2V
//   V' = V + b1 U + b2 DU + b3 DV + b4 D^2U + b5 D^2V
// Forward:  a = (dt, dt^2/2h^2, dt^3/6h^2, dt^4/24h^4, 0),  b = (0, dt/h^2, dt^2/2h^2, dt^3/6h^4, dt^4/24h^4)
// Adjoint (A^T = [[0, L], [I, 0]]):
//           a = (0, dt^2/2h^2, dt/h^2, dt^4/24h^4, dt^3/6h^4), b = (dt, dt^3/6h^2, dt^2/2h^2, 0, dt^4/24h^4)
template <typename T> struct StepCoefT {
    T a1, a2, a3, a4, a5;
    T b1, b2, b3, b4, b5;
};
// Both precisions are carried so that a kernel never converts a coefficient on the device
// (a double -> float conversion runs on the FP64 pipe, which is narrow on this part).
struct StepCoef {
    StepCoefT<double> d;
    StepCoefT<float> f;
};
template <typename T> __host__ __device__ __forceinline__ const StepCoefT<T> &coef_of(const StepCoef &c);
template <> __host__ __device__ __forceinline__ const StepCoefT<double> &coef_of<double>(const StepCoef &c) { return c.d; }
template <> __host__ __device__ __forceinline__ const StepCoefT<float> &coef_of<float>(const StepCoef &c) { return c.f; }

// Constants of the layer kernels (1/h, 1/h^2, 1/(2h) and the Horner coefficients
// dt/4, dt/3, dt/2, dt), in both precisions.
template <typename T> struct LayerConstT {
    T ih, ih2, i2h, c4, c3, c2, c1;
};
struct LayerConst {
    LayerConstT<double> d;
    LayerConstT<float> f;
};
template <typename T> __host__ __device__ __forceinline__ const LayerConstT<T> &lconst_of(const LayerConst &c);
template <> __host__ __device__ __forceinline__ const LayerConstT<double> &lconst_of<double>(const LayerConst &c) { return c.d; }
template <> __host__ __device__ __forceinline__ const LayerConstT<float> &lconst_of<float>(const LayerConst &c) { return c.f; }

// One output tile of a layer kernel (2D: z fields unused).
struct LayerTile {
    int32_t x0, y0, z0;        // tile origin (x0 multiple of 4)
    int32_t xlo, xhi;          // inclusive output clamp (rectangle of the frame)
    int32_t ylo, yhi;
    int32_t zlo, zhi;
    int32_t flags;             // bit a: aux fields of axis a are active in the footprint
};

struct DeviceError {
    int code;                  // 0 = ok, 1 = a bounded mbarrier wait gave up, 2 = the finiteness
                               // scan met a non-finite value
    int where;                 // code 1: wait site; code 2: field (0 U, 1 V)
    long long step;            // code 2: step counter when the scan ran
};

// ---------------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------------
#ifdef __CUDACC__

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// The dynamic shared memory `base` rounded up to a 128-byte boundary (TMA destinations).  The
// result is an offset from `base`, not a round trip through an integer, so the compiler still
// knows that accesses through it are shared-memory accesses (32-bit addresses).
template <typename T> __device__ __forceinline__ T *smem_align128(unsigned char *base)
{
    return reinterpret_cast<T *>(base + ((128u - (smem_u32(base) & 127u)) & 127u));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
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

// Bounded wait: gives up after `limit_ns` nanoseconds of the global timer (checked every
// 256 polls), records the failure and returns false.  No wait in this library can spin
// forever.  limit_ns = 0 means the default, far above any legitimate wait (a few
// microseconds); a limit below kImmediateNs gives up at once without probing (the
// context's wait-limit setting uses this to exercise the error path of every kernel on
// purpose: each kernel then waits, bounded by kDrainLimitNs, for the copies it has in
// flight, including the one it gave up on, before it ends).
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s
constexpr uint64_t kDrainLimitNs = 100000000ull;   // 0.1 s, waits on the error path
constexpr uint64_t kImmediateNs = 1000ull;

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, DeviceError *err, int where,
                                          uint64_t limit_ns = 0)
{
    if (limit_ns != 0 && limit_ns < kImmediateNs) {
        // give up at once, landed or not: the caller's error path then lets the copy land
    } else {
        if (mbar_try_wait(bar, parity)) return true;
        const uint64_t lim = limit_ns ? limit_ns : kWaitLimitNs;
        const uint64_t t0 = global_ns();
        for (;;) {
            for (int i = 0; i < 256; ++i)
                if (mbar_try_wait(bar, parity)) return true;
            if (global_ns() - t0 > lim) break;
        }
    }
    if (err) {
        atomicCAS(&err->code, 0, 1);
        err->where = where;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int32_t x, int32_t y,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int32_t x, int32_t y,
                                            int32_t z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Four consecutive x values of one row owned by one lane.
template <typename T> struct V4 {
    T x, y, z, w;
};

template <typename T> __device__ __forceinline__ V4<T> lds4(const T *p);
template <> __device__ __forceinline__ V4<float> lds4<float>(const float *p)
{
    float4 v = *reinterpret_cast<const float4 *>(p);
    return {v.x, v.y, v.z, v.w};
}
template <> __device__ __forceinline__ V4<double> lds4<double>(const double *p)
{
    double2 a = reinterpret_cast<const double2 *>(p)[0];
    double2 b = reinterpret_cast<const double2 *>(p)[1];
    return {a.x, a.y, b.x, b.y};
}

template <typename T> __device__ __forceinline__ void stg4(T *p, const V4<T> &v);
template <> __device__ __forceinline__ void stg4<float>(float *p, const V4<float> &v)
{
    *reinterpret_cast<float4 *>(p) = make_float4(v.x, v.y, v.z, v.w);
}
template <> __device__ __forceinline__ void stg4<double>(double *p, const V4<double> &v)
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(v.x, v.y);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v.z, v.w);
}

template <typename T> __device__ __forceinline__ T get4(const V4<T> &v, int k)
{
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// Store one value at logical (x, y, z) and at every periodic image that falls inside the
// ghost ring, so that the next step's tile loads see a periodic field.
template <typename T>
__device__ __forceinline__ void store_wrapped(T *base, const Geom &g, int64_t x, int64_t y, int64_t z,
                                              T v)
{
    int64_t xs[2] = {x, x}, ys[2] = {y, y}, zs[2] = {z, z};
    int nx = 1, ny = 1, nz = 1;
    if (x < G) xs[nx++] = x + g.wrap[0];
    else if (x >= g.T[0] - G) xs[nx++] = x - g.wrap[0];
    if (y < G) ys[ny++] = y + g.wrap[1];
    else if (y >= g.T[1] - G) ys[ny++] = y - g.wrap[1];
    if (g.ndim == 3) {
        if (z < G) zs[nz++] = z + g.wrap[2];
        else if (z >= g.T[2] - G) zs[nz++] = z - g.wrap[2];
    }
    for (int c = 0; c < nz; ++c)
        for (int b = 0; b < ny; ++b)
            for (int a = 0; a < nx; ++a) base[g.origin + xs[a] + ys[b] * g.P + zs[c] * g.PS] = v;
}

// Programmatic dependent launch: let the next kernel in the stream start (its CTAs only
// start once every CTA of this grid has called this), and wait for the previous kernel's
// grid to complete (so that completion of this grid implies completion of that one).
__device__ __forceinline__ void allow_dependent_launch()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void wait_prerequisite_grid()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ bool near_edge(const Geom &g, int64_t x, int64_t y, int64_t z)
{
    bool e = x < G || x >= g.T[0] - G || y < G || y >= g.T[1] - G;
    if (g.ndim == 3) e = e || z < G || z >= g.T[2] - G;
    return e;
}

#endif  // __CUDACC__

// ---------------------------------------------------------------------------------
// kernel launchers (defined in the kernel translation units)
// ---------------------------------------------------------------------------------

// Interior (layer-free) step of a 2D field pair: reads (U, V) through the tensor maps,
// writes (Uo, Vo) on the output rectangle xr x yr.  Persistent kernel fed by a work
// queue: this launch counts on queue[parity] and clears queue[1 - parity].
struct Interior2DArgs {
    Geom g;
    Range xr, yr;
    StepCoef c;
    DeviceError *err;
    uint64_t wait_ns;          // limit of every bounded wait (0: the default 2 s)
    int *queue;
    int parity;
    int rows;                  // rows per work item of the warp-streaming shape (0: its default)
};
// Variant v of the 2D interior kernel (see kI2Vars32 / kI2Vars64 in step2d.cu): its TMA
// box is interior2d_box_cols(prec, v) x interior2d_box_rows(prec, v).
int interior2d_variants(int prec);
int interior2d_box_cols(int prec, int v);
int interior2d_box_rows(int prec, int v);
int interior2d_max_blocks_per_sm(int prec, bool adjoint, int v);
// overlap_previous: the launch may start while the previous kernel of the stream (the
// layer kernel of the same step, whose outputs it does not read) is still running
cudaError_t launch_interior2d(int prec, bool adjoint, int v, const CUtensorMap *tmU, const CUtensorMap *tmV,
                              void *Uo, void *Vo, const Interior2DArgs &a, int grid, cudaStream_t st,
                              bool overlap_previous);
// Two steps per pass (temporal blocking depth 2; forward or transposed) over the run given
// in a.xr, a.yr (the layer-free run shrunk by 2 where a layer bounds it); FP32 only
// (variants() = 0 for FP64).  Its TMA box is interior2d_tb2_box_cols(prec, v) x interior2d_tb2_box_rows(prec, v).
int interior2d_tb2_variants(int prec);
int interior2d_tb2_box_rows(int prec, int v);
int interior2d_tb2_box_cols(int prec, int v);
int interior2d_tb2_max_blocks_per_sm(int prec, bool adjoint, int v);
cudaError_t launch_interior2d_tb2(int prec, bool adjoint, int v, const CUtensorMap *tmU, const CUtensorMap *tmV,
                                  void *Uo, void *Vo, const Interior2DArgs &a, int grid, cudaStream_t st,
                                  bool overlap_previous);

// Layer step of 2D strips (Horner form of the RK4 polynomial with the full operator).
struct Layer2DArgs {
    Geom g;
    LayerConst k;
    const void *sig[2];        // device sigma per axis (context precision), length T[a]
    const LayerTile *tiles;
    int ntiles;
    DeviceError *err;
    uint64_t wait_ns;          // limit of every bounded wait (0: the default 2 s)
    int *queue;                // work counters (this launch: queue[parity]; clears the other)
    int parity;
};
// 2D layer work items: one strip of layer2d_tile_cols() output columns (one warp, halo
// 4 columns per side) by a run of rows, taken by the warps from a work queue
constexpr int kLayer2BandRows = 32;  // most output rows of one item of the y band
constexpr int kLayer2SlabRows = 24;  // most output rows of one item of an x slab
constexpr int kLayer2BandRowsTB = 32;  // the same for the frames of two-step blocks
constexpr int kLayer2SlabRowsTB = 24;
constexpr int kLayer2MinOffRows = 8;   // shorter inactive row runs next to active rows join them
constexpr int kLayer2SlabRowsWall = 32;    // x-slab items of a wall-backed box (two short bands, no seam)
constexpr int kLayer2BandRowsBatch = 40;   // items of a batch (many frames, many items per warp)
constexpr int kLayer2SlabRowsBatch = 40;
int layer2d_grid(int prec, int ntiles, int sm_count);   // CTAs of one layer launch (warps loop over items)
int layer2d_box_rows();               // rows of the layer kernel's TMA box
int layer2d_box_cols(int prec);       // columns of the layer kernel's TMA box (one strip)
int layer2d_tile_cols(int prec);      // output columns of one layer strip (box minus the halo)
// overlap_previous: the launch may start while the previous kernel of the stream runs; the
// kernel waits for that kernel to complete before it reads anything (its inputs may be
// that kernel's outputs), but the kernel after it may start early
cudaError_t launch_layer2d(int prec, bool adjoint, const CUtensorMap *tm /*[6] U,V,Px,Qx,Py,Qy*/,
                           void *const *out /*[6]*/, const Layer2DArgs &a, int grid, cudaStream_t st,
                           bool overlap_previous = false);

// Batched 2D step over many independent grids: one interior launch and one layer launch
// per step for the whole batch.  Per-grid descriptors (tensor maps included) live in device
// memory; work items of all grids share one queue.
struct GridDesc2 {   // aligned as CUtensorMap
    CUtensorMap tm_int[2][2];  // [input parity][U, V], interior box of the batch's variant
    CUtensorMap tm_lay[2][6];  // [input parity][field], layer box
    CUtensorMap tm_tb[2][2];   // [input parity][U, V], box of the two-step interior shape
    CUtensorMap tm_mid[6];     // first-step values of a two-step block, layer box
    void *out[2][6];           // output buffers when the input parity is p
    void *mid[6];              // first-step values of a two-step block
    Interior2DArgs in;         // geometry, layer-free ranges, coefficients
    Interior2DArgs in2;        // the same with the run shrunk by 2 (two-step interior)
    Layer2DArgs lay;           // geometry, constants, sigma (tiles: the batch list)
    int rblocks, nstrips;      // interior work items of this grid: nstrips x rblocks
    int rblocks2, nstrips2;    // two-step interior work items of this grid
};
struct Batch2DArgs {
    const GridDesc2 *desc;
    const int *item_off;       // [ngrid + 1] first interior item of each grid (of this launch's kind)
    const LayerTile *tiles;    // layer tiles of all grids (of this launch's frame)
    const int *tile_grid;      // grid of each tile
    int ngrid, n_items, ntiles;
    int *queue;                // work counters: interior [2], layer [2], second layer pass [2]
    int parity;                // input parity of every grid; a launch counts on counter [parity]
    int pass;                  // layer launch: 0 one step (fields -> fields), 1 first pass of a
                               // two-step block (fields -> mid), 2 second pass (mid -> fields)
    int qparity;               // counter parity of a second pass (its own launch count)
};
int batch2d_variants(int prec);
int batch2d_box_cols(int prec, int v);     // interior tensor-map box of variant v
int batch2d_box_rows(int prec, int v);
int batch2d_item_rows(int prec, int v);    // output rows per interior work item
int batch2d_strip_cols(int prec, int v);   // output columns per interior work item
int batch2d_interior_blocks_per_sm(int prec, int v);
cudaError_t launch_batch2d_interior(int prec, int v, const Batch2DArgs &a, int grid, cudaStream_t st,
                                    bool overlap_previous);
cudaError_t launch_batch2d_layer(int prec, const Batch2DArgs &a, int grid, bool wall, cudaStream_t st,
                                 bool overlap_previous = false);
// Two-step (temporally blocked) batched interior shapes (FP32 only).
int batch2d_tb2_variants(int prec);
int batch2d_tb2_box_cols(int prec, int v);
int batch2d_tb2_box_rows(int prec, int v);
int batch2d_tb2_item_rows(int prec, int v);
int batch2d_tb2_strip_cols(int prec, int v);
int batch2d_tb2_blocks_per_sm(int prec, int v);
cudaError_t launch_batch2d_tb2(int prec, int v, const Batch2DArgs &a, int grid, cudaStream_t st,
                               bool overlap_previous);

// 3D counterparts.
struct Interior3DArgs {
    Geom g;
    Range xr, yr, zr;
    StepCoef c;
    DeviceError *err;
    uint64_t wait_ns;          // limit of every bounded wait (0: the default 2 s)
    int *queue;                // work counters (this launch: queue[parity])
    int parity;
    float2 pf[11];             // FP32 kernel: a1..a5, b1..b5, -6 as pairs (set by the launcher)
};
cudaError_t launch_interior3d(int prec, bool adjoint, const CUtensorMap *tmU, const CUtensorMap *tmV,
                              void *Uo, void *Vo, const Interior3DArgs &a, int grid, bool overlap_previous,
                              cudaStream_t st);
int interior3d_box_rows(int prec);
int interior3d_tile_y(int prec);   // output rows of a CTA tile
int interior3d_box_cols(int prec);   // box width of the 3D interior kernel (one strip plus halo)
int interior3d_max_blocks_per_sm(int prec, bool adjoint);

struct Layer3DArgs {
    Geom g;
    LayerConst k;
    const void *sig[3];
    const LayerTile *tiles;    // sorted by flags (set of axes with active aux fields)
    int ntiles;
    int class_off[9];          // tiles of flags m are [class_off[m], class_off[m+1])
    DeviceError *err;
    uint64_t wait_ns;          // limit of every bounded wait (0: the default 2 s)
};
// 3D layer column tiles (x, y output extent; halo 4 on each side) and z segment length
constexpr int kLayer3TXf = 28, kLayer3TYf = 9;   // FP32: 36 x 17 region columns (20 warps)
constexpr int kLayer3TXd = 12, kLayer3TYd = 4;   // FP64: 20 x 12 region columns
constexpr int kLayer3LZ = 32;
// The 3D frame by level passes (frame3d.cu): one Horner level per launch over dense
// scratch buffers, on the frame widened by level - 1; tiles of kLevel3TX x kLevel3TY
// columns by kLevel3TZ planes, one CTA each.
struct Level3Args {
    Geom g;
    LayerConst k;
    const void *sig[3];
    const void *in[8];         // the level's operand (the state y for level 4), by global field id
    const void *base[8];       // the state y
    void *out[8];
    const LayerTile *tiles;    // flags: axes whose aux fields reach the tile
    int ntiles;
    int level;                 // 4, 3, 2, 1: out = y + (dt / level) A in
};
constexpr int kLevel3TX = 32, kLevel3TY = 8, kLevel3TZ = 16;
cudaError_t launch_level3d(int prec, bool adjoint, const Level3Args &a, cudaStream_t st);
int layer3d_tile_x(int prec);
int layer3d_tile_y(int prec);
// The 3D layer frame by slab tiles (slab3d.cuh, FP32 only): tiles of class m (bit a: aux
// fields of axis a within reach of the tile's outputs) have a region of rx x ry columns,
// outputs inset by hx, hy (4 along active axes, 2 along the others) and z items of at most
// kSlabItemZ output planes; tensor maps [class m][field f] with box rx x ry x 1.
void slab3d_shape(int mask, int *rx, int *ry, int *hx, int *hy);
// per class: threads, registers, the largest block the registers allow, shared memory
std::string slab3d_describe(bool adjoint, bool wall);
constexpr int kSlabItemZ = 64;
cudaError_t launch_slab3d(bool adjoint, const CUtensorMap *tm /*[8][8]*/, void *const *out /*[8]*/,
                          const Layer3DArgs &a, cudaStream_t st);
cudaError_t launch_slab3d_wall(bool adjoint, const CUtensorMap *tm /*[8][8]*/, void *const *out /*[8]*/,
                               const Layer3DArgs &a, cudaStream_t st);
// The eight class launches follow each other with programmatic dependent launch (their
// outputs are disjoint), the first one after all earlier work of the stream.
cudaError_t launch_layer3d(int prec, bool adjoint, const CUtensorMap *tm /*[8]*/,
                           void *const *out /*[8]*/, const Layer3DArgs &a, cudaStream_t st);
cudaError_t launch_layer3d_wall(int prec, bool adjoint, const CUtensorMap *tm /*[8]*/,
                                void *const *out /*[8]*/, const Layer3DArgs &a, cudaStream_t st);

// Launch with programmatic stream serialization when overlap_previous: the kernel may
// start while the previous kernel of the stream still runs (their outputs must be
// disjoint); the kernel calls wait_prerequisite_grid() before it finishes.
template <typename K, typename... Args>
inline cudaError_t launch_pdl(K kernel, int grid, int threads, size_t smem, cudaStream_t st, bool overlap_previous,
                              Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(unsigned(threads));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = overlap_previous ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Damping gradient (grad_sigma.cu): explicit stage evaluations on lists of row chunks
// {x0, x1, y, z} (inclusive x range of row (y, z), at most kStageChunkMax vertices each) and
// the per-edge contraction kbar^T (dA/dsigma_a[e]) Y of the four stage pairs of a step.
constexpr int kStageChunkMax = 64;
struct SigmaPtrs {
    const void *p[3];          // device sigma per axis (context precision)
};
// out = alpha base + cop Op(in) on the segments (Op = A or A^T)
cudaError_t launch_stage(int prec, bool adjoint, void *const *in, void *const *base, void *const *out, int nf,
                         const Geom &g, const SigmaPtrs &s, double h, double alpha, double cop, const int4 *seg,
                         int nseg, cudaStream_t st);
// acc[edge] += sum_i scale[i] kb[i]^T (dA/dsigma) Y[i], i = 0..3
cudaError_t launch_contract4(int prec, void *const *const *kb, void *const *const *Y, const double *scale, int nf,
                             const Geom &g, const SigmaPtrs &s, double h, double *acc, cudaStream_t st);
cudaError_t launch_residual(int prec, const void *trace, const void *target, void *res, int64_t count,
                            double *misfit, cudaStream_t st);

// Sources and receivers after a forward step; receiver injection and source-amplitude
// gradients before an adjoint step.
struct PointArgs {
    Geom g;
    int ns;
    const int64_t *src_off;    // element offsets (origin-relative flat index) of sources
    const int32_t *src_xyz;    // logical coordinates [ns][3]
    const double *src_amp;
    double f_peak, t_delay;
    int nr;
    const int64_t *rec_off;
    double dt, h;
    // Points whose updates touch a common vertex must add in index order: every source has
    // a level one above the highest level of the earlier sources whose stencils (the
    // vertex and its 2 d neighbours) meet its own, every receiver one above the earlier
    // receivers at its vertex; the kernels run level after level, each level in parallel.
    const int32_t *src_level;
    int src_levels;
    const int32_t *rec_xyz;    // logical coordinates [nr][3]
    const int32_t *rec_level;
    int rec_levels;
};
cudaError_t launch_post_step(int prec, void *U, void *V, const PointArgs &a, int64_t step,
                             void *trace_row, cudaStream_t st);
cudaError_t launch_adjoint_points(int prec, void *Ub, void *Vb, const PointArgs &a, int64_t m,
                                  const void *residual_row, double *grad_amp, cudaStream_t st);

// Finiteness scan of U and V over the box (ghost ring and row padding excluded): the
// first non-finite value found sets err->code = 2 (where = field, step = `step`).
cudaError_t launch_check_finite(int prec, const void *U, const void *V, const Geom &g, DeviceError *err,
                                int64_t step, cudaStream_t st);

// Ghost ring refresh, dense <-> padded copies and FP64 norms.
cudaError_t launch_fill_ghosts(int prec, void *f, const Geom &g, cudaStream_t st);
cudaError_t launch_norms(int prec, const void *U, const void *V, const Geom &g, const int64_t *wlo,
                         const int64_t *whi, double h, const double *ref, double *partials,
                         int nblocks, double *out, cudaStream_t st);
constexpr int kNormBlocks = 592;   // fixed partition (4 x 148): deterministic sums
constexpr int kNormVals = 5;

}  // namespace pml
