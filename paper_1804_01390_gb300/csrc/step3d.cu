// 3D kernels of one RK4 step of the discrete PML system (eq:DiscretePML, Sec. 1.1.2) on
// sm_103a.  Same evaluation of the RK4 polynomial as the 2D kernels (closed form in the
// layer-free region, Horner form with the full operator in the layer frame), with the
// 7-point difference and streaming along z.
//
//  * k_interior3d_rows (FP32, interior3d_rows.cuh): several rows per warp, see there.
//
//  * k_interior3d (FP64): a CTA owns a 30 NC-column x strip by kBY3 output rows and streams z.
//    One warp per region row (kBY3 + 4 rows: halo 2 in y); TMA brings one z-plane box of
//    U and V per stage; each lane keeps three planes of U, V, DU, DV in registers (z
//    neighbours; NC = 2 columns per lane, so two CTAs fit on an SM), y neighbours come
//    from the shared-memory plane, x neighbours from shuffles.  DU/DV planes go through a 3-slot shared ring for the second difference.
//
//  * k_layer3d: a CTA owns an (x, y) column tile of the frame and streams z; one thread
//    per region column (halo 4 in x and y).  The four Horner levels run pipelined in z:
//    when input plane p arrives, level 4 produces plane p-1, level 3 plane p-2, level 2
//    plane p-3 and level 1 (the output) plane p-4.  Own-column z neighbours live in
//    register rings, x/y neighbours in one shared plane per level; one block barrier per
//    plane.  Templated on the set of axes whose aux fields are active in the tile, so
//    face tiles carry 4 fields, edge tiles 6 and corner tiles 8.
#include <cstdio>

#include "common.cuh"

namespace pml {

constexpr int kBY3 = 8;        // interior output rows per CTA
constexpr int kS3 = 4;         // interior TMA plane stages
constexpr int kZSeg3 = 64;     // z planes per interior work item
template <typename T> struct I3Cfg {
    static constexpr int NC = 2;                         // columns per lane
    static constexpr int MINB = sizeof(T) == 4 ? 2 : 1;  // resident CTAs per SM
};

int interior3d_box_rows(int) { return 1; }
int interior3d_tile_y(int prec);   // defined after the FP32 kernel's shape
int interior3d_box_cols(int prec) { return 32 * (prec == 32 ? I3Cfg<float>::NC : I3Cfg<double>::NC); }

// NC adjacent columns of one lane
template <typename T, int NC> struct VN {
    T c[NC];
};
template <typename T, int NC> __device__ __forceinline__ VN<T, NC> ldsN(const T *p)
{
    VN<T, NC> v;
    if constexpr (sizeof(T) * NC == 8) {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        v.c[0] = t.x;
        v.c[1] = t.y;
    } else {
#pragma unroll
        for (int q = 0; q < NC; q += 16 / int(sizeof(T))) {
            if constexpr (sizeof(T) == 4) {
                const float4 t = *reinterpret_cast<const float4 *>(p + q);
                v.c[q] = t.x; v.c[q + 1] = t.y; v.c[q + 2] = t.z; v.c[q + 3] = t.w;
            } else {
                const double2 t = *reinterpret_cast<const double2 *>(p + q);
                v.c[q] = t.x; v.c[q + 1] = t.y;
            }
        }
    }
    return v;
}
template <typename T, int NC> __device__ __forceinline__ void stN(T *p, const VN<T, NC> &v)
{
    if constexpr (sizeof(T) * NC == 8) {
        *reinterpret_cast<float2 *>(p) = make_float2(v.c[0], v.c[1]);
    } else {
#pragma unroll
        for (int q = 0; q < NC; q += 16 / int(sizeof(T))) {
            if constexpr (sizeof(T) == 4)
                *reinterpret_cast<float4 *>(p + q) = make_float4(v.c[q], v.c[q + 1], v.c[q + 2], v.c[q + 3]);
            else
                *reinterpret_cast<double2 *>(p + q) = make_double2(v.c[q], v.c[q + 1]);
        }
    }
}

// Unscaled 7-point difference of one lane's NC columns; x neighbours beyond the lane from
// the neighbouring lanes.
template <typename T, int NC>
__device__ __forceinline__ VN<T, NC> diff7(const VN<T, NC> &c, const VN<T, NC> &ym, const VN<T, NC> &yp,
                                           const VN<T, NC> &zm, const VN<T, NC> &zp)
{
    const T l = __shfl_up_sync(0xffffffffu, c.c[NC - 1], 1);
    const T r = __shfl_down_sync(0xffffffffu, c.c[0], 1);
    VN<T, NC> o;
    if constexpr (sizeof(T) == 4 && NC == 2) {   // packed FP32x2: one instruction per pair
        const float2 cc = make_float2(c.c[0], c.c[1]);
        float2 t = __fadd2_rn(make_float2(l, c.c[0]), make_float2(c.c[1], r));
        t = __fadd2_rn(t, __fadd2_rn(make_float2(ym.c[0], ym.c[1]), make_float2(yp.c[0], yp.c[1])));
        t = __fadd2_rn(t, __fadd2_rn(make_float2(zm.c[0], zm.c[1]), make_float2(zp.c[0], zp.c[1])));
        t = __ffma2_rn(make_float2(-6.f, -6.f), cc, t);
        o.c[0] = t.x;
        o.c[1] = t.y;
    } else {
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            const T left = q == 0 ? l : c.c[q - 1], right = q == NC - 1 ? r : c.c[q + 1];
            o.c[q] = (((left + right) + (ym.c[q] + yp.c[q])) + (zm.c[q] + zp.c[q])) - T(6) * c.c[q];
        }
    }
    return o;
}

template <typename T> struct I3 {
    static constexpr int NC = I3Cfg<T>::NC;
    static constexpr int NW = kBY3 + 4;
    static constexpr int ROW = 32 * NC;         // box width (lane 0 and lane 31 hold the x halo)
    static constexpr int STRIP = 30 * NC;       // output columns per CTA
    static constexpr uint32_t FIELD = NW * ROW * sizeof(T);
    static constexpr uint32_t STAGE = 2 * FIELD;
    static constexpr uint32_t DPLANE = 2 * (kBY3 + 2) * ROW * sizeof(T);
    static constexpr size_t SMEM = size_t(kS3) * STAGE + 3 * DPLANE + 128;
};

template <typename T, bool ADJ>
__global__ void __launch_bounds__(32 * (kBY3 + 4), I3Cfg<T>::MINB)
    k_interior3d(const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmV,
                 T *__restrict__ Uo, T *__restrict__ Vo, const Interior3DArgs a)
{
    using C = I3<T>;
    constexpr int NC = C::NC, ROW = C::ROW, NW = C::NW, S = kS3, DR = kBY3 + 2;
    using VT = VN<T, NC>;
    __shared__ __align__(8) uint64_t bars[S];
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *smem =
        smem_align128<unsigned char>(smem_dyn);
    T *dbuf = reinterpret_cast<T *>(smem + S * C::STAGE);   // [3][2][DR][ROW]

    const int tid = threadIdx.x, k = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        prefetch_tmap(&tmU);
        prefetch_tmap(&tmV);
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    const Geom &g = a.g;
    // strips start where the box's first column (xs - NC) is a multiple of 4 (TMA alignment)
    const int64_t xs0 = a.xr.lo - ((a.xr.lo - NC + G) & 3);
    const int64_t nstrips = (a.xr.hi - xs0) / C::STRIP + 1;
    const int64_t nty = (a.yr.hi - a.yr.lo) / kBY3 + 1;
    const int64_t nz = a.zr.hi - a.zr.lo + 1;
    const int nzs = int((nz + kZSeg3 - 1) / kZSeg3);
    const int n_items = int(nstrips * nty) * nzs;
    __shared__ int item_sh;
    if (blockIdx.x == 0 && tid == 0) a.queue[1 - a.parity] = 0;

    const StepCoefT<T> &kc = coef_of<T>(a.c);
    const T a1 = kc.a1, a2 = kc.a2, a3 = kc.a3, a4 = kc.a4, a5 = kc.a5;
    const T b1 = kc.b1, b2 = kc.b2, b3 = kc.b3, b4 = kc.b4, b5 = kc.b5;
    uint32_t use = 0;

    for (;;) {
        // work item: (x strip s, y tile t, z segment) taken from the queue
        if (tid == 0) item_sh = atomicAdd(&a.queue[a.parity], 1);
        __syncthreads();
        const int item = item_sh;
        __syncthreads();
        if (item >= n_items) break;
        const int64_t col = item / nzs, zs = item - col * nzs;
        const int64_t zi = zs * kZSeg3;
        const int64_t cnt = (nz - zi) < kZSeg3 ? (nz - zi) : kZSeg3;
        const int64_t s = col / nty, t = col - s * nty;
        const int64_t xs = xs0 + C::STRIP * s, y0 = a.yr.lo + kBY3 * t, z0 = a.zr.lo + zi;
        const int n_in = int(cnt) + 4;
        const int32_t tx = int32_t(xs - NC + G), ty = int32_t(y0 - 2 + G), tz = int32_t(z0 - 2 + G);

        if (tid == 0) {
            fence_proxy_async();
            const int npro = n_in < S ? n_in : S;
            for (int p = 0; p < npro; ++p) {
                const int st = (use + p) % S;
                unsigned char *dst = smem + st * C::STAGE;
                mbar_arrive_expect_tx(&bars[st], C::STAGE);
                tma_load_3d(dst, &tmU, tx, ty, tz + p, &bars[st]);
                tma_load_3d(dst + C::FIELD, &tmV, tx, ty, tz + p, &bars[st]);
            }
        }

        const int64_t x0 = xs - NC + NC * lane;
        const int64_t y = y0 - 2 + k;
        const bool out_lane = lane >= 1 && lane <= 30;
        const bool full_vec =
            out_lane && x0 >= a.xr.lo && x0 + NC - 1 <= a.xr.hi && x0 >= G && x0 + NC - 1 < g.T[0] - G;
        // the lane's columns and row lie more than G from every box edge: no ghost images
        const bool row_inner = x0 >= G && x0 + NC - 1 < g.T[0] - G && y >= G && y < g.T[1] - G;
        const bool d_row = k >= 1 && k <= kBY3 + 2;
        const bool o_row = k >= 2 && k <= kBY3 + 1 && y <= a.yr.hi;
        // the thread's offsets in a stage plane (rows k, k - 1, k + 1) and in a difference plane
        // (rows k - 1, k - 2, k), and its output offset without the plane term
        const int lo = NC * lane;
        const int o_c = k * ROW + lo, o_m = (k - 1) * ROW + lo, o_p = (k + 1) * ROW + lo;
        const int d_c = (k - 1) * ROW + lo, d_m = (k - 2) * ROW + lo, d_p = k * ROW + lo;
        const int64_t obase = g.origin + y * g.P + x0;
        VT u[3], v[3], du[3], dv[3];
        bool ok = true;
        int pfail = n_in;   // first plane whose wait gave up

        for (int p0 = 0; p0 < n_in && ok; p0 += 3) {
#pragma unroll
            for (int PH = 0; PH < 3; ++PH) {
                const int p = p0 + PH;
                if (p < n_in && ok) {
                    const uint32_t uu = use + p;
                    const int st = uu % S;
                    if (!mbar_wait(&bars[st], (uu / S) & 1u, a.err, 3, a.wait_ns)) {
                        ok = false;
                    } else {
                        const T *sU = reinterpret_cast<const T *>(smem + st * C::STAGE);
                        const T *sV = sU + NW * ROW;
                        u[PH] = ldsN<T, NC>(sU + o_c);
                        v[PH] = ldsN<T, NC>(sV + o_c);
                        const int J1 = (PH + 2) % 3, J2 = (PH + 1) % 3;   // planes p-1, p-2
                        if (p >= 2 && d_row) {
                            const int sp = (use + p - 1) % S;
                            const T *pU = reinterpret_cast<const T *>(smem + sp * C::STAGE);
                            const T *pV = pU + NW * ROW;
                            du[J1] = diff7(u[J1], ldsN<T, NC>(pU + o_m), ldsN<T, NC>(pU + o_p), u[J2], u[PH]);
                            dv[J1] = diff7(v[J1], ldsN<T, NC>(pV + o_m), ldsN<T, NC>(pV + o_p), v[J2], v[PH]);
                            T *db = dbuf + ((PH + 2) % 3) * 2 * DR * ROW;   // plane p - 1 (p0 is a multiple of 3)
                            stN(db + d_c, du[J1]);
                            stN(db + DR * ROW + d_c, dv[J1]);
                        }
                    }
                }
                ok = __syncthreads_and(ok);
                if (!ok && pfail == n_in) pfail = p;
                if (p < n_in && ok) {
                    if (tid == 0 && p >= 1 && p - 1 + S < n_in) {
                        fence_proxy_async();
                        const int st2 = (use + p - 1) % S;
                        unsigned char *dst = smem + st2 * C::STAGE;
                        mbar_arrive_expect_tx(&bars[st2], C::STAGE);
                        tma_load_3d(dst, &tmU, tx, ty, tz + p - 1 + S, &bars[st2]);
                        tma_load_3d(dst + C::FIELD, &tmV, tx, ty, tz + p - 1 + S, &bars[st2]);
                    }
                    if (p >= 4 && o_row) {
                        const int J1 = (PH + 2) % 3, J2 = (PH + 1) % 3;
                        const T *db = dbuf + ((PH + 1) % 3) * 2 * DR * ROW;   // plane p - 2
                        const VT d2u = diff7(du[J2], ldsN<T, NC>(db + d_m), ldsN<T, NC>(db + d_p), du[PH], du[J1]);
                        const VT d2v = diff7(dv[J2], ldsN<T, NC>(db + DR * ROW + d_m), ldsN<T, NC>(db + DR * ROW + d_p),
                                             dv[PH], dv[J1]);
                        const VT &uc = u[J2], &vc = v[J2], &duc = du[J2], &dvc = dv[J2];
                        VT uo, vo;
                        if constexpr (sizeof(T) == 4 && NC == 2) {   // packed FP32x2
                            auto P = [](const VT &x) { return make_float2(x.c[0], x.c[1]); };
                            auto B = [](T x) { return make_float2(x, x); };
                            float2 tu, tv;
                            if (!ADJ) {
                                tu = __ffma2_rn(B(a1), P(vc), __ffma2_rn(B(a2), P(duc), __ffma2_rn(B(a3), P(dvc), __fmul2_rn(B(a4), P(d2u)))));
                                tv = __ffma2_rn(B(b2), P(duc), __ffma2_rn(B(b3), P(dvc), __ffma2_rn(B(b4), P(d2u), __fmul2_rn(B(b5), P(d2v)))));
                            } else {
                                tu = __ffma2_rn(B(a2), P(duc), __ffma2_rn(B(a3), P(dvc), __ffma2_rn(B(a4), P(d2u), __fmul2_rn(B(a5), P(d2v)))));
                                tv = __ffma2_rn(B(b1), P(uc), __ffma2_rn(B(b2), P(duc), __ffma2_rn(B(b3), P(dvc), __fmul2_rn(B(b5), P(d2v)))));
                            }
                            tu = __fadd2_rn(P(uc), tu);
                            tv = __fadd2_rn(P(vc), tv);
                            uo.c[0] = tu.x; uo.c[1] = tu.y;
                            vo.c[0] = tv.x; vo.c[1] = tv.y;
                        } else
#pragma unroll
                        for (int q = 0; q < NC; ++q) {
                            if (!ADJ) {
                                uo.c[q] = uc.c[q] + (a1 * vc.c[q] + (a2 * duc.c[q] + (a3 * dvc.c[q] + a4 * d2u.c[q])));
                                vo.c[q] = vc.c[q] + (b2 * duc.c[q] + (b3 * dvc.c[q] + (b4 * d2u.c[q] + b5 * d2v.c[q])));
                            } else {
                                uo.c[q] = uc.c[q] + (a2 * duc.c[q] + (a3 * dvc.c[q] + (a4 * d2u.c[q] + a5 * d2v.c[q])));
                                vo.c[q] = vc.c[q] + (b1 * uc.c[q] + (b2 * duc.c[q] + (b3 * dvc.c[q] + b5 * d2v.c[q])));
                            }
                        }
                        const int64_t z = z0 + p - 4;
                        const bool inner = row_inner && z >= G && z < g.T[2] - G;
                        const int64_t off = obase + z * g.PS;
                        if (full_vec && inner) {
                            stN(Uo + off, uo);
                            stN(Vo + off, vo);
                        } else if (out_lane && inner) {   // a strip's end: plain stores of its columns in the run
#pragma unroll
                            for (int q = 0; q < NC; ++q)
                                if (x0 + q >= a.xr.lo && x0 + q <= a.xr.hi) {
                                    Uo[off + q] = uo.c[q];
                                    Vo[off + q] = vo.c[q];
                                }
                        } else if (out_lane) {
#pragma unroll
                            for (int q = 0; q < NC; ++q) {
                                const int64_t x = x0 + q;
                                if (x >= a.xr.lo && x <= a.xr.hi) {
                                    store_wrapped(Uo, g, x, y, z, uo.c[q]);
                                    store_wrapped(Vo, g, x, y, z, vo.c[q]);
                                }
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (!ok) {   // let the copies in flight (planes pfail .. pfail + S - 2 at most) land
            if (tid == 0)
                for (int q = pfail; q < n_in && q < pfail + S; ++q)
                    mbar_wait(&bars[(use + q) % S], ((use + q) / S) & 1u, nullptr, 0, kDrainLimitNs);
            return;
        }
        use += n_in;
    }
    // When this launch overlapped the layer kernels, finish only after them.
    wait_prerequisite_grid();
}

}  // namespace pml

#include "interior3d_rows.cuh"

namespace pml {

int interior3d_tile_y(int prec) { return prec == 32 ? I3Rf::TY : kBY3; }

template <bool ADJ> static cudaError_t prep_interior3d_rows()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_interior3d_rows<ADJ, kI3R, kI3W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(I3Rf::SMEM));
    if (e == cudaSuccess) done = true;
    return e;
}

template <bool ADJ> static int occ_interior3d_rows()
{
    if (prep_interior3d_rows<ADJ>() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_interior3d_rows<ADJ, kI3R, kI3W>, 32 * kI3W, I3Rf::SMEM) !=
        cudaSuccess)
        return 0;
    return n;
}

template <typename T, bool ADJ> static cudaError_t prep_interior3d()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_interior3d<T, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(I3<T>::SMEM));
    if (e == cudaSuccess) done = true;
    return e;
}

template <typename T, bool ADJ> static int occ_interior3d()
{
    if (prep_interior3d<T, ADJ>() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_interior3d<T, ADJ>, 32 * (kBY3 + 4), I3<T>::SMEM) !=
        cudaSuccess)
        return 0;
    return n;
}

int interior3d_max_blocks_per_sm(int prec, bool adjoint)
{
    if (prec == 32) return adjoint ? occ_interior3d_rows<true>() : occ_interior3d_rows<false>();
    return adjoint ? occ_interior3d<double, true>() : occ_interior3d<double, false>();
}

cudaError_t launch_interior3d(int prec, bool adjoint, const CUtensorMap *tmU, const CUtensorMap *tmV,
                              void *Uo, void *Vo, const Interior3DArgs &a, int grid, bool overlap_previous,
                              cudaStream_t st)
{
    if (a.xr.lo > a.xr.hi || a.yr.lo > a.yr.hi || a.zr.lo > a.zr.hi || grid <= 0) return cudaSuccess;
    cudaError_t e;
    const int threads = 32 * (kBY3 + 4);
#define PML_LAUNCH(TT, AA)                                                                              \
    if ((e = prep_interior3d<TT, AA>()) != cudaSuccess) return e;                                       \
    return launch_pdl(k_interior3d<TT, AA>, grid, threads, I3<TT>::SMEM, st, overlap_previous, *tmU, *tmV, \
                      (TT *)Uo, (TT *)Vo, a);
    if (prec == 32) {
        Interior3DArgs b = a;
        const StepCoefT<float> &k = a.c.f;
        const float cf[11] = {k.a1, k.a2, k.a3, k.a4, k.a5, k.b1, k.b2, k.b3, k.b4, k.b5, -6.f};
        for (int i = 0; i < 11; ++i) b.pf[i] = make_float2(cf[i], cf[i]);
        if (adjoint) {
            if ((e = prep_interior3d_rows<true>()) != cudaSuccess) return e;
            return launch_pdl(k_interior3d_rows<true, kI3R, kI3W>, grid, 32 * kI3W, I3Rf::SMEM, st, overlap_previous,
                              *tmU, *tmV, (float *)Uo, (float *)Vo, b);
        }
        if ((e = prep_interior3d_rows<false>()) != cudaSuccess) return e;
        return launch_pdl(k_interior3d_rows<false, kI3R, kI3W>, grid, 32 * kI3W, I3Rf::SMEM, st, overlap_previous,
                          *tmU, *tmV, (float *)Uo, (float *)Vo, b);
    } else {
        if (adjoint) { PML_LAUNCH(double, true) } else { PML_LAUNCH(double, false) }
    }
#undef PML_LAUNCH
}

}  // namespace pml

#include "layer3d.cuh"
#include "slab3d.cuh"

namespace pml {

void slab3d_shape(int mask, int *rx, int *ry, int *hx, int *hy)
{
    switch (mask & 7) {
#define PML_SHAPE(M) \
    case M: *rx = Slab<M>::RX; *ry = Slab<M>::RY; *hx = Slab<M>::HX; *hy = Slab<M>::HY; break;
        PML_SHAPE(0) PML_SHAPE(1) PML_SHAPE(2) PML_SHAPE(3) PML_SHAPE(4) PML_SHAPE(5) PML_SHAPE(6)
        default: *rx = Slab<7>::RX; *ry = Slab<7>::RY; *hx = Slab<7>::HX; *hy = Slab<7>::HY; break;
#undef PML_SHAPE
    }
}

template <bool ADJ, bool WALL, int M> static void describe_one(std::string &out)
{
    cudaFuncAttributes fa{};
    const cudaError_t e = cudaFuncGetAttributes(&fa, k_slab3d<ADJ, M, WALL>);
    char buf[160];
    if (e != cudaSuccess) std::snprintf(buf, sizeof buf, "class %d: %s; ", M, cudaGetErrorString(e));
    else
        std::snprintf(buf, sizeof buf, "class %d: %d threads, %d regs, max block %d, smem %zu+%zu; ", M, Slab<M>::NT,
                      fa.numRegs, fa.maxThreadsPerBlock, size_t(fa.sharedSizeBytes), Slab<M>::SMEM);
    out += buf;
}
template <bool ADJ, bool WALL> static std::string describe_all()
{
    std::string s;
    describe_one<ADJ, WALL, 0>(s); describe_one<ADJ, WALL, 1>(s); describe_one<ADJ, WALL, 2>(s);
    describe_one<ADJ, WALL, 3>(s); describe_one<ADJ, WALL, 4>(s); describe_one<ADJ, WALL, 5>(s);
    describe_one<ADJ, WALL, 6>(s); describe_one<ADJ, WALL, 7>(s);
    return s;
}
std::string slab3d_describe_wall(bool adjoint);   // layer3d_wall.cu
std::string slab3d_describe(bool adjoint, bool wall)
{
    if (wall) return slab3d_describe_wall(adjoint);
    return adjoint ? describe_all<true, false>() : describe_all<false, false>();
}

cudaError_t launch_slab3d(bool adjoint, const CUtensorMap *tm, void *const *outp, const Layer3DArgs &a,
                          cudaStream_t st)
{
    if (a.g.wall) return launch_slab3d_wall(adjoint, tm, outp, a, st);   // layer3d_wall.cu
    return launch_slab3d_impl<false>(adjoint, tm, outp, a, st);
}

int layer3d_tile_x(int prec) { return prec == 32 ? kLayer3TXf : kLayer3TXd; }
int layer3d_tile_y(int prec) { return prec == 32 ? kLayer3TYf : kLayer3TYd; }

cudaError_t launch_layer3d(int prec, bool adjoint, const CUtensorMap *tm, void *const *outp, const Layer3DArgs &a,
                           cudaStream_t st)
{
    if (a.g.wall) return launch_layer3d_wall(prec, adjoint, tm, outp, a, st);   // layer3d_wall.cu
    return launch_layer3d_impl<false>(prec, adjoint, tm, outp, a, st);
}

}  // namespace pml
