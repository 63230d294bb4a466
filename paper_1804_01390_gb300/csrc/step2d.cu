// 2D kernels of one RK4 step of the discrete PML system (eq:DiscretePML, Sec. 1.1.2) on
// sm_103a.
//
// One RK4 step of a linear autonomous system is the Taylor polynomial
//   y' = P(dt A) y,  P(z) = 1 + z + z^2/2 + z^3/6 + z^4/24
// (classic RK4 with b = (1/6, 1/3, 1/3, 1/6), c = (0, 1/2, 1/2, 1), Sec. 1.1.3).
// Two kernels evaluate it in one pass over HBM:
//
//  * k_interior2d: vertices whose step never sees a damping term.  There
//    A = [[0, I], [L, 0]] and P(dt A) expands to U, V, DU, DV, D^2U, D^2V with D the
//    unscaled 5-point difference (coefficients in StepCoef).  Each warp streams a
//    128-column strip (32 lanes x 4 columns; lanes 0 and 31 are halo lanes) down the
//    rows: TMA brings 6-row boxes of U and V into a shared-memory ring, each lane keeps
//    three rows of U, V, DU, DV in registers, and x neighbours come from warp
//    shuffles.  HBM traffic is one read and one write of U and V per vertex.
//
//  * k_layer2d: tiles of the layer frame.  The polynomial is evaluated in Horner form
//    y' = y + dt A (y + dt/2 A (y + dt/3 A (y + dt/4 A y)))
//    with the full operator (Laplacian + damping terms + Phi/Psi recurrences), four
//    applications of A on a shrinking shared-memory region (halo 4).
#include "common.cuh"

namespace pml {

constexpr int kRows2D = 6;   // rows per TMA box; multiple of 3 (register ring period)
constexpr int kStrip = 120;  // output columns per warp strip (lanes 1..30)

template <typename T> struct Stages2D {
    static constexpr int S = sizeof(T) == 4 ? 3 : 2;
};

int interior2d_box_rows(int) { return kRows2D; }

// Unscaled 5-point difference of one lane's 4 columns: c is the centre row, up/dn the
// rows above/below; x neighbours across lanes by shuffles.
template <typename T>
__device__ __forceinline__ V4<T> diff5(const V4<T> &c, const V4<T> &up, const V4<T> &dn)
{
    const T l = __shfl_up_sync(0xffffffffu, c.w, 1);
    const T r = __shfl_down_sync(0xffffffffu, c.x, 1);
    V4<T> o;
    o.x = ((l + c.y) + (up.x + dn.x)) - T(4) * c.x;
    o.y = ((c.x + c.z) + (up.y + dn.y)) - T(4) * c.y;
    o.z = ((c.y + c.w) + (up.z + dn.z)) - T(4) * c.z;
    o.w = ((c.z + r) + (up.w + dn.w)) - T(4) * c.w;
    return o;
}

template <typename T, bool ADJ>
__global__ void __launch_bounds__(128)
    k_interior2d(const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmV,
                 T *__restrict__ Uo, T *__restrict__ Vo, const Interior2DArgs a)
{
    constexpr int CH = kRows2D;
    constexpr int S = Stages2D<T>::S;
    constexpr int ROW = 128;
    constexpr uint32_t FIELD_BYTES = CH * ROW * sizeof(T);
    constexpr uint32_t STAGE_BYTES = 2 * FIELD_BYTES;
    __shared__ __align__(8) uint64_t bars[4][S];
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_dyn) + 127) & ~uintptr_t(127));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wbase = smem + warp * S * STAGE_BYTES;
    if (lane == 0) {
        prefetch_tmap(&tmU);
        prefetch_tmap(&tmV);
        for (int s = 0; s < S; ++s) mbar_init(&bars[warp][s], 1);
        fence_mbar_init();
    }
    __syncwarp();

    const Geom &g = a.g;
    const int64_t xs0 = a.xr.lo & ~int64_t(3);
    const int64_t nstrips = (a.xr.hi - xs0) / kStrip + 1;
    const int64_t nrows = a.yr.hi - a.yr.lo + 1;
    const int64_t total = nstrips * nrows;
    const int64_t nw = int64_t(gridDim.x) * 4, gw = int64_t(blockIdx.x) * 4 + warp;
    int64_t cur = total * gw / nw;
    const int64_t end = total * (gw + 1) / nw;

    const T a1 = T(a.c.a1), a2 = T(a.c.a2), a3 = T(a.c.a3), a4 = T(a.c.a4), a5 = T(a.c.a5);
    const T b1 = T(a.c.b1), b2 = T(a.c.b2), b3 = T(a.c.b3), b4 = T(a.c.b4), b5 = T(a.c.b5);
    uint32_t use = 0;

    while (cur < end) {
        const int64_t s = cur / nrows, r0 = cur - s * nrows;
        const int64_t cnt = (nrows - r0) < (end - cur) ? (nrows - r0) : (end - cur);
        const int64_t y0 = a.yr.lo + r0;
        const int64_t xs = xs0 + kStrip * s;
        const int n_in = int(cnt) + 4;
        const int nch = (n_in + CH - 1) / CH;
        const int32_t tx = int32_t(xs - 4 + G);
        const int32_t ty = int32_t(y0 - 2 + G);

        if (lane == 0) {
            fence_proxy_async();   // earlier generic reads of the ring before async writes
            const int npro = nch < S ? nch : S;
            for (int c = 0; c < npro; ++c) {
                const int slot = (use + c) % S;
                unsigned char *dst = wbase + slot * STAGE_BYTES;
                mbar_arrive_expect_tx(&bars[warp][slot], STAGE_BYTES);
                tma_load_2d(dst, &tmU, tx, ty + c * CH, &bars[warp][slot]);
                tma_load_2d(dst + FIELD_BYTES, &tmV, tx, ty + c * CH, &bars[warp][slot]);
            }
        }

        const int64_t x0 = xs - 4 + 4 * lane;
        const bool out_lane = lane >= 1 && lane <= 30;
        const bool full_vec = out_lane && x0 >= a.xr.lo && x0 + 3 <= a.xr.hi && x0 >= G &&
                              x0 + 3 < g.T[0] - G;
        V4<T> u[3], v[3], du[3], dv[3];

        for (int c = 0; c < nch; ++c) {
            const uint32_t uu = use + c;
            const int slot = uu % S;
            if (!mbar_wait(&bars[warp][slot], (uu / S) & 1u, a.err, 1)) {
                // give the copies still in flight a bounded chance to land, then stop
                for (int c2 = c + 1; c2 < nch && c2 < c + S; ++c2)
                    mbar_wait(&bars[warp][(use + c2) % S], ((use + c2) / S) & 1u, nullptr, 0);
                return;
            }
            const T *sU = reinterpret_cast<const T *>(wbase + slot * STAGE_BYTES) + 4 * lane;
            const T *sV = sU + CH * ROW;
#pragma unroll
            for (int j = 0; j < CH; ++j) {
                const int q = c * CH + j;
                if (q < n_in) {
                    const int J0 = j % 3, J1 = (j + 2) % 3, J2 = (j + 1) % 3;  // rows q, q-1, q-2
                    u[J0] = lds4(sU + j * ROW);
                    v[J0] = lds4(sV + j * ROW);
                    if (q >= 2) {
                        du[J1] = diff5(u[J1], u[J2], u[J0]);
                        dv[J1] = diff5(v[J1], v[J2], v[J0]);
                    }
                    if (q >= 4) {
                        // second differences at row q-2 from DU rows q-3 (slot J0), q-2, q-1
                        const V4<T> d2u = diff5(du[J2], du[J0], du[J1]);
                        const V4<T> d2v = diff5(dv[J2], dv[J0], dv[J1]);
                        const V4<T> &uc = u[J2], &vc = v[J2], &duc = du[J2], &dvc = dv[J2];
                        V4<T> uo, vo;
#define PML_OUT(k)                                                                            \
    if (!ADJ) {                                                                               \
        uo.k = uc.k + (a1 * vc.k + (a2 * duc.k + (a3 * dvc.k + a4 * d2u.k)));                \
        vo.k = vc.k + (b2 * duc.k + (b3 * dvc.k + (b4 * d2u.k + b5 * d2v.k)));               \
    } else {                                                                                  \
        uo.k = uc.k + (a2 * duc.k + (a3 * dvc.k + (a4 * d2u.k + a5 * d2v.k)));               \
        vo.k = vc.k + (b1 * uc.k + (b2 * duc.k + (b3 * dvc.k + b5 * d2v.k)));                \
    }
                        PML_OUT(x) PML_OUT(y) PML_OUT(z) PML_OUT(w)
#undef PML_OUT
                        const int64_t r = y0 + q - 4;
                        if (full_vec && r >= G && r < g.T[1] - G) {
                            const int64_t off = g.origin + r * g.P + x0;
                            stg4(Uo + off, uo);
                            stg4(Vo + off, vo);
                        } else if (out_lane) {
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const int64_t x = x0 + k;
                                if (x >= a.xr.lo && x <= a.xr.hi) {
                                    store_wrapped(Uo, g, x, r, 0, get4(uo, k));
                                    store_wrapped(Vo, g, x, r, 0, get4(vo, k));
                                }
                            }
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0 && c + S < nch) {
                fence_proxy_async();
                const int slot2 = (use + c + S) % S;
                unsigned char *dst = wbase + slot2 * STAGE_BYTES;
                mbar_arrive_expect_tx(&bars[warp][slot2], STAGE_BYTES);
                tma_load_2d(dst, &tmU, tx, ty + (c + S) * CH, &bars[warp][slot2]);
                tma_load_2d(dst + FIELD_BYTES, &tmV, tx, ty + (c + S) * CH, &bars[warp][slot2]);
            }
        }
        use += nch;
        cur += cnt;
    }
}

template <typename T> static size_t interior2d_smem()
{
    return size_t(4) * Stages2D<T>::S * 2 * kRows2D * 128 * sizeof(T) + 128;
}

template <typename T, bool ADJ> static cudaError_t prep_interior2d()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_interior2d<T, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(interior2d_smem<T>()));
    if (e == cudaSuccess) done = true;
    return e;
}

int interior2d_max_blocks_per_sm(int prec, bool adjoint)
{
    int n = 0;
    cudaError_t e;
    if (prec == 32) {
        if (adjoint) {
            prep_interior2d<float, true>();
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_interior2d<float, true>, 128, interior2d_smem<float>());
        } else {
            prep_interior2d<float, false>();
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_interior2d<float, false>, 128, interior2d_smem<float>());
        }
    } else {
        if (adjoint) {
            prep_interior2d<double, true>();
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_interior2d<double, true>, 128, interior2d_smem<double>());
        } else {
            prep_interior2d<double, false>();
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_interior2d<double, false>, 128, interior2d_smem<double>());
        }
    }
    return e == cudaSuccess ? n : 0;
}

cudaError_t launch_interior2d(int prec, bool adjoint, const CUtensorMap *tmU, const CUtensorMap *tmV,
                              void *Uo, void *Vo, const Interior2DArgs &a, int grid, cudaStream_t st)
{
    if (a.xr.lo > a.xr.hi || a.yr.lo > a.yr.hi || grid <= 0) return cudaSuccess;
    cudaError_t e;
    if (prec == 32) {
        if (adjoint) {
            if ((e = prep_interior2d<float, true>()) != cudaSuccess) return e;
            k_interior2d<float, true><<<grid, 128, interior2d_smem<float>(), st>>>(*tmU, *tmV, (float *)Uo, (float *)Vo, a);
        } else {
            if ((e = prep_interior2d<float, false>()) != cudaSuccess) return e;
            k_interior2d<float, false><<<grid, 128, interior2d_smem<float>(), st>>>(*tmU, *tmV, (float *)Uo, (float *)Vo, a);
        }
    } else {
        if (adjoint) {
            if ((e = prep_interior2d<double, true>()) != cudaSuccess) return e;
            k_interior2d<double, true><<<grid, 128, interior2d_smem<double>(), st>>>(*tmU, *tmV, (double *)Uo, (double *)Vo, a);
        } else {
            if ((e = prep_interior2d<double, false>()) != cudaSuccess) return e;
            k_interior2d<double, false><<<grid, 128, interior2d_smem<double>(), st>>>(*tmU, *tmV, (double *)Uo, (double *)Vo, a);
        }
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Layer frame: Horner form with the full operator of Eq. 3 (or its transpose), streamed
// down the rows by independent warps.
//
// A warp owns 32 consecutive columns (lane = column; lanes 4..27 are its kL2W outputs,
// lanes 0..3 and 28..31 the halo of the four applications of A) and a run of rows of one
// frame rectangle.  When input row p arrives, level 4 (z4 = y + dt/4 A y) produces row
// p-1, level 3 row p-2, level 2 row p-3 and level 1 (y' = y + dt A z2) the output row
// p-4.  Row neighbours of each level come from three-row register rings, column
// neighbours from shuffles, the base y of every level from the warp's TMA ring; no block
// barrier is needed.  Templated on the axes whose aux fields are active in the strip.
// ------------------------------------------------------------------------------------

constexpr int kL2CH = 6;     // rows per TMA box (multiple of 3: the register ring period)
constexpr int kL2S = 4;      // TMA stages per warp

template <int MASK> struct Fields2 {
    static constexpr int NAX = ((MASK >> 0) & 1) + ((MASK >> 1) & 1);
    static constexpr int NF = 2 + 2 * NAX;
    static __device__ __forceinline__ constexpr int axis(int k)
    {
        return (MASK & 1) ? k : 1;   // k-th active axis
    }
    static __device__ __forceinline__ constexpr int gid(int f)
    {
        return f < 2 ? f : 2 + 2 * axis((f - 2) >> 1) + ((f - 2) & 1);
    }
};

template <typename T> struct Sig2 {
    T si[2], sm[2];   // sigma_a[i_a], sigma_a[i_a - 1]
};

// A z (or A^T z) at one vertex; N(f, d): d = 0 centre, 1 x-, 2 x+, 3 y-, 4 y+.
template <typename T, bool ADJ, int MASK, typename Get>
__device__ __forceinline__ void apply_A2(const Get &N, const Sig2<T> &s, T ih, T ih2, T i2h, T *o)
{
    using F = Fields2<MASK>;
    const T half = T(0.5);
    if (!ADJ) {
        const T U0 = N(0, 0);
        const T lap = ((N(0, 2) + N(0, 1)) - T(2) * U0) + ((N(0, 4) + N(0, 3)) - T(2) * U0);
        T aV = lap * ih2;
        o[0] = N(1, 0);
#pragma unroll
        for (int k = 0; k < F::NAX; ++k) {
            const int ax = F::axis(k), fp = 2 + 2 * k, fq = 3 + 2 * k, dm = 1 + 2 * ax, dp = 2 + 2 * ax;
            const T si = s.si[ax], sm = s.sm[ax];
            aV += (si * N(fq, dp) - sm * N(fp, dm)) * ih;
            const T dU = (N(0, dp) - N(0, dm)) * i2h;
            o[fp] = si != T(0) ? -half * (sm * N(fp, dm) + si * N(fp, 0)) - dU : T(0);
            o[fq] = sm != T(0) ? -half * (sm * N(fq, 0) + si * N(fq, dp)) - dU : T(0);
        }
        o[1] = aV;
    } else {
        const T V0 = N(1, 0);
        const T lap = ((N(1, 2) + N(1, 1)) - T(2) * V0) + ((N(1, 4) + N(1, 3)) - T(2) * V0);
        T aU = lap * ih2;
        o[1] = N(0, 0);
#pragma unroll
        for (int k = 0; k < F::NAX; ++k) {
            const int ax = F::axis(k), fp = 2 + 2 * k, fq = 3 + 2 * k, dm = 1 + 2 * ax, dp = 2 + 2 * ax;
            const T si = s.si[ax], sm = s.sm[ax];
            aU += ((N(fp, dp) - N(fp, dm)) + (N(fq, dp) - N(fq, dm))) * i2h;
            o[fp] = si != T(0) ? -si * N(1, dp) * ih - half * si * (N(fp, dp) + N(fp, 0)) : T(0);
            o[fq] = sm != T(0) ? sm * N(1, dm) * ih - half * sm * (N(fq, 0) + N(fq, dm)) : T(0);
        }
        o[0] = aU;
    }
}

struct Maps6 {
    CUtensorMap m[6];
};
struct Out6 {
    void *p[6];
};

template <typename T, int MASK>
__device__ __forceinline__ void issue_chunk2(T *dst, const Maps6 &maps, int32_t x, int32_t y, uint64_t *bar)
{
    using F = Fields2<MASK>;
    constexpr int FE = kL2CH * 32;
    mbar_arrive_expect_tx(bar, uint32_t(F::NF * FE * sizeof(T)));
#pragma unroll
    for (int f = 0; f < F::NF; ++f) tma_load_2d(dst + f * FE, &maps.m[F::gid(f)], x, y, bar);
}

template <typename T, bool ADJ, int MASK>
__global__ void __launch_bounds__(128)
    k_layer2d(const __grid_constant__ Maps6 maps, const Out6 out, const Layer2DArgs a, int base, int count)
{
    using F = Fields2<MASK>;
    constexpr int NF = F::NF, CH = kL2CH, S = kL2S, FE = CH * 32, SE = NF * FE;
    __shared__ __align__(8) uint64_t bars[4][S];
    extern __shared__ unsigned char smem_dyn[];
    T *smem = reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(smem_dyn) + 127) & ~uintptr_t(127));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = blockIdx.x * 4 + warp;
    if (item >= count) return;   // whole warp; the kernel has no block barrier
    T *ring = smem + warp * S * SE;
    const LayerTile tile = a.tiles[base + item];
    const Geom &g = a.g;
    const int nout = tile.yhi - tile.ylo + 1, nin = nout + 8;
    const int nch = (nin + CH - 1) / CH;
    const int32_t tx = tile.x0 - 4 + G, ty = tile.ylo - 4 + G;
    if (lane == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[warp][s], 1);
        fence_mbar_init();
        const int npro = nch < S ? nch : S;
        for (int c = 0; c < npro; ++c) issue_chunk2<T, MASK>(ring + c * SE, maps, tx, ty + c * CH, &bars[warp][c]);
    }
    __syncwarp();

    const T *sgx = static_cast<const T *>(a.sig[0]);
    const T *sgy = static_cast<const T *>(a.sig[1]);
    const int64_t gx = int64_t(tile.x0) - 4 + lane;
    Sig2<T> sg;
    {
        const int64_t xi = ((gx % g.T[0]) + g.T[0]) % g.T[0];
        sg.si[0] = sgx[xi];
        sg.sm[0] = sgx[xi == 0 ? g.T[0] - 1 : xi - 1];
    }
    auto ysig = [&](int q) {
        int64_t yi = (int64_t(tile.ylo) - 4 + q) % g.T[1];
        if (yi < 0) yi += g.T[1];
        sg.si[1] = sgy[yi];
        sg.sm[1] = sgy[yi == 0 ? g.T[1] - 1 : yi - 1];
    };
    const bool out_lane = lane >= 4 && lane <= 27 && gx >= tile.xlo && gx <= tile.xhi;
    const T ih = T(1.0 / a.h), ih2 = T(1.0 / (a.h * a.h)), i2h = T(0.5 / a.h);
    const T c4 = T(a.dt / 4.0), c3 = T(a.dt / 3.0), c2 = T(a.dt / 2.0), c1 = T(a.dt);
    T z4[3][NF], z3[3][NF], z2[3][NF];

    for (int c = 0; c < nch; ++c) {
        if (!mbar_wait(&bars[warp][c % S], (c / S) & 1, a.err, 2)) {
            for (int c2 = c + 1; c2 < nch && c2 < c + S; ++c2) mbar_wait(&bars[warp][c2 % S], (c2 / S) & 1, nullptr, 0);
            return;
        }
        const T *cur = ring + (c % S) * SE + lane;
        const T *prv = ring + ((c + S - 1) % S) * SE + lane;
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const int p = c * CH + j;
            if (p < nin) {
                const int PH = j % 3;
                // own-column value of input row p - k, field f (rows of this or the previous chunk)
                auto Y = [&](int k, int f) -> T {
                    const int r = j - k;
                    return r >= 0 ? cur[f * FE + r * 32] : prv[f * FE + (r + CH) * 32];
                };
                if (p >= 2) {   // level 4 at row p-1
                    T cen[NF], xm[NF], xp[NF];
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        cen[f] = Y(1, f);
                        xm[f] = __shfl_up_sync(0xffffffffu, cen[f], 1);
                        xp[f] = __shfl_down_sync(0xffffffffu, cen[f], 1);
                    }
                    auto N = [&](int f, int d) -> T {
                        switch (d) {
                        case 0: return cen[f];
                        case 1: return xm[f];
                        case 2: return xp[f];
                        case 3: return Y(2, f);
                        default: return Y(0, f);
                        }
                    };
                    ysig(p - 1);
                    T r[NF];
                    apply_A2<T, ADJ, MASK>(N, sg, ih, ih2, i2h, r);
#pragma unroll
                    for (int f = 0; f < NF; ++f) z4[(PH + 2) % 3][f] = cen[f] + c4 * r[f];
                }
                if (p >= 4) {   // level 3 at row p-2
                    T xm[NF], xp[NF];
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        xm[f] = __shfl_up_sync(0xffffffffu, z4[(PH + 1) % 3][f], 1);
                        xp[f] = __shfl_down_sync(0xffffffffu, z4[(PH + 1) % 3][f], 1);
                    }
                    auto N = [&](int f, int d) -> T {
                        switch (d) {
                        case 0: return z4[(PH + 1) % 3][f];
                        case 1: return xm[f];
                        case 2: return xp[f];
                        case 3: return z4[PH][f];
                        default: return z4[(PH + 2) % 3][f];
                        }
                    };
                    ysig(p - 2);
                    T r[NF];
                    apply_A2<T, ADJ, MASK>(N, sg, ih, ih2, i2h, r);
#pragma unroll
                    for (int f = 0; f < NF; ++f) z3[(PH + 1) % 3][f] = Y(2, f) + c3 * r[f];
                }
                if (p >= 6) {   // level 2 at row p-3
                    T xm[NF], xp[NF];
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        xm[f] = __shfl_up_sync(0xffffffffu, z3[PH][f], 1);
                        xp[f] = __shfl_down_sync(0xffffffffu, z3[PH][f], 1);
                    }
                    auto N = [&](int f, int d) -> T {
                        switch (d) {
                        case 0: return z3[PH][f];
                        case 1: return xm[f];
                        case 2: return xp[f];
                        case 3: return z3[(PH + 2) % 3][f];
                        default: return z3[(PH + 1) % 3][f];
                        }
                    };
                    ysig(p - 3);
                    T r[NF];
                    apply_A2<T, ADJ, MASK>(N, sg, ih, ih2, i2h, r);
#pragma unroll
                    for (int f = 0; f < NF; ++f) z2[PH][f] = Y(3, f) + c2 * r[f];
                }
                if (p >= 8) {   // level 1: output row p-4
                    T xm[NF], xp[NF];
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        xm[f] = __shfl_up_sync(0xffffffffu, z2[(PH + 2) % 3][f], 1);
                        xp[f] = __shfl_down_sync(0xffffffffu, z2[(PH + 2) % 3][f], 1);
                    }
                    auto N = [&](int f, int d) -> T {
                        switch (d) {
                        case 0: return z2[(PH + 2) % 3][f];
                        case 1: return xm[f];
                        case 2: return xp[f];
                        case 3: return z2[(PH + 1) % 3][f];
                        default: return z2[PH][f];
                        }
                    };
                    ysig(p - 4);
                    T r[NF];
                    apply_A2<T, ADJ, MASK>(N, sg, ih, ih2, i2h, r);
                    if (out_lane) {
                        const int64_t y = int64_t(tile.ylo) + p - 8;
                        const bool edge = near_edge(g, gx, y, 0);
#pragma unroll
                        for (int f = 0; f < NF; ++f) {
                            const T val = Y(4, f) + c1 * r[f];
                            T *dst = static_cast<T *>(out.p[F::gid(f)]);
                            if (edge) store_wrapped(dst, g, gx, y, 0, val);
                            else dst[g.origin + gx + y * g.P] = val;
                        }
                    }
                }
            }
        }
        __syncwarp();
        // chunk c-1 is no longer needed (rows >= c*CH - 4 remain in use): refill it
        if (lane == 0 && c >= 1 && c - 1 + S < nch) {
            fence_proxy_async();
            const int st = (c - 1) % S;
            issue_chunk2<T, MASK>(ring + st * SE, maps, tx, ty + (c - 1 + S) * CH, &bars[warp][st]);
        }
    }
}

template <typename T, int MASK> static size_t layer2d_smem()
{
    return size_t(4) * kL2S * Fields2<MASK>::NF * kL2CH * 32 * sizeof(T) + 128;
}

template <typename T, bool ADJ, int MASK>
static cudaError_t launch_l2(const Maps6 &m, const Out6 &o, const Layer2DArgs &a, cudaStream_t st)
{
    const int n = a.class_off[MASK + 1] - a.class_off[MASK];
    if (n <= 0) return cudaSuccess;
    static bool done = false;
    const size_t sm = layer2d_smem<T, MASK>();
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(k_layer2d<T, ADJ, MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        if (e != cudaSuccess) return e;
        done = true;
    }
    k_layer2d<T, ADJ, MASK><<<(n + 3) / 4, 128, sm, st>>>(m, o, a, a.class_off[MASK], n);
    return cudaGetLastError();
}

template <typename T, bool ADJ>
static cudaError_t launch_l2_all(const Maps6 &m, const Out6 &o, const Layer2DArgs &a, cudaStream_t st)
{
    cudaError_t e;
    if ((e = launch_l2<T, ADJ, 0>(m, o, a, st)) != cudaSuccess) return e;
    if ((e = launch_l2<T, ADJ, 1>(m, o, a, st)) != cudaSuccess) return e;
    if ((e = launch_l2<T, ADJ, 2>(m, o, a, st)) != cudaSuccess) return e;
    return launch_l2<T, ADJ, 3>(m, o, a, st);
}

cudaError_t launch_layer2d(int prec, bool adjoint, const CUtensorMap *tm, void *const *outp,
                           const Layer2DArgs &a, cudaStream_t st)
{
    if (a.ntiles <= 0) return cudaSuccess;
    Maps6 m;
    Out6 o;
    for (int f = 0; f < 6; ++f) {
        m.m[f] = tm[f];
        o.p[f] = outp[f];
    }
    if (prec == 32) return adjoint ? launch_l2_all<float, true>(m, o, a, st) : launch_l2_all<float, false>(m, o, a, st);
    return adjoint ? launch_l2_all<double, true>(m, o, a, st) : launch_l2_all<double, false>(m, o, a, st);
}

}  // namespace pml
