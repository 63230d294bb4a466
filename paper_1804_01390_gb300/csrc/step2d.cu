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
// Layer frame: Horner form with the full operator of Eq. 3 (or its transpose).
// ------------------------------------------------------------------------------------

constexpr int kLR = kLayerTH + 8;   // region rows (halo 4 = one per application of A)
constexpr int kLC = kLayerTW + 8;   // region columns
constexpr int kLN = kLR * kLC;
constexpr int kLThreads = 256;
constexpr int kLPts = (kLN + kLThreads - 1) / kLThreads;

struct Out6 {
    void *p[6];
};

// Field order in shared memory and in the tensor maps: U, V, Phi_x, Psi_x, Phi_y, Psi_y.
template <typename T, bool ADJ>
__device__ __forceinline__ void apply_A2(const T *__restrict__ Z, const T *sx, const T *sy, int r,
                                         int c, bool ax, bool ay, T ih, T ih2, T i2h, T o[6])
{
#define F(f, rr, cc) Z[(f) * kLN + (rr) * kLC + (cc)]
    const T half = T(0.5);
    if (!ADJ) {
        const T zU = F(0, r, c);
        const T lap = ((F(0, r, c + 1) + F(0, r, c - 1)) - T(2) * zU) +
                      ((F(0, r + 1, c) + F(0, r - 1, c)) - T(2) * zU);
        T aV = lap * ih2;
        o[0] = F(1, r, c);
        if (ax) {
            const T si = sx[c + 1], sm = sx[c];
            aV += (si * F(3, r, c + 1) - sm * F(2, r, c - 1)) * ih;
            const T dU = (F(0, r, c + 1) - F(0, r, c - 1)) * i2h;
            o[2] = si != T(0) ? -half * (sm * F(2, r, c - 1) + si * F(2, r, c)) - dU : T(0);
            o[3] = sm != T(0) ? -half * (sm * F(3, r, c) + si * F(3, r, c + 1)) - dU : T(0);
        }
        if (ay) {
            const T si = sy[r + 1], sm = sy[r];
            aV += (si * F(5, r + 1, c) - sm * F(4, r - 1, c)) * ih;
            const T dU = (F(0, r + 1, c) - F(0, r - 1, c)) * i2h;
            o[4] = si != T(0) ? -half * (sm * F(4, r - 1, c) + si * F(4, r, c)) - dU : T(0);
            o[5] = sm != T(0) ? -half * (sm * F(5, r, c) + si * F(5, r + 1, c)) - dU : T(0);
        }
        o[1] = aV;
    } else {
        // transpose of the operator above (entries collected column by column)
        const T zV = F(1, r, c);
        const T lap = ((F(1, r, c + 1) + F(1, r, c - 1)) - T(2) * zV) +
                      ((F(1, r + 1, c) + F(1, r - 1, c)) - T(2) * zV);
        T aU = lap * ih2;
        o[1] = F(0, r, c);
        if (ax) {
            const T si = sx[c + 1], sm = sx[c];
            aU += ((F(2, r, c + 1) - F(2, r, c - 1)) + (F(3, r, c + 1) - F(3, r, c - 1))) * i2h;
            o[2] = si != T(0) ? -si * F(1, r, c + 1) * ih - half * si * (F(2, r, c + 1) + F(2, r, c)) : T(0);
            o[3] = sm != T(0) ? sm * F(1, r, c - 1) * ih - half * sm * (F(3, r, c) + F(3, r, c - 1)) : T(0);
        }
        if (ay) {
            const T si = sy[r + 1], sm = sy[r];
            aU += ((F(4, r + 1, c) - F(4, r - 1, c)) + (F(5, r + 1, c) - F(5, r - 1, c))) * i2h;
            o[4] = si != T(0) ? -si * F(1, r + 1, c) * ih - half * si * (F(4, r + 1, c) + F(4, r, c)) : T(0);
            o[5] = sm != T(0) ? sm * F(1, r - 1, c) * ih - half * sm * (F(5, r, c) + F(5, r - 1, c)) : T(0);
        }
        o[0] = aU;
    }
#undef F
}

template <typename T, bool ADJ>
__global__ void __launch_bounds__(kLThreads)
    k_layer2d(const __grid_constant__ CUtensorMap t0, const __grid_constant__ CUtensorMap t1,
              const __grid_constant__ CUtensorMap t2, const __grid_constant__ CUtensorMap t3,
              const __grid_constant__ CUtensorMap t4, const __grid_constant__ CUtensorMap t5, const Out6 out,
              const Layer2DArgs a)
{
    extern __shared__ unsigned char smem_dyn[];
    T *Y = reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(smem_dyn) + 127) & ~uintptr_t(127));
    T *Z = Y + 6 * kLN;
    __shared__ T sx[kLC + 1], sy[kLR + 1];
    __shared__ __align__(8) uint64_t bar;

    const LayerTile tile = a.tiles[blockIdx.x];
    const bool ax = tile.flags & 1, ay = tile.flags & 2;
    const Geom &g = a.g;
    const int tid = threadIdx.x;

    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        constexpr uint32_t FB = kLN * sizeof(T);
        const uint32_t bytes = FB * (2 + (ax ? 2 : 0) + (ay ? 2 : 0));
        mbar_arrive_expect_tx(&bar, bytes);
        const int32_t x = tile.x0 - 4 + G, y = tile.y0 - 4 + G;
        tma_load_2d(Y + 0 * kLN, &t0, x, y, &bar);
        tma_load_2d(Y + 1 * kLN, &t1, x, y, &bar);
        if (ax) {
            tma_load_2d(Y + 2 * kLN, &t2, x, y, &bar);
            tma_load_2d(Y + 3 * kLN, &t3, x, y, &bar);
        }
        if (ay) {
            tma_load_2d(Y + 4 * kLN, &t4, x, y, &bar);
            tma_load_2d(Y + 5 * kLN, &t5, x, y, &bar);
        }
    }
    // damping of the edges to the left of / below each region vertex and of the vertex
    const T *sgx = static_cast<const T *>(a.sig[0]);
    const T *sgy = static_cast<const T *>(a.sig[1]);
    for (int k = tid; k <= kLC; k += kLThreads) {
        int64_t i = (int64_t(tile.x0) - 5 + k) % g.T[0];
        if (i < 0) i += g.T[0];
        sx[k] = sgx[i];
    }
    for (int k = tid; k <= kLR; k += kLThreads) {
        int64_t i = (int64_t(tile.y0) - 5 + k) % g.T[1];
        if (i < 0) i += g.T[1];
        sy[k] = sgy[i];
    }
    __syncthreads();
    if (!__syncthreads_and(mbar_wait(&bar, 0, a.err, 2))) return;

    const T ih = T(1.0 / a.h), ih2 = T(1.0 / (a.h * a.h)), i2h = T(0.5 / a.h);
    const T cl[4] = {T(a.dt / 4.0), T(a.dt / 3.0), T(a.dt / 2.0), T(a.dt)};
    const int nfl = 2;
#pragma unroll 1
    for (int L = 0; L < 4; ++L) {
        const int rad = 3 - L;
        const int rlo = 4 - rad, clo = 4 - rad;
        const int nr = kLayerTH + 2 * rad, nc = kLayerTW + 2 * rad, np = nr * nc;
        const T *src = L == 0 ? Y : Z;
        T res[kLPts][6];
#pragma unroll
        for (int k = 0; k < kLPts; ++k) {
            const int p = tid + k * kLThreads;
            if (p < np) {
                const int r = rlo + p / nc, c = clo + p % nc;
                apply_A2<T, ADJ>(src, sx, sy, r, c, ax, ay, ih, ih2, i2h, res[k]);
            }
        }
        __syncthreads();
        if (L < 3) {
            const T cL = cl[L];
#pragma unroll
            for (int k = 0; k < kLPts; ++k) {
                const int p = tid + k * kLThreads;
                if (p < np) {
                    const int o = (rlo + p / nc) * kLC + clo + p % nc;
                    for (int f = 0; f < nfl; ++f) Z[f * kLN + o] = Y[f * kLN + o] + cL * res[k][f];
                    if (ax)
                        for (int f = 2; f < 4; ++f) Z[f * kLN + o] = Y[f * kLN + o] + cL * res[k][f];
                    if (ay)
                        for (int f = 4; f < 6; ++f) Z[f * kLN + o] = Y[f * kLN + o] + cL * res[k][f];
                }
            }
            __syncthreads();
        } else {
            const T cL = cl[3];
#pragma unroll
            for (int k = 0; k < kLPts; ++k) {
                const int p = tid + k * kLThreads;
                if (p < np) {
                    const int rr = rlo + p / nc, cc = clo + p % nc;
                    const int64_t x = int64_t(tile.x0) + cc - 4, y = int64_t(tile.y0) + rr - 4;
                    if (x >= tile.xlo && x <= tile.xhi && y >= tile.ylo && y <= tile.yhi) {
                        const int o = rr * kLC + cc;
                        const bool edge = near_edge(g, x, y, 0);
                        for (int f = 0; f < 6; ++f) {
                            if ((f == 2 || f == 3) && !ax) continue;
                            if ((f == 4 || f == 5) && !ay) continue;
                            const T val = Y[f * kLN + o] + cL * res[k][f];
                            T *dst = static_cast<T *>(out.p[f]);
                            if (edge) store_wrapped(dst, g, x, y, 0, val);
                            else dst[g.origin + x + y * g.P] = val;
                        }
                    }
                }
            }
        }
    }
}

template <typename T> static size_t layer2d_smem() { return size_t(12) * kLN * sizeof(T) + 128; }

template <typename T, bool ADJ> static cudaError_t prep_layer2d()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_layer2d<T, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(layer2d_smem<T>()));
    if (e == cudaSuccess) done = true;
    return e;
}

cudaError_t launch_layer2d(int prec, bool adjoint, const CUtensorMap *tm, void *const *outp,
                           const Layer2DArgs &a, cudaStream_t st)
{
    if (a.ntiles <= 0) return cudaSuccess;
    Out6 o;
    for (int f = 0; f < 6; ++f) o.p[f] = outp[f];
    cudaError_t e;
#define PML_LAUNCH(TT, AA)                                                                           \
    if ((e = prep_layer2d<TT, AA>()) != cudaSuccess) return e;                                       \
    k_layer2d<TT, AA><<<a.ntiles, kLThreads, layer2d_smem<TT>(), st>>>(tm[0], tm[1], tm[2], tm[3], \
                                                                        tm[4], tm[5], o, a);
    if (prec == 32) {
        if (adjoint) { PML_LAUNCH(float, true) } else { PML_LAUNCH(float, false) }
    } else {
        if (adjoint) { PML_LAUNCH(double, true) } else { PML_LAUNCH(double, false) }
    }
#undef PML_LAUNCH
    return cudaGetLastError();
}

}  // namespace pml
