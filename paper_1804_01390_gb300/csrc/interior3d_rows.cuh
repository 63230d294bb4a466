// FP32 3D interior kernel with several rows per warp (included by step3d.cu).
//
// The layer-free region advances by the closed form of the RK4 polynomial P(dtA) (Sec. 1.1.2:
// with sigma = 0 the system is the plain wave equation and P(dtA) has the coefficients a1..a5,
// b1..b5 of the first and second powers of the 7-point Laplacian D):
//     U' = U + a1 V + a2 DU + a3 DV + a4 D^2 U,   V' = V + b2 DU + b3 DV + b4 D^2 U + b5 D^2 V
// (the transposed system for the adjoint).  A CTA owns a 60-column x strip by TY = NWP R - 2
// output rows and streams z.  Box rows b = 0 .. NWP R + 1 map to y = y0 - 2 + b; warp w owns
// rows 1 + wR .. wR + R: it forms D U, D V there and the outputs of those that are output rows
// (2 .. NWP R - 1).  Two adjacent columns per lane in packed FP32x2; x neighbours by
// shuffles; y neighbours inside the warp from its own registers, across warps from the
// shared stage plane (U, V) or the shared difference plane (D U, D V: only the warp's first
// and last rows go there); z neighbours from three-plane register rings.  One block barrier
// per plane.
//
// Against the one-row-per-warp kernel this removes the two warps that only load halo rows,
// shares the wait, barrier and addressing of a plane between R rows, and halves the shared
// loads of y neighbours.

namespace pml {

template <int R, int NWP> struct I3R {
    static constexpr int BY = NWP * R + 2;     // box rows
    static constexpr int TY = NWP * R - 2;     // output rows
    static constexpr int ROW = 64;             // box columns (lanes 0 and 31 hold the x halo)
    static constexpr int STRIP = 60;           // output columns
    static constexpr uint32_t FIELD = BY * ROW * 4;
    static constexpr uint32_t STAGE = 2 * FIELD;
    static constexpr uint32_t DPLANE = 2 * BY * ROW * 4;   // D U and D V of one plane, by box row
    static constexpr size_t SMEM = size_t(kS3) * STAGE + 3 * DPLANE + 128;
};
constexpr int kI3R = 2;     // rows per warp
constexpr int kI3W = 8;     // warps per CTA
using I3Rf = I3R<kI3R, kI3W>;

__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void st2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }

// Unscaled 7-point difference of a lane's two columns: x neighbours of the pair from the
// neighbouring lanes (scalar sums, so no pair has to be assembled), the rest packed.
__device__ __forceinline__ float2 lap7_pair(float2 c, float2 ym, float2 yp, float2 zm, float2 zp, float2 m6)
{
    const float l = __shfl_up_sync(0xffffffffu, c.y, 1);
    const float r = __shfl_down_sync(0xffffffffu, c.x, 1);
    float2 t;
    t.x = l + c.y;
    t.y = c.x + r;
    t = __fadd2_rn(t, __fadd2_rn(ym, yp));
    t = __fadd2_rn(t, __fadd2_rn(zm, zp));
    return __ffma2_rn(m6, c, t);
}

template <bool ADJ, int R, int NWP>
__global__ void __launch_bounds__(32 * NWP, 2)
    k_interior3d_rows(const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmV,
                      float *__restrict__ Uo, float *__restrict__ Vo, const Interior3DArgs a)
{
    using C = I3R<R, NWP>;
    constexpr int S = kS3, ROW = C::ROW, BY = C::BY;
    constexpr int FS = BY * ROW;                 // field stride in a stage and in a difference plane
    __shared__ __align__(8) uint64_t bars[S];
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *smem =
        smem_align128<unsigned char>(smem_dyn);
    float *dbuf = reinterpret_cast<float *>(smem + S * C::STAGE);   // [3][2][BY][ROW]

    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        prefetch_tmap(&tmU);
        prefetch_tmap(&tmV);
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    const Geom &g = a.g;
    // strips start where the box's first column (xs - 2) is a multiple of 4 (TMA alignment)
    const int64_t xs0 = a.xr.lo - ((a.xr.lo - 2 + G) & 3);
    const int64_t nstrips = (a.xr.hi - xs0) / C::STRIP + 1;
    const int64_t nty = (a.yr.hi - a.yr.lo) / C::TY + 1;
    const int64_t nz = a.zr.hi - a.zr.lo + 1;
    const int nzs = int((nz + kZSeg3 - 1) / kZSeg3);
    const int n_items = int(nstrips * nty) * nzs;
    __shared__ int item_sh;
    if (blockIdx.x == 0 && tid == 0) a.queue[1 - a.parity] = 0;

    // coefficient pairs (both halves equal), read from the launch parameters
    const float2 *cp = a.pf;
    const int b0 = 1 + w * R;   // the warp's first box row
    const int lo = 2 * lane;
    const int o_own = b0 * ROW + lo;   // the lane's offset in the warp's first row of a plane
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
        const int64_t xs = xs0 + C::STRIP * s, y0 = a.yr.lo + C::TY * t, z0 = a.zr.lo + zi;
        const int n_in = int(cnt) + 4;
        const int32_t tx = int32_t(xs - 2 + G), ty = int32_t(y0 - 2 + G), tz = int32_t(z0 - 2 + G);

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

        const int64_t x0 = xs - 2 + 2 * lane;
        const bool out_lane = lane >= 1 && lane <= 30;
        const bool col_inner = x0 >= G && x0 + 1 < g.T[0] - G;
        const bool full_vec = out_lane && x0 >= a.xr.lo && x0 + 1 <= a.xr.hi && col_inner;
        // per own row: an output row (warp-uniform), and the lane's columns in that row more
        // than G from the x and y box edges (no ghost images)
        uint32_t omask = 0, imask = 0;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int b = b0 + j;
            const int64_t y = y0 - 2 + b;
            if (b >= 2 && b <= BY - 3 && y <= a.yr.hi) omask |= 1u << j;
            if (col_inner && y >= G && y < g.T[1] - G) imask |= 1u << j;
        }
        const int64_t obase = g.origin + (y0 - 2 + b0) * g.P + x0;
        // every own row and both columns of the lane stored by one vector store, no images
        const bool lane_fast = full_vec && imask == (1u << R) - 1u;
        // input planes whose output plane (z = z0 + p - 4) lies more than G from the z box edges
        const int pin_lo = int(G - z0 + 4), pin_hi = int(g.T[2] - G - z0 + 4);
        // the lane's output pointers at input plane p = 0 (z = z0 - 4), advanced by one plane
        // per iteration
        float *ou = Uo + (obase + (z0 - 4) * g.PS), *ov = Vo + (obase + (z0 - 4) * g.PS);
        float2 U[3][R], V[3][R], DU[3][R], DV[3][R];
        bool ok = true;
        int pfail = n_in;   // first plane whose wait gave up

        for (int p0 = 0; p0 < n_in && ok; p0 += 3) {
#pragma unroll
            for (int PH = 0; PH < 3; ++PH) {
                const int p = p0 + PH;
                // ring slots (p0 is a multiple of 3): plane q lives in slot q mod 3
                const int s0 = PH, s1 = (PH + 2) % 3, s2 = (PH + 1) % 3;   // planes p, p-1, p-2 (and p-3 in s0)
                if (p < n_in && ok) {
                    const uint32_t uu = use + p;
                    const int st = uu % S;
                    if (!mbar_wait(&bars[st], (uu / S) & 1u, a.err, 3, a.wait_ns)) {
                        ok = false;
                    } else {
                        const float *sU = reinterpret_cast<const float *>(smem + st * C::STAGE) + o_own;
#pragma unroll
                        for (int j = 0; j < R; ++j) {
                            U[s0][j] = ld2(sU + j * ROW);
                            V[s0][j] = ld2(sU + FS + j * ROW);
                        }
                        if (p >= 2) {   // D U, D V at plane p - 1
                            const float *pU =
                                reinterpret_cast<const float *>(smem + ((use + p - 1) % S) * C::STAGE) + o_own;
                            const float2 um = ld2(pU - ROW), up = ld2(pU + R * ROW);
                            const float2 vm = ld2(pU + FS - ROW), vp = ld2(pU + FS + R * ROW);
#pragma unroll
                            for (int j = 0; j < R; ++j) {
                                DU[s1][j] = lap7_pair(U[s1][j], j > 0 ? U[s1][j - 1] : um, j < R - 1 ? U[s1][j + 1] : up,
                                                      U[s2][j], U[s0][j], cp[10]);
                                DV[s1][j] = lap7_pair(V[s1][j], j > 0 ? V[s1][j - 1] : vm, j < R - 1 ? V[s1][j + 1] : vp,
                                                      V[s2][j], V[s0][j], cp[10]);
                            }
                            float *db = dbuf + s1 * (2 * FS) + o_own;   // slot of plane p - 1
                            st2(db, DU[s1][0]);
                            st2(db + FS, DV[s1][0]);
                            if (R > 1) {
                                st2(db + (R - 1) * ROW, DU[s1][R - 1]);
                                st2(db + FS + (R - 1) * ROW, DV[s1][R - 1]);
                            }
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
                    if (p >= 4 && omask) {   // outputs at plane p - 2
                        const float *db = dbuf + s2 * (2 * FS) + o_own;   // slot of plane p - 2
                        const float2 gum = ld2(db - ROW), gup = ld2(db + R * ROW);
                        const float2 gvm = ld2(db + FS - ROW), gvp = ld2(db + FS + R * ROW);
                        const bool zin = p >= pin_lo && p < pin_hi;
                        const bool fast = lane_fast && zin;
#pragma unroll
                        for (int j = 0; j < R; ++j) {
                            if (!(omask >> j & 1u)) continue;
                            const float2 d2u = lap7_pair(DU[s2][j], j > 0 ? DU[s2][j - 1] : gum,
                                                         j < R - 1 ? DU[s2][j + 1] : gup, DU[s0][j], DU[s1][j], cp[10]);
                            const float2 d2v = lap7_pair(DV[s2][j], j > 0 ? DV[s2][j - 1] : gvm,
                                                         j < R - 1 ? DV[s2][j + 1] : gvp, DV[s0][j], DV[s1][j], cp[10]);
                            const float2 uc = U[s2][j], vc = V[s2][j], duc = DU[s2][j], dvc = DV[s2][j];
                            float2 tu, tv;
                            if (!ADJ) {
                                tu = __ffma2_rn(cp[0], vc, __ffma2_rn(cp[1], duc, __ffma2_rn(cp[2], dvc, __fmul2_rn(cp[3], d2u))));
                                tv = __ffma2_rn(cp[6], duc, __ffma2_rn(cp[7], dvc, __ffma2_rn(cp[8], d2u, __fmul2_rn(cp[9], d2v))));
                            } else {
                                tu = __ffma2_rn(cp[1], duc, __ffma2_rn(cp[2], dvc, __ffma2_rn(cp[3], d2u, __fmul2_rn(cp[4], d2v))));
                                tv = __ffma2_rn(cp[5], uc, __ffma2_rn(cp[6], duc, __ffma2_rn(cp[7], dvc, __fmul2_rn(cp[9], d2v))));
                            }
                            const float2 uo = __fadd2_rn(uc, tu), vo = __fadd2_rn(vc, tv);
                            float *pu = ou + int64_t(j) * g.P, *pv = ov + int64_t(j) * g.P;
                            if (fast) {
                                st2(pu, uo);
                                st2(pv, vo);
                                continue;
                            }
                            const bool inner = zin && (imask >> j & 1u);
                            if (full_vec && inner) {
                                st2(pu, uo);
                                st2(pv, vo);
                            } else if (out_lane && inner) {   // a strip's end: plain stores of its columns in the run
                                if (x0 >= a.xr.lo && x0 <= a.xr.hi) {
                                    pu[0] = uo.x;
                                    pv[0] = vo.x;
                                }
                                if (x0 + 1 >= a.xr.lo && x0 + 1 <= a.xr.hi) {
                                    pu[1] = uo.y;
                                    pv[1] = vo.y;
                                }
                            } else if (out_lane) {
                                const int64_t y = y0 - 2 + b0 + j, z = z0 + p - 4;
                                if (x0 >= a.xr.lo && x0 <= a.xr.hi) {
                                    store_wrapped(Uo, g, x0, y, z, uo.x);
                                    store_wrapped(Vo, g, x0, y, z, vo.x);
                                }
                                if (x0 + 1 >= a.xr.lo && x0 + 1 <= a.xr.hi) {
                                    store_wrapped(Uo, g, x0 + 1, y, z, uo.y);
                                    store_wrapped(Vo, g, x0 + 1, y, z, vo.y);
                                }
                            }
                        }
                    }
                }
                ou += g.PS;
                ov += g.PS;
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
