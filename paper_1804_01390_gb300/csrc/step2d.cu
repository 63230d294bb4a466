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
#include <utility>

#include "common.cuh"

namespace pml {

// Interior kernel variants.
//  kind 0 (row-parallel): a CTA of BY warps streams one strip of 120 output columns in
//     blocks of BY rows, one warp per row; U/V rows come through an S-chunk TMA ring,
//     first differences through a shared row ring; block barriers twice per block.
//  kind 1 (warp-streaming): each warp streams its own strip down the rows with register
//     row rings; NC columns per lane (30 NC outputs per strip), CH rows per TMA box,
//     S stages per warp.
// minb: resident CTAs per SM the launch bounds ask for.
struct I2Var {
    int kind, nc, ch, s, minb;   // kind 0: ch = BY (rows per block / warps per CTA)
};
constexpr I2Var kI2Vars32[] = {{1, 4, 6, 3, 3}, {0, 4, 8, 8, 2}, {0, 4, 4, 8, 4}, {1, 4, 6, 2, 4}, {1, 8, 3, 3, 2}};
constexpr I2Var kI2Vars64[] = {{0, 4, 4, 8, 3}, {0, 4, 8, 4, 1}, {1, 4, 6, 2, 2}, {1, 4, 3, 3, 2}};
constexpr int kNI2Vars32 = sizeof(kI2Vars32) / sizeof(I2Var);
constexpr int kNI2Vars64 = sizeof(kI2Vars64) / sizeof(I2Var);
constexpr int kI2Rows = 64;     // rows per work item, warp-streaming kind
constexpr int kI2RowsR = 128;   // rows per work item, row-parallel kind

int interior2d_variants(int prec) { return prec == 32 ? kNI2Vars32 : kNI2Vars64; }
int interior2d_box_cols(int prec, int v) { return 32 * (prec == 32 ? kI2Vars32[v].nc : kI2Vars64[v].nc); }
int interior2d_threads(int prec, int v)
{
    const I2Var &q = prec == 32 ? kI2Vars32[v] : kI2Vars64[v];
    return q.kind == 0 ? 32 * q.ch : 128;
}
int interior2d_box_rows(int prec, int v) { return prec == 32 ? kI2Vars32[v].ch : kI2Vars64[v].ch; }




// Pairs of adjacent columns.  FP32 uses the packed FP32x2 instructions of this
// architecture (one instruction rounds each lane of the pair exactly like the scalar
// one); FP64 uses two scalar operations.
template <typename T> struct Pair;
template <> struct Pair<float> {
    using P = float2;
    static __device__ __forceinline__ P mk(float a, float b) { return make_float2(a, b); }
    static __device__ __forceinline__ P add(P a, P b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ P mul(P a, P b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ P fma(P a, P b, P c) { return __ffma2_rn(a, b, c); }
};
template <> struct Pair<double> {
    using P = double2;
    static __device__ __forceinline__ P mk(double a, double b) { return make_double2(a, b); }
    static __device__ __forceinline__ P add(P a, P b) { return make_double2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ P mul(P a, P b) { return make_double2(a.x * b.x, a.y * b.y); }
    static __device__ __forceinline__ P fma(P a, P b, P c) { return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y)); }
};

// Unscaled 5-point difference of one lane's NC columns held as NC/2 pairs; l / r are the
// values left of column 0 and right of column NC-1 (neighbouring lanes), up / dn the rows
// above and below.  o = ((x-1 + x+1) + (up + dn)) - 4 x.
template <typename T, int NH>
__device__ __forceinline__ void diff5p(const typename Pair<T>::P (&c)[NH], T l, T r, const typename Pair<T>::P (&up)[NH],
                                       const typename Pair<T>::P (&dn)[NH], typename Pair<T>::P (&o)[NH])
{
    using M = Pair<T>;
    const typename M::P m4 = M::mk(T(-4), T(-4));
#pragma unroll
    for (int k = 0; k < NH; ++k) {
        // x-neighbour sums of the pair's two columns as two scalar additions (the packed
        // form would first assemble the straddling pairs (x-1) and (x+1) with moves)
        const T lv = k == 0 ? l : c[k - 1].y, rv = k == NH - 1 ? r : c[k + 1].x;
        const typename M::P xs = M::mk(lv + c[k].y, c[k].x + rv);
        o[k] = M::fma(m4, c[k], M::add(xs, M::add(up[k], dn[k])));
    }
}

// One interior work item: output rows y0 .. y0+cnt-1 of the strip starting at column xs,
// streamed by one warp through its TMA ring (`wbase`, S stages).  The warp's barriers are
// initialised once per kernel; `use` counts the ring stages this warp has consumed so far
// and gives each stage's slot and phase parity.
template <typename T, bool ADJ, int NC, int CH, int S>
__device__ __forceinline__ bool interior2d_seg(const CUtensorMap *tmU, const CUtensorMap *tmV, T *__restrict__ Uo,
                                               T *__restrict__ Vo, const Interior2DArgs &a, int64_t xs, int64_t y0,
                                               int cnt, unsigned char *wbase, uint64_t *bars, int lane,
                                               uint32_t &use)
{
    using M = Pair<T>;
    using PT = typename M::P;
    constexpr int NH = NC / 2;
    constexpr int ROW = 32 * NC;
    constexpr uint32_t FIELD_BYTES = CH * ROW * sizeof(T);
    constexpr uint32_t STAGE_BYTES = 2 * FIELD_BYTES;
    const Geom &g = a.g;
    const StepCoefT<T> &kc = coef_of<T>(a.c);
    const PT A1 = M::mk(kc.a1, kc.a1), A2 = M::mk(kc.a2, kc.a2), A3 = M::mk(kc.a3, kc.a3), A4 = M::mk(kc.a4, kc.a4),
             A5 = M::mk(kc.a5, kc.a5);
    const PT B1 = M::mk(kc.b1, kc.b1), B2 = M::mk(kc.b2, kc.b2), B3 = M::mk(kc.b3, kc.b3), B4 = M::mk(kc.b4, kc.b4),
             B5 = M::mk(kc.b5, kc.b5);
    const int n_in = cnt + 4;
    const int nch = (n_in + CH - 1) / CH;
    const int32_t tx = int32_t(xs - NC + G);
    const int32_t ty = int32_t(y0 - 2 + G);

    if (lane == 0) {
        fence_proxy_async();   // earlier generic reads of the ring before async writes
        const int npro = nch < S ? nch : S;
        for (int c = 0; c < npro; ++c) {
            const int slot = (use + c) % S;
            unsigned char *dst = wbase + slot * STAGE_BYTES;
            mbar_arrive_expect_tx(&bars[slot], STAGE_BYTES);
            tma_load_2d(dst, tmU, tx, ty + c * CH, &bars[slot]);
            tma_load_2d(dst + FIELD_BYTES, tmV, tx, ty + c * CH, &bars[slot]);
        }
    }
    __syncwarp();

    const int64_t x0 = xs - NC + NC * lane;
    const bool out_lane = lane >= 1 && lane <= 30;
    // every output row of this segment can use vector stores (the common case)
    const bool seg_vec = out_lane && x0 >= a.xr.lo && x0 + NC - 1 <= a.xr.hi && x0 >= G &&
                         x0 + NC - 1 < g.T[0] - G && y0 >= G && y0 + cnt <= g.T[1] - G;
    T *const pU = Uo + g.origin + (y0 - 4) * g.P + x0;   // output row of input row q: pU + q P
    T *const pV = Vo + g.origin + (y0 - 4) * g.P + x0;
    PT u[3][NH], v[3][NH], du[3][NH], dv[3][NH];
    T ul[3], ur[3], vl[3], vr[3], dul[3], dur[3], dvl[3], dvr[3];

    // one input row q at ring position j (compile-time after unrolling)
    auto row = [&](const T *sU, const T *sV, int j, int q, bool d1, bool d2) {
        const int J0 = j % 3, J1 = (j + 2) % 3, J2 = (j + 1) % 3;   // rows q, q-1, q-2
#pragma unroll
        for (int k = 0; k < NH; k += 2) {
            const V4<T> tu = lds4(sU + 2 * k), tv = lds4(sV + 2 * k);
            u[J0][k] = M::mk(tu.x, tu.y);
            u[J0][k + 1] = M::mk(tu.z, tu.w);
            v[J0][k] = M::mk(tv.x, tv.y);
            v[J0][k + 1] = M::mk(tv.z, tv.w);
        }
        // edges of row q for its difference at the next row
        ul[J0] = __shfl_up_sync(0xffffffffu, u[J0][NH - 1].y, 1);
        ur[J0] = __shfl_down_sync(0xffffffffu, u[J0][0].x, 1);
        vl[J0] = __shfl_up_sync(0xffffffffu, v[J0][NH - 1].y, 1);
        vr[J0] = __shfl_down_sync(0xffffffffu, v[J0][0].x, 1);
        if (d1) {
            diff5p<T, NH>(u[J1], ul[J1], ur[J1], u[J2], u[J0], du[J1]);
            diff5p<T, NH>(v[J1], vl[J1], vr[J1], v[J2], v[J0], dv[J1]);
            dul[J1] = __shfl_up_sync(0xffffffffu, du[J1][NH - 1].y, 1);
            dur[J1] = __shfl_down_sync(0xffffffffu, du[J1][0].x, 1);
            dvl[J1] = __shfl_up_sync(0xffffffffu, dv[J1][NH - 1].y, 1);
            dvr[J1] = __shfl_down_sync(0xffffffffu, dv[J1][0].x, 1);
        }
        if (d2) {
            // second differences at row q-2 from DU rows q-3 (slot J0), q-2, q-1
            PT d2u[NH], d2v[NH], uo[NH], vo[NH];
            diff5p<T, NH>(du[J2], dul[J2], dur[J2], du[J0], du[J1], d2u);
            diff5p<T, NH>(dv[J2], dvl[J2], dvr[J2], dv[J0], dv[J1], d2v);
#pragma unroll
            for (int k = 0; k < NH; ++k) {
                const PT uc = u[J2][k], vc = v[J2][k], duc = du[J2][k], dvc = dv[J2][k];
                if (!ADJ) {
                    uo[k] = M::add(uc, M::fma(A1, vc, M::fma(A2, duc, M::fma(A3, dvc, M::mul(A4, d2u[k])))));
                    vo[k] = M::add(vc, M::fma(B2, duc, M::fma(B3, dvc, M::fma(B4, d2u[k], M::mul(B5, d2v[k])))));
                } else {
                    uo[k] = M::add(uc, M::fma(A2, duc, M::fma(A3, dvc, M::fma(A4, d2u[k], M::mul(A5, d2v[k])))));
                    vo[k] = M::add(vc, M::fma(B1, uc, M::fma(B2, duc, M::fma(B3, dvc, M::mul(B5, d2v[k])))));
                }
            }
            if (seg_vec) {
                T *ru = pU + int64_t(q) * g.P, *rv = pV + int64_t(q) * g.P;
#pragma unroll
                for (int k = 0; k < NH; k += 2) {
                    stg4(ru + 2 * k, V4<T>{uo[k].x, uo[k].y, uo[k + 1].x, uo[k + 1].y});
                    stg4(rv + 2 * k, V4<T>{vo[k].x, vo[k].y, vo[k + 1].x, vo[k + 1].y});
                }
            } else if (out_lane) {
                const int64_t r = y0 + q - 4;
#pragma unroll
                for (int k = 0; k < NC; ++k) {
                    const int64_t x = x0 + k;
                    if (x >= a.xr.lo && x <= a.xr.hi) {
                        const T vu = (k & 1) ? uo[k >> 1].y : uo[k >> 1].x;
                        const T vv = (k & 1) ? vo[k >> 1].y : vo[k >> 1].x;
                        if (x >= G && x < g.T[0] - G && r >= G && r < g.T[1] - G) {
                            Uo[g.origin + r * g.P + x] = vu;
                            Vo[g.origin + r * g.P + x] = vv;
                        } else {
                            store_wrapped(Uo, g, x, r, 0, vu);
                            store_wrapped(Vo, g, x, r, 0, vv);
                        }
                    }
                }
            }
        }
    };

    for (int c = 0; c < nch; ++c) {
        const uint32_t uu = use + c;
        const int slot = uu % S;
        if (!mbar_wait(&bars[slot], (uu / S) & 1u, a.err, 1, a.wait_ns)) {
            // give the copies still in flight (this box's included) a bounded chance to
            // land, then stop
            for (int c2 = c; c2 < nch && c2 < c + S; ++c2)
                mbar_wait(&bars[(use + c2) % S], ((use + c2) / S) & 1u, nullptr, 0, kDrainLimitNs);
            return false;
        }
        const T *sU = reinterpret_cast<const T *>(wbase + slot * STAGE_BYTES) + NC * lane;
        const T *sV = sU + CH * ROW;
        if (c * CH < 4) {   // priming rows 0..3: differences start at q = 2, outputs at q = 4
            if constexpr (CH >= 4) {   // box 0 holds them all
#pragma unroll
                for (int j = 0; j < CH; ++j)
                    if (j < n_in) row(sU + j * ROW, sV + j * ROW, j, j, j >= 2, j >= 4);
            } else {                   // shallower boxes: every box that holds one of them
#pragma unroll
                for (int j = 0; j < CH; ++j) {
                    const int q = c * CH + j;
                    if (q < n_in) row(sU + j * ROW, sV + j * ROW, j, q, q >= 2, q >= 4);
                }
            }
        } else if (c < nch - 1) {   // steady state: every row complete, no guards
#pragma unroll
            for (int j = 0; j < CH; ++j) row(sU + j * ROW, sV + j * ROW, j, c * CH + j, true, true);
        } else {
#pragma unroll
            for (int j = 0; j < CH; ++j)
                if (c * CH + j < n_in) row(sU + j * ROW, sV + j * ROW, j, c * CH + j, true, true);
        }
        __syncwarp();
        if (lane == 0 && c + S < nch) {   // slot (use + c + S) % S == slot
            fence_proxy_async();
            unsigned char *dst = wbase + slot * STAGE_BYTES;
            mbar_arrive_expect_tx(&bars[slot], STAGE_BYTES);
            tma_load_2d(dst, tmU, tx, ty + (c + S) * CH, &bars[slot]);
            tma_load_2d(dst + FIELD_BYTES, tmV, tx, ty + (c + S) * CH, &bars[slot]);
        }
    }
    __syncwarp();
    use += uint32_t(nch);
    return true;
}

// ------------------------------------------------------------------------------------
// Temporal blocking, depth 2: two forward RK4 steps in one pass over HBM.
//
// The layer-free run shrunk by 2 vertices per side is advanced by two closed-form steps:
// the first step's values are needed two vertices beyond the outputs, and the closed form
// holds there (the first step only reads the run itself plus its halo).  One warp streams
// its 128-column strip as before, but the rows of the first step (two rows behind the
// input) feed a second copy of the one-step pipeline, whose rows (two more behind) are the
// outputs.  The two steps reach 4 columns to each side: with 4 columns per lane, lanes 0
// and 31 carry exactly that halo and a 128-column strip still has 120 outputs; with 2
// columns per lane (half the registers, more warps per SM) lanes 0-1 and 30-31 do and a
// 64-column strip has 56.  Each output row needs 4 input rows above and below.  Every
// vertex is read and written once per two steps.
// ------------------------------------------------------------------------------------

// Three consecutive rows of U, V and of their 5-point differences, for one step.
template <typename T, int NH> struct StepRing {
    typename Pair<T>::P u[3][NH], v[3][NH], du[3][NH], dv[3][NH];
    T ul[3], ur[3], vl[3], vr[3], dul[3], dur[3], dvl[3], dvr[3];
};

template <typename T> struct StepCoefP {
    typename Pair<T>::P A1, A2, A3, A4, A5, B1, B2, B3, B4, B5;
};

// Row q of one step's input sits in R.u[j % 3], R.v[j % 3] (j = q mod 3 after unrolling):
// its edge columns go to the neighbouring lanes; with d1 the differences of row q-1
// follow, with d2 the step's new values of row q-2 are returned in uo, vo.  Same
// arithmetic, in the same order, as interior2d_seg (ADJ: the transposed step).
template <typename T, bool ADJ, int NH>
__device__ __forceinline__ void ring_push(StepRing<T, NH> &R, const StepCoefP<T> &k, int j, bool d1, bool d2,
                                          typename Pair<T>::P (&uo)[NH], typename Pair<T>::P (&vo)[NH])
{
    using M = Pair<T>;
    using PT = typename M::P;
    const int J0 = j % 3, J1 = (j + 2) % 3, J2 = (j + 1) % 3;   // rows q, q-1, q-2
    R.ul[J0] = __shfl_up_sync(0xffffffffu, R.u[J0][NH - 1].y, 1);
    R.ur[J0] = __shfl_down_sync(0xffffffffu, R.u[J0][0].x, 1);
    R.vl[J0] = __shfl_up_sync(0xffffffffu, R.v[J0][NH - 1].y, 1);
    R.vr[J0] = __shfl_down_sync(0xffffffffu, R.v[J0][0].x, 1);
    if (d1) {
        diff5p<T, NH>(R.u[J1], R.ul[J1], R.ur[J1], R.u[J2], R.u[J0], R.du[J1]);
        diff5p<T, NH>(R.v[J1], R.vl[J1], R.vr[J1], R.v[J2], R.v[J0], R.dv[J1]);
        R.dul[J1] = __shfl_up_sync(0xffffffffu, R.du[J1][NH - 1].y, 1);
        R.dur[J1] = __shfl_down_sync(0xffffffffu, R.du[J1][0].x, 1);
        R.dvl[J1] = __shfl_up_sync(0xffffffffu, R.dv[J1][NH - 1].y, 1);
        R.dvr[J1] = __shfl_down_sync(0xffffffffu, R.dv[J1][0].x, 1);
    }
    if (d2) {
        PT d2u[NH], d2v[NH];
        diff5p<T, NH>(R.du[J2], R.dul[J2], R.dur[J2], R.du[J0], R.du[J1], d2u);
        diff5p<T, NH>(R.dv[J2], R.dvl[J2], R.dvr[J2], R.dv[J0], R.dv[J1], d2v);
#pragma unroll
        for (int c = 0; c < NH; ++c) {
            const PT uc = R.u[J2][c], vc = R.v[J2][c], duc = R.du[J2][c], dvc = R.dv[J2][c];
            if (!ADJ) {
                uo[c] = M::add(uc, M::fma(k.A1, vc, M::fma(k.A2, duc, M::fma(k.A3, dvc, M::mul(k.A4, d2u[c])))));
                vo[c] = M::add(vc, M::fma(k.B2, duc, M::fma(k.B3, dvc, M::fma(k.B4, d2u[c], M::mul(k.B5, d2v[c])))));
            } else {
                uo[c] = M::add(uc, M::fma(k.A2, duc, M::fma(k.A3, dvc, M::fma(k.A4, d2u[c], M::mul(k.A5, d2v[c])))));
                vo[c] = M::add(vc, M::fma(k.B1, uc, M::fma(k.B2, duc, M::fma(k.B3, dvc, M::mul(k.B5, d2v[c])))));
            }
        }
    }
}

// NH pairs of one lane's row from shared memory / to global memory (16-byte accesses for
// two pairs, 8-byte for one).
template <typename T, int NH>
__device__ __forceinline__ void lds_pairs(const T *p, typename Pair<T>::P (&o)[NH])
{
    if constexpr (NH == 1) {
        o[0] = *reinterpret_cast<const typename Pair<T>::P *>(p);
    } else {
#pragma unroll
        for (int c = 0; c < NH; c += 2) {
            const V4<T> t = lds4(p + 2 * c);
            o[c] = Pair<T>::mk(t.x, t.y);
            o[c + 1] = Pair<T>::mk(t.z, t.w);
        }
    }
}
template <typename T, int NH>
__device__ __forceinline__ void stg_pairs(T *p, const typename Pair<T>::P (&v)[NH])
{
    if constexpr (NH == 1) {
        *reinterpret_cast<typename Pair<T>::P *>(p) = v[0];
    } else {
#pragma unroll
        for (int c = 0; c < NH; c += 2) stg4(p + 2 * c, V4<T>{v[c].x, v[c].y, v[c + 1].x, v[c + 1].y});
    }
}

// One work item of the two-step kernel: output rows y0 .. y0+cnt-1 of the strip starting
// at column xs (ring and barrier conventions as in interior2d_seg).  NC = 4 columns per
// lane (lanes 0 and 31 carry the 4-column halo, 120 outputs) or NC = 2 (lanes 0-1 and
// 30-31, 56 outputs).
template <typename T, bool ADJ, int NC, int CH, int S>
__device__ __forceinline__ bool interior2d_seg2(const CUtensorMap *tmU, const CUtensorMap *tmV, T *__restrict__ Uo,
                                                T *__restrict__ Vo, const Interior2DArgs &a, int64_t xs, int64_t y0,
                                                int cnt, unsigned char *wbase, uint64_t *bars, int lane,
                                                uint32_t &use)
{
    using M = Pair<T>;
    using PT = typename M::P;
    constexpr int NH = NC / 2;
    constexpr int ROW = 32 * NC;
    constexpr uint32_t FIELD_BYTES = CH * ROW * sizeof(T);
    constexpr uint32_t STAGE_BYTES = 2 * FIELD_BYTES;
    static_assert((NC == 4 || NC == 2) && CH % 3 == 0, "2 or 4 columns per lane; ring positions repeat every 3 rows");
    constexpr int HL = 4 / NC;   // halo lanes per side
    const Geom &g = a.g;
    const StepCoefT<T> &kc = coef_of<T>(a.c);
    const StepCoefP<T> k{M::mk(kc.a1, kc.a1), M::mk(kc.a2, kc.a2), M::mk(kc.a3, kc.a3), M::mk(kc.a4, kc.a4),
                         M::mk(kc.a5, kc.a5), M::mk(kc.b1, kc.b1), M::mk(kc.b2, kc.b2), M::mk(kc.b3, kc.b3),
                         M::mk(kc.b4, kc.b4), M::mk(kc.b5, kc.b5)};
    const int n_in = cnt + 8;
    const int nch = (n_in + CH - 1) / CH;
    const int32_t tx = int32_t(xs - 4 + G);
    const int32_t ty = int32_t(y0 - 4 + G);

    if (lane == 0) {
        fence_proxy_async();   // earlier generic reads of the ring before async writes
        const int npro = nch < S ? nch : S;
        for (int c = 0; c < npro; ++c) {
            const int slot = (use + c) % S;
            unsigned char *dst = wbase + slot * STAGE_BYTES;
            mbar_arrive_expect_tx(&bars[slot], STAGE_BYTES);
            tma_load_2d(dst, tmU, tx, ty + c * CH, &bars[slot]);
            tma_load_2d(dst + FIELD_BYTES, tmV, tx, ty + c * CH, &bars[slot]);
        }
    }
    __syncwarp();

    const int64_t x0 = xs - 4 + NC * lane;
    const bool out_lane = lane >= HL && lane <= 31 - HL;
    const bool seg_vec = out_lane && x0 >= a.xr.lo && x0 + NC - 1 <= a.xr.hi && x0 >= G &&
                         x0 + NC - 1 < g.T[0] - G && y0 >= G && y0 + cnt <= g.T[1] - G;
    T *const pU = Uo + g.origin + (y0 - 8) * g.P + x0;   // output row of input row q: pU + q P
    T *const pV = Vo + g.origin + (y0 - 8) * g.P + x0;
    StepRing<T, NH> RA, RB;

    // every output lane of this item can use vector stores (the common case): the steady
    // rows then store without a branch, so the unrolled box stays one basic block
    const bool fast = __all_sync(0xffffffffu, !out_lane || seg_vec);
    // input row q at ring position j; `guard`: the first boxes (stages start at rows 2, 4,
    // 6, 8), the last (rows past the input) and items at the edges of the run or the box
    auto row = [&](const T *sU, const T *sV, int j, int q, bool guard) {
        if (guard && q >= n_in) return;
        const int J0 = j % 3;
        lds_pairs<T, NH>(sU, RA.u[J0]);
        lds_pairs<T, NH>(sV, RA.v[J0]);
        PT u1[NH], v1[NH];
        const bool a2 = !guard || q >= 4;
        ring_push<T, ADJ, NH>(RA, k, j, !guard || q >= 2, a2, u1, v1);
        if (!a2) return;
        const int jb = j + 2;   // first-step row q-2 is row q-4 of the second step's input
#pragma unroll
        for (int c = 0; c < NH; ++c) {
            RB.u[jb % 3][c] = u1[c];
            RB.v[jb % 3][c] = v1[c];
        }
        PT uo[NH], vo[NH];
        const bool b2 = !guard || q >= 8;
        ring_push<T, ADJ, NH>(RB, k, jb, !guard || q >= 6, b2, uo, vo);
        if (!b2) return;
        if (!guard) {   // fast item: predicated vector stores
            if (out_lane) {
                stg_pairs<T, NH>(pU + int64_t(q) * g.P, uo);
                stg_pairs<T, NH>(pV + int64_t(q) * g.P, vo);
            }
        } else if (seg_vec) {
            stg_pairs<T, NH>(pU + int64_t(q) * g.P, uo);
            stg_pairs<T, NH>(pV + int64_t(q) * g.P, vo);
        } else if (out_lane) {
            const int64_t r = y0 + q - 8;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int64_t x = x0 + c;
                if (x >= a.xr.lo && x <= a.xr.hi) {
                    const T vu = (c & 1) ? uo[c >> 1].y : uo[c >> 1].x;
                    const T vv = (c & 1) ? vo[c >> 1].y : vo[c >> 1].x;
                    if (x >= G && x < g.T[0] - G && r >= G && r < g.T[1] - G) {
                        Uo[g.origin + r * g.P + x] = vu;
                        Vo[g.origin + r * g.P + x] = vv;
                    } else {
                        store_wrapped(Uo, g, x, r, 0, vu);
                        store_wrapped(Vo, g, x, r, 0, vv);
                    }
                }
            }
        }
    };

    for (int c = 0; c < nch; ++c) {
        const uint32_t uu = use + c;
        const int slot = uu % S;
        if (!mbar_wait(&bars[slot], (uu / S) & 1u, a.err, 6, a.wait_ns)) {
            for (int c2 = c; c2 < nch && c2 < c + S; ++c2)
                mbar_wait(&bars[(use + c2) % S], ((use + c2) / S) & 1u, nullptr, 0, kDrainLimitNs);
            return false;
        }
        const T *sU = reinterpret_cast<const T *>(wbase + slot * STAGE_BYTES) + NC * lane;
        const T *sV = sU + CH * ROW;
        if (c * CH < 8 || c == nch - 1 || !fast) {
#pragma unroll
            for (int j = 0; j < CH; ++j) row(sU + j * ROW, sV + j * ROW, j, c * CH + j, true);
        } else {
#pragma unroll
            for (int j = 0; j < CH; ++j) row(sU + j * ROW, sV + j * ROW, j, c * CH + j, false);
        }
        __syncwarp();
        if (lane == 0 && c + S < nch) {
            fence_proxy_async();
            unsigned char *dst = wbase + slot * STAGE_BYTES;
            mbar_arrive_expect_tx(&bars[slot], STAGE_BYTES);
            tma_load_2d(dst, tmU, tx, ty + (c + S) * CH, &bars[slot]);
            tma_load_2d(dst + FIELD_BYTES, tmV, tx, ty + (c + S) * CH, &bars[slot]);
        }
    }
    __syncwarp();
    use += uint32_t(nch);
    return true;
}

// ------------------------------------------------------------------------------------
// Layer frame: Horner form with the full operator of Eq. 3 (or its transpose), streamed
// down the rows by independent warps.
//
// A warp owns 32 consecutive columns (lane = column; lanes 4..27 are its 24 outputs,
// lanes 0..3 and 28..31 the halo of the four applications of A) and a run of rows of the
// frame.  Input rows arrive through the warp's TMA ring, kL2CH rows per box.  The four
// Horner levels z4 = y + dt/4 A y, z3 = y + dt/3 A z4, z2 = y + dt/2 A z3 and
// y' = y + dt A z2 are skewed by two rows each: when input row p arrives, level 4 gives
// row p-1, level 3 row p-3, level 2 row p-5 and level 1 the output row p-7.  Each level
// then reads only rows finished in earlier iterations, so the four evaluations of one
// iteration are independent and overlap in the pipeline.  Row neighbours of each level
// come from four-row register rings, column neighbours from shuffles, the base y of
// every level from the TMA ring; no block barrier is needed.  Templated on the axes whose
// aux fields are active in the strip.
// ------------------------------------------------------------------------------------

constexpr int kL2CH = 4;         // rows per TMA box
constexpr int kL2SigRows = 80;   // sigma_y table rows per warp (input rows of an item)
template <typename T> struct L2Cfg {
    static constexpr int W = 1;                         // columns per lane
    static constexpr int COLS = 32 * W;                 // columns of one strip (box width)
    static constexpr int OUT = COLS - 8;                // output columns of one strip
    // TMA ring per warp: S boxes of kL2CH rows, RR = S kL2CH rows (a power of two) per
    // field; boxes c-2, c-1, c are being read, the others are in flight
    static constexpr int S = 4;
    static constexpr int RR = S * kL2CH;
    static constexpr int MINB = sizeof(T) == 4 ? 4 : 2;   // resident CTAs per SM (the launch's cap)
    static constexpr int WE = 6 * RR * COLS;   // ring elements per warp, sized for the largest class
    static constexpr size_t smem() { return size_t(4) * WE * sizeof(T) + 128; }
    static_assert((RR & (RR - 1)) == 0, "ring rows must be a power of two");
};

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

// Lane vectors: W adjacent columns per lane.  W = 2 (FP32) uses the packed FP32x2
// instructions (each lane of the pair rounds exactly like the scalar operation).
template <typename T, int W> struct LV;
template <typename T> struct LV<T, 1> {
    using V = T;
    static __device__ __forceinline__ V bc(T a) { return a; }
    static __device__ __forceinline__ V add(V a, V b) { return a + b; }
    static __device__ __forceinline__ V sub(V a, V b) { return a - b; }
    static __device__ __forceinline__ V mul(V a, V b) { return a * b; }
    static __device__ __forceinline__ V fma(V a, V b, V c) { return ::fma(a, b, c); }
    static __device__ __forceinline__ V sel(V m, V x) { return m != T(0) ? x : T(0); }   // x where m != 0
    static __device__ __forceinline__ V left(V c) { return __shfl_up_sync(0xffffffffu, c, 1); }
    static __device__ __forceinline__ V right(V c) { return __shfl_down_sync(0xffffffffu, c, 1); }
    static __device__ __forceinline__ V ld(const T *p) { return *p; }
};
template <> struct LV<float, 2> {
    using V = float2;
    static __device__ __forceinline__ V bc(float a) { return make_float2(a, a); }
    static __device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ V sub(V a, V b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
    static __device__ __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ V sel(V m, V x) { return make_float2(m.x != 0.f ? x.x : 0.f, m.y != 0.f ? x.y : 0.f); }
    static __device__ __forceinline__ V left(V c) { return make_float2(__shfl_up_sync(0xffffffffu, c.y, 1), c.x); }
    static __device__ __forceinline__ V right(V c) { return make_float2(c.y, __shfl_down_sync(0xffffffffu, c.x, 1)); }
    static __device__ __forceinline__ V ld(const float *p) { return *reinterpret_cast<const float2 *>(p); }
};

// Whether apply_A2 reads field f at the x neighbour d (1: x-, 2: x+): only those
// neighbours are fetched by shuffles.  Forward: U on both sides, Phi_x on the left, Psi_x
// on the right; transposed: V, Phi_x and Psi_x on both sides.
template <bool ADJ, int MASK> __device__ __forceinline__ constexpr bool need_x2(int f, int d)
{
    if (f == 0) return !ADJ;
    if (f == 1) return ADJ;
    if (Fields2<MASK>::axis((f - 2) >> 1) != 0) return false;
    if (ADJ) return true;
    return ((f - 2) & 1) == 0 ? d == 1 : d == 2;
}
template <typename O, bool ADJ, int MASK, int F, typename V>
__device__ __forceinline__ void x_neighbour(const V *c, V *xm, V *xp)
{
    if constexpr (need_x2<ADJ, MASK>(F, 1)) xm[F] = O::left(c[F]);
    else xm[F] = c[F];
    if constexpr (need_x2<ADJ, MASK>(F, 2)) xp[F] = O::right(c[F]);
    else xp[F] = c[F];
}
template <typename O, bool ADJ, int MASK, typename V, int... F>
__device__ __forceinline__ void x_neighbours(const V *c, V *xm, V *xp, std::integer_sequence<int, F...>)
{
    (x_neighbour<O, ADJ, MASK, F>(c, xm, xp), ...);
}

template <typename V> struct Sig2 {
    V si[2], sm[2];   // sigma_a[i_a], sigma_a[i_a - 1]
};

// A z (or A^T z) at the lane's vertices; N(f, d): d = 0 centre, 1 x-, 2 x+, 3 y-, 4 y+.
template <typename O, bool ADJ, int MASK, typename Get>
__device__ __forceinline__ void apply_A2(const Get &N, const Sig2<typename O::V> &s, typename O::V ih,
                                         typename O::V ih2, typename O::V i2h, typename O::V *o)
{
    using F = Fields2<MASK>;
    using V = typename O::V;
    const V m2 = O::bc(-2), mhalf = O::bc(-0.5);
    if (!ADJ) {
        const V U0 = N(0, 0);
        const V lap = O::add(O::fma(m2, U0, O::add(N(0, 2), N(0, 1))), O::fma(m2, U0, O::add(N(0, 4), N(0, 3))));
        V aV = O::mul(lap, ih2);
        o[0] = N(1, 0);
#pragma unroll
        for (int k = 0; k < F::NAX; ++k) {
            const int ax = F::axis(k), fp = 2 + 2 * k, fq = 3 + 2 * k, dm = 1 + 2 * ax, dp = 2 + 2 * ax;
            const V si = s.si[ax], sm = s.sm[ax];
            const V phm = N(fp, dm), psp = N(fq, dp);
            aV = O::fma(O::sub(O::mul(si, psp), O::mul(sm, phm)), ih, aV);
            const V ndU = O::mul(O::sub(N(0, dm), N(0, dp)), i2h);   // -(U(+) - U(-)) / 2h
            o[fp] = O::sel(si, O::fma(mhalf, O::fma(sm, phm, O::mul(si, N(fp, 0))), ndU));
            o[fq] = O::sel(sm, O::fma(mhalf, O::fma(sm, N(fq, 0), O::mul(si, psp)), ndU));
        }
        o[1] = aV;
    } else {
        const V V0 = N(1, 0);
        const V lap = O::add(O::fma(m2, V0, O::add(N(1, 2), N(1, 1))), O::fma(m2, V0, O::add(N(1, 4), N(1, 3))));
        V aU = O::mul(lap, ih2);
        o[1] = N(0, 0);
#pragma unroll
        for (int k = 0; k < F::NAX; ++k) {
            const int ax = F::axis(k), fp = 2 + 2 * k, fq = 3 + 2 * k, dm = 1 + 2 * ax, dp = 2 + 2 * ax;
            const V si = s.si[ax], sm = s.sm[ax];
            aU = O::fma(O::add(O::sub(N(fp, dp), N(fp, dm)), O::sub(N(fq, dp), N(fq, dm))), i2h, aU);
            // -si V(+)/h - si/2 (Phi(+) + Phi),  sm V(-)/h - sm/2 (Psi + Psi(-))
            o[fp] = O::sel(si, O::mul(si, O::fma(mhalf, O::add(N(fp, dp), N(fp, 0)), O::mul(O::bc(-1), O::mul(N(1, dp), ih)))));
            o[fq] = O::sel(sm, O::mul(sm, O::fma(mhalf, O::add(N(fq, 0), N(fq, dm)), O::mul(N(1, dm), ih))));
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
__device__ __forceinline__ void issue_rows2(T *ring, const Maps6 &maps, int32_t x, int32_t y, int row0, uint64_t *bar)
{
    using F = Fields2<MASK>;
    constexpr int RR = L2Cfg<T>::RR, COLS = L2Cfg<T>::COLS;
    mbar_arrive_expect_tx(bar, uint32_t(F::NF * kL2CH * COLS * sizeof(T)));
#pragma unroll
    for (int f = 0; f < F::NF; ++f) tma_load_2d(ring + (f * RR + row0) * COLS, &maps.m[F::gid(f)], x, y, bar);
}

// One work item (a strip of the frame) streamed by one warp.  Lane l holds columns
// x0 - 4 + W l .. + W - 1 (W = L2Cfg::W); the outputs are the columns x0 .. x0 + OUT - 1
// of lanes 4/W .. 31 - 4/W.  `ring` is the warp's row ring ([NF][RR][COLS]; input row q
// of the item sits in ring row (kL2CH use + q) mod RR), `sy` its sigma_y table
// (2 x kL2SigRows).  The warp's barriers are initialised once per kernel; `use` counts
// the boxes this warp has consumed and gives each box's slot and phase parity.  Output
// rows ylo..yhi may run past T1 - 1 (the band across the periodic seam of y): rows and
// box coordinates wrap by T1.  One loop iteration handles one input row p; the register
// rings hold three rows of each level and rotate by one row per iteration (a compact loop
// body keeps the instruction stream in cache).
template <typename T, bool ADJ, int MASK, bool WALL>
__device__ __forceinline__ bool layer2d_item(const Maps6 &maps, const Out6 &out, const Layer2DArgs &a,
                                             const LayerTile &tile, T *ring, T *sy, uint64_t *bars, int lane,
                                             uint32_t &use)
{
    using F = Fields2<MASK>;
    constexpr int W = L2Cfg<T>::W, COLS = L2Cfg<T>::COLS;
    using O = LV<T, W>;
    using V = typename O::V;
    constexpr int NF = F::NF, CH = kL2CH, S = L2Cfg<T>::S, RR = L2Cfg<T>::RR;
    // halo of 4 along a damped axis, 2 along an undamped one (there U and V of every Horner
    // level depend on the level above only through the Laplacian of V)
    constexpr int HX = (MASK & 1) ? 4 : 2, HY = (MASK & 2) ? 4 : 2, OUT = COLS - 2 * HX;
    const Geom &g = a.g;
    const int T1 = int(g.T[1]);
    const int nout = tile.yhi - tile.ylo + 1, nin = nout + 2 * HY;
    const int nch = (nin + CH - 1) / CH;          // boxes that hold input rows
    const int32_t tx = tile.x0 - HX + G;
    auto box_y = [&](int c) -> int32_t {          // box row of box c (rows stay in -4 .. T1 + 3)
        int y = tile.ylo - HY + c * CH;
        if (!WALL && y > T1) y -= T1;              // with a wall, items never cross the seam and
        return int32_t(y + G);                     // rows beyond the ghost ring load as zeros
    };
    auto issue = [&](int c) {
        const uint32_t k = use + uint32_t(c);
        issue_rows2<T, MASK>(ring, maps, tx, box_y(c), int((k % S) * CH), &bars[k % S]);
    };
    if (lane == 0) {
        fence_proxy_async();   // earlier generic reads of the ring before async writes
        for (int c = 0; c < nch && c < S; ++c) issue(c);
    }
    if (MASK & 2) {   // sigma_y[row], sigma_y[row - 1] of every input row
        const T *sgy = static_cast<const T *>(a.sig[1]);
        for (int q = lane; q < nin; q += 32) {
            int yi = tile.ylo - HY + q;
            yi += yi < 0 ? T1 : 0;
            yi -= yi >= T1 ? T1 : 0;
            yi -= yi >= T1 ? T1 : 0;
            sy[q] = sgy[yi];
            sy[kL2SigRows + q] = sgy[yi == 0 ? T1 - 1 : yi - 1];
        }
    }
    __syncwarp();

    const int64_t gx0 = int64_t(tile.x0) - HX + W * lane;   // first column of the lane
    Sig2<V> sgx;
    {
        const T *sgxp = static_cast<const T *>(a.sig[0]);
        const int T0 = int(g.T[0]);
        T si[W], sm[W];
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const int xi = int((((gx0 + k) % T0) + T0) % T0);
            si[k] = sgxp[xi];
            sm[k] = sgxp[xi == 0 ? T0 - 1 : xi - 1];
        }
        if constexpr (W == 1) {
            sgx.si[0] = si[0];
            sgx.sm[0] = sm[0];
        } else {
            sgx.si[0] = make_float2(si[0], si[W - 1]);
            sgx.sm[0] = make_float2(sm[0], sm[W - 1]);
        }
        sgx.si[1] = O::bc(T(0));
        sgx.sm[1] = O::bc(T(0));
    }
    auto sig_at = [&](int q) {   // sigma of input row q (clamped: rows outside feed nothing)
        Sig2<V> s = sgx;
        if (MASK & 2) {
            q = q < 0 ? 0 : (q >= nin ? nin - 1 : q);
            s.si[1] = O::bc(sy[q]);
            s.sm[1] = O::bc(sy[kL2SigRows + q]);
        }
        return s;
    };
    bool out_col[W];
#pragma unroll
    for (int k = 0; k < W; ++k)
        out_col[k] = gx0 + k >= tile.x0 && gx0 + k < tile.x0 + OUT && gx0 + k >= tile.xlo &&
                     gx0 + k <= tile.xhi;
    bool any_out = false;
#pragma unroll
    for (int k = 0; k < W; ++k) any_out = any_out || out_col[k];
    const LayerConstT<T> &lk = lconst_of<T>(a.k);
    const V ih = O::bc(lk.ih), ih2 = O::bc(lk.ih2), i2h = O::bc(lk.i2h), c4 = O::bc(lk.c4), c3 = O::bc(lk.c3),
            c2 = O::bc(lk.c2), c1 = O::bc(lk.c1);
    // with a wall every stage value beyond the ends of the box is zero: the lane's columns
    // and a row's validity as masks for the level values
    V xmask = O::bc(T(1));
    if (WALL) {
        T m[W];
#pragma unroll
        for (int k = 0; k < W; ++k) m[k] = (gx0 + k >= 0 && gx0 + k < g.T[0]) ? T(1) : T(0);
        if constexpr (W == 1) xmask = m[0];
        else xmask = make_float2(m[0], m[W - 1]);
    }
    auto wall_mask = [&](V v, int q) -> V {        // level value at input row q
        if (!WALL) return v;
        const int y = tile.ylo - HY + q;
        return (y >= 0 && y < T1) ? O::sel(xmask, v) : O::bc(T(0));
    };
    const int qmax = nch * CH - 1;                 // last row the boxes brought in
    const uint32_t rbase = uint32_t(CH) * use;
    // the lane's values of input row q (clamped into the rows brought in), field f at + f RR COLS
    auto rowp = [&](int q) -> const T * {
        q = q < 0 ? 0 : (q > qmax ? qmax : q);
        return ring + int((rbase + uint32_t(q)) & uint32_t(RR - 1)) * COLS + W * lane;
    };
    // level rings: [0] row r-1, [1] row r, [2] row r+1 of the row r the level reads
    V z4[3][NF], z3[3][NF], z2[3][NF];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int f = 0; f < NF; ++f) z4[k][f] = z3[k][f] = z2[k][f] = O::bc(T(0));

    // ghost images of the lane's columns (a vertex within G of the box edge is also stored
    // at its periodic image in the ghost ring; 0: none, and with a wall the ring stays zero)
    int64_t dxk[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const int64_t x = gx0 + k;
        dxk[k] = g.wrap[0] == 0 ? 0 : (x < G ? g.wrap[0] : (x >= g.T[0] - G ? -g.wrap[0] : 0));
    }
    bool all = true;
#pragma unroll
    for (int k = 0; k < W; ++k) all = all && out_col[k];

    // iteration p reads input rows p .. p - 7; the output row of input row r is formed in
    // iteration r + 7
#pragma unroll 1
    for (int p = 0; p < nin + 7 - HY; ++p) {
        if ((p & (CH - 1)) == 0) {
            const int c = p / CH;
            // box c - 3 was last read in iteration p - 2: refill its slot with box c - 3 + S
            if (c >= 3 && c - 3 + S < nch) {
                __syncwarp();
                if (lane == 0) {
                    fence_proxy_async();
                    issue(c - 3 + S);
                }
            }
            if (c < nch) {
                const uint32_t k = use + uint32_t(c);
                if (!mbar_wait(&bars[k % S], (k / S) & 1, a.err, 2, a.wait_ns)) {
                    for (int c2 = c; c2 < nch && c2 < c + S; ++c2) {
                        const uint32_t k2 = use + uint32_t(c2);
                        mbar_wait(&bars[k2 % S], (k2 / S) & 1, nullptr, 0, kDrainLimitNs);
                    }
                    return false;
                }
            }
        }
        const T *y0 = rowp(p), *y1 = rowp(p - 1), *y2 = rowp(p - 2), *y3 = rowp(p - 3), *y5 = rowp(p - 5),
                *y7 = rowp(p - 7);
        constexpr int FS = RR * COLS;   // field stride in the ring
        V n4[NF], n3[NF], n2[NF], r[NF];
        // level 4 at row p-1 (input rows p-2, p-1, p)
        {
            V cen[NF], xm[NF], xp[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) cen[f] = O::ld(y1 + f * FS);
            x_neighbours<O, ADJ, MASK>(cen, xm, xp, std::make_integer_sequence<int, NF>{});
            auto N = [&](int f, int d) -> V {
                switch (d) {
                case 0: return cen[f];
                case 1: return xm[f];
                case 2: return xp[f];
                case 3: return O::ld(y2 + f * FS);
                default: return O::ld(y0 + f * FS);
                }
            };
            apply_A2<O, ADJ, MASK>(N, sig_at(p - 1), ih, ih2, i2h, r);
#pragma unroll
            for (int f = 0; f < NF; ++f) n4[f] = wall_mask(O::fma(c4, r[f], cen[f]), p - 1);
        }
        // level 3 at row p-3 (z4 rows p-4, p-3, p-2)
        {
            V xm[NF], xp[NF];
            x_neighbours<O, ADJ, MASK>(z4[1], xm, xp, std::make_integer_sequence<int, NF>{});
            auto N = [&](int f, int d) -> V {
                switch (d) {
                case 0: return z4[1][f];
                case 1: return xm[f];
                case 2: return xp[f];
                case 3: return z4[0][f];
                default: return z4[2][f];
                }
            };
            apply_A2<O, ADJ, MASK>(N, sig_at(p - 3), ih, ih2, i2h, r);
#pragma unroll
            for (int f = 0; f < NF; ++f) n3[f] = wall_mask(O::fma(c3, r[f], O::ld(y3 + f * FS)), p - 3);
        }
        // level 2 at row p-5 (z3 rows p-6, p-5, p-4)
        {
            V xm[NF], xp[NF];
            x_neighbours<O, ADJ, MASK>(z3[1], xm, xp, std::make_integer_sequence<int, NF>{});
            auto N = [&](int f, int d) -> V {
                switch (d) {
                case 0: return z3[1][f];
                case 1: return xm[f];
                case 2: return xp[f];
                case 3: return z3[0][f];
                default: return z3[2][f];
                }
            };
            apply_A2<O, ADJ, MASK>(N, sig_at(p - 5), ih, ih2, i2h, r);
#pragma unroll
            for (int f = 0; f < NF; ++f) n2[f] = wall_mask(O::fma(c2, r[f], O::ld(y5 + f * FS)), p - 5);
        }
        // level 1 at row p-7 (z2 rows p-8, p-7, p-6): output row p-11 of the item
        {
            V xm[NF], xp[NF];
            x_neighbours<O, ADJ, MASK>(z2[1], xm, xp, std::make_integer_sequence<int, NF>{});
            auto N = [&](int f, int d) -> V {
                switch (d) {
                case 0: return z2[1][f];
                case 1: return xm[f];
                case 2: return xp[f];
                case 3: return z2[0][f];
                default: return z2[2][f];
                }
            };
            apply_A2<O, ADJ, MASK>(N, sig_at(p - 7), ih, ih2, i2h, r);
            const int ro = p - 7 - HY;
            if (any_out && ro >= 0 && ro < nout) {
                int64_t y = int64_t(tile.ylo) + ro;
                if (y >= T1) y -= T1;
                const int64_t dy = g.wrap[1] == 0 ? 0 : (y < G ? g.wrap[1] : (y >= T1 - G ? -g.wrap[1] : 0)) * g.P;
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const V val = O::fma(c1, r[f], O::ld(y7 + f * FS));
                    T *b = static_cast<T *>(out.p[F::gid(f)]) + g.origin + gx0 + y * g.P;
                    const T *vv = reinterpret_cast<const T *>(&val);
                    if (all) {
                        *reinterpret_cast<V *>(b) = val;
                        if (dy) *reinterpret_cast<V *>(b + dy) = val;
                    } else {
#pragma unroll
                        for (int k = 0; k < W; ++k)
                            if (out_col[k]) {
                                b[k] = vv[k];
                                if (dy) b[k + dy] = vv[k];
                            }
                    }
#pragma unroll
                    for (int k = 0; k < W; ++k)
                        if (out_col[k] && dxk[k]) {
                            b[k + dxk[k]] = vv[k];
                            if (dy) b[k + dxk[k] + dy] = vv[k];
                        }
                }
            }
        }
        // rotate the rings by one row
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            z4[0][f] = z4[1][f]; z4[1][f] = z4[2][f]; z4[2][f] = n4[f];
            z3[0][f] = z3[1][f]; z3[1][f] = z3[2][f]; z3[2][f] = n3[f];
            z2[0][f] = z2[1][f]; z2[1][f] = z2[2][f]; z2[2][f] = n2[f];
        }
    }
    __syncwarp();
    use += uint32_t(nch);
    return true;
}

// ------------------------------------------------------------------------------------
// Row-parallel interior kernel (kind 0).  Input row i of a work item is row y0 - 2 + i.
// U and V live in circular rings of RR = 32 rows (row i in slot (base + i) & 31, base
// advancing by whole chunks across work items); TMA chunk c brings input rows
// [c BY, c BY + BY) into one contiguous run of slots.  Block b (outputs y0 + b BY + w,
// w = warp) needs U/V rows [b BY, b BY + BY + 4) (chunks b, b+1) and first differences of
// rows [b BY + 1, b BY + BY + 3); it computes those of rows [b BY + 3, b BY + BY + 3)
// (block 0 also rows 1, 2) into a second 32-row ring, and after one block barrier the
// second differences and outputs of its BY rows.
// ------------------------------------------------------------------------------------
template <typename T, int BY, int NCH> struct I2R {
    // U/V ring: NCH chunks of BY rows (two resident, NCH - 2 in flight); DU/DV ring: at
    // least the 2 BY + 2 rows one block reads; both powers of two
    static constexpr int ROW = 128, RR = NCH * BY, RD = BY <= 4 ? 16 : (BY <= 8 ? 32 : 64);
    static constexpr uint32_t FB = BY * ROW * sizeof(T);      // one field of one chunk
    static constexpr size_t SMEM = (2 * size_t(RR) + 2 * size_t(RD)) * ROW * sizeof(T) + 128;
    static_assert((RR & (RR - 1)) == 0 && NCH >= 3 && RD >= 2 * BY + 2, "ring sizes");
};

template <typename T, bool ADJ, int BY, int NCH, int MINB>
__global__ void __launch_bounds__(32 * BY, MINB)
    k_interior2d_rows(const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmV,
                      T *__restrict__ Uo, T *__restrict__ Vo, const Interior2DArgs a)
{
    using C = I2R<T, BY, NCH>;
    using M = Pair<T>;
    using PT = typename M::P;
    constexpr int ROW = C::ROW, RR = C::RR, RD = C::RD, NH = 2;
    __shared__ __align__(8) uint64_t bars[NCH];
    __shared__ int item_sh;
    extern __shared__ unsigned char smem_dyn[];
    T *ring = smem_align128<T>(smem_dyn);
    T *const ringU = ring, *const ringV = ring + RR * ROW, *const ringDU = ring + 2 * RR * ROW,
          *const ringDV = ring + (2 * RR + RD) * ROW;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    if (blockIdx.x == 0 && tid == 0) a.queue[1 - a.parity] = 0;
    if (tid == 0) {
        prefetch_tmap(&tmU);
        prefetch_tmap(&tmV);
        for (int k = 0; k < NCH; ++k) mbar_init(&bars[k], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const Geom &g = a.g;
    const StepCoefT<T> &kc = coef_of<T>(a.c);
    const int64_t xs0 = a.xr.lo & ~int64_t(3);
    const int64_t nrows = a.yr.hi - a.yr.lo + 1;
    const int rblocks = int((nrows + kI2RowsR - 1) / kI2RowsR);
    const int nstrips = int((a.xr.hi - xs0) / 120 + 1);
    const int n_items = nstrips * rblocks;
    uint32_t use = 0;   // chunks consumed by this CTA so far
    bool ok = true;
    const int lo4 = 4 * lane;

    auto ld2 = [&](const T *p, PT (&o)[NH]) {
        const V4<T> t = lds4(p);
        o[0] = M::mk(t.x, t.y);
        o[1] = M::mk(t.z, t.w);
    };
    // first differences of U and V at input row i into the DU / DV rings
    auto diff_row = [&](int i) {
        const int s0 = (int(use) * BY + i) & (RR - 1), sm = (s0 - 1) & (RR - 1), sp = (s0 + 1) & (RR - 1);
        const int d0 = i & (RD - 1);
        PT c[NH], up[NH], dn[NH], o[NH];
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const T *R = f == 0 ? ringU : ringV;
            ld2(R + s0 * ROW + lo4, c);
            ld2(R + sm * ROW + lo4, up);
            ld2(R + sp * ROW + lo4, dn);
            const T l = __shfl_up_sync(0xffffffffu, c[NH - 1].y, 1), r = __shfl_down_sync(0xffffffffu, c[0].x, 1);
            diff5p<T, NH>(c, l, r, up, dn, o);
            stg4((f == 0 ? ringDU : ringDV) + d0 * ROW + lo4, V4<T>{o[0].x, o[0].y, o[1].x, o[1].y});
        }
    };

    for (;;) {
        if (tid == 0) item_sh = atomicAdd(&a.queue[a.parity], 1);
        __syncthreads();
        const int item = item_sh;
        if (item >= n_items) break;
        const int st = item / rblocks, rb = item - st * rblocks;
        const int64_t xs = xs0 + int64_t(120) * st;
        const int64_t y0 = a.yr.lo + int64_t(rb) * kI2RowsR;
        const int64_t rem = a.yr.hi - y0 + 1;
        const int cnt = int(rem < kI2RowsR ? rem : kI2RowsR);
        const int nblk = (cnt + BY - 1) / BY;
        const int nch = nblk + 1;   // input rows nblk BY + 4 <= (nblk + 1) BY
        const int32_t tx = int32_t(xs - 4 + G), ty = int32_t(y0 - 2 + G);
        auto issue = [&](int c) {
            const int slot = (use + c) % NCH;
            const int row0 = (int(use) * BY + c * BY) & (RR - 1);
            mbar_arrive_expect_tx(&bars[slot], 2 * C::FB);
            tma_load_2d(ringU + row0 * ROW, &tmU, tx, ty + c * BY, &bars[slot]);
            tma_load_2d(ringV + row0 * ROW, &tmV, tx, ty + c * BY, &bars[slot]);
        };
        auto wait_chunk = [&](int c) {
            const uint32_t uu = use + c;
            return mbar_wait(&bars[uu % NCH], (uu / NCH) & 1u, a.err, 5, a.wait_ns);
        };
        if (tid == 0) {
            fence_proxy_async();
            for (int c = 0; c < nch && c < NCH; ++c) issue(c);
        }
        const int64_t x0 = xs - 4 + lo4;
        const bool out_lane = lane >= 1 && lane <= 30;
        const bool col_vec = out_lane && x0 >= a.xr.lo && x0 + 3 <= a.xr.hi && x0 >= G && x0 + 3 < g.T[0] - G;
        for (int b = 0; b < nblk; ++b) {
            bool okw = true;
            if (b == 0) okw = wait_chunk(0);
            if (okw && b + 1 < nch) okw = wait_chunk(b + 1);
            ok = __syncthreads_and(okw);
            if (!ok) {   // let the copies in flight (chunks b .. b + NCH - 2 at most) land
                if (tid == 0)
                    for (int c = b; c < nch && c < b + NCH; ++c) {
                        const uint32_t uu = use + c;
                        mbar_wait(&bars[uu % NCH], (uu / NCH) & 1u, nullptr, 0, kDrainLimitNs);
                    }
                break;
            }
            // chunk b - 1 was last read by block b - 1 (all warps are past it): refill its slots
            if (tid == 0 && b >= 1 && b - 1 + NCH < nch) {
                fence_proxy_async();
                issue(b - 1 + NCH);
            }
            if (b == 0) {
                diff_row(1 + w);
                if (w < 2) diff_row(BY + 1 + w);
            } else {
                diff_row(b * BY + 3 + w);
            }
            __syncthreads();
            // second differences and outputs of input row i = b BY + 2 + w
            const int i = b * BY + 2 + w;
            const int64_t y = y0 + b * BY + w;
            if (y < y0 + cnt) {
                const int s0 = (int(use) * BY + i) & (RR - 1);
                const int d0 = i & (RD - 1), dm = (i - 1) & (RD - 1), dp = (i + 1) & (RD - 1);
                PT uc[NH], vc[NH], duc[NH], dvc[NH], d2u[NH], d2v[NH], up[NH], dn[NH], uo[NH], vo[NH];
                ld2(ringU + s0 * ROW + lo4, uc);
                ld2(ringV + s0 * ROW + lo4, vc);
                ld2(ringDU + d0 * ROW + lo4, duc);
                ld2(ringDU + dm * ROW + lo4, up);
                ld2(ringDU + dp * ROW + lo4, dn);
                {
                    const T l = __shfl_up_sync(0xffffffffu, duc[NH - 1].y, 1), r = __shfl_down_sync(0xffffffffu, duc[0].x, 1);
                    diff5p<T, NH>(duc, l, r, up, dn, d2u);
                }
                ld2(ringDV + d0 * ROW + lo4, dvc);
                ld2(ringDV + dm * ROW + lo4, up);
                ld2(ringDV + dp * ROW + lo4, dn);
                {
                    const T l = __shfl_up_sync(0xffffffffu, dvc[NH - 1].y, 1), r = __shfl_down_sync(0xffffffffu, dvc[0].x, 1);
                    diff5p<T, NH>(dvc, l, r, up, dn, d2v);
                }
                const PT A1 = M::mk(kc.a1, kc.a1), A2 = M::mk(kc.a2, kc.a2), A3 = M::mk(kc.a3, kc.a3),
                         A4 = M::mk(kc.a4, kc.a4), A5 = M::mk(kc.a5, kc.a5);
                const PT B1 = M::mk(kc.b1, kc.b1), B2 = M::mk(kc.b2, kc.b2), B3 = M::mk(kc.b3, kc.b3),
                         B4 = M::mk(kc.b4, kc.b4), B5 = M::mk(kc.b5, kc.b5);
#pragma unroll
                for (int k = 0; k < NH; ++k) {
                    if (!ADJ) {
                        uo[k] = M::add(uc[k], M::fma(A1, vc[k], M::fma(A2, duc[k], M::fma(A3, dvc[k], M::mul(A4, d2u[k])))));
                        vo[k] = M::add(vc[k], M::fma(B2, duc[k], M::fma(B3, dvc[k], M::fma(B4, d2u[k], M::mul(B5, d2v[k])))));
                    } else {
                        uo[k] = M::add(uc[k], M::fma(A2, duc[k], M::fma(A3, dvc[k], M::fma(A4, d2u[k], M::mul(A5, d2v[k])))));
                        vo[k] = M::add(vc[k], M::fma(B1, uc[k], M::fma(B2, duc[k], M::fma(B3, dvc[k], M::mul(B5, d2v[k])))));
                    }
                }
                if (col_vec && y >= G && y < g.T[1] - G) {
                    const int64_t off = g.origin + y * g.P + x0;
                    stg4(Uo + off, V4<T>{uo[0].x, uo[0].y, uo[1].x, uo[1].y});
                    stg4(Vo + off, V4<T>{vo[0].x, vo[0].y, vo[1].x, vo[1].y});
                } else if (out_lane) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int64_t x = x0 + k;
                        if (x >= a.xr.lo && x <= a.xr.hi) {
                            store_wrapped(Uo, g, x, y, 0, (k & 1) ? uo[k >> 1].y : uo[k >> 1].x);
                            store_wrapped(Vo, g, x, y, 0, (k & 1) ? vo[k >> 1].y : vo[k >> 1].x);
                        }
                    }
                }
            }
        }
        if (!ok) break;
        use += uint32_t(nch);
        __syncthreads();   // the next item's prologue reuses the rings
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ------------------------------------------------------------------------------------
// Launch structure of one 2D step (two kernels, disjoint outputs):
//  1. k_layer2d: one warp per frame strip (latency bound, long); it lets the next
//     kernel start right away (programmatic dependent launch).
//  2. k_interior2d: persistent; warps take interior segments of kI2Rows rows from a work
//     queue (atomic counter), so SMs that start late, while layer warps still run, or
//     that run slower simply take fewer segments.  The counter of this launch is
//     queue[parity]; block 0 clears queue[1 - parity] for the next launch (the next launch
//     follows the next layer kernel, which waits for this one to finish).
// ------------------------------------------------------------------------------------


// Each warp takes items from a work queue (atomic counter) until the list is done; tiles
// are sorted by class, so warps run the same class at the same time.
template <typename T, bool ADJ, bool WALL>
__global__ void __launch_bounds__(128, L2Cfg<T>::MINB)
    k_layer2d(const __grid_constant__ Maps6 maps, const Out6 out, const Layer2DArgs a)
{
    constexpr int S = L2Cfg<T>::S, WE = L2Cfg<T>::WE;
    __shared__ __align__(8) uint64_t bars[4][S];
    __shared__ T sig_sh[4][2 * kL2SigRows];
    extern __shared__ unsigned char smem_dyn[];
    T *smem = smem_align128<T>(smem_dyn);
    allow_dependent_launch();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        for (int k = 0; k < S; ++k) mbar_init(&bars[warp][k], 1);
        fence_mbar_init();
    }
    // launched early (second layer pass of a two-step block): the inputs are the previous
    // kernel's outputs; a no-op for a launch without programmatic overlap
    wait_prerequisite_grid();
    __syncwarp();
    T *ring = smem + warp * WE;
    uint32_t use = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.queue[1 - a.parity] = 0;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&a.queue[a.parity], 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= a.ntiles) break;
        const LayerTile tile = a.tiles[item];
        bool ok;
        switch (tile.flags & 3) {
        case 0: ok = layer2d_item<T, ADJ, 0, WALL>(maps, out, a, tile, ring, sig_sh[warp], bars[warp], lane, use); break;
        case 1: ok = layer2d_item<T, ADJ, 1, WALL>(maps, out, a, tile, ring, sig_sh[warp], bars[warp], lane, use); break;
        case 2: ok = layer2d_item<T, ADJ, 2, WALL>(maps, out, a, tile, ring, sig_sh[warp], bars[warp], lane, use); break;
        default: ok = layer2d_item<T, ADJ, 3, WALL>(maps, out, a, tile, ring, sig_sh[warp], bars[warp], lane, use); break;
        }
        if (!ok) break;
    }
}

template <typename T> static size_t layer2d_smem() { return L2Cfg<T>::smem(); }

int layer2d_box_rows() { return kL2CH; }
int layer2d_box_cols(int prec) { return prec == 32 ? L2Cfg<float>::COLS : L2Cfg<double>::COLS; }
int layer2d_tile_cols(int prec) { return prec == 32 ? L2Cfg<float>::OUT : L2Cfg<double>::OUT; }

template <typename T, bool ADJ, bool WALL>
static cudaError_t launch_l2w(const Maps6 &m, const Out6 &o, const Layer2DArgs &a, int grid, cudaStream_t st,
                              bool overlap)
{
    static bool done = false;
    const size_t sm = layer2d_smem<T>();
    if (!done) {
        cudaError_t e =
            cudaFuncSetAttribute(k_layer2d<T, ADJ, WALL>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        if (e != cudaSuccess) return e;
        done = true;
    }
    if (!overlap) {
        k_layer2d<T, ADJ, WALL><<<grid, 128, sm, st>>>(m, o, a);
        return cudaGetLastError();
    }
    return launch_pdl(k_layer2d<T, ADJ, WALL>, grid, 128, sm, st, true, m, o, a);
}

template <typename T, bool ADJ>
static cudaError_t launch_l2(const Maps6 &m, const Out6 &o, const Layer2DArgs &a, int grid, cudaStream_t st,
                             bool overlap)
{
    return a.g.wall ? launch_l2w<T, ADJ, true>(m, o, a, grid, st, overlap)
                    : launch_l2w<T, ADJ, false>(m, o, a, grid, st, overlap);
}

int layer2d_grid(int prec, int ntiles, int sm_count)
{
    const int need = (ntiles + 3) / 4;
    const int cap = (prec == 32 ? L2Cfg<float>::MINB : L2Cfg<double>::MINB) * sm_count;
    return need < cap ? need : cap;
}

cudaError_t launch_layer2d(int prec, bool adjoint, const CUtensorMap *tm, void *const *outp, const Layer2DArgs &a,
                           int grid, cudaStream_t st, bool overlap_previous)
{
    if (a.ntiles <= 0 || grid <= 0) return cudaSuccess;
    Maps6 m;
    Out6 o;
    for (int f = 0; f < 6; ++f) {
        m.m[f] = tm[f];
        o.p[f] = outp[f];
    }
    const bool ov = overlap_previous;
    if (prec == 32)
        return adjoint ? launch_l2<float, true>(m, o, a, grid, st, ov) : launch_l2<float, false>(m, o, a, grid, st, ov);
    return adjoint ? launch_l2<double, true>(m, o, a, grid, st, ov) : launch_l2<double, false>(m, o, a, grid, st, ov);
}

template <typename T, bool ADJ, int NC, int CH, int S, int MINB>
__global__ void __launch_bounds__(128, MINB)
    k_interior2d(const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmV,
                 T *__restrict__ Uo, T *__restrict__ Vo, const Interior2DArgs a)
{
    constexpr size_t WB = size_t(S) * 2 * CH * 32 * NC * sizeof(T);
    __shared__ __align__(8) uint64_t bars[4][S];
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *smem =
        smem_align128<unsigned char>(smem_dyn);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wbase = smem + warp * WB;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.queue[1 - a.parity] = 0;
    if (lane == 0) {
        prefetch_tmap(&tmU);
        prefetch_tmap(&tmV);
        for (int s = 0; s < S; ++s) mbar_init(&bars[warp][s], 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t use = 0;
    const int64_t xs0 = a.xr.lo & ~int64_t(3);
    const int64_t nrows = a.yr.hi - a.yr.lo + 1;
    const int R = a.rows > 0 ? a.rows : kI2Rows;
    const int rblocks = int((nrows + R - 1) / R);
    const int nstrips = int((a.xr.hi - xs0) / (30 * NC) + 1);
    const int n_items = nstrips * rblocks;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&a.queue[a.parity], 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        const int st = item / rblocks, rb = item - st * rblocks;
        const int64_t y0 = a.yr.lo + int64_t(rb) * R;
        const int64_t rem = a.yr.hi - y0 + 1;
        if (!interior2d_seg<T, ADJ, NC, CH, S>(&tmU, &tmV, Uo, Vo, a, xs0 + int64_t(30 * NC) * st, y0,
                                               int(rem < R ? rem : R), wbase, bars[warp], lane, use))
            break;
    }
    // When this launch overlapped the layer kernel, finish only after it: later work in the
    // stream then sees both halves of the step.  (Every layer CTA has started before this
    // kernel could, so the wait cannot block a layer CTA from running.)
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename T, bool ADJ, int NC, int CH, int S, int MINB> struct I2Kernel {
    static constexpr size_t smem() { return size_t(4) * S * 2 * CH * 32 * NC * sizeof(T) + 128; }
    static cudaError_t prep()
    {
        static bool done = false;
        if (done) return cudaSuccess;
        cudaError_t e = cudaFuncSetAttribute(k_interior2d<T, ADJ, NC, CH, S, MINB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem()));
        if (e == cudaSuccess) done = true;
        return e;
    }
    static int occupancy()
    {
        if (prep() != cudaSuccess) return 0;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_interior2d<T, ADJ, NC, CH, S, MINB>, 128, smem()) !=
            cudaSuccess)
            return 0;
        return n;
    }
    static cudaError_t launch(const CUtensorMap *tmU, const CUtensorMap *tmV, void *Uo, void *Vo,
                              const Interior2DArgs &a, int grid, cudaStream_t st, bool overlap_previous)
    {
        cudaError_t e = prep();
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(unsigned(grid));
        cfg.blockDim = dim3(128);
        cfg.dynamicSmemBytes = smem();
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = overlap_previous ? 1 : 0;
        return cudaLaunchKernelEx(&cfg, k_interior2d<T, ADJ, NC, CH, S, MINB>, *tmU, *tmV, (T *)Uo, (T *)Vo, a);
    }
};

template <typename T, bool ADJ, int BY, int NCH, int MINB> struct I2RKernel {
    static constexpr size_t smem() { return I2R<T, BY, NCH>::SMEM; }
    static cudaError_t prep()
    {
        static bool done = false;
        if (done) return cudaSuccess;
        cudaError_t e = cudaFuncSetAttribute(k_interior2d_rows<T, ADJ, BY, NCH, MINB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem()));
        if (e == cudaSuccess) done = true;
        return e;
    }
    static int occupancy()
    {
        if (prep() != cudaSuccess) return 0;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_interior2d_rows<T, ADJ, BY, NCH, MINB>, 32 * BY, smem()) !=
            cudaSuccess)
            return 0;
        return n;
    }
    static cudaError_t launch(const CUtensorMap *tmU, const CUtensorMap *tmV, void *Uo, void *Vo,
                              const Interior2DArgs &a, int grid, cudaStream_t st, bool overlap_previous)
    {
        cudaError_t e = prep();
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(unsigned(grid));
        cfg.blockDim = dim3(32 * BY);
        cfg.dynamicSmemBytes = smem();
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = overlap_previous ? 1 : 0;
        return cudaLaunchKernelEx(&cfg, k_interior2d_rows<T, ADJ, BY, NCH, MINB>, *tmU, *tmV, (T *)Uo, (T *)Vo, a);
    }
};

// dispatch over the variant tables (index v of kI2Vars32 / kI2Vars64)
template <bool ADJ, typename F> static auto with_i2(int prec, int v, F &&f)
{
    if (prec == 32) {
        switch (v) {
        case 0: return f(I2Kernel<float, ADJ, 4, 6, 3, 3>{});
        case 1: return f(I2RKernel<float, ADJ, 8, 8, 2>{});
        case 2: return f(I2RKernel<float, ADJ, 4, 8, 4>{});
        case 3: return f(I2Kernel<float, ADJ, 4, 6, 2, 4>{});
        default: return f(I2Kernel<float, ADJ, 8, 3, 3, 2>{});
        }
    }
    switch (v) {
    case 0: return f(I2RKernel<double, ADJ, 4, 8, 3>{});
    case 1: return f(I2RKernel<double, ADJ, 8, 4, 1>{});
    case 2: return f(I2Kernel<double, ADJ, 4, 6, 2, 2>{});
    default: return f(I2Kernel<double, ADJ, 4, 3, 3, 2>{});
    }
}

int interior2d_max_blocks_per_sm(int prec, bool adjoint, int v)
{
    auto occ = [](auto k) { return decltype(k)::occupancy(); };
    return adjoint ? with_i2<true>(prec, v, occ) : with_i2<false>(prec, v, occ);
}

cudaError_t launch_interior2d(int prec, bool adjoint, int v, const CUtensorMap *tmU, const CUtensorMap *tmV,
                              void *Uo, void *Vo, const Interior2DArgs &a, int grid, cudaStream_t st,
                              bool overlap_previous)
{
    if (a.xr.lo > a.xr.hi || a.yr.lo > a.yr.hi || grid <= 0) return cudaSuccess;
    auto go = [&](auto k) { return decltype(k)::launch(tmU, tmV, Uo, Vo, a, grid, st, overlap_previous); };
    return adjoint ? with_i2<true>(prec, v, go) : with_i2<false>(prec, v, go);
}

// Two-step interior kernel: persistent CTAs of 4 warps take ROWS-row strip segments of
// the shrunk run from the work queue, as k_interior2d does.
template <typename T, bool ADJ, int NC, int CH, int S, int MINB, int ROWS>
__global__ void __launch_bounds__(128, MINB)
    k_interior2d_tb2(const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmV,
                     T *__restrict__ Uo, T *__restrict__ Vo, const Interior2DArgs a)
{
    constexpr size_t WB = size_t(S) * 2 * CH * 32 * NC * sizeof(T);
    __shared__ __align__(8) uint64_t bars[4][S];
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *smem =
        smem_align128<unsigned char>(smem_dyn);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wbase = smem + warp * WB;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.queue[1 - a.parity] = 0;
    if (lane == 0) {
        prefetch_tmap(&tmU);
        prefetch_tmap(&tmV);
        for (int s = 0; s < S; ++s) mbar_init(&bars[warp][s], 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t use = 0;
    const int64_t xs0 = a.xr.lo & ~int64_t(3);
    const int64_t nrows = a.yr.hi - a.yr.lo + 1;
    constexpr int OUT = (32 - 2 * (4 / NC)) * NC;   // output columns per strip
    const int nstrips = int((a.xr.hi - xs0) / OUT + 1);
    // Items: every strip's first rows in ROWS-row segments, then its last rows in
    // SR-row segments, queued after all the long ones, so that the launch ends with about
    // two rounds of short items over all warps instead of a ragged round of long ones.
    constexpr int SR = ROWS / 4;
    const int64_t nwarps = int64_t(gridDim.x) * 4;
    int64_t small = int64_t(SR) * ((2 * nwarps + nstrips - 1) / nstrips);
    small = small < nrows ? small : nrows;
    const int64_t big = nrows - small;
    const int nbig = int((big + ROWS - 1) / ROWS), nsmall = int((small + SR - 1) / SR);
    const int items_big = nstrips * nbig, n_items = items_big + nstrips * nsmall;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&a.queue[a.parity], 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        int st;
        int64_t y0, cnt;
        if (item < items_big) {
            st = item / nbig;
            const int rb = item - st * nbig;
            y0 = int64_t(rb) * ROWS;
            cnt = big - y0 < ROWS ? big - y0 : ROWS;
        } else {
            const int i = item - items_big;
            st = i / nsmall;
            const int sb = i - st * nsmall;
            y0 = big + int64_t(sb) * SR;
            cnt = nrows - y0 < SR ? nrows - y0 : SR;
        }
        if (!interior2d_seg2<T, ADJ, NC, CH, S>(&tmU, &tmV, Uo, Vo, a, xs0 + int64_t(OUT) * st, a.yr.lo + y0,
                                           int(cnt), wbase, bars[warp], lane, use))
            break;
    }
    // finish only after the layer kernels of the same two steps (launched before this one)
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename T, bool ADJ, int NC, int CH, int S, int MINB, int ROWS> struct I2TKernel {
    static constexpr size_t smem() { return size_t(4) * S * 2 * CH * 32 * NC * sizeof(T) + 128; }
    static cudaError_t prep()
    {
        static bool done = false;
        if (done) return cudaSuccess;
        cudaError_t e = cudaFuncSetAttribute(k_interior2d_tb2<T, ADJ, NC, CH, S, MINB, ROWS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem()));
        if (e == cudaSuccess) done = true;
        return e;
    }
    static int occupancy()
    {
        if (prep() != cudaSuccess) return 0;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_interior2d_tb2<T, ADJ, NC, CH, S, MINB, ROWS>, 128,
                                                          smem()) != cudaSuccess)
            return 0;
        return n;
    }
    static cudaError_t launch(const CUtensorMap *tmU, const CUtensorMap *tmV, void *Uo, void *Vo,
                              const Interior2DArgs &a, int grid, cudaStream_t st, bool overlap_previous)
    {
        cudaError_t e = prep();
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(unsigned(grid));
        cfg.blockDim = dim3(128);
        cfg.dynamicSmemBytes = smem();
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = overlap_previous ? 1 : 0;
        return cudaLaunchKernelEx(&cfg, k_interior2d_tb2<T, ADJ, NC, CH, S, MINB, ROWS>, *tmU, *tmV, (T *)Uo, (T *)Vo, a);
    }
};

// Two-step variants (FP32 only: FP64 is bound by its arithmetic, not by HBM, so a second
// step per pass gains nothing there): rows per TMA box, ring stages, resident CTAs per
// SM, rows per work item.
struct I2TVar {
    int nc, ch, s, minb, rows;
};
constexpr I2TVar kI2TVars32[] = {{4, 6, 4, 2, 128}, {4, 3, 6, 2, 128}, {2, 3, 6, 3, 128}};
constexpr int kNI2TVars32 = sizeof(kI2TVars32) / sizeof(I2TVar);

template <bool ADJ, typename F> static auto with_i2t(int v, F &&f)
{
    switch (v) {
    case 0: return f(I2TKernel<float, ADJ, 4, 6, 4, 2, 128>{});
    case 1: return f(I2TKernel<float, ADJ, 4, 3, 6, 2, 128>{});
    default: return f(I2TKernel<float, ADJ, 2, 3, 6, 3, 128>{});
    }
}

int interior2d_tb2_variants(int prec) { return prec == 32 ? kNI2TVars32 : 0; }
int interior2d_tb2_box_rows(int prec, int v) { return prec == 32 ? kI2TVars32[v].ch : 0; }
int interior2d_tb2_box_cols(int prec, int v) { return prec == 32 ? 32 * kI2TVars32[v].nc : 0; }
int interior2d_tb2_max_blocks_per_sm(int prec, bool adjoint, int v)
{
    if (prec != 32) return 0;
    auto occ = [](auto k) { return decltype(k)::occupancy(); };
    return adjoint ? with_i2t<true>(v, occ) : with_i2t<false>(v, occ);
}

cudaError_t launch_interior2d_tb2(int prec, bool adjoint, int v, const CUtensorMap *tmU, const CUtensorMap *tmV,
                                  void *Uo, void *Vo, const Interior2DArgs &a, int grid, cudaStream_t st,
                                  bool overlap_previous)
{
    if (prec != 32 || v < 0 || v >= kNI2TVars32) return cudaErrorInvalidValue;
    if (a.xr.lo > a.xr.hi || a.yr.lo > a.yr.hi || grid <= 0) return cudaSuccess;
    auto go = [&](auto k) { return decltype(k)::launch(tmU, tmV, Uo, Vo, a, grid, st, overlap_previous); };
    return adjoint ? with_i2t<true>(v, go) : with_i2t<false>(v, go);
}

// ------------------------------------------------------------------------------------
// Batched 2D step: the per-item code above, with the grid of each work item read from a
// descriptor table in device memory.  Interior items of all grids form one queue (the
// owning grid found by binary search over item_off); layer tiles of all grids form one
// list.  Variants differ in the warp-streaming shape and in the rows per work item.
// ------------------------------------------------------------------------------------
struct BVar {
    int nc, ch, s, minb, rows;
};
constexpr BVar kB32[] = {{4, 6, 3, 3, 64}, {4, 6, 2, 4, 64}, {8, 3, 3, 2, 64}, {4, 6, 3, 3, 32}};
constexpr BVar kB64[] = {{4, 6, 2, 2, 64}, {4, 3, 3, 2, 64}, {4, 6, 2, 2, 32}};
constexpr int kNB32 = sizeof(kB32) / sizeof(BVar), kNB64 = sizeof(kB64) / sizeof(BVar);

int batch2d_variants(int prec) { return prec == 32 ? kNB32 : kNB64; }
static const BVar &bvar(int prec, int v) { return prec == 32 ? kB32[v] : kB64[v]; }
int batch2d_box_cols(int prec, int v) { return 32 * bvar(prec, v).nc; }
int batch2d_box_rows(int prec, int v) { return bvar(prec, v).ch; }
int batch2d_item_rows(int prec, int v) { return bvar(prec, v).rows; }
int batch2d_strip_cols(int prec, int v) { return 30 * bvar(prec, v).nc; }

template <typename T, bool ADJ, int NC, int CH, int S, int MINB, int ROWS>
__global__ void __launch_bounds__(128, MINB) k_interior2d_batch(const Batch2DArgs b)
{
    constexpr size_t WB = size_t(S) * 2 * CH * 32 * NC * sizeof(T);
    __shared__ __align__(8) uint64_t bars[4][S];
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *smem =
        smem_align128<unsigned char>(smem_dyn);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wbase = smem + warp * WB;
    if (blockIdx.x == 0 && threadIdx.x == 0) b.queue[1 - b.parity] = 0;
    if (lane == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[warp][s], 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t use = 0;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&b.queue[b.parity], 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= b.n_items) break;
        int lo = 0, hi = b.ngrid - 1;   // last grid whose first item is <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (b.item_off[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const GridDesc2 &d = b.desc[lo];
        const Interior2DArgs a = d.in;   // a local copy: stores to the fields cannot alias it
        const int k = item - b.item_off[lo];
        const int st = k / d.rblocks, rb = k - st * d.rblocks;
        const int64_t y0 = a.yr.lo + int64_t(rb) * ROWS;
        const int64_t rem = a.yr.hi - y0 + 1;
        const int64_t xs = (a.xr.lo & ~int64_t(3)) + int64_t(30 * NC) * st;
        if (!interior2d_seg<T, ADJ, NC, CH, S>(&d.tm_int[b.parity][0], &d.tm_int[b.parity][1],
                                               static_cast<T *>(d.out[b.parity][0]),
                                               static_cast<T *>(d.out[b.parity][1]), a, xs, y0,
                                               int(rem < ROWS ? rem : ROWS), wbase, bars[warp], lane, use))
            break;
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename T, bool ADJ, bool WALL>
__global__ void __launch_bounds__(128, L2Cfg<T>::MINB) k_layer2d_batch(const Batch2DArgs b)
{
    constexpr int S = L2Cfg<T>::S, WE = L2Cfg<T>::WE;
    __shared__ __align__(8) uint64_t bars[4][S];
    __shared__ T sig_sh[4][2 * kL2SigRows];
    extern __shared__ unsigned char smem_dyn[];
    T *smem = smem_align128<T>(smem_dyn);
    allow_dependent_launch();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        for (int k = 0; k < S; ++k) mbar_init(&bars[warp][k], 1);
        fence_mbar_init();
    }
    // launched early (second layer pass of a two-step block): the inputs are the previous
    // kernel's outputs; a no-op for a launch without programmatic overlap
    wait_prerequisite_grid();
    __syncwarp();
    T *ring = smem + warp * WE;
    uint32_t use = 0;
    // the second pass of a two-step block has its own counters (it starts before the first
    // pass has finished with its own)
    int *const lq = b.queue + (b.pass == 2 ? 4 : 2);
    const int qp = b.pass == 2 ? b.qparity : b.parity;
    if (blockIdx.x == 0 && threadIdx.x == 0) lq[1 - qp] = 0;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&lq[qp], 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= b.ntiles) break;
        const LayerTile tile = b.tiles[item];
        const GridDesc2 &d = b.desc[b.tile_grid[item]];
        const Maps6 &maps = *reinterpret_cast<const Maps6 *>(b.pass == 2 ? &d.tm_mid[0] : &d.tm_lay[b.parity][0]);
        const Out6 out = *reinterpret_cast<const Out6 *>(b.pass == 1 ? &d.mid[0] : &d.out[b.parity][0]);
        const Layer2DArgs la = d.lay;   // local copies: stores to the fields cannot alias them
        bool ok;
        switch (tile.flags & 3) {
        case 0: ok = layer2d_item<T, ADJ, 0, WALL>(maps, out, la, tile, ring, sig_sh[warp], bars[warp], lane, use); break;
        case 1: ok = layer2d_item<T, ADJ, 1, WALL>(maps, out, la, tile, ring, sig_sh[warp], bars[warp], lane, use); break;
        case 2: ok = layer2d_item<T, ADJ, 2, WALL>(maps, out, la, tile, ring, sig_sh[warp], bars[warp], lane, use); break;
        default: ok = layer2d_item<T, ADJ, 3, WALL>(maps, out, la, tile, ring, sig_sh[warp], bars[warp], lane, use); break;
        }
        if (!ok) break;
    }
}

template <typename T, int NC, int CH, int S, int MINB, int ROWS> struct BKernel {
    static constexpr size_t smem() { return size_t(4) * S * 2 * CH * 32 * NC * sizeof(T) + 128; }
    static auto fn() { return k_interior2d_batch<T, false, NC, CH, S, MINB, ROWS>; }
    static cudaError_t prep()
    {
        static bool done = false;
        if (done) return cudaSuccess;
        cudaError_t e = cudaFuncSetAttribute(fn(), cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem()));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_layer2d_batch<T, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(layer2d_smem<T>()));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_layer2d_batch<T, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(layer2d_smem<T>()));
        if (e == cudaSuccess) done = true;
        return e;
    }
    static int occupancy()
    {
        if (prep() != cudaSuccess) return 0;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn(), 128, smem()) != cudaSuccess) return 0;
        return n;
    }
    static cudaError_t launch(const Batch2DArgs &a, int grid, cudaStream_t st, bool overlap_previous)
    {
        cudaError_t e = prep();
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(unsigned(grid));
        cfg.blockDim = dim3(128);
        cfg.dynamicSmemBytes = smem();
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = overlap_previous ? 1 : 0;
        return cudaLaunchKernelEx(&cfg, fn(), a);
    }
};

// dispatch over kB32 / kB64
template <typename F> static auto with_b2(int prec, int v, F &&f)
{
    if (prec == 32) {
        switch (v) {
        case 0: return f(BKernel<float, 4, 6, 3, 3, 64>{});
        case 1: return f(BKernel<float, 4, 6, 2, 4, 64>{});
        case 2: return f(BKernel<float, 8, 3, 3, 2, 64>{});
        default: return f(BKernel<float, 4, 6, 3, 3, 32>{});
        }
    }
    switch (v) {
    case 0: return f(BKernel<double, 4, 6, 2, 2, 64>{});
    case 1: return f(BKernel<double, 4, 3, 3, 2, 64>{});
    default: return f(BKernel<double, 4, 6, 2, 2, 32>{});
    }
}

int batch2d_interior_blocks_per_sm(int prec, int v)
{
    return with_b2(prec, v, [](auto k) { return decltype(k)::occupancy(); });
}

cudaError_t launch_batch2d_interior(int prec, int v, const Batch2DArgs &a, int grid, cudaStream_t st,
                                    bool overlap_previous)
{
    if (a.n_items <= 0 || grid <= 0) return cudaSuccess;
    return with_b2(prec, v, [&](auto k) { return decltype(k)::launch(a, grid, st, overlap_previous); });
}

cudaError_t launch_batch2d_layer(int prec, const Batch2DArgs &a, int grid, bool wall, cudaStream_t st,
                                 bool overlap_previous)
{
    if (a.ntiles <= 0 || grid <= 0) return cudaSuccess;
    cudaError_t e = with_b2(prec, 0, [](auto k) { return decltype(k)::prep(); });
    if (e != cudaSuccess) return e;
    const bool ov = overlap_previous;
    if (prec == 32) {
        if (wall) return launch_pdl(k_layer2d_batch<float, false, true>, grid, 128, layer2d_smem<float>(), st, ov, a);
        return launch_pdl(k_layer2d_batch<float, false, false>, grid, 128, layer2d_smem<float>(), st, ov, a);
    }
    if (wall) return launch_pdl(k_layer2d_batch<double, false, true>, grid, 128, layer2d_smem<double>(), st, ov, a);
    return launch_pdl(k_layer2d_batch<double, false, false>, grid, 128, layer2d_smem<double>(), st, ov, a);
}

// ------------------------------------------------------------------------------------
// Batched two-step interior kernel: interior2d_seg2 over the shrunk runs of all grids, one
// queue of ROWS-row strip segments (owning grid by binary search over item_off).
// ------------------------------------------------------------------------------------
template <typename T, int NC, int CH, int S, int MINB, int ROWS>
__global__ void __launch_bounds__(128, MINB) k_interior2d_tb2_batch(const Batch2DArgs b)
{
    constexpr size_t WB = size_t(S) * 2 * CH * 32 * NC * sizeof(T);
    constexpr int OUT = (32 - 2 * (4 / NC)) * NC;
    __shared__ __align__(8) uint64_t bars[4][S];
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *smem =
        smem_align128<unsigned char>(smem_dyn);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wbase = smem + warp * WB;
    if (blockIdx.x == 0 && threadIdx.x == 0) b.queue[1 - b.parity] = 0;
    if (lane == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[warp][s], 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t use = 0;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&b.queue[b.parity], 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= b.n_items) break;
        int lo = 0, hi = b.ngrid - 1;   // last grid whose first item is <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (b.item_off[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const GridDesc2 &d = b.desc[lo];
        const Interior2DArgs a = d.in2;   // a local copy: stores to the fields cannot alias it
        const int k = item - b.item_off[lo];
        const int st = k / d.rblocks2, rb = k - st * d.rblocks2;
        const int64_t y0 = a.yr.lo + int64_t(rb) * ROWS;
        const int64_t rem = a.yr.hi - y0 + 1;
        const int64_t xs = (a.xr.lo & ~int64_t(3)) + int64_t(OUT) * st;
        if (!interior2d_seg2<T, false, NC, CH, S>(&d.tm_tb[b.parity][0], &d.tm_tb[b.parity][1],
                                           static_cast<T *>(d.out[b.parity][0]), static_cast<T *>(d.out[b.parity][1]),
                                           a, xs, y0, int(rem < ROWS ? rem : ROWS), wbase, bars[warp], lane, use))
            break;
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename T, int NC, int CH, int S, int MINB, int ROWS> struct BTKernel {
    static constexpr size_t smem() { return size_t(4) * S * 2 * CH * 32 * NC * sizeof(T) + 128; }
    static auto fn() { return k_interior2d_tb2_batch<T, NC, CH, S, MINB, ROWS>; }
    static cudaError_t prep()
    {
        static bool done = false;
        if (done) return cudaSuccess;
        cudaError_t e = cudaFuncSetAttribute(fn(), cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem()));
        if (e == cudaSuccess) done = true;
        return e;
    }
    static int occupancy()
    {
        if (prep() != cudaSuccess) return 0;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn(), 128, smem()) != cudaSuccess) return 0;
        return n;
    }
    static cudaError_t launch(const Batch2DArgs &a, int grid, cudaStream_t st, bool overlap_previous)
    {
        cudaError_t e = prep();
        if (e != cudaSuccess) return e;
        return launch_pdl(fn(), grid, 128, smem(), st, overlap_previous, a);
    }
};

struct BTVar {
    int nc, ch, s, minb, rows;
};
constexpr BTVar kBT32[] = {{4, 3, 6, 2, 64}, {4, 3, 6, 2, 128}};
constexpr int kNBT32 = sizeof(kBT32) / sizeof(BTVar);

template <typename F> static auto with_bt2(int v, F &&f)
{
    switch (v) {
    case 0: return f(BTKernel<float, 4, 3, 6, 2, 64>{});
    default: return f(BTKernel<float, 4, 3, 6, 2, 128>{});
    }
}

int batch2d_tb2_variants(int prec) { return prec == 32 ? kNBT32 : 0; }
int batch2d_tb2_box_cols(int prec, int v) { return prec == 32 ? 32 * kBT32[v].nc : 0; }
int batch2d_tb2_box_rows(int prec, int v) { return prec == 32 ? kBT32[v].ch : 0; }
int batch2d_tb2_item_rows(int prec, int v) { return prec == 32 ? kBT32[v].rows : 0; }
int batch2d_tb2_strip_cols(int prec, int v) { return prec == 32 ? (32 - 2 * (4 / kBT32[v].nc)) * kBT32[v].nc : 0; }
int batch2d_tb2_blocks_per_sm(int prec, int v)
{
    if (prec != 32) return 0;
    return with_bt2(v, [](auto k) { return decltype(k)::occupancy(); });
}

cudaError_t launch_batch2d_tb2(int prec, int v, const Batch2DArgs &a, int grid, cudaStream_t st, bool overlap_previous)
{
    if (prec != 32 || v < 0 || v >= kNBT32) return cudaErrorInvalidValue;
    if (a.n_items <= 0 || grid <= 0) return cudaSuccess;
    return with_bt2(v, [&](auto k) { return decltype(k)::launch(a, grid, st, overlap_previous); });
}

}  // namespace pml
