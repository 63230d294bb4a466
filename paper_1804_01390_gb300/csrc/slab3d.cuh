// 3D layer frame by slab tiles (FP32): the z-streaming Horner pipeline of one RK4 step
// with the full operator of Eq. 3, in tiles whose halo depends on which axes carry
// damping.  Included by step3d.cu (periodic box) and layer3d_wall.cu (walls).
//
// Halo per axis.  Along an axis whose aux fields are inactive in a tile's reach (no
// damping term within 4 vertices of its outputs), the operator couples vertices only
// through the Laplacian row of V, and U' = V is local.  So along that axis a value of
// U or V at level k of the Horner form y + dt A(y + dt/2 A(y + dt/3 A(y + dt/4 A y)))
// depends on level k + 1 within distance 1 only every second application: the outputs
// need U, V of the input within distance 2 (Phi, Psi of the other axes within 1), not 4.
// The tile region is therefore the outputs widened by 4 along active axes and by 2 along
// inactive ones; intermediate values beyond that reach are computed but never feed an
// output.
//
// Layout.  A CTA owns a region of RX x RY columns (x, y), two adjacent columns per thread
// (packed FP32x2 arithmetic), and streams z one plane per iteration: when input plane p
// has landed, level 4 produces plane p-1, level 3 plane p-2, level 2 plane p-3 and level
// 1 (the output) plane p-4.  A thread keeps its own columns' level values of three
// consecutive planes in registers (its z neighbours); x and y neighbours come from one
// shared-memory plane per level, double-buffered by plane parity, written one iteration
// before they are read; one block barrier per plane.  Input planes arrive by TMA into a
// ring of S slots (one box of RX x RY per field): planes p-4 .. p are read in iteration p,
// the next two are in flight.
#ifndef PML_SLAB3D_CUH_
#define PML_SLAB3D_CUH_

#include <type_traits>

#include "common.cuh"
#include "layer3d.cuh"

namespace pml {

// Shape of the tiles of class MASK (bit a: aux fields of axis a active): region columns
// RX x RY and the halos HX, HY (4 along an active axis, 2 otherwise); the z halo is 4.
template <int MASK> struct Slab {
    static constexpr int AX = MASK & 1, AY = (MASK >> 1) & 1, AZ = (MASK >> 2) & 1;
    static constexpr int NAX = AX + AY + AZ;
    static constexpr int NF = 2 + 2 * NAX;
    static constexpr int HX = AX ? 4 : 2, HY = AY ? 4 : 2;
    static constexpr int RX = AX ? 36 : (AY && NAX == 1 ? 28 : 32);
    // rows: as many as the shared memory of 13 planes per field (NF = 4: up to ~1100
    // columns, NF = 6: ~740, NF = 8: ~550) and the registers of one CTA per SM allow
    // without spilling; the y-active one-axis class covers a 25-row layer slab with one tile;
    // the x-active one takes 21 rows (378 threads, 152 registers) rather than 26 (468
    // threads, 128 registers with spills): 17 % more halo rows, but no spills
    static constexpr int RY = NF == 2 ? 32 : NF == 4 ? (AY ? 33 : (AX ? 21 : 32)) : NF == 6 ? (AX ? 18 : 20) : 14;
    static constexpr int TPR = RX / 2;                    // threads per region row
    static constexpr int NT = TPR * RY;                   // threads
    // registers per thread of one resident CTA: the warps spread over the SM's four
    // sub-partitions, each with 16384 registers, allocated in 8-register steps per thread
    static constexpr int WARPS_PER_SUB = ((NT + 31) / 32 + 3) / 4;
    static constexpr int MAXREG_ = 16384 / (32 * WARPS_PER_SUB) / 8 * 8;
    static constexpr int MAXREG = MAXREG_ > 248 ? 248 : MAXREG_;
    static constexpr int PLS = (RX * RY + 31) / 32 * 32;  // field plane stride (128-byte TMA destinations)
    static constexpr int S = 7;                           // input plane slots (p-4 .. p resident, two in flight)
    static constexpr size_t SMEM = size_t(S + 6) * NF * PLS * sizeof(float) + 128;
    static_assert(SMEM <= 227 * 1024 - 1024, "slab tile exceeds shared memory");
    static_assert(RX - 2 * HX > 0 && RY - 2 * HY > 0, "slab tile without outputs");
};
constexpr int kSlabMaxZ = 128;    // most output planes of one slab work item

// Packed pairs of adjacent columns (each half rounds exactly like the scalar operation).
struct Pf {
    using V = float2;
    static __device__ __forceinline__ V bc(float a) { return make_float2(a, a); }
    static __device__ __forceinline__ V mk(float a, float b) { return make_float2(a, b); }
    static __device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ V sub(V a, V b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
    static __device__ __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ V sel(V m, V x) { return make_float2(m.x != 0.f ? x.x : 0.f, m.y != 0.f ? x.y : 0.f); }
    static __device__ __forceinline__ V ld(const float *p) { return *reinterpret_cast<const float2 *>(p); }
    static __device__ __forceinline__ void st(float *p, V v) { *reinterpret_cast<float2 *>(p) = v; }
};

// local field f of class MASK -> global field id (0 U, 1 V, 2 + 2a Phi_a, 3 + 2a Psi_a)
template <int MASK> __device__ __forceinline__ constexpr int slab_gid(int f)
{
    if (f < 2) return f;
    int k = (f - 2) >> 1;
    for (int a = 0; a < 3; ++a)
        if ((MASK >> a) & 1) {
            if (k == 0) return 2 + 2 * a + ((f - 2) & 1);
            --k;
        }
    return 0;
}
template <int MASK> __device__ __forceinline__ constexpr int slab_axis(int k)   // k-th active axis
{
    for (int a = 0; a < 3; ++a)
        if ((MASK >> a) & 1) {
            if (k == 0) return a;
            --k;
        }
    return 0;
}

struct SlabSig {
    float2 si[3], sm[3];   // sigma_a[i_a], sigma_a[i_a - 1] of the thread's two columns
    float2 mi[3], mm[3];   // 1 where sigma_a[i_a] (sigma_a[i_a - 1]) != 0, else 0: Phi_a (Psi_a)
                           // lives there; elsewhere it stays zero
};

// A z (or A^T z) at the thread's two columns; N(f, d): local field f at direction d
// (0 centre, 1 x-, 2 x+, 3 y-, 4 y+, 5 z-, 6 z+).
template <bool ADJ, int MASK, typename Get>
__device__ __forceinline__ void slab_apply(const Get &N, const SlabSig &s, float2 ih, float2 ih2, float2 i2h,
                                           float2 *o)
{
    using P = Pf;
    constexpr int NAX = Slab<MASK>::NAX;
    const float2 m2 = P::bc(-2.f), mhalf = P::bc(-0.5f);
    if (!ADJ) {
        const float2 U0 = N(0, 0);
        float2 lap = P::fma(m2, U0, P::add(N(0, 2), N(0, 1)));
        lap = P::add(lap, P::fma(m2, U0, P::add(N(0, 4), N(0, 3))));
        lap = P::add(lap, P::fma(m2, U0, P::add(N(0, 6), N(0, 5))));
        float2 aV = P::mul(lap, ih2);
        o[0] = N(1, 0);
#pragma unroll
        for (int k = 0; k < NAX; ++k) {
            const int ax = slab_axis<MASK>(k), fp = 2 + 2 * k, fq = 3 + 2 * k, dm = 1 + 2 * ax, dp = 2 + 2 * ax;
            const float2 si = s.si[ax], sm = s.sm[ax];
            const float2 phm = N(fp, dm), psp = N(fq, dp);
            aV = P::fma(P::sub(P::mul(si, psp), P::mul(sm, phm)), ih, aV);
            const float2 ndU = P::mul(P::sub(N(0, dm), N(0, dp)), i2h);   // -(U(+) - U(-)) / 2h
            o[fp] = P::mul(s.mi[ax], P::fma(mhalf, P::fma(sm, phm, P::mul(si, N(fp, 0))), ndU));
            o[fq] = P::mul(s.mm[ax], P::fma(mhalf, P::fma(sm, N(fq, 0), P::mul(si, psp)), ndU));
        }
        o[1] = aV;
    } else {
        const float2 V0 = N(1, 0);
        float2 lap = P::fma(m2, V0, P::add(N(1, 2), N(1, 1)));
        lap = P::add(lap, P::fma(m2, V0, P::add(N(1, 4), N(1, 3))));
        lap = P::add(lap, P::fma(m2, V0, P::add(N(1, 6), N(1, 5))));
        float2 aU = P::mul(lap, ih2);
        o[1] = N(0, 0);
#pragma unroll
        for (int k = 0; k < NAX; ++k) {
            const int ax = slab_axis<MASK>(k), fp = 2 + 2 * k, fq = 3 + 2 * k, dm = 1 + 2 * ax, dp = 2 + 2 * ax;
            const float2 si = s.si[ax], sm = s.sm[ax];
            aU = P::fma(P::add(P::sub(N(fp, dp), N(fp, dm)), P::sub(N(fq, dp), N(fq, dm))), i2h, aU);
            // -si V(+)/h - si/2 (Phi(+) + Phi),  sm V(-)/h - sm/2 (Psi + Psi(-))
            o[fp] = P::mul(si, P::fma(mhalf, P::add(N(fp, dp), N(fp, 0)), P::mul(P::bc(-1.f), P::mul(N(1, dp), ih))));
            o[fq] = P::mul(sm, P::fma(mhalf, P::add(N(fq, 0), N(fq, dm)), P::mul(N(1, dm), ih)));
        }
        o[0] = aU;
    }
}

struct SlabMaps {
    CUtensorMap m[8];   // by global field id, box RX x RY x 1 of the class
};

template <int MASK, bool WALL>
__device__ __forceinline__ void slab_issue(float *slot, const SlabMaps &maps, int32_t bx, int32_t by, int64_t zin,
                                           const Geom &g, uint64_t *bar)
{
    using SH = Slab<MASK>;
    int64_t z = zin;
    if (!WALL) z += z < 0 ? g.T[2] : (z >= g.T[2] ? -g.T[2] : 0);   // a wall keeps the zero ghost planes
    mbar_arrive_expect_tx(bar, uint32_t(SH::NF * SH::RX * SH::RY * sizeof(float)));
#pragma unroll
    for (int f = 0; f < SH::NF; ++f)
        tma_load_3d(slot + f * SH::PLS, &maps.m[slab_gid<MASK>(f)], bx, by, int32_t(z + G), bar);
}

// One tile: region origin (tile.x0, tile.y0) (x0 a multiple of 4), outputs in
// [xlo, xhi] x [ylo, yhi] x [zlo, zhi] (z unwrapped across the periodic seam).
template <bool ADJ, int MASK, bool WALL>
__global__ void __maxnreg__(Slab<MASK>::MAXREG)
    k_slab3d(const __grid_constant__ SlabMaps maps, const Out8 out, const Layer3DArgs a, int tile_base)
{
    using SH = Slab<MASK>;
    using P = Pf;
    constexpr int NF = SH::NF, RX = SH::RX, RY = SH::RY, TPR = SH::TPR, NT = SH::NT, PLS = SH::PLS, S = SH::S;
    constexpr int FPL = NF * PLS;   // one plane of all fields
    extern __shared__ unsigned char smem_dyn[];
    float *stage = smem_align128<float>(smem_dyn);
    float *lvl = stage + S * FPL;   // [3 levels: 4, 3, 2][2 plane parities][NF][PLS]
    __shared__ float sz[kSlabMaxZ + 10], mz[kSlabMaxZ + 10];
    __shared__ __align__(8) uint64_t bars[S];

    allow_dependent_launch();
    const LayerTile tile = a.tiles[tile_base + blockIdx.x];
    const Geom &g = a.g;
    const int tid = threadIdx.x, cp = tid % TPR, r = tid / TPR;
    const int e = r * RX + 2 * cp;   // the thread's first column in a plane
    const int nout = tile.zhi - tile.zlo + 1;
    const int nin = nout + 8;
    const int64_t zin0 = int64_t(tile.zlo) - 4;
    const int32_t bx = tile.x0 + G, by = tile.y0 + G;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
        const int npro = nin < S ? nin : S;
        for (int p = 0; p < npro; ++p) slab_issue<MASK, WALL>(stage + p * FPL, maps, bx, by, zin0 + p, g, &bars[p]);
    }
    // sigma of the thread's columns (x), its row (y) and of the item's planes (z)
    const int64_t gx = int64_t(tile.x0) + 2 * cp, gy = int64_t(tile.y0) + r;
    SlabSig sg;
    {
        const float *sgx = static_cast<const float *>(a.sig[0]);
        const float *sgy = static_cast<const float *>(a.sig[1]);
        const int64_t T0 = g.T[0], T1 = g.T[1];
        auto wx = [&](int64_t i) { i %= T0; return i < 0 ? i + T0 : i; };
        auto wy = [&](int64_t i) { i %= T1; return i < 0 ? i + T1 : i; };
        const float s0 = sgx[wx(gx - 1)], s1 = sgx[wx(gx)], s2 = sgx[wx(gx + 1)];
        auto m = [](float v) { return v != 0.f ? 1.f : 0.f; };
        sg.si[0] = P::mk(s1, s2);
        sg.sm[0] = P::mk(s0, s1);
        sg.mi[0] = P::mk(m(s1), m(s2));
        sg.mm[0] = P::mk(m(s0), m(s1));
        const float y0 = sgy[wy(gy - 1)], y1 = sgy[wy(gy)];
        sg.si[1] = P::bc(y1);
        sg.sm[1] = P::bc(y0);
        sg.mi[1] = P::bc(m(y1));
        sg.mm[1] = P::bc(m(y0));
        sg.si[2] = sg.sm[2] = sg.mi[2] = sg.mm[2] = P::bc(0.f);
    }
    for (int k = tid; k <= nin; k += NT) {   // sz[k] = sigma_z[zin0 - 1 + k], mz[k] its support
        const float *sgz = static_cast<const float *>(a.sig[2]);
        int64_t i = (zin0 - 1 + k) % g.T[2];
        if (i < 0) i += g.T[2];
        sz[k] = sgz[i];
        mz[k] = sgz[i] != 0.f ? 1.f : 0.f;
    }
    __syncthreads();

    const LayerConstT<float> &lk = lconst_of<float>(a.k);
    const float2 ih = P::bc(lk.ih), ih2 = P::bc(lk.ih2), i2h = P::bc(lk.i2h), c4 = P::bc(lk.c4), c3 = P::bc(lk.c3),
                 c2 = P::bc(lk.c2), c1 = P::bc(lk.c1);
    // neighbour offsets in a plane (edge threads read themselves: their values are halo)
    const int oxm = cp > 0 ? e - 1 : e, oxp = cp < TPR - 1 ? e + 2 : e + 1;
    const int oym = r > 0 ? e - RX : e, oyp = r < RY - 1 ? e + RX : e;
    auto zsig = [&](int q) {   // plane zin0 + q of the item
        SlabSig s2 = sg;
        if (Slab<MASK>::AZ) {
            s2.si[2] = P::bc(sz[q + 1]);
            s2.sm[2] = P::bc(sz[q]);
            s2.mi[2] = P::bc(mz[q + 1]);
            s2.mm[2] = P::bc(mz[q]);
        }
        return s2;
    };
    // with a wall every stage value beyond the ends of the box is zero
    float2 xymask = P::bc(1.f);
    if (WALL) {
        const bool iny = gy >= 0 && gy < g.T[1];
        xymask = P::mk((iny && gx >= 0 && gx < g.T[0]) ? 1.f : 0.f, (iny && gx + 1 >= 0 && gx + 1 < g.T[0]) ? 1.f : 0.f);
    }
    auto keep = [&](float2 v, int q) -> float2 {
        if (!WALL) return v;
        return (zin0 + q >= 0 && zin0 + q < g.T[2]) ? P::sel(xymask, v) : P::bc(0.f);
    };
    // outputs of this thread's columns, and the offsets of their ghost images (a vertex
    // within G of the box edge is also stored at its periodic image in the ghost ring; 0:
    // no image, and with a wall the ring stays zero)
    const bool oy = gy >= tile.ylo && gy <= tile.yhi;
    const bool ox0 = oy && gx >= tile.xlo && gx <= tile.xhi, ox1 = oy && gx + 1 >= tile.xlo && gx + 1 <= tile.xhi;
    auto img = [&](int64_t c, int a) -> int64_t {
        if (g.wrap[a] == 0) return 0;
        return c < G ? g.wrap[a] : (c >= g.T[a] - G ? -g.wrap[a] : 0);
    };
    const int64_t dx0 = img(gx, 0), dx1 = img(gx + 1, 0), dy = img(gy, 1) * g.P;
    const int64_t off_xy = g.origin + gx + gy * g.P;

    // x and y neighbours of local field f at a shared plane `pl`, centre c (the thread's own)
    auto xm = [&](const float *pl, int f, float2 c) { return P::mk(pl[f * PLS + oxm], c.x); };
    auto xp = [&](const float *pl, int f, float2 c) { return P::mk(c.y, pl[f * PLS + oxp]); };
    auto ym = [&](const float *pl, int f) { return P::ld(pl + f * PLS + oym); };
    auto yp = [&](const float *pl, int f) { return P::ld(pl + f * PLS + oyp); };

    float2 z4r[3][NF], z3r[3][NF], z2r[3][NF];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int f = 0; f < NF; ++f) z4r[k][f] = z3r[k][f] = z2r[k][f] = P::bc(0.f);

    bool ok = true;
    int pfail = nin;   // first plane whose wait gave up
    // One iteration per input plane p.  Every shared-memory read of an iteration sees planes
    // written in earlier iterations (the level planes alternate by plane parity), so in the
    // x- and z-active classes (and the class without damping) the stores of levels 4, 3 and
    // 2 are made after all four levels are formed: the loads of a later level then need not
    // wait behind the stores of an earlier one, and their STEADY iterations (p >= 8: every
    // level has its planes) run as one block without the start-up guards.  The other
    // classes keep one guarded body that stores each level at once (a second body, or values
    // held to the end, spill there).
    // Level planes: [3 levels: 4, 3, 2][2 plane parities][NF][PLS].
    auto store_level = [&](int lv, int q, const float2 *v) {
        float *zo = lvl + ((lv * 2 + (q & 1)) * NF) * PLS;
#pragma unroll
        for (int f = 0; f < NF; ++f) P::st(zo + f * PLS + e, v[f]);
    };
    auto iter = [&](const int p, auto phc, auto stc) -> bool {
        constexpr int PH = decltype(phc)::value;   // p mod 3: position in the register rings
        constexpr bool STEADY = decltype(stc)::value;
        constexpr bool DEFER = SH::NAX <= 1 && !SH::AY;   // the other classes store each level at once
        const int sp = p % S;   // slot of input plane p; plane p - k sits in slot (sp - k) mod S
        auto slot = [&](int k) { return sp - k < 0 ? sp - k + S : sp - k; };
        if (p < nin) {
            if (!mbar_wait(&bars[sp], (p / S) & 1, a.err, 7, a.wait_ns)) ok = false;
            if (ok) {
                // level 4 at plane q = p-1 from the input planes (stage slots)
                if (STEADY || p >= 2) {
                    const int q = p - 1;
                    const float *Pc = stage + slot(1) * FPL, *Pm = stage + slot(2) * FPL, *Pp = stage + sp * FPL;
                    float2 cen[NF];
#pragma unroll
                    for (int f = 0; f < NF; ++f) cen[f] = P::ld(Pc + f * PLS + e);
                    auto N = [&](int f, int d) -> float2 {
                        switch (d) {
                        case 0: return cen[f];
                        case 1: return xm(Pc, f, cen[f]);
                        case 2: return xp(Pc, f, cen[f]);
                        case 3: return ym(Pc, f);
                        case 4: return yp(Pc, f);
                        case 5: return P::ld(Pm + f * PLS + e);
                        default: return P::ld(Pp + f * PLS + e);
                        }
                    };
                    float2 rr[NF];
                    slab_apply<ADJ, MASK>(N, zsig(q), ih, ih2, i2h, rr);
#pragma unroll
                    for (int f = 0; f < NF; ++f) z4r[(PH + 2) % 3][f] = keep(P::fma(c4, rr[f], cen[f]), q);
                    if (!DEFER) store_level(0, q, z4r[(PH + 2) % 3]);
                }
                // level 3 at plane q = p-2 (z neighbours: own ring; x, y: level-4 plane)
                if (STEADY || p >= 4) {
                    const int q = p - 2;
                    const float *zb = lvl + ((0 * 2 + (q & 1)) * NF) * PLS;
                    auto N = [&](int f, int d) -> float2 {
                        switch (d) {
                        case 0: return z4r[(PH + 1) % 3][f];
                        case 1: return xm(zb, f, z4r[(PH + 1) % 3][f]);
                        case 2: return xp(zb, f, z4r[(PH + 1) % 3][f]);
                        case 3: return ym(zb, f);
                        case 4: return yp(zb, f);
                        case 5: return z4r[PH][f];
                        default: return z4r[(PH + 2) % 3][f];
                        }
                    };
                    float2 rr[NF];
                    slab_apply<ADJ, MASK>(N, zsig(q), ih, ih2, i2h, rr);
                    const float *Y = stage + slot(2) * FPL;
#pragma unroll
                    for (int f = 0; f < NF; ++f)
                        z3r[(PH + 1) % 3][f] = keep(P::fma(c3, rr[f], P::ld(Y + f * PLS + e)), q);
                    if (!DEFER) store_level(1, q, z3r[(PH + 1) % 3]);
                }
                // level 2 at plane q = p-3
                if (STEADY || p >= 6) {
                    const int q = p - 3;
                    const float *zb = lvl + ((1 * 2 + (q & 1)) * NF) * PLS;
                    auto N = [&](int f, int d) -> float2 {
                        switch (d) {
                        case 0: return z3r[PH][f];
                        case 1: return xm(zb, f, z3r[PH][f]);
                        case 2: return xp(zb, f, z3r[PH][f]);
                        case 3: return ym(zb, f);
                        case 4: return yp(zb, f);
                        case 5: return z3r[(PH + 2) % 3][f];
                        default: return z3r[(PH + 1) % 3][f];
                        }
                    };
                    float2 rr[NF];
                    slab_apply<ADJ, MASK>(N, zsig(q), ih, ih2, i2h, rr);
                    const float *Y = stage + slot(3) * FPL;
#pragma unroll
                    for (int f = 0; f < NF; ++f) z2r[PH][f] = keep(P::fma(c2, rr[f], P::ld(Y + f * PLS + e)), q);
                    if (!DEFER) store_level(2, q, z2r[PH]);
                }
                // level 1 (the output) at plane q = p-4
                if ((STEADY || p >= 8) && (ox0 || ox1)) {
                    const int q = p - 4;
                    const float *zb = lvl + ((2 * 2 + (q & 1)) * NF) * PLS;
                    auto N = [&](int f, int d) -> float2 {
                        switch (d) {
                        case 0: return z2r[(PH + 2) % 3][f];
                        case 1: return xm(zb, f, z2r[(PH + 2) % 3][f]);
                        case 2: return xp(zb, f, z2r[(PH + 2) % 3][f]);
                        case 3: return ym(zb, f);
                        case 4: return yp(zb, f);
                        case 5: return z2r[(PH + 1) % 3][f];
                        default: return z2r[PH][f];
                        }
                    };
                    float2 rr[NF];
                    slab_apply<ADJ, MASK>(N, zsig(q), ih, ih2, i2h, rr);
                    const float *Y = stage + slot(4) * FPL;
                    int64_t z = zin0 + q;
                    z += z < 0 ? g.T[2] : (z >= g.T[2] ? -g.T[2] : 0);
                    const int64_t off = off_xy + z * g.PS, dz = img(z, 2) * g.PS;
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const float2 v = P::fma(c1, rr[f], P::ld(Y + f * PLS + e));
                        float *b = static_cast<float *>(out.p[slab_gid<MASK>(f)]) + off;
                        auto put = [&](float *q2) {
                            if (ox0 && ox1) P::st(q2, v);
                            else if (ox0) q2[0] = v.x;
                            else q2[1] = v.y;
                        };
                        put(b);
                        if (dy) put(b + dy);
                        if (dz) {
                            put(b + dz);
                            if (dy) put(b + dy + dz);
                        }
                        if (ox0 && dx0) {
                            b[dx0] = v.x;
                            if (dy) b[dx0 + dy] = v.x;
                            if (dz) {
                                b[dx0 + dz] = v.x;
                                if (dy) b[dx0 + dy + dz] = v.x;
                            }
                        }
                        if (ox1 && dx1) {
                            b[1 + dx1] = v.y;
                            if (dy) b[1 + dx1 + dy] = v.y;
                            if (dz) {
                                b[1 + dx1 + dz] = v.y;
                                if (dy) b[1 + dx1 + dy + dz] = v.y;
                            }
                        }
                    }
                }
                // x and y neighbours for the next iteration: levels 4, 3, 2 of planes p-1, p-2, p-3
                if (DEFER && (STEADY || p >= 2)) store_level(0, p - 1, z4r[(PH + 2) % 3]);
                if (DEFER && (STEADY || p >= 4)) store_level(1, p - 2, z3r[(PH + 1) % 3]);
                if (DEFER && (STEADY || p >= 6)) store_level(2, p - 3, z2r[PH]);
            }
        }
        ok = __syncthreads_and(ok);
        if (!ok) {
            pfail = p;
            return false;
        }
        // input plane p-4 was last read in this iteration: refill its slot
        if (p < nin && tid == 0 && p >= 4 && p - 4 + S < nin) {
            fence_proxy_async();
            const int st = slot(4);
            slab_issue<MASK, WALL>(stage + st * FPL, maps, bx, by, zin0 + p - 4 + S, g, &bars[st]);
        }
        return true;
    };
    using I0 = std::integral_constant<int, 0>;
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    using Fs = std::false_type;
    using Ts = std::true_type;
    if constexpr (SH::NAX <= 1 && !SH::AY) {
        int p0 = 0;
        for (; p0 < 9 && p0 < nin; p0 += 3)   // start-up: planes 0 .. 8
            if (!iter(p0, I0{}, Fs{}) || !iter(p0 + 1, I1{}, Fs{}) || !iter(p0 + 2, I2{}, Fs{})) break;
        if (ok)
            for (; p0 < nin; p0 += 3)
                if (!iter(p0, I0{}, Ts{}) || !iter(p0 + 1, I1{}, Ts{}) || !iter(p0 + 2, I2{}, Ts{})) break;
    } else {   // the y-active and multi-axis classes keep one guarded body (two copies spill)
        for (int p0 = 0; p0 < nin; p0 += 3)
            if (!iter(p0, I0{}, Fs{}) || !iter(p0 + 1, I1{}, Fs{}) || !iter(p0 + 2, I2{}, Fs{})) break;
    }
    if (!ok && tid == 0)   // let the copies in flight land (planes pfail .. pfail + S - 1 at most)
        for (int q = pfail; q < nin && q < pfail + S; ++q)
            mbar_wait(&bars[q % S], (q / S) & 1, nullptr, 0, kDrainLimitNs);
    // a class launched to overlap the previous one finishes only after it
    wait_prerequisite_grid();
}

template <bool ADJ, int MASK, bool WALL>
static cudaError_t launch_slab_class(const SlabMaps *maps, const Out8 &o, const Layer3DArgs &a, cudaStream_t st,
                                     bool &first)
{
    const int n = a.class_off[MASK + 1] - a.class_off[MASK];
    if (n <= 0) return cudaSuccess;
    static bool done = false;
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(k_slab3d<ADJ, MASK, WALL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(Slab<MASK>::SMEM));
        if (e != cudaSuccess) return e;
        cudaFuncAttributes fa{};
        if ((e = cudaFuncGetAttributes(&fa, k_slab3d<ADJ, MASK, WALL>)) != cudaSuccess) return e;
        if (fa.maxThreadsPerBlock < Slab<MASK>::NT) return cudaErrorLaunchOutOfResources;   // registers
        done = true;
    }
    const bool overlap = !first;
    first = false;
    return launch_pdl(k_slab3d<ADJ, MASK, WALL>, n, Slab<MASK>::NT, Slab<MASK>::SMEM, st, overlap, maps[MASK], o, a,
                      a.class_off[MASK]);
}

// Classes with the most fields per tile first, so that the short face tiles fill the tail.
template <bool ADJ, bool WALL>
static cudaError_t launch_slab_all(const SlabMaps *maps, const Out8 &o, const Layer3DArgs &a, cudaStream_t st)
{
    cudaError_t e;
    bool first = true;
    if ((e = launch_slab_class<ADJ, 7, WALL>(maps, o, a, st, first)) != cudaSuccess) return e;
    if ((e = launch_slab_class<ADJ, 6, WALL>(maps, o, a, st, first)) != cudaSuccess) return e;
    if ((e = launch_slab_class<ADJ, 5, WALL>(maps, o, a, st, first)) != cudaSuccess) return e;
    if ((e = launch_slab_class<ADJ, 3, WALL>(maps, o, a, st, first)) != cudaSuccess) return e;
    if ((e = launch_slab_class<ADJ, 4, WALL>(maps, o, a, st, first)) != cudaSuccess) return e;
    if ((e = launch_slab_class<ADJ, 2, WALL>(maps, o, a, st, first)) != cudaSuccess) return e;
    if ((e = launch_slab_class<ADJ, 1, WALL>(maps, o, a, st, first)) != cudaSuccess) return e;
    return launch_slab_class<ADJ, 0, WALL>(maps, o, a, st, first);
}

template <bool WALL>
cudaError_t launch_slab3d_impl(bool adjoint, const CUtensorMap *tm /*[8 classes][8 fields]*/, void *const *outp,
                               const Layer3DArgs &a, cudaStream_t st)
{
    if (a.ntiles <= 0) return cudaSuccess;
    SlabMaps maps[8];
    Out8 o;
    for (int m = 0; m < 8; ++m)
        for (int f = 0; f < 8; ++f) maps[m].m[f] = tm[m * 8 + f];
    for (int f = 0; f < 8; ++f) o.p[f] = outp[f];
    return adjoint ? launch_slab_all<true, WALL>(maps, o, a, st) : launch_slab_all<false, WALL>(maps, o, a, st);
}

}  // namespace pml

#endif  // PML_SLAB3D_CUH_
