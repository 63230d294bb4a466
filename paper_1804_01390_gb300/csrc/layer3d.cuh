// 3D layer frame kernel (z-streaming Horner pipeline), templated on the boundary of the
// box: WALL = false for the periodic box, true for reflecting walls.  Included by
// step3d.cu (periodic) and layer3d_wall.cu (walls), so the two sets of kernels compile in
// parallel.
#ifndef PML_LAYER3D_CUH_
#define PML_LAYER3D_CUH_

#include "common.cuh"

namespace pml {

// ------------------------------------------------------------------------------------
// layer frame, z-streaming Horner pipeline
// ------------------------------------------------------------------------------------

template <typename T> struct L3 {
    // region (x, y) = tile + halo 4 on each side; one thread per region column
    static constexpr int RX = sizeof(T) == 4 ? kLayer3TXf + 8 : kLayer3TXd + 8;
    static constexpr int RY = sizeof(T) == 4 ? kLayer3TYf + 8 : kLayer3TYd + 8;
    static constexpr int PL = RX * RY;                 // threads; elements of one TMA box
    static constexpr int PLS = (PL + 31) / 32 * 32;    // shared-memory stride of one field plane
                                                       // (TMA destinations must be 128-byte aligned)
    // plane ring: resident planes p-4..p plus one in flight; the 8-field FP32 class keeps
    // none in flight so that its shared memory fits
    static constexpr int stages(int nf) { return sizeof(T) == 4 && nf == 8 ? 5 : 6; }
};

template <int MASK> struct Fields {
    static constexpr int NAX = ((MASK >> 0) & 1) + ((MASK >> 1) & 1) + ((MASK >> 2) & 1);
    static constexpr int NF = 2 + 2 * NAX;
    // global field id of local field f (0 U, 1 V, then Phi/Psi of the active axes)
    static __device__ __forceinline__ constexpr int gid(int f)
    {
        if (f < 2) return f;
        int k = (f - 2) >> 1, ax = 0;
        for (int a = 0; a < 3; ++a)
            if ((MASK >> a) & 1) {
                if (k == 0) { ax = a; break; }
                --k;
            }
        return 2 + 2 * ax + ((f - 2) & 1);
    }
    static __device__ __forceinline__ constexpr int axis(int k)   // k-th active axis
    {
        for (int a = 0; a < 3; ++a)
            if ((MASK >> a) & 1) {
                if (k == 0) return a;
                --k;
            }
        return 0;
    }
};

template <typename T> struct Sig3 {
    T si[3], sm[3];   // sigma_a[i_a], sigma_a[i_a - 1]
};

// A z (or A^T z) at one vertex; N(f, d) returns local field f at direction d:
// 0 centre, 1 x-, 2 x+, 3 y-, 4 y+, 5 z-, 6 z+.
template <typename T, bool ADJ, int MASK, typename Get>
__device__ __forceinline__ void apply_A3(const Get &N, const Sig3<T> &s, T ih, T ih2, T i2h, T *o)
{
    using F = Fields<MASK>;
    const T half = T(0.5);
    if (!ADJ) {
        const T U0 = N(0, 0);
        const T lap = (((N(0, 2) + N(0, 1)) - T(2) * U0) + ((N(0, 4) + N(0, 3)) - T(2) * U0)) +
                      ((N(0, 6) + N(0, 5)) - T(2) * U0);
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
        const T lap = (((N(1, 2) + N(1, 1)) - T(2) * V0) + ((N(1, 4) + N(1, 3)) - T(2) * V0)) +
                      ((N(1, 6) + N(1, 5)) - T(2) * V0);
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

struct Maps8 {
    CUtensorMap m[8];
};
struct Out8 {
    void *p[8];
};

template <typename T, int MASK, bool WALL>
__device__ __forceinline__ void issue_plane3(T *stage_base, const Maps8 &maps, const LayerTile &tile, int64_t zin,
                                             const Geom &g, uint64_t *bar)
{
    using F = Fields<MASK>;
    constexpr int PL = L3<T>::PL, PLS = L3<T>::PLS;
    int64_t z = zin;
    if (!WALL) z += z < 0 ? g.T[2] : (z >= g.T[2] ? -g.T[2] : 0);   // a wall keeps the zero ghost planes
    mbar_arrive_expect_tx(bar, uint32_t(F::NF * PL * sizeof(T)));
#pragma unroll
    for (int f = 0; f < F::NF; ++f)
        tma_load_3d(stage_base + f * PLS, &maps.m[F::gid(f)], tile.x0 - 4 + G, tile.y0 - 4 + G, int32_t(z + G), bar);
}

template <typename T, bool ADJ, int MASK, bool WALL>
__global__ void __launch_bounds__(L3<T>::PL, 1)
    k_layer3d(const __grid_constant__ Maps8 maps, const Out8 out, const Layer3DArgs a, int tile_base)
{
    using F = Fields<MASK>;
    constexpr int NF = F::NF, RX = L3<T>::RX, RY = L3<T>::RY, PL = L3<T>::PL, PLS = L3<T>::PLS, S = L3<T>::stages(F::NF);
    extern __shared__ unsigned char smem_dyn[];
    T *stage = smem_align128<T>(smem_dyn);
    T *Zb = stage + S * NF * PLS;   // [3 levels][2 slots][NF][PLS]
    __shared__ T sx[RX + 1], sy[RY + 1], sz[kLayer3LZ + 9];
    __shared__ __align__(8) uint64_t bars[S];

    allow_dependent_launch();
    const LayerTile tile = a.tiles[tile_base + blockIdx.x];
    const Geom &g = a.g;
    const int tid = threadIdx.x, cx = tid % RX, cy = tid / RX;
    const int nout = tile.zhi - tile.zlo + 1;
    const int nin = nout + 8;
    const int64_t zin0 = int64_t(tile.zlo) - 4;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
        const int npro = nin < S ? nin : S;
        for (int p = 0; p < npro; ++p) issue_plane3<T, MASK, WALL>(stage + p * NF * PLS, maps, tile, zin0 + p, g, &bars[p]);
    }
    const T *sgx = static_cast<const T *>(a.sig[0]);
    const T *sgy = static_cast<const T *>(a.sig[1]);
    const T *sgz = static_cast<const T *>(a.sig[2]);
    for (int k = tid; k <= RX; k += PL) {
        int64_t i = (int64_t(tile.x0) - 5 + k) % g.T[0];
        if (i < 0) i += g.T[0];
        sx[k] = sgx[i];
    }
    for (int k = tid; k <= RY; k += PL) {
        int64_t i = (int64_t(tile.y0) - 5 + k) % g.T[1];
        if (i < 0) i += g.T[1];
        sy[k] = sgy[i];
    }
    for (int k = tid; k <= nin; k += PL) {   // sz[k] = sigma_z[zin0 - 1 + k]
        int64_t i = (zin0 - 1 + k) % g.T[2];
        if (i < 0) i += g.T[2];
        sz[k] = sgz[i];
    }
    __syncthreads();

    const LayerConstT<T> &lk = lconst_of<T>(a.k);
    const T ih = lk.ih, ih2 = lk.ih2, i2h = lk.i2h, c4 = lk.c4, c3 = lk.c3, c2 = lk.c2, c1 = lk.c1;
    T z4r[3][NF], z3r[3][NF], z2r[3][NF];
    Sig3<T> sg;
    sg.si[0] = sx[cx + 1];
    sg.sm[0] = sx[cx];
    sg.si[1] = sy[cy + 1];
    sg.sm[1] = sy[cy];
    const int T2 = int(g.T[2]);
    auto zsig = [&](int64_t zl, Sig3<T> &s) {   // plane zl = zin0 + q of the work item
        const int q = int(zl - zin0);
        s.si[2] = sz[q + 1];
        s.sm[2] = sz[q];
    };
    const bool v4 = cx >= 1 && cx <= RX - 2 && cy >= 1 && cy <= RY - 2;
    const bool v3 = cx >= 2 && cx <= RX - 3 && cy >= 2 && cy <= RY - 3;
    const bool v2 = cx >= 3 && cx <= RX - 4 && cy >= 3 && cy <= RY - 4;
    const bool v1 = cx >= 4 && cx <= RX - 5 && cy >= 4 && cy <= RY - 5;
    const int64_t gx = int64_t(tile.x0) - 4 + cx, gy = int64_t(tile.y0) - 4 + cy;
    const bool in_rect = v1 && gx >= tile.xlo && gx <= tile.xhi && gy >= tile.ylo && gy <= tile.yhi;
    // with a wall every stage value beyond the ends of the box is zero
    const bool in_xy = !WALL || (gx >= 0 && gx < g.T[0] && gy >= 0 && gy < g.T[1]);
    auto keep = [&](int q) { return !WALL || (in_xy && zin0 + q >= 0 && zin0 + q < g.T[2]); };

    bool ok = true;
    int pfail = nin;   // first plane whose wait gave up
    for (int p0 = 0; p0 < nin && ok; p0 += 3) {
#pragma unroll
        for (int PH = 0; PH < 3; ++PH) {
            const int p = p0 + PH;
            if (p < nin) {
                if (!mbar_wait(&bars[p % S], (p / S) & 1, a.err, 4, a.wait_ns)) ok = false;
                if (ok) {
                    // level 4 at plane q = p-1 from the input planes in the stage ring
                    if (p >= 2 && v4) {
                        const int q = p - 1;
                        const T *Pc = stage + (q % S) * NF * PLS, *Pm = stage + ((q - 1) % S) * NF * PLS,
                                *Pp = stage + (p % S) * NF * PLS;
                        auto N = [&](int f, int d) -> T {
                            const int o = f * PLS + tid;
                            switch (d) {
                            case 0: return Pc[o];
                            case 1: return Pc[o - 1];
                            case 2: return Pc[o + 1];
                            case 3: return Pc[o - RX];
                            case 4: return Pc[o + RX];
                            case 5: return Pm[o];
                            default: return Pp[o];
                            }
                        };
                        zsig(zin0 + q, sg);
                        T r[NF];
                        apply_A3<T, ADJ, MASK>(N, sg, ih, ih2, i2h, r);
                        T *zb = Zb + ((0 * 2 + (q & 1)) * NF) * PLS;
                        const bool kq = keep(q);
#pragma unroll
                        for (int f = 0; f < NF; ++f) {
                            const T val = kq ? Pc[f * PLS + tid] + c4 * r[f] : T(0);
                            z4r[(PH + 2) % 3][f] = val;
                            zb[f * PLS + tid] = val;
                        }
                    }
                    // level 3 at plane q = p-2 (z neighbours: own ring; x/y: level-4 plane)
                    if (p >= 4 && v3) {
                        const int q = p - 2;
                        const T *zb = Zb + ((0 * 2 + (q & 1)) * NF) * PLS;
                        auto N = [&](int f, int d) -> T {
                            switch (d) {
                            case 0: return z4r[(PH + 1) % 3][f];
                            case 1: return zb[f * PLS + tid - 1];
                            case 2: return zb[f * PLS + tid + 1];
                            case 3: return zb[f * PLS + tid - RX];
                            case 4: return zb[f * PLS + tid + RX];
                            case 5: return z4r[PH][f];
                            default: return z4r[(PH + 2) % 3][f];
                            }
                        };
                        zsig(zin0 + q, sg);
                        T r[NF];
                        apply_A3<T, ADJ, MASK>(N, sg, ih, ih2, i2h, r);
                        const T *Y = stage + (q % S) * NF * PLS;
                        T *zo = Zb + ((1 * 2 + (q & 1)) * NF) * PLS;
                        const bool kq = keep(q);
#pragma unroll
                        for (int f = 0; f < NF; ++f) {
                            const T val = kq ? Y[f * PLS + tid] + c3 * r[f] : T(0);
                            z3r[(PH + 1) % 3][f] = val;
                            zo[f * PLS + tid] = val;
                        }
                    }
                    // level 2 at plane q = p-3
                    if (p >= 6 && v2) {
                        const int q = p - 3;
                        const T *zb = Zb + ((1 * 2 + (q & 1)) * NF) * PLS;
                        auto N = [&](int f, int d) -> T {
                            switch (d) {
                            case 0: return z3r[PH][f];
                            case 1: return zb[f * PLS + tid - 1];
                            case 2: return zb[f * PLS + tid + 1];
                            case 3: return zb[f * PLS + tid - RX];
                            case 4: return zb[f * PLS + tid + RX];
                            case 5: return z3r[(PH + 2) % 3][f];
                            default: return z3r[(PH + 1) % 3][f];
                            }
                        };
                        zsig(zin0 + q, sg);
                        T r[NF];
                        apply_A3<T, ADJ, MASK>(N, sg, ih, ih2, i2h, r);
                        const T *Y = stage + (q % S) * NF * PLS;
                        T *zo = Zb + ((2 * 2 + (q & 1)) * NF) * PLS;
                        const bool kq = keep(q);
#pragma unroll
                        for (int f = 0; f < NF; ++f) {
                            const T val = kq ? Y[f * PLS + tid] + c2 * r[f] : T(0);
                            z2r[PH][f] = val;
                            zo[f * PLS + tid] = val;
                        }
                    }
                    // level 1 (output) at plane q = p-4
                    if (p >= 8 && in_rect) {
                        const int q = p - 4;
                        const T *zb = Zb + ((2 * 2 + (q & 1)) * NF) * PLS;
                        auto N = [&](int f, int d) -> T {
                            switch (d) {
                            case 0: return z2r[(PH + 2) % 3][f];
                            case 1: return zb[f * PLS + tid - 1];
                            case 2: return zb[f * PLS + tid + 1];
                            case 3: return zb[f * PLS + tid - RX];
                            case 4: return zb[f * PLS + tid + RX];
                            case 5: return z2r[(PH + 1) % 3][f];
                            default: return z2r[PH][f];
                            }
                        };
                        const int64_t zl = zin0 + q;
                        zsig(zl, sg);
                        T r[NF];
                        apply_A3<T, ADJ, MASK>(N, sg, ih, ih2, i2h, r);
                        const T *Y = stage + (q % S) * NF * PLS;
                        int64_t z = zl;
                        z += z < 0 ? T2 : (z >= T2 ? -T2 : 0);
                        const bool edge = near_edge(g, gx, gy, z);
#pragma unroll
                        for (int f = 0; f < NF; ++f) {
                            const T val = Y[f * PLS + tid] + c1 * r[f];
                            T *dst = static_cast<T *>(out.p[F::gid(f)]);
                            if (edge) store_wrapped(dst, g, gx, gy, z, val);
                            else dst[g.origin + gx + gy * g.P + z * g.PS] = val;
                        }
                    }
                }
            }
            ok = __syncthreads_and(ok);
            if (!ok) {
                pfail = p;
                break;
            }
            if (p < nin && tid == 0 && p >= 4 && p - 4 + S < nin) {
                fence_proxy_async();
                const int st = (p - 4) % S;
                issue_plane3<T, MASK, WALL>(stage + st * NF * PLS, maps, tile, zin0 + p - 4 + S, g, &bars[st]);
            }
        }
    }
    if (!ok && tid == 0)   // let the copies in flight (planes pfail .. pfail + S - 5 at most) land
        for (int q = pfail; q < nin && q < pfail + S; ++q)
            mbar_wait(&bars[q % S], (q / S) & 1, nullptr, 0, kDrainLimitNs);
    // a class launched to overlap the previous one finishes only after it
    wait_prerequisite_grid();
}

template <typename T, int MASK> static size_t layer3d_smem()
{
    return (size_t(L3<T>::stages(Fields<MASK>::NF)) + 6) * Fields<MASK>::NF * L3<T>::PLS * sizeof(T) + 128;
}

// One class's launch; `first` marks the first class launch of the step (fully ordered
// after earlier work), later ones overlap their predecessor.
template <typename T, bool ADJ, int MASK, bool WALL>
static cudaError_t launch_l3(const Maps8 &m, const Out8 &o, const Layer3DArgs &a, cudaStream_t st, bool &first)
{
    const int n = a.class_off[MASK + 1] - a.class_off[MASK];
    if (n <= 0) return cudaSuccess;
    static bool done = false;
    const size_t sm = layer3d_smem<T, MASK>();
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(k_layer3d<T, ADJ, MASK, WALL>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        if (e != cudaSuccess) return e;
        done = true;
    }
    const bool overlap = !first;
    first = false;
    return launch_pdl(k_layer3d<T, ADJ, MASK, WALL>, n, L3<T>::PL, sm, st, overlap, m, o, a, a.class_off[MASK]);
}

// Classes with the most fields per tile (the longest tiles) first, so that the short
// face tiles fill the tail.
template <typename T, bool ADJ, bool WALL>
static cudaError_t launch_l3_all(const Maps8 &m, const Out8 &o, const Layer3DArgs &a, cudaStream_t st)
{
    cudaError_t e;
    bool first = true;
    if ((e = launch_l3<T, ADJ, 7, WALL>(m, o, a, st, first)) != cudaSuccess) return e;
    if ((e = launch_l3<T, ADJ, 6, WALL>(m, o, a, st, first)) != cudaSuccess) return e;
    if ((e = launch_l3<T, ADJ, 5, WALL>(m, o, a, st, first)) != cudaSuccess) return e;
    if ((e = launch_l3<T, ADJ, 3, WALL>(m, o, a, st, first)) != cudaSuccess) return e;
    if ((e = launch_l3<T, ADJ, 4, WALL>(m, o, a, st, first)) != cudaSuccess) return e;
    if ((e = launch_l3<T, ADJ, 2, WALL>(m, o, a, st, first)) != cudaSuccess) return e;
    if ((e = launch_l3<T, ADJ, 1, WALL>(m, o, a, st, first)) != cudaSuccess) return e;
    return launch_l3<T, ADJ, 0, WALL>(m, o, a, st, first);
}


template <bool WALL>
cudaError_t launch_layer3d_impl(int prec, bool adjoint, const CUtensorMap *tm, void *const *outp,
                                const Layer3DArgs &a, cudaStream_t st)
{
    if (a.ntiles <= 0) return cudaSuccess;
    Maps8 m;
    Out8 o;
    for (int f = 0; f < 8; ++f) {
        m.m[f] = tm[f];
        o.p[f] = outp[f];
    }
    if (prec == 32) return adjoint ? launch_l3_all<float, true, WALL>(m, o, a, st) : launch_l3_all<float, false, WALL>(m, o, a, st);
    return adjoint ? launch_l3_all<double, true, WALL>(m, o, a, st) : launch_l3_all<double, false, WALL>(m, o, a, st);
}

}  // namespace pml

#endif  // PML_LAYER3D_CUH_
