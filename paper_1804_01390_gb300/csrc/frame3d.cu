// 3D layer frame by level passes: the Horner form of the RK4 polynomial
//   z4 = y + dt/4 A y,  z3 = y + dt/3 A z4,  z2 = y + dt/2 A z3,  y' = y + dt A z2
// (eq:DiscretePML, Sec. 1.1.3) evaluated one level per launch over dense scratch buffers.
// Each level is a radius-1 stencil, so level k is needed on the frame widened by k - 1
// vertices (the frame of the layer-free run shrunk by k - 1): the passes cover the frame
// widened by 3, 2, 1 and 0.  Unlike the z-streaming tile kernel (layer3d.cuh), whose
// register rings limit its tiles to a 36 x 17 column region per 28 x 9 outputs, every
// thread here produces one vertex per plane; the price is one read of the operand and of
// y and one write per field and level (memory-bound instead of latency-bound).
//
// A CTA of 32 x 8 threads owns a tile of (x, y) columns and walks its z range; the
// operand's neighbours come through the read-only cache (consecutive planes of one tile
// reuse each other's rows).  The tile's class (axes whose aux fields reach it) selects the
// field count, as in the tile kernel.
#include "layer3d.cuh"

namespace pml {

template <typename T, bool ADJ, int MASK>
__device__ __forceinline__ void level3d_tile(const Level3Args &a, const LayerTile &tile)
{
    using F = Fields<MASK>;
    constexpr int NF = F::NF;
    const Geom &g = a.g;
    const int64_t x = int64_t(tile.x0) + (threadIdx.x & 31), y = int64_t(tile.y0) + (threadIdx.x >> 5);
    if (x < tile.xlo || x > tile.xhi || y < tile.ylo || y > tile.yhi) return;
    const LayerConstT<T> &lk = lconst_of<T>(a.k);
    const T ih = lk.ih, ih2 = lk.ih2, i2h = lk.i2h;
    const T c = a.level == 4 ? lk.c4 : (a.level == 3 ? lk.c3 : (a.level == 2 ? lk.c2 : lk.c1));
    const int64_t T0 = g.T[0], T1 = g.T[1], T2 = g.T[2];
    const T *sgx = static_cast<const T *>(a.sig[0]);
    const T *sgy = static_cast<const T *>(a.sig[1]);
    const T *sgz = static_cast<const T *>(a.sig[2]);
    Sig3<T> sg;
    sg.si[0] = sgx[x];
    sg.sm[0] = sgx[x == 0 ? T0 - 1 : x - 1];
    sg.si[1] = sgy[y];
    sg.sm[1] = sgy[y == 0 ? T1 - 1 : y - 1];
    const T *in[NF];
    const T *bs[NF];
    T *out[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        in[f] = static_cast<const T *>(a.in[F::gid(f)]);
        bs[f] = static_cast<const T *>(a.base[F::gid(f)]);
        out[f] = static_cast<T *>(a.out[F::gid(f)]);
    }
    const int64_t P = g.P, PS = g.PS;
    for (int64_t zu = tile.zlo; zu <= tile.zhi; ++zu) {
        const int64_t z = zu >= T2 ? zu - T2 : zu;   // the z band of a periodic box crosses the seam
        sg.si[2] = sgz[z];
        sg.sm[2] = sgz[z == 0 ? T2 - 1 : z - 1];
        const int64_t o = g.origin + x + y * P + z * PS;
        auto N = [&](int f, int d) -> T {
            const T *p = in[f] + o;
            switch (d) {
            case 0: return __ldg(p);
            case 1: return __ldg(p - 1);
            case 2: return __ldg(p + 1);
            case 3: return __ldg(p - P);
            case 4: return __ldg(p + P);
            case 5: return __ldg(p - PS);
            default: return __ldg(p + PS);
            }
        };
        T r[NF];
        apply_A3<T, ADJ, MASK>(N, sg, ih, ih2, i2h, r);
        const bool edge = near_edge(g, x, y, z);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const T v = __ldg(bs[f] + o) + c * r[f];
            if (!edge) out[f][o] = v;
            else store_wrapped(out[f], g, x, y, z, v);
        }
    }
}

template <typename T, bool ADJ>
__global__ void __launch_bounds__(kLevel3TX * kLevel3TY) k_level3d(const Level3Args a)
{
    allow_dependent_launch();
    const LayerTile tile = a.tiles[blockIdx.x];
    switch (tile.flags & 7) {
    case 0: level3d_tile<T, ADJ, 0>(a, tile); break;
    case 1: level3d_tile<T, ADJ, 1>(a, tile); break;
    case 2: level3d_tile<T, ADJ, 2>(a, tile); break;
    case 3: level3d_tile<T, ADJ, 3>(a, tile); break;
    case 4: level3d_tile<T, ADJ, 4>(a, tile); break;
    case 5: level3d_tile<T, ADJ, 5>(a, tile); break;
    case 6: level3d_tile<T, ADJ, 6>(a, tile); break;
    default: level3d_tile<T, ADJ, 7>(a, tile); break;
    }
}

cudaError_t launch_level3d(int prec, bool adjoint, const Level3Args &a, cudaStream_t st)
{
    if (a.ntiles <= 0) return cudaSuccess;
    const dim3 grid(unsigned(a.ntiles)), block(kLevel3TX * kLevel3TY);
    if (prec == 32) {
        if (adjoint) k_level3d<float, true><<<grid, block, 0, st>>>(a);
        else k_level3d<float, false><<<grid, block, 0, st>>>(a);
    } else {
        if (adjoint) k_level3d<double, true><<<grid, block, 0, st>>>(a);
        else k_level3d<double, false><<<grid, block, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace pml
