// Kernels of the damping gradient: dJ/dsigma_a[e] of the receiver misfit.
//
// Per RK4 step n -> n+1 the gradient gains sum_i kbar_i^T (dA/dsigma) Y_i, where Y_i are
// the stage inputs of the forward step (Y1 = y_n, Y2 = y_n + dt/2 k1, Y3 = y_n + dt/2 k2,
// Y4 = y_n + dt k3, k_i = A Y_i) and kbar_i the stage cotangents of the reverse stage
// graph driven by the adjoint state ybar_{n+1} (kbar4 = dt/6 ybar, kbar3 = dt/3 ybar +
// dt A^T kbar4, kbar2 = dt/3 ybar + dt/2 A^T kbar3, kbar1 = dt/6 ybar + dt/2 A^T kbar2).
// The contraction reads kbar_i and Y_i only on the vertices next to an edge with nonzero
// sigma (the set C: along each axis a, the slab of coordinates e, e + 1 of those edges).
// Since the stencil of A is a cross, C widened by r stencil steps is the union of those
// slabs widened by r along their own axis (C_r), so Y2 is formed on C_2, Y3 on C_1, Y4 on
// C, and likewise kbar3 on C_2, kbar2 on C_1, kbar1 on C (kbar4 = dt/6 ybar is a scaling,
// applied inside the kernels).  The kernels evaluate these stages explicitly on host-built
// lists of row segments of C_r (plain global loads; neighbours by index wrap, or zero
// beyond the ends of a box with walls, so ghost cells are never read), and contract them
// edge by edge.  Source terms are left out of the stages: a source sits where sigma is
// zero on the edges within two of it, so it never reaches the vertices the contraction
// reads (those next to an edge with nonzero sigma) within one step.
#include "common.cuh"

namespace pml {

namespace {

struct Idx {
    int64_t T[3];
    int64_t P, PS, origin;
    int nd;
    __device__ __forceinline__ int64_t off(int64_t x, int64_t y, int64_t z) const { return origin + x + y * P + z * PS; }
};

__device__ __forceinline__ int64_t wrap(int64_t v, int64_t T) { return v < 0 ? v + T : (v >= T ? v - T : v); }

template <typename T> struct Fld {
    const T *f[8];
};
template <typename T> struct FldW {
    T *f[8];
};

// out = alpha base + cop Op(in) (Op = A, the forward operator of Eq. 3, or its
// transpose) on chunks {x0, x1, y, z} of at most kStageChunk consecutive vertices of a row,
// one block per chunk and one thread per vertex.  Every value of `in` the stencil reads
// must be valid: the caller's chunks for `out` lie one vertex inside those on which `in`
// was formed.  Neighbours by offset, wrapped only at the ends of an axis (or zero beyond
// them with a wall); the ghost ring is never read.
constexpr int kStageChunk = kStageChunkMax;

template <typename T, bool ADJ, int ND>
__global__ void __launch_bounds__(kStageChunk) k_stage(const Fld<T> in, const Fld<T> base, const FldW<T> out,
                                                       const Idx ix, SigmaPtrs s, T ih, T ih2, T i2h, T alpha,
                                                       T cop, const int4 *seg, int wall)
{
    const int4 sg4 = seg[blockIdx.x];
    const int64_t x = sg4.x + int64_t(threadIdx.x);
    if (x > sg4.y) return;
    const int64_t c[3] = {x, sg4.z, sg4.w};
    const int64_t st[3] = {1, ix.P, ix.PS};
    const int64_t o = ix.off(c[0], c[1], c[2]);
    T acc = T(0);   // V row (forward) or U row (transpose)
#pragma unroll
    for (int a = 0; a < ND; ++a) {
        const int64_t Ta = ix.T[a];
        const bool okp = c[a] + 1 < Ta || !wall, okm = c[a] > 0 || !wall;
        const int64_t op = o + (c[a] + 1 < Ta ? st[a] : -(Ta - 1) * st[a]);
        const int64_t om = o + (c[a] > 0 ? -st[a] : (Ta - 1) * st[a]);
        const T *sgm = static_cast<const T *>(s.p[a]);
        const T si = sgm[c[a]], sm = sgm[c[a] > 0 ? c[a] - 1 : Ta - 1];
        const T *L = in.f[ADJ ? 1 : 0];
        const T Lc = L[o];
        acc += ((okp ? L[op] : T(0)) - T(2) * Lc + (okm ? L[om] : T(0))) * ih2;
        const T *Ph = in.f[2 + 2 * a], *Ps = in.f[3 + 2 * a];
        const T php = okp ? Ph[op] : T(0), phm = okm ? Ph[om] : T(0);
        const T psp = okp ? Ps[op] : T(0), psm = okm ? Ps[om] : T(0);
        T oph, ops;
        if (!ADJ) {
            const T *U = in.f[0];
            const T dU = ((okp ? U[op] : T(0)) - (okm ? U[om] : T(0))) * i2h;
            acc += (si * psp - sm * phm) * ih;
            oph = si != T(0) ? -T(0.5) * (sm * phm + si * Ph[o]) - dU : T(0);
            ops = sm != T(0) ? -T(0.5) * (sm * Ps[o] + si * psp) - dU : T(0);
        } else {
            const T *Vb = in.f[1];
            acc += ((php - phm) + (psp - psm)) * i2h;
            oph = si != T(0) ? -si * (okp ? Vb[op] : T(0)) * ih - T(0.5) * si * (php + Ph[o]) : T(0);
            ops = sm != T(0) ? sm * (okm ? Vb[om] : T(0)) * ih - T(0.5) * sm * (Ps[o] + psm) : T(0);
        }
        out.f[2 + 2 * a][o] = alpha * base.f[2 + 2 * a][o] + cop * oph;
        out.f[3 + 2 * a][o] = alpha * base.f[3 + 2 * a][o] + cop * ops;
    }
    if (!ADJ) {
        out.f[0][o] = alpha * base.f[0][o] + cop * in.f[1][o];
        out.f[1][o] = alpha * base.f[1][o] + cop * acc;
    } else {
        out.f[0][o] = alpha * base.f[0][o] + cop * acc;
        out.f[1][o] = alpha * base.f[1][o] + cop * in.f[0][o];
    }
}

// The four stage pairs of one step in one launch: one block per edge (a, e) with
// sigma_a[e] != 0, acc[a-block + e] += sum_i scale_i kb_i^T (dA/dsigma_a[e]) Y_i over the
// vertices with i_a = e and i_a = e + 1 (FP64, fixed order, no atomics).
struct Pairs4 {
    const void *kb[4][8];
    const void *Y[4][8];
    double scale[4];
};

template <typename T>
__global__ void __launch_bounds__(256) k_contract4(const Pairs4 pr, const Idx ix, SigmaPtrs s, double ih, int wall,
                                                   double *acc)
{
    int a = 0, e = int(blockIdx.x), off = 0;
    while (a < ix.nd - 1 && e >= ix.T[a]) {
        e -= int(ix.T[a]);
        off += int(ix.T[a]);
        ++a;
    }
    const T *sg = static_cast<const T *>(s.p[a]);
    const int64_t Ta = ix.T[a];
    if (sg[e] == T(0)) return;   // whole block: no barrier below is reached
    // (with a wall sigma_a[T - 1] = 0, so e + 1 never leaves the box here)
    const bool psi_at_e = sg[wrap(e - 1, Ta)] != T(0);    // Psi row active at i_a = e
    const bool phi_at_e1 = sg[wrap(e + 1, Ta)] != T(0);   // Phi row active at i_a = e + 1
    const int b1 = a == 0 ? 1 : 0, b2 = a == 2 ? 1 : 2;   // the other axes
    const int64_t n1 = ix.T[b1], n2 = ix.nd == 3 ? ix.T[b2] : 1;
    double sum = 0.0;
    for (int i = 0; i < 4; ++i) {
        const T *kV = static_cast<const T *>(pr.kb[i][1]), *kPh = static_cast<const T *>(pr.kb[i][2 + 2 * a]),
                *kPs = static_cast<const T *>(pr.kb[i][3 + 2 * a]);
        const T *Ph = static_cast<const T *>(pr.Y[i][2 + 2 * a]), *Ps = static_cast<const T *>(pr.Y[i][3 + 2 * a]);
        double part = 0.0;
        for (int64_t j = threadIdx.x; j < n1 * n2; j += blockDim.x) {
            int64_t c[3] = {0, 0, 0};
            c[b1] = j % n1;
            if (ix.nd == 3) c[b2] = j / n1;
            // i_a = e: sigma_a[i_a] terms
            c[a] = e;
            int64_t cp[3] = {c[0], c[1], c[2]};
            cp[a] = wrap(e + 1, Ta);
            const int64_t o = ix.off(c[0], c[1], c[2]), op = ix.off(cp[0], cp[1], cp[2]);
            part += double(kV[o]) * double(Ps[op]) * ih;
            part += -0.5 * double(kPh[o]) * double(Ph[o]);
            if (psi_at_e) part += -0.5 * double(kPs[o]) * double(Ps[op]);
            // i_a = e + 1: sigma_a[i_a - 1] terms (o is now the vertex i - e_a)
            part += -double(kV[op]) * double(Ph[o]) * ih;
            if (phi_at_e1) part += -0.5 * double(kPh[op]) * double(Ph[o]);
            part += -0.5 * double(kPs[op]) * double(Ps[op]);
        }
        sum += pr.scale[i] * part;
    }
    __shared__ double red[256];
    red[threadIdx.x] = sum;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (int(threadIdx.x) < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) acc[off + e] += red[0];
}

// res[k] = trace[k] - target[k] (k < count); misfit[0] = 1/2 sum res^2 (one block, FP64)
template <typename T>
__global__ void __launch_bounds__(256) k_residual(const T *trace, const T *target, T *res, int64_t count, double *misfit)
{
    double s = 0.0;
    for (int64_t k = threadIdx.x; k < count; k += blockDim.x) {
        const T d = trace[k] - target[k];
        res[k] = d;
        s += double(d) * double(d);
    }
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (int(threadIdx.x) < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) misfit[0] = 0.5 * red[0];
}

Idx make_idx(const Geom &g)
{
    Idx ix;
    for (int a = 0; a < 3; ++a) ix.T[a] = g.T[a];
    ix.P = g.P;
    ix.PS = g.PS;
    ix.origin = g.origin;
    ix.nd = g.ndim;
    return ix;
}

template <typename T> Fld<T> fld(void *const *p, int nf)
{
    Fld<T> r{};
    for (int f = 0; f < nf; ++f) r.f[f] = static_cast<const T *>(p[f]);
    return r;
}
template <typename T> FldW<T> fldw(void *const *p, int nf)
{
    FldW<T> r{};
    for (int f = 0; f < nf; ++f) r.f[f] = static_cast<T *>(p[f]);
    return r;
}

}  // namespace

cudaError_t launch_stage(int prec, bool adjoint, void *const *in, void *const *base, void *const *out, int nf,
                         const Geom &g, const SigmaPtrs &s, double h, double alpha, double cop, const int4 *seg,
                         int nseg, cudaStream_t st)
{
    if (nseg <= 0) return cudaSuccess;
    const Idx ix = make_idx(g);
    const int wall = g.wall;
#define PML_STAGE(TT, AA, DD, IH, IH2, I2H, AL, CO)                                                              \
    k_stage<TT, AA, DD><<<nseg, kStageChunk, 0, st>>>(fld<TT>(in, nf), fld<TT>(base, nf), fldw<TT>(out, nf), ix, s, \
                                                      IH, IH2, I2H, AL, CO, seg, wall)
    if (prec == 32) {
        const float ih = float(1.0 / h), ih2 = float(1.0 / (h * h)), i2h = float(0.5 / h), al = float(alpha),
                    co = float(cop);
        if (g.ndim == 2) {
            if (adjoint) PML_STAGE(float, true, 2, ih, ih2, i2h, al, co);
            else PML_STAGE(float, false, 2, ih, ih2, i2h, al, co);
        } else {
            if (adjoint) PML_STAGE(float, true, 3, ih, ih2, i2h, al, co);
            else PML_STAGE(float, false, 3, ih, ih2, i2h, al, co);
        }
    } else {
        const double ih = 1.0 / h, ih2 = 1.0 / (h * h), i2h = 0.5 / h;
        if (g.ndim == 2) {
            if (adjoint) PML_STAGE(double, true, 2, ih, ih2, i2h, alpha, cop);
            else PML_STAGE(double, false, 2, ih, ih2, i2h, alpha, cop);
        } else {
            if (adjoint) PML_STAGE(double, true, 3, ih, ih2, i2h, alpha, cop);
            else PML_STAGE(double, false, 3, ih, ih2, i2h, alpha, cop);
        }
    }
#undef PML_STAGE
    return cudaGetLastError();
}

cudaError_t launch_contract4(int prec, void *const *const *kb, void *const *const *Y, const double *scale, int nf,
                             const Geom &g, const SigmaPtrs &s, double h, double *acc, cudaStream_t st)
{
    const Idx ix = make_idx(g);
    Pairs4 pr{};
    for (int i = 0; i < 4; ++i) {
        for (int f = 0; f < nf; ++f) {
            pr.kb[i][f] = kb[i][f];
            pr.Y[i][f] = Y[i][f];
        }
        pr.scale[i] = scale[i];
    }
    int nblk = 0;
    for (int a = 0; a < g.ndim; ++a) nblk += int(g.T[a]);
    if (prec == 32) k_contract4<float><<<nblk, 256, 0, st>>>(pr, ix, s, 1.0 / h, g.wall, acc);
    else k_contract4<double><<<nblk, 256, 0, st>>>(pr, ix, s, 1.0 / h, g.wall, acc);
    return cudaGetLastError();
}

cudaError_t launch_residual(int prec, const void *trace, const void *target, void *res, int64_t count, double *misfit,
                            cudaStream_t st)
{
    if (prec == 32)
        k_residual<float><<<1, 256, 0, st>>>((const float *)trace, (const float *)target, (float *)res, count, misfit);
    else
        k_residual<double><<<1, 256, 0, st>>>((const double *)trace, (const double *)target, (double *)res, count, misfit);
    return cudaGetLastError();
}

}  // namespace pml
