// Kernels of the damping gradient: dJ/dsigma_a[e] of the receiver misfit.
//
// Per RK4 step n -> n+1 the gradient gains sum_i kbar_i^T (dA/dsigma) Y_i, where Y_i are
// the stage inputs of the forward step (Y1 = y_n, Y2 = y_n + dt/2 k1, Y3 = y_n + dt/2 k2,
// Y4 = y_n + dt k3, k_i = A Y_i) and kbar_i the stage cotangents of the reverse stage
// graph driven by the adjoint state ybar_{n+1} (kbar4 = dt/6 ybar, kbar3 = dt/3 ybar +
// dt A^T kbar4, kbar2 = dt/3 ybar + dt/2 A^T kbar3, kbar1 = dt/6 ybar + dt/2 A^T kbar2).
// These kernels evaluate the stages explicitly over the whole box (plain global loads,
// periodic neighbours by index wrap, so ghost cells are never read), and contract them
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

// out = A in (forward operator of Eq. 3) or A^T in, at every vertex of the box.
template <typename T, bool ADJ>
__global__ void __launch_bounds__(256) k_apply(const Fld<T> in, const FldW<T> out, const Idx ix, SigmaPtrs s, T ih,
                                               T ih2, T i2h)
{
    // boxes handled here have fewer than 2^31 vertices (checked by the caller): 32-bit index math
    const uint32_t T0 = uint32_t(ix.T[0]), T1 = uint32_t(ix.T[1]);
    const uint32_t n = T0 * T1 * uint32_t(ix.T[2]);
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int64_t c[3];
        const uint32_t q = v / T0;
        c[0] = v - q * T0;
        c[1] = q % T1;
        c[2] = q / T1;
        const int64_t o = ix.off(c[0], c[1], c[2]);
        T acc = T(0);   // V row (forward) or U row (transpose)
        const int lapf = ADJ ? 1 : 0;
        for (int a = 0; a < ix.nd; ++a) {
            int64_t cp[3] = {c[0], c[1], c[2]}, cm[3] = {c[0], c[1], c[2]};
            cp[a] = wrap(c[a] + 1, ix.T[a]);
            cm[a] = wrap(c[a] - 1, ix.T[a]);
            const int64_t op = ix.off(cp[0], cp[1], cp[2]), om = ix.off(cm[0], cm[1], cm[2]);
            const T *sg = static_cast<const T *>(s.p[a]);
            const T si = sg[c[a]], sm = sg[wrap(c[a] - 1, ix.T[a])];
            const T *L = in.f[lapf];
            acc += (L[op] - T(2) * L[o] + L[om]) * ih2;
            const T *Ph = in.f[2 + 2 * a], *Ps = in.f[3 + 2 * a];
            T *oPh = out.f[2 + 2 * a], *oPs = out.f[3 + 2 * a];
            if (!ADJ) {
                const T *U = in.f[0];
                const T dU = (U[op] - U[om]) * i2h;
                acc += (si * Ps[op] - sm * Ph[om]) * ih;
                oPh[o] = si != T(0) ? -T(0.5) * (sm * Ph[om] + si * Ph[o]) - dU : T(0);
                oPs[o] = sm != T(0) ? -T(0.5) * (sm * Ps[o] + si * Ps[op]) - dU : T(0);
            } else {
                const T *Vb = in.f[1];
                acc += ((Ph[op] - Ph[om]) + (Ps[op] - Ps[om])) * i2h;
                oPh[o] = si != T(0) ? -si * Vb[op] * ih - T(0.5) * si * (Ph[op] + Ph[o]) : T(0);
                oPs[o] = sm != T(0) ? sm * Vb[om] * ih - T(0.5) * sm * (Ps[o] + Ps[om]) : T(0);
            }
        }
        if (!ADJ) {
            out.f[0][o] = in.f[1][o];
            out.f[1][o] = acc;
        } else {
            out.f[0][o] = acc;
            out.f[1][o] = in.f[0][o];
        }
    }
}

// out = alpha x + beta y over the nf padded arrays (elementwise, ghosts included)
template <typename T>
__global__ void __launch_bounds__(256) k_axpby(const Fld<T> x, const Fld<T> y, const FldW<T> out, T alpha, T beta,
                                               int nf, int64_t elems)
{
    for (int f = 0; f < nf; ++f)
        for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < elems;
             i += int64_t(gridDim.x) * blockDim.x)
            out.f[f][i] = alpha * x.f[f][i] + beta * y.f[f][i];
}

// One block per edge (a, e) with sigma_a[e] != 0: acc[a-block + e] += kb^T (dA/dsigma_a[e]) Y
// over the vertices with i_a = e and i_a = e + 1 (FP64, fixed order, no atomics).
template <typename T>
__global__ void __launch_bounds__(256) k_contract(const Fld<T> kb, const Fld<T> Y, const Idx ix, SigmaPtrs s, double ih,
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
    const bool psi_at_e = sg[wrap(e - 1, Ta)] != T(0);    // Psi row active at i_a = e
    const bool phi_at_e1 = sg[wrap(e + 1, Ta)] != T(0);   // Phi row active at i_a = e + 1
    const int b1 = a == 0 ? 1 : 0, b2 = a == 2 ? 1 : 2;   // the other axes
    const int64_t n1 = ix.T[b1], n2 = ix.nd == 3 ? ix.T[b2] : 1;
    const T *kV = kb.f[1], *kPh = kb.f[2 + 2 * a], *kPs = kb.f[3 + 2 * a];
    const T *Ph = Y.f[2 + 2 * a], *Ps = Y.f[3 + 2 * a];
    double sum = 0.0;
    for (int64_t j = threadIdx.x; j < n1 * n2; j += blockDim.x) {
        int64_t c[3] = {0, 0, 0};
        c[b1] = j % n1;
        if (ix.nd == 3) c[b2] = j / n1;
        // i_a = e: sigma_a[i_a] terms
        c[a] = e;
        int64_t cp[3] = {c[0], c[1], c[2]};
        cp[a] = wrap(e + 1, Ta);
        const int64_t o = ix.off(c[0], c[1], c[2]), op = ix.off(cp[0], cp[1], cp[2]);
        sum += double(kV[o]) * double(Ps[op]) * ih;
        sum += -0.5 * double(kPh[o]) * double(Ph[o]);
        if (psi_at_e) sum += -0.5 * double(kPs[o]) * double(Ps[op]);
        // i_a = e + 1: sigma_a[i_a - 1] terms (o is now the vertex i - e_a)
        sum += -double(kV[op]) * double(Ph[o]) * ih;
        if (phi_at_e1) sum += -0.5 * double(kPh[op]) * double(Ph[o]);
        sum += -0.5 * double(kPs[op]) * double(Ps[op]);
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

int grid_for(int64_t n)
{
    const int64_t b = (n + 255) / 256;
    return int(b < 4096 ? (b > 0 ? b : 1) : 4096);
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

cudaError_t launch_apply_op(int prec, bool adjoint, void *const *in, void *const *out, int nf, const Geom &g,
                            const SigmaPtrs &s, double h, cudaStream_t st)
{
    if (g.T[0] * g.T[1] * g.T[2] >= (int64_t(1) << 31)) return cudaErrorInvalidValue;
    const Idx ix = make_idx(g);
    const int grid = grid_for(g.T[0] * g.T[1] * g.T[2]);
    if (prec == 32) {
        const float ih = float(1.0 / h), ih2 = float(1.0 / (h * h)), i2h = float(0.5 / h);
        if (adjoint) k_apply<float, true><<<grid, 256, 0, st>>>(fld<float>(in, nf), fldw<float>(out, nf), ix, s, ih, ih2, i2h);
        else k_apply<float, false><<<grid, 256, 0, st>>>(fld<float>(in, nf), fldw<float>(out, nf), ix, s, ih, ih2, i2h);
    } else {
        const double ih = 1.0 / h, ih2 = 1.0 / (h * h), i2h = 0.5 / h;
        if (adjoint) k_apply<double, true><<<grid, 256, 0, st>>>(fld<double>(in, nf), fldw<double>(out, nf), ix, s, ih, ih2, i2h);
        else k_apply<double, false><<<grid, 256, 0, st>>>(fld<double>(in, nf), fldw<double>(out, nf), ix, s, ih, ih2, i2h);
    }
    return cudaGetLastError();
}

cudaError_t launch_axpby(int prec, void *const *x, void *const *y, void *const *out, double alpha, double beta, int nf,
                         int64_t elems, cudaStream_t st)
{
    const int grid = grid_for(elems);
    if (prec == 32)
        k_axpby<float><<<grid, 256, 0, st>>>(fld<float>(x, nf), fld<float>(y, nf), fldw<float>(out, nf), float(alpha),
                                            float(beta), nf, elems);
    else
        k_axpby<double><<<grid, 256, 0, st>>>(fld<double>(x, nf), fld<double>(y, nf), fldw<double>(out, nf), alpha,
                                             beta, nf, elems);
    return cudaGetLastError();
}

cudaError_t launch_contract(int prec, void *const *kb, void *const *Y, int nf, const Geom &g, const SigmaPtrs &s,
                            double h, double *acc, cudaStream_t st)
{
    const Idx ix = make_idx(g);
    int nblk = 0;
    for (int a = 0; a < g.ndim; ++a) nblk += int(g.T[a]);
    if (prec == 32) k_contract<float><<<nblk, 256, 0, st>>>(fld<float>(kb, nf), fld<float>(Y, nf), ix, s, 1.0 / h, acc);
    else k_contract<double><<<nblk, 256, 0, st>>>(fld<double>(kb, nf), fld<double>(Y, nf), ix, s, 1.0 / h, acc);
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
