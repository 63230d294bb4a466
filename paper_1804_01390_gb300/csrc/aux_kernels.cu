// Small kernels around the step: periodic ghost refresh, point sources / receivers,
// adjoint injection and source-amplitude gradients, and FP64 reductions (energy
// eq:Energy of Sec. 1.1.5 and error norms).
#include "common.cuh"

namespace pml {

// ---------------------------------------------------------------------------------
// ghost ring: every stored vertex outside [0, T) of some axis takes the value of its
// periodic image inside the box.
// ---------------------------------------------------------------------------------
template <typename T> __global__ void k_fill_ghosts(T *f, const Geom g)
{
    const int64_t nx = g.T[0] + 2 * G, ny = g.T[1] + 2 * G, nz = g.ndim == 3 ? g.T[2] + 2 * G : 1;
    const int64_t total = nx * ny * nz;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t x = i % nx - G, y = (i / nx) % ny - G;
        const int64_t z = g.ndim == 3 ? i / (nx * ny) - G : 0;
        const bool inside = x >= 0 && x < g.T[0] && y >= 0 && y < g.T[1] &&
                            (g.ndim == 2 || (z >= 0 && z < g.T[2]));
        if (inside) continue;
        const int64_t xs = (x + g.T[0]) % g.T[0], ys = (y + g.T[1]) % g.T[1];
        const int64_t zs = g.ndim == 3 ? (z + g.T[2]) % g.T[2] : 0;
        f[g.origin + x + y * g.P + z * g.PS] = f[g.origin + xs + ys * g.P + zs * g.PS];
    }
}

cudaError_t launch_fill_ghosts(int prec, void *f, const Geom &g, cudaStream_t st)
{
    const int blocks = 1024, threads = 256;
    if (prec == 32) k_fill_ghosts<float><<<blocks, threads, 0, st>>>((float *)f, g);
    else k_fill_ghosts<double><<<blocks, threads, 0, st>>>((double *)f, g);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// finiteness scan: one block per row (y, z) of the box, threads along x; the first
// non-finite value sets the error word (code 2) that the host reads at its next
// synchronising call
// ---------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_check_finite(const T *U, const T *V, const Geom g, DeviceError *err,
                                                      long long step)
{
    const int64_t rows = g.T[1] * g.T[2];
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const int64_t y = r % g.T[1], z = r / g.T[1];
        const int64_t o = g.origin + y * g.P + z * g.PS;
        int bad = 0;
        for (int64_t x = threadIdx.x; x < g.T[0]; x += blockDim.x)
            bad |= (isfinite(U[o + x]) ? 0 : 1) | (isfinite(V[o + x]) ? 0 : 2);
        if (__syncthreads_or(bad)) {   // the same answer in every thread: a uniform return
            if (bad && atomicCAS(&err->code, 0, 2) == 0) {
                err->where = (bad & 1) ? 0 : 1;
                err->step = step;
            }
            return;
        }
    }
}

cudaError_t launch_check_finite(int prec, const void *U, const void *V, const Geom &g, DeviceError *err,
                                int64_t step, cudaStream_t st)
{
    const int64_t rows = g.T[1] * g.T[2];
    const int blocks = int(rows < 2048 ? rows : 2048);
    if (prec == 32) k_check_finite<float><<<blocks, 256, 0, st>>>((const float *)U, (const float *)V, g, err, step);
    else k_check_finite<double><<<blocks, 256, 0, st>>>((const double *)U, (const double *)V, g, err, step);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// point sources and receivers
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double ricker(double t, double f, double t0)
{
    const double a = (3.14159265358979323846 * f * (t - t0)) * (3.14159265358979323846 * f * (t - t0));
    return (1.0 - 2.0 * a) * exp(-a);
}

template <typename T>
__device__ __forceinline__ void add_wrapped(T *base, const Geom &g, int64_t x, int64_t y, int64_t z, double v)
{
    const int64_t o = g.origin + x + y * g.P + z * g.PS;
    const T nv = T(double(base[o]) + v);
    store_wrapped(base, g, x, y, z, nv);
}

// Adds the exact RK4 contribution of the sources over one step (step index n, times
// t = n dt, t + dt/2, t + dt).  With forcing b(t) = a g(t) e_V(x_s), classic RK4 adds
//   S = dt (b1 + 4 b2 + b4)/6 + dt^2 A (b1 + 2 b2)/6 + dt^3 A^2 (b1 + b2)/12 + dt^4 A^3 b1/24
// to P(dt A) y, and near the source (where no damping term is within reach)
// A e_V = e_U, A^2 e_V = (0, L delta), A^3 e_V = (L delta, 0).  Then the receivers read U.
// One thread per source; sources whose stencils meet are in different levels (PointArgs),
// so every vertex receives its additions in source order.
template <typename T>
__global__ void k_post_step(T *U, T *V, const PointArgs a, int64_t step, T *trace_row)
{
    const Geom &g = a.g;
    const double dt = a.dt, t = double(step) * dt, ih2 = 1.0 / (a.h * a.h);
    const int nd = g.ndim;
    for (int lv = 0; lv < a.src_levels; ++lv) {   // one thread per source of the level
        for (int s = threadIdx.x; s < a.ns; s += blockDim.x) {
            if (a.src_level[s] != lv) continue;
            const double am = a.src_amp[s];
            const double b1 = am * ricker(t, a.f_peak, a.t_delay);
            const double b2 = am * ricker(t + 0.5 * dt, a.f_peak, a.t_delay);
            const double b4 = am * ricker(t + dt, a.f_peak, a.t_delay);
            const double sV0 = dt * (b1 + 4.0 * b2 + b4) / 6.0;
            const double cV = dt * dt * dt * (b1 + b2) / 12.0;
            const double sU0 = dt * dt * (b1 + 2.0 * b2) / 6.0;
            const double cU = dt * dt * dt * dt * b1 / 24.0;
            // the stencil: the vertex and its 2 nd neighbours, all distinct, so every load can
            // be issued before the first store
            int64_t cc[7][3];
            const int nk = 1 + 2 * nd;
            cc[0][0] = a.src_xyz[3 * s];
            cc[0][1] = a.src_xyz[3 * s + 1];
            cc[0][2] = a.src_xyz[3 * s + 2];
            for (int ax = 0, k = 1; ax < nd; ++ax) {
                for (int sg = -1; sg <= 1; sg += 2, ++k) {
                    cc[k][0] = cc[0][0];
                    cc[k][1] = cc[0][1];
                    cc[k][2] = cc[0][2];
                    int64_t v = cc[0][ax] + sg;
                    v += v < 0 ? g.T[ax] : 0;
                    v -= v >= g.T[ax] ? g.T[ax] : 0;
                    cc[k][ax] = v;
                }
            }
            T ov[7], ou[7];
            for (int k = 0; k < nk; ++k) {
                const int64_t o = g.origin + cc[k][0] + cc[k][1] * g.P + cc[k][2] * g.PS;
                ov[k] = V[o];
                ou[k] = U[o];
            }
            for (int k = 0; k < nk; ++k) {
                const double dv = k == 0 ? sV0 - cV * 2.0 * nd * ih2 : cV * ih2;
                const double du = k == 0 ? sU0 - cU * 2.0 * nd * ih2 : cU * ih2;
                store_wrapped(V, g, cc[k][0], cc[k][1], cc[k][2], T(double(ov[k]) + dv));
                store_wrapped(U, g, cc[k][0], cc[k][1], cc[k][2], T(double(ou[k]) + du));
            }
        }
        __syncthreads();
    }
    if (trace_row)
        for (int r = threadIdx.x; r < a.nr; r += blockDim.x) trace_row[r] = U[g.origin + a.rec_off[r]];
}

cudaError_t launch_post_step(int prec, void *U, void *V, const PointArgs &a, int64_t step, void *trace_row,
                             cudaStream_t st)
{
    if (prec == 32) k_post_step<float><<<1, 128, 0, st>>>((float *)U, (float *)V, a, step, (float *)trace_row);
    else k_post_step<double><<<1, 128, 0, st>>>((double *)U, (double *)V, a, step, (double *)trace_row);
    return cudaGetLastError();
}

// Adjoint counterpart, run on the adjoint state of forward step index m before the
// reverse step m-1 -> m:
//   1. Ub(x_r) += residual_row[r]  (dJ/dU_m at the receivers)
//   2. dJ/da_s += ybar^T S / a_s = dt (g1 + 4 g2 + g4)/6 Vb + dt^2 (g1 + 2 g2)/6 Ub
//                 + dt^3 (g1 + g2)/12 (L Vb) + dt^4 g1/24 (L Ub)   at x_s
//      with g_i the Ricker values at t = (m-1) dt, t + dt/2, t + dt.
template <typename T>
__global__ void k_adjoint_points(T *Ub, T *Vb, const PointArgs a, int64_t m, const T *residual_row,
                                 double *grad_amp)
{
    const Geom &g = a.g;
    if (residual_row) {
        for (int lv = 0; lv < a.rec_levels; ++lv) {   // one thread per receiver of the level
            for (int r = threadIdx.x; r < a.nr; r += blockDim.x)
                if (a.rec_level[r] == lv)
                    add_wrapped(Ub, g, a.rec_xyz[3 * r], a.rec_xyz[3 * r + 1], a.rec_xyz[3 * r + 2],
                                double(residual_row[r]));
            __syncthreads();
        }
    }
    __syncthreads();
    if (grad_amp) {
        const double dt = a.dt, t = double(m - 1) * dt, ih2 = 1.0 / (a.h * a.h);
        for (int s = threadIdx.x; s < a.ns; s += blockDim.x) {
            const double g1 = ricker(t, a.f_peak, a.t_delay);
            const double g2 = ricker(t + 0.5 * dt, a.f_peak, a.t_delay);
            const double g4 = ricker(t + dt, a.f_peak, a.t_delay);
            const int64_t x = a.src_xyz[3 * s], y = a.src_xyz[3 * s + 1], z = a.src_xyz[3 * s + 2];
            const int64_t o = g.origin + x + y * g.P + z * g.PS;
            const double u = Ub[o], v = Vb[o];
            double lu = -2.0 * g.ndim * u, lv = -2.0 * g.ndim * v;
            const int64_t st[3] = {1, g.P, g.PS};
            for (int ax = 0; ax < g.ndim; ++ax) {
                lu += double(Ub[o + st[ax]]) + double(Ub[o - st[ax]]);
                lv += double(Vb[o + st[ax]]) + double(Vb[o - st[ax]]);
            }
            lu *= ih2;
            lv *= ih2;
            grad_amp[s] += dt * (g1 + 4.0 * g2 + g4) / 6.0 * v + dt * dt * (g1 + 2.0 * g2) / 6.0 * u +
                           dt * dt * dt * (g1 + g2) / 12.0 * lv + dt * dt * dt * dt * g1 / 24.0 * lu;
        }
    }
}

cudaError_t launch_adjoint_points(int prec, void *Ub, void *Vb, const PointArgs &a, int64_t m,
                                  const void *residual_row, double *grad_amp, cudaStream_t st)
{
    if (prec == 32)
        k_adjoint_points<float><<<1, 128, 0, st>>>((float *)Ub, (float *)Vb, a, m, (const float *)residual_row, grad_amp);
    else
        k_adjoint_points<double><<<1, 128, 0, st>>>((double *)Ub, (double *)Vb, a, m, (const double *)residual_row, grad_amp);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// FP64 norms over the physical window (deterministic: fixed block partition, fixed
// per-thread order, fixed tree).
//   v[0] = sum V^2 + sum_a ((U(i+e_a) - U(i))/h)^2    (2 E, eq:Energy)
//   v[1] = max |U|, v[2] = sum U^2, v[3] = sum (U - ref)^2, v[4] = max |U - ref|
// ---------------------------------------------------------------------------------
struct NormArgs {
    Geom g;
    int64_t wlo[3], whi[3];
    double ih;
    const double *ref;
};

template <typename T> __global__ void __launch_bounds__(256) k_norms_partial(const T *U, const T *V, const NormArgs a, double *part)
{
    const Geom &g = a.g;
    const int64_t nxw = a.whi[0] - a.wlo[0] + 1, nyw = a.whi[1] - a.wlo[1] + 1;
    const int64_t nzw = g.ndim == 3 ? a.whi[2] - a.wlo[2] + 1 : 1;
    const int64_t rows = nyw * nzw;
    const int64_t r0 = rows * blockIdx.x / gridDim.x, r1 = rows * (blockIdx.x + 1) / gridDim.x;
    double e = 0.0, mx = 0.0, s2 = 0.0, d2 = 0.0, dm = 0.0;
    const int64_t st[3] = {1, g.P, g.PS};
    for (int64_t row = r0; row < r1; ++row) {
        const int64_t y = a.wlo[1] + row % nyw, z = g.ndim == 3 ? a.wlo[2] + row / nyw : 0;
        for (int64_t xi = threadIdx.x; xi < nxw; xi += blockDim.x) {
            const int64_t x = a.wlo[0] + xi;
            const int64_t o = g.origin + x + y * g.P + z * g.PS;
            const double u = U[o], v = V[o];
            double el = 0.0;
            for (int ax = 0; ax < g.ndim; ++ax) {
                const double d = (double(U[o + st[ax]]) - u) * a.ih;
                el += d * d;
            }
            e += v * v + el;
            mx = fmax(mx, fabs(u));
            s2 += u * u;
            if (a.ref) {
                const double rf = a.ref[xi + nxw * ((y - a.wlo[1]) + nyw * (z - (g.ndim == 3 ? a.wlo[2] : 0)))];
                const double d = u - rf;
                d2 += d * d;
                dm = fmax(dm, fabs(d));
            }
        }
    }
    __shared__ double sh[kNormVals][256];
    sh[0][threadIdx.x] = e;
    sh[1][threadIdx.x] = mx;
    sh[2][threadIdx.x] = s2;
    sh[3][threadIdx.x] = d2;
    sh[4][threadIdx.x] = dm;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + w]);
            sh[2][threadIdx.x] += sh[2][threadIdx.x + w];
            sh[3][threadIdx.x] += sh[3][threadIdx.x + w];
            sh[4][threadIdx.x] = fmax(sh[4][threadIdx.x], sh[4][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x < kNormVals) part[blockIdx.x * kNormVals + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(256) k_norms_final(const double *part, int nblocks, double *out)
{
    double e = 0.0, mx = 0.0, s2 = 0.0, d2 = 0.0, dm = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        e += part[b * kNormVals + 0];
        mx = fmax(mx, part[b * kNormVals + 1]);
        s2 += part[b * kNormVals + 2];
        d2 += part[b * kNormVals + 3];
        dm = fmax(dm, part[b * kNormVals + 4]);
    }
    __shared__ double sh[kNormVals][256];
    sh[0][threadIdx.x] = e;
    sh[1][threadIdx.x] = mx;
    sh[2][threadIdx.x] = s2;
    sh[3][threadIdx.x] = d2;
    sh[4][threadIdx.x] = dm;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + w]);
            sh[2][threadIdx.x] += sh[2][threadIdx.x + w];
            sh[3][threadIdx.x] += sh[3][threadIdx.x + w];
            sh[4][threadIdx.x] = fmax(sh[4][threadIdx.x], sh[4][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = 0.5 * sh[0][0];
        out[1] = sh[1][0];
        out[2] = sqrt(sh[2][0]);
        out[3] = sqrt(sh[3][0]);
        out[4] = sh[4][0];
    }
}

cudaError_t launch_norms(int prec, const void *U, const void *V, const Geom &g, const int64_t *wlo,
                         const int64_t *whi, double h, const double *ref, double *partials, int nblocks,
                         double *out, cudaStream_t st)
{
    NormArgs a;
    a.g = g;
    for (int k = 0; k < 3; ++k) {
        a.wlo[k] = wlo[k];
        a.whi[k] = whi[k];
    }
    a.ih = 1.0 / h;
    a.ref = ref;
    if (prec == 32) k_norms_partial<float><<<nblocks, 256, 0, st>>>((const float *)U, (const float *)V, a, partials);
    else k_norms_partial<double><<<nblocks, 256, 0, st>>>((const double *)U, (const double *)V, a, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_norms_final<<<1, 256, 0, st>>>(partials, nblocks, out);
    return cudaGetLastError();
}

}  // namespace pml
