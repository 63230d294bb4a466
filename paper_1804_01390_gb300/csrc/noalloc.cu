// Energy and norms of a dense field pair without any device allocation.
//
// pml_norms needs a context, and a context needs a workspace.  Some callers cannot
// allocate device memory at the point where they want these numbers: services that
// reserve all their memory at start-up and must not allocate afterwards (so that latency
// stays predictable and an allocation failure cannot happen mid-run), and processes whose
// device memory is owned entirely by another allocator or capped by a fixed budget (for
// example a framework's caching allocator that already holds the free memory).  This file
// gives them pml_norms_dense_static: the caller passes the fields and receives the five
// numbers; the per-row partial sums go to a fixed array in this library's own device
// memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "pml.h"

namespace pml {
void set_global_error(const char *msg);   // runtime.cu: text for pml_last_error(NULL)
}

namespace {

constexpr int kMaxRows = 16384;   // window rows (y, z) one call may reduce
constexpr int kVals = 5;
constexpr int kMaxDevices = 64;

// Per-row partial sums of every call (kMaxRows x 5) followed by the 5 results.  Every
// process that loads the library holds this array on each device it touches, until exit.
static __device__ __align__(256) double g_scratch[kMaxRows * kVals + 8];

std::mutex g_mutex;

// Device address of g_scratch in the context current on device `dev`.  The host-side name
// of the array is not a device address; the address is looked up with the device current,
// once per device and context: after cudaDeviceReset, or with another context made current
// on the same device, the array lives at a new address, so the cached one is replaced.
struct ScratchEntry {
    CUcontext ctx;
    double *addr;
};
ScratchEntry g_scratch_addr[kMaxDevices] = {};
PFN_cuCtxGetCurrent_v4000 g_ctx_current = nullptr;

CUcontext current_context()
{
    if (!g_ctx_current) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return nullptr;
        g_ctx_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
    }
    CUcontext c = nullptr;
    if (g_ctx_current(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

cudaError_t scratch_address(int dev, double **out)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    ScratchEntry &e = g_scratch_addr[dev];
    const CUcontext before = current_context();
    if (before && e.addr && e.ctx == before) {
        *out = e.addr;
        return cudaSuccess;
    }
    void *p = nullptr;
    const cudaError_t r = cudaGetSymbolAddress(&p, g_scratch);   // makes the device's context current
    if (r != cudaSuccess) return r;
    e.ctx = current_context();
    e.addr = e.ctx ? static_cast<double *>(p) : nullptr;          // no context to key on: look up again next time
    *out = static_cast<double *>(p);
    return cudaSuccess;
}

struct DenseArgs {
    int ndim;
    int64_t T[3];
    int64_t lo[3], hi[3];
    double ih;
    const double *ref;   // dense FP64 array of the window shape, or NULL
};

// One block per window row: fixed per-thread order, fixed tree; every call overwrites the
// partial of every row it uses, so nothing carries over from an earlier call.
template <typename T>
__global__ void __launch_bounds__(256) k_rows(const T *U, const T *V, const DenseArgs a, double *part)
{
    const int64_t nxw = a.hi[0] - a.lo[0] + 1, nyw = a.hi[1] - a.lo[1] + 1;
    const int64_t row = blockIdx.x;
    const int64_t y = a.lo[1] + row % nyw, z = a.ndim == 3 ? a.lo[2] + row / nyw : 0;
    const int64_t T0 = a.T[0], T1 = a.T[1], T2 = a.ndim == 3 ? a.T[2] : 1;
    const int64_t yp = (y + 1) % T1, zp = (z + 1) % T2;
    double e = 0.0, mx = 0.0, s2 = 0.0, d2 = 0.0, dm = 0.0;
    for (int64_t xi = threadIdx.x; xi < nxw; xi += blockDim.x) {
        const int64_t x = a.lo[0] + xi, xp = (x + 1) % T0;
        const int64_t o = x + T0 * (y + T1 * z);
        const double u = U[o], v = V[o];
        double el = 0.0, d;
        d = (double(U[xp + T0 * (y + T1 * z)]) - u) * a.ih;
        el += d * d;
        d = (double(U[x + T0 * (yp + T1 * z)]) - u) * a.ih;
        el += d * d;
        if (a.ndim == 3) {
            d = (double(U[x + T0 * (y + T1 * zp)]) - u) * a.ih;
            el += d * d;
        }
        e += v * v + el;
        mx = fmax(mx, fabs(u));
        s2 += u * u;
        if (a.ref) {
            const double r = a.ref[xi + nxw * row];
            d2 += (u - r) * (u - r);
            dm = fmax(dm, fabs(u - r));
        }
    }
    __shared__ double sh[kVals][256];
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
    if (threadIdx.x < kVals) part[row * kVals + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(256) k_rows_final(const double *part, int nrows, double *out)
{
    double e = 0.0, mx = 0.0, s2 = 0.0, d2 = 0.0, dm = 0.0;
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
        e += part[r * kVals + 0];
        mx = fmax(mx, part[r * kVals + 1]);
        s2 += part[r * kVals + 2];
        d2 += part[r * kVals + 3];
        dm = fmax(dm, part[r * kVals + 4]);
    }
    __shared__ double sh[kVals][256];
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

pml_status fail(pml_status s, const char *msg)
{
    pml::set_global_error(msg);
    return s;
}

}  // namespace

extern "C" pml_status pml_norms_dense_static(int ndim, const int64_t *T, int precision, const void *U, const void *V,
                                              const int64_t *wlo, const int64_t *whi, double h, const double *ref,
                                              void *cuda_stream, double *out)
{
    if (ndim != 2 && ndim != 3) return fail(PML_EINVAL, "pml_norms_dense_static: ndim must be 2 or 3");
    if (precision != 32 && precision != 64) return fail(PML_EINVAL, "pml_norms_dense_static: precision must be 32 or 64");
    if (!T || !U || !V || !wlo || !whi || !out) return fail(PML_EINVAL, "pml_norms_dense_static: NULL argument");
    if (!(h > 0.0)) return fail(PML_EINVAL, "pml_norms_dense_static: h must be > 0");
    DenseArgs a{};
    a.ndim = ndim;
    a.ih = 1.0 / h;
    a.ref = ref;
    int64_t rows = 1;
    for (int k = 0; k < 3; ++k) {
        a.T[k] = k < ndim ? T[k] : 1;
        a.lo[k] = k < ndim ? wlo[k] : 0;
        a.hi[k] = k < ndim ? whi[k] : 0;
        if (a.T[k] < 1 || a.lo[k] < 0 || a.hi[k] < a.lo[k] || a.hi[k] >= a.T[k])
            return fail(PML_EINVAL, "pml_norms_dense_static: window must satisfy 0 <= lo <= hi < T on every axis");
        if (k >= 1) rows *= a.hi[k] - a.lo[k] + 1;
    }
    if (rows > kMaxRows)
        return fail(PML_EINVAL, "pml_norms_dense_static: the window has more than 16384 rows (y extent times z "
                                "extent); its fixed scratch holds one partial sum per row");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(PML_ECUDA, "pml_norms_dense_static: no usable current CUDA device");
    double *scratch = nullptr;
    cudaError_t e = scratch_address(dev, &scratch);
    if (e != cudaSuccess) return fail(PML_ECUDA, "pml_norms_dense_static: cudaGetSymbolAddress failed");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    double *result = scratch + size_t(kMaxRows) * kVals;
    if (precision == 32) k_rows<float><<<unsigned(rows), 256, 0, st>>>((const float *)U, (const float *)V, a, scratch);
    else k_rows<double><<<unsigned(rows), 256, 0, st>>>((const double *)U, (const double *)V, a, scratch);
    k_rows_final<<<1, 256, 0, st>>>(scratch, int(rows), result);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, result, kVals * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(PML_ECUDA, cudaGetErrorString(e));
    return PML_OK;
}
