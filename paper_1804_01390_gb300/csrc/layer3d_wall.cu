// 3D layer kernels for boxes ended by reflecting walls (see layer3d.cuh, slab3d.cuh).
#include <cstdio>

#include "layer3d.cuh"
#include "slab3d.cuh"

namespace pml {

cudaError_t launch_layer3d_wall(int prec, bool adjoint, const CUtensorMap *tm, void *const *outp,
                                const Layer3DArgs &a, cudaStream_t st)
{
    return launch_layer3d_impl<true>(prec, adjoint, tm, outp, a, st);
}

template <bool ADJ, int M> static void describe_one_wall(std::string &out)
{
    cudaFuncAttributes fa{};
    const cudaError_t e = cudaFuncGetAttributes(&fa, k_slab3d<ADJ, M, true>);
    char buf[160];
    if (e != cudaSuccess) std::snprintf(buf, sizeof buf, "class %d: %s; ", M, cudaGetErrorString(e));
    else
        std::snprintf(buf, sizeof buf, "class %d: %d threads, %d regs, max block %d, smem %zu+%zu; ", M, Slab<M>::NT,
                      fa.numRegs, fa.maxThreadsPerBlock, size_t(fa.sharedSizeBytes), Slab<M>::SMEM);
    out += buf;
}
std::string slab3d_describe_wall(bool adjoint)
{
    std::string s;
    if (adjoint) {
        describe_one_wall<true, 0>(s); describe_one_wall<true, 1>(s); describe_one_wall<true, 2>(s);
        describe_one_wall<true, 3>(s); describe_one_wall<true, 4>(s); describe_one_wall<true, 5>(s);
        describe_one_wall<true, 6>(s); describe_one_wall<true, 7>(s);
    } else {
        describe_one_wall<false, 0>(s); describe_one_wall<false, 1>(s); describe_one_wall<false, 2>(s);
        describe_one_wall<false, 3>(s); describe_one_wall<false, 4>(s); describe_one_wall<false, 5>(s);
        describe_one_wall<false, 6>(s); describe_one_wall<false, 7>(s);
    }
    return s;
}

cudaError_t launch_slab3d_wall(bool adjoint, const CUtensorMap *tm, void *const *outp, const Layer3DArgs &a,
                               cudaStream_t st)
{
    return launch_slab3d_impl<true>(adjoint, tm, outp, a, st);
}

}  // namespace pml
