// 3D layer kernels for boxes ended by reflecting walls (see layer3d.cuh).
#include "layer3d.cuh"

namespace pml {

cudaError_t launch_layer3d_wall(int prec, bool adjoint, const CUtensorMap *tm, void *const *outp,
                                const Layer3DArgs &a, cudaStream_t st)
{
    return launch_layer3d_impl<true>(prec, adjoint, tm, outp, a, st);
}

}  // namespace pml
