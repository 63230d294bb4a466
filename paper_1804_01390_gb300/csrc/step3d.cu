// 3D kernels of one RK4 step of the discrete PML system.
#include "common.cuh"

namespace pml {

int interior3d_box_rows(int) { return 1; }
int interior3d_tile_y() { return 16; }
int interior3d_max_blocks_per_sm(int, bool) { return 0; }

cudaError_t launch_interior3d(int, bool, const CUtensorMap *, const CUtensorMap *, void *, void *,
                              const Interior3DArgs &, int, cudaStream_t)
{
    return cudaErrorNotSupported;
}

cudaError_t launch_layer3d(int, bool, const CUtensorMap *, void *const *, const Layer3DArgs &, cudaStream_t)
{
    return cudaErrorNotSupported;
}

}  // namespace pml
