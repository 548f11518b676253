// Tiled window gather (K3): the gaussian kernels' instantiations.
#include "k3_tiled_kernels.cuh"

namespace swih {

cudaError_t tiled_dispatch_gaussian(int elem_bytes, int gdx, int gdy, int tx, int bb, TiledOp &op)
{
    return dispatch_kind<kGatherGaussian>(elem_bytes, gdx, gdy, tx, bb, op);
}

}  // namespace swih
