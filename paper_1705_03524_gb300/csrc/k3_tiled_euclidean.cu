// Tiled window gather (K3): the euclidean kernels' instantiations.
#include "k3_tiled_kernels.cuh"

namespace swih {

cudaError_t tiled_dispatch_euclidean(int elem_bytes, int gdx, int gdy, int tx, int bb, TiledOp &op)
{
    return dispatch_kind<kGatherEuclidean>(elem_bytes, gdx, gdy, tx, bb, op);
}

}  // namespace swih
