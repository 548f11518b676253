// Instantiation entry points of the tiled window gather (K3), one translation
// unit per kernel kind so that they compile in parallel. Host code only.
#pragma once

#include "swih_internal.h"

namespace swih {

// What to do with the kernel of one (kind, element type, tile width, degrees,
// bins per step) shape: report its registers, launch it for one job, or launch
// it over a device table of jobs.
struct TiledOp {
    enum What { kRegs, kSingle, kTable } what = kRegs;
    const GatherParams *p = nullptr;  // kSingle: the job (host copy, passed by value)
    const GatherShape *sh = nullptr;
    const GatherParams *d_jobs = nullptr;  // kTable
    const int *d_items = nullptr;
    int n_jobs = 0, n_items = 0;
    cudaStream_t s = nullptr;
    int regs = 255;  // kRegs: the answer
};

cudaError_t tiled_dispatch_plain(int elem_bytes, int gdx, int gdy, int tx, int bb, TiledOp &op);
cudaError_t tiled_dispatch_manhattan(int elem_bytes, int gdx, int gdy, int tx, int bb, TiledOp &op);
cudaError_t tiled_dispatch_euclidean(int elem_bytes, int gdx, int gdy, int tx, int bb, TiledOp &op);
cudaError_t tiled_dispatch_gaussian(int elem_bytes, int gdx, int gdy, int tx, int bb, TiledOp &op);

inline cudaError_t tiled_dispatch(int kind, int elem_bytes, int gdx, int gdy, int tx, int bb, TiledOp &op)
{
    switch (kind) {
    case kGatherPlain: return tiled_dispatch_plain(elem_bytes, gdx, gdy, tx, bb, op);
    case kGatherManhattan: return tiled_dispatch_manhattan(elem_bytes, gdx, gdy, tx, bb, op);
    case kGatherEuclidean: return tiled_dispatch_euclidean(elem_bytes, gdx, gdy, tx, bb, op);
    case kGatherGaussian: return tiled_dispatch_gaussian(elem_bytes, gdx, gdy, tx, bb, op);
    default: return cudaErrorInvalidValue;
    }
}

// shared-memory layout constants of the tiled gather
constexpr int kTiledMaxStages = 8;
constexpr int kTiledDefaultStages = 4;

}  // namespace swih
