// Ragged batches in one persistent launch.
//
// A cooperative grid (every block resident) walks three stages over all
// volumes of all orders of the batch, separated by grid-wide barriers:
//
//   1. orbit mixing Z = S x     unit = kMixWarps tiles of one volume
//   2. slab DFT (two fast axes) unit = one n x n slab of one volume
//   3. pencil DFT (slow axis)   unit = one middle index x column block
//
// Units of every stage are numbered order by order (the order of a unit is
// found from the per-order unit offsets), each block takes units
// blockIdx.x, blockIdx.x + gridDim.x, ... and the DFT bodies are the same
// register-radix code as the per-order kernels, dispatched on n.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mix_tiled.cuh"

namespace fcc {

constexpr int kRaggedMaxOrders = 16;
constexpr int kRaggedThreads = 256;   // = kMixThreads = kFastThreads = 8 warps

struct RaggedOrder {
    TiledMixArgs mix;        // this order's orbit tables (forward mode)
    int ntiles;              // mixing tiles per volume
    int nvol;                // volumes of this order
    const float2* tw;        // exp(+2 pi i j / n), j < n
    const int64_t* voff;     // point offsets of this order's volumes (device)
    int64_t first[3];        // first unit of this order in each stage
};

struct RaggedArgs {
    int norders;
    int real_in;             // 1: real FP32 volumes in, 0: complex
    int64_t units[3];        // units per stage
    RaggedOrder o[kRaggedMaxOrders];
};

// Host side (ragged.cu).  smem_for: dynamic shared memory the launch needs
// for the given orders; upload: the constant-memory tables of this
// translation unit (same contents as the per-order kernels').
size_t ragged_smem_for(const int* orders, int count);
int64_t ragged_units(int n, int ntiles, int nvol, int stage);
bool ragged_order_supported(int n);
cudaError_t ragged_upload_constants(const float2* cores, const int* W, const int* u);
// grid_blocks: 0 = as many as can be resident; returns the error of the
// cooperative launch (too large a grid is refused, never run)
cudaError_t launch_ragged_persistent(const RaggedArgs& args, const float* in, float* out, size_t smem,
                                     int grid_blocks, cudaStream_t st);

}  // namespace fcc
