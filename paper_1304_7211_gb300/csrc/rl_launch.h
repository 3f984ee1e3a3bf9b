// rl_launch.h -- host-side launch entry points of the RL kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "rl_common.cuh"

namespace rl {

enum Storage { ST_F32 = 0, ST_BF16 = 1, ST_F16 = 2 };
enum TileMode { TILE_SPAN = 0, TILE_STENCIL = 1 };

// Running-sum box filter along x (Sec. 3 "Linear motion blur"): one fused RL
// iteration, whole rows resident in shared memory.
cudaError_t launch_motion_x(const IterArgs &a, int storage, bool thin, cudaStream_t s);
size_t motion_x_smem_bytes(int W, int L);
bool motion_x_fits(int W, int L);

// Running-sum box filter along y: column strips streamed through shared
// memory, one fused RL iteration.
cudaError_t launch_motion_y(const IterArgs &a, int storage, bool thin, cudaStream_t s);

// 2D tile kernel: per-row span sums of a uniform PSF (Sec. 3 "generic box
// filter") or direct summation over dense taps (naive / list filter).
struct TileShape { int tx, ty; };
TileShape tile_shape_for(int ax, int bx, int ay, int by);
cudaError_t launch_tile(const IterArgs &a, int storage, bool thin, int mode, TileShape ts,
                        cudaStream_t s);

}  // namespace rl
