// 2D tile kernels, storage __nv_bfloat16 (see k_tile.cuh).
#include "k_tile.cuh"
RL_TILE_TU(launch_tile_bf16, __nv_bfloat16)
