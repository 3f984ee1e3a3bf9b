// 2D tile kernels, storage __half (see k_tile.cuh).
#include "k_tile.cuh"
RL_TILE_TU(launch_tile_f16, __half)
