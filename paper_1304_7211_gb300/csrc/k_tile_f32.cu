// 2D tile kernels, storage float (see k_tile.cuh).
#include "k_tile.cuh"
RL_TILE_TU(launch_tile_f32, float)
