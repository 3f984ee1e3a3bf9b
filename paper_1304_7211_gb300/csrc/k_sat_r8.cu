// Summed-area-table rectangle kernel, halo 8 (see k_disc.cuh).
#include "k_disc.cuh"
RL_SAT_TU(8)
