// Rectangle kernel, halo 8 (see k_disc.cuh).
#include "k_disc.cuh"
RL_RECT_TU(8)
