// Disc kernel instantiation for radius 1 (see k_disc.cuh).
#include "k_disc.cuh"
RL_DISC_RADIUS_TU(1)
