// Register-blocked stencil instantiation for 3x3 taps (see k_disc.cuh).
#include "k_disc.cuh"
RL_STENCIL_TU(3)
