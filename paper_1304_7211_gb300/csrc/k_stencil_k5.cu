// Register-blocked stencil instantiation for 5x5 taps (see k_disc.cuh).
#include "k_disc.cuh"
RL_STENCIL_TU(5)
