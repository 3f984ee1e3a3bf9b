// Register-blocked stencil instantiation for 9x9 taps (see k_disc.cuh).
#include "k_disc.cuh"
RL_STENCIL_TU(9)
