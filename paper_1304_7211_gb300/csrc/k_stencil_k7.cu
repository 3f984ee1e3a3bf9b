// Register-blocked stencil instantiation for 7x7 taps (see k_disc.cuh).
#include "k_disc.cuh"
RL_STENCIL_TU(7)
