// Box kernel instantiations for radii 5..8 (see k_disc.cuh).
#include "k_disc.cuh"
RL_BOX_TU(5)
RL_BOX_TU(6)
RL_BOX_TU(7)
RL_BOX_TU(8)
