// Box kernel instantiations for radii 1..4 (see k_disc.cuh).
#include "k_disc.cuh"
RL_BOX_TU(1)
RL_BOX_TU(2)
RL_BOX_TU(3)
RL_BOX_TU(4)
