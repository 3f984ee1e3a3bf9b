// Box kernel instantiations for radii 9..12 (see k_disc.cuh).
#include "k_disc.cuh"
RL_BOX_TU(9)
RL_BOX_TU(10)
RL_BOX_TU(11)
RL_BOX_TU(12)
