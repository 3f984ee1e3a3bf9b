// Box kernel instantiations for radii 13..16 (see k_disc.cuh).
#include "k_disc.cuh"
RL_BOX_TU(13)
RL_BOX_TU(14)
RL_BOX_TU(15)
RL_BOX_TU(16)
