// Resident running-sum kernel instantiation: storage __half, thinning false (see k_motion_tb.cuh).
#include "k_motion_tb.cuh"
RL_MOTION_TB_TU(launch_motion_tb_f16, __half, false)
