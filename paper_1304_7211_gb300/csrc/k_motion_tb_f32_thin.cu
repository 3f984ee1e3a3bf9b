// Resident running-sum kernel instantiation: storage float, thinning true (see k_motion_tb.cuh).
#include "k_motion_tb.cuh"
RL_MOTION_TB_TU(launch_motion_tb_f32_thin, float, true)
