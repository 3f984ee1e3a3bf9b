// Resident running-sum kernel instantiation: storage __nv_bfloat16, thinning true (see k_motion_tb.cuh).
#include "k_motion_tb.cuh"
RL_MOTION_TB_TU(launch_motion_tb_bf16_thin, __nv_bfloat16, true)
