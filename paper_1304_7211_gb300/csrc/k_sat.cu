// k_sat.cu -- halo-class dispatch of the summed-area-table rectangle kernel.
#include <algorithm>
#include <cstdlib>

#include "k_disc.cuh"

RL_SAT_TU(4)

namespace rl {

cudaError_t launch_sat(const IterArgs &a, int lox, int hix, int loy, int hiy, int storage, float *qplane,
                       long long q_pitch, cudaStream_t s) {
    if (lox > hix || loy > hiy) return cudaErrorInvalidValue;
    const int reach = std::max(std::max(std::abs(lox), std::abs(hix)), std::max(std::abs(loy), std::abs(hiy)));
    switch (rect_halo(reach)) {
    case 4: return launch_sat_r4(a, lox, hix, loy, hiy, storage, qplane, q_pitch, s);
    case 8: return launch_sat_r8(a, lox, hix, loy, hiy, storage, qplane, q_pitch, s);
    case 16: return launch_sat_r16(a, lox, hix, loy, hiy, storage, qplane, q_pitch, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace rl
