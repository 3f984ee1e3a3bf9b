// k_rect.cu -- halo-class dispatch of the register-blocked rectangle kernel.
#include <algorithm>
#include <cstdlib>

#include "k_disc.cuh"

RL_RECT_TU(4)

namespace rl {

int rect_halo(int reach) { return reach <= 4 ? 4 : reach <= 8 ? 8 : reach <= kRectMaxReach ? 16 : 0; }

cudaError_t launch_rect(const IterArgs &a, int lox, int hix, int loy, int hiy, int storage, bool thin,
                        float *qplane, long long q_pitch, cudaStream_t s) {
    if (lox > hix || loy > hiy) return cudaErrorInvalidValue;
    const int reach = std::max(std::max(std::abs(lox), std::abs(hix)), std::max(std::abs(loy), std::abs(hiy)));
    switch (rect_halo(reach)) {
    case 4: return launch_rect_r4(a, lox, hix, loy, hiy, storage, thin, qplane, q_pitch, s);
    case 8: return launch_rect_r8(a, lox, hix, loy, hiy, storage, thin, qplane, q_pitch, s);
    case 16: return launch_rect_r16(a, lox, hix, loy, hiy, storage, thin, qplane, q_pitch, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace rl
