// k_disc.cu -- radius / size dispatch of the register-blocked disc, box and stencil kernels.
#include "rl_launch.h"

namespace rl {

cudaError_t launch_disc(const IterArgs &a, int storage, bool thin, int radius, float *qplane,
                        long long q_pitch, cudaStream_t s) {
    switch (radius) {
#define RL_DISC_CASE(R) \
    case R: return launch_disc_r##R(a, storage, thin, qplane, q_pitch, s);
    RL_DISC_CASE(1) RL_DISC_CASE(2) RL_DISC_CASE(3) RL_DISC_CASE(4) RL_DISC_CASE(5)
    RL_DISC_CASE(6) RL_DISC_CASE(7) RL_DISC_CASE(8) RL_DISC_CASE(9) RL_DISC_CASE(10)
    RL_DISC_CASE(11) RL_DISC_CASE(12) RL_DISC_CASE(13) RL_DISC_CASE(14) RL_DISC_CASE(15)
    RL_DISC_CASE(16)
#undef RL_DISC_CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_box(const IterArgs &a, int storage, bool thin, int radius, float *qplane, long long q_pitch,
                       cudaStream_t s) {
    switch (radius) {
#define RL_BOX_CASE(R) \
    case R: return launch_box_r##R(a, storage, thin, qplane, q_pitch, s);
    RL_BOX_CASE(1) RL_BOX_CASE(2) RL_BOX_CASE(3) RL_BOX_CASE(4) RL_BOX_CASE(5)
    RL_BOX_CASE(6) RL_BOX_CASE(7) RL_BOX_CASE(8) RL_BOX_CASE(9) RL_BOX_CASE(10)
    RL_BOX_CASE(11) RL_BOX_CASE(12) RL_BOX_CASE(13) RL_BOX_CASE(14) RL_BOX_CASE(15)
    RL_BOX_CASE(16)
#undef RL_BOX_CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_tiles(int op, int radius, const TileJob *jobs, const int2 *items, int n_items, int phase,
                         cudaStream_t s) {
    switch (radius) {
#define RL_TILES_CASE(R)                                                                    \
    case R:                                                                                 \
        return op == 0 ? launch_disc_tiles_r##R(jobs, items, n_items, phase, s)             \
                       : launch_box_tiles_r##R(jobs, items, n_items, phase, s);
    RL_TILES_CASE(1) RL_TILES_CASE(2) RL_TILES_CASE(3) RL_TILES_CASE(4) RL_TILES_CASE(5)
    RL_TILES_CASE(6) RL_TILES_CASE(7) RL_TILES_CASE(8) RL_TILES_CASE(9) RL_TILES_CASE(10)
    RL_TILES_CASE(11) RL_TILES_CASE(12) RL_TILES_CASE(13) RL_TILES_CASE(14) RL_TILES_CASE(15)
    RL_TILES_CASE(16)
#undef RL_TILES_CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_tiles_persist(int op, int radius, const TilesPersistArgs &p, cudaStream_t s) {
    switch (radius) {
#define RL_TP_CASE(R)                                                                       \
    case R:                                                                                 \
        return op == 0 ? launch_disc_tiles_persist_r##R(p, s) : launch_box_tiles_persist_r##R(p, s);
    RL_TP_CASE(1) RL_TP_CASE(2) RL_TP_CASE(3) RL_TP_CASE(4) RL_TP_CASE(5) RL_TP_CASE(6) RL_TP_CASE(7)
    RL_TP_CASE(8) RL_TP_CASE(9) RL_TP_CASE(10) RL_TP_CASE(11) RL_TP_CASE(12) RL_TP_CASE(13) RL_TP_CASE(14)
    RL_TP_CASE(15) RL_TP_CASE(16)
#undef RL_TP_CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_disc_persist(const PersistArgs &p, int storage, int radius, cudaStream_t s) {
    switch (radius) {
#define RL_PERSIST_CASE(R) \
    case R: return launch_disc_persist_r##R(p, storage, s);
    RL_PERSIST_CASE(1) RL_PERSIST_CASE(2) RL_PERSIST_CASE(3) RL_PERSIST_CASE(4) RL_PERSIST_CASE(5)
    RL_PERSIST_CASE(6) RL_PERSIST_CASE(7) RL_PERSIST_CASE(8) RL_PERSIST_CASE(9) RL_PERSIST_CASE(10)
    RL_PERSIST_CASE(11) RL_PERSIST_CASE(12) RL_PERSIST_CASE(13) RL_PERSIST_CASE(14) RL_PERSIST_CASE(15)
    RL_PERSIST_CASE(16)
#undef RL_PERSIST_CASE
    }
    return cudaErrorNotSupported;
}

cudaError_t launch_stencil(const IterArgs &a, const float *taps, int K, int storage, bool thin,
                           float *qplane, long long q_pitch, cudaStream_t s) {
    switch (K) {
    case 3: return launch_stencil_k3(a, taps, storage, thin, qplane, q_pitch, s);
    case 5: return launch_stencil_k5(a, taps, storage, thin, qplane, q_pitch, s);
    case 7: return launch_stencil_k7(a, taps, storage, thin, qplane, q_pitch, s);
    case 9: return launch_stencil_k9(a, taps, storage, thin, qplane, q_pitch, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace rl
