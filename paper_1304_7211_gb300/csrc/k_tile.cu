// k_tile.cu -- tile shape choice and storage dispatch of the 2D tile kernels
// (k_tile.cuh; one translation unit per storage type).
#include "rl_launch.h"

namespace rl {

TileShape tile_shape_for(int ax, int bx, int ay, int by) {
    const int e = ax + bx > ay + by ? ax + bx : ay + by;
    if (e <= 8) return {64, 32};
    if (e <= 20) return {64, 64};
    return {128, 64};
}

cudaError_t launch_tile(const IterArgs &a, int storage, bool thin, int mode, TileShape ts,
                        cudaStream_t s) {
    switch (storage) {
    case ST_F32: return launch_tile_f32(a, thin, mode, ts, s);
    case ST_BF16: return launch_tile_bf16(a, thin, mode, ts, s);
    case ST_F16: return launch_tile_f16(a, thin, mode, ts, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace rl
