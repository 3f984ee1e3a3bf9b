// k_transpose.cu -- tiled transpose of image planes (32 x 32 tiles staged in
// shared memory, coalesced on both sides).  Motion blur along y runs as
// motion blur along x on the transposed image.
#include "rl_launch.h"

namespace rl {

namespace {

template <typename E>
__global__ void __launch_bounds__(256) k_transpose(const E *src, long long sp, long long s_plane,
                                                   E *dst, long long dp, long long d_plane, int W,
                                                   int H) {
    __shared__ E tile[32][33];
    const E *sb = src + (long long)blockIdx.z * s_plane;
    E *db = dst + (long long)blockIdx.z * d_plane;
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    for (int r = ty; r < 32; r += 8) {
        const int x = bx + tx, y = by + r;
        if (x < W && y < H) tile[r][tx] = sb[(long long)y * sp + x];
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int x = by + tx, y = bx + r;  // dst is H wide, W tall
        if (x < H && y < W) db[(long long)y * dp + x] = tile[tx][r];
    }
}

template <typename E>
cudaError_t launch_e(const void *src, long long sp, long long s_plane, void *dst, long long dp,
                     long long d_plane, int W, int H, int n, cudaStream_t s) {
    dim3 grid((W + 31) / 32, (H + 31) / 32, n);
    k_transpose<E><<<grid, 256, 0, s>>>((const E *)src, sp, s_plane, (E *)dst, dp, d_plane, W, H);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_transpose(const void *src, long long sp, long long s_plane, void *dst,
                             long long dp, long long d_plane, int W, int H, int n_planes,
                             int elem_bytes, cudaStream_t s) {
    if (n_planes < 1 || n_planes > 65535) return cudaErrorInvalidValue;
    switch (elem_bytes) {
    case 4: return launch_e<unsigned>(src, sp, s_plane, dst, dp, d_plane, W, H, n_planes, s);
    case 2: return launch_e<unsigned short>(src, sp, s_plane, dst, dp, d_plane, W, H, n_planes, s);
    case 1: return launch_e<unsigned char>(src, sp, s_plane, dst, dp, d_plane, W, H, n_planes, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace rl
