// k_reduce.cu -- FP64 sums of an image plane (diagnostics: total flux).
// Deterministic: per-block partial sums in a fixed order, then one block
// adds the partials in index order.
#include "rl_launch.h"

namespace rl {

namespace {

constexpr int RT = 256;

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[RT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < RT / 32; ++i) s += ws[i];
    return s;
}

template <typename T>
__global__ void __launch_bounds__(RT) k_sum_partial(const T *p, long long pitch, int W, int H,
                                                    double *partial) {
    double s = 0.0;
    const long long n = (long long)W * H;
    for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        const long long y = i / W, x = i - y * W;
        s += (double)Stor<T>::ld(p, y * pitch + x);
    }
    s = block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(RT) k_sum_final(const double *partial, int n, double *out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += RT) s += partial[i];
    s = block_sum(s);
    if (threadIdx.x == 0) *out = s;
}

}  // namespace

int flux_blocks() { return 608; }

cudaError_t launch_flux(const void *p, long long pitch, int W, int H, int storage, double *partial,
                        double *out, cudaStream_t s) {
    const int nb = flux_blocks();
    switch (storage) {
    case ST_F32: k_sum_partial<float><<<nb, RT, 0, s>>>((const float *)p, pitch, W, H, partial); break;
    case ST_BF16: k_sum_partial<__nv_bfloat16><<<nb, RT, 0, s>>>((const __nv_bfloat16 *)p, pitch, W, H, partial); break;
    case ST_F16: k_sum_partial<__half><<<nb, RT, 0, s>>>((const __half *)p, pitch, W, H, partial); break;
    default: return cudaErrorInvalidValue;
    }
    k_sum_final<<<1, RT, 0, s>>>(partial, nb, out);
    return cudaGetLastError();
}

}  // namespace rl
