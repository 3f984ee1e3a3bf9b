// k_motion_tb.cuh -- the resident running-sum kernel for a motion blur along
// x (Sec. 3 "Linear motion blur"), all K iterations of Eq. 3 in one launch,
// instantiated per storage type and thinning mode in k_motion_tb_*.cu (the
// instantiations are many; separate translation units compile in parallel).
#pragma once

#include "rl_launch.h"

namespace rl {
namespace mtb {

__device__ __forceinline__ void warp_count_add(unsigned long long *ctr, unsigned cnt) {
    unsigned s = __reduce_add_sync(0xffffffffu, cnt);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(ctr, (unsigned long long)s);
}

// ---- motion along x, all iterations with the rows resident -------------------
// Rows are independent under a motion PSF along x for every iteration, so a
// CTA keeps its rows of u, q and f (and the selective-convolution mask) in
// shared memory for all K iterations: HBM sees f and u0 read once and u_K
// written once.  Each iteration is the same arithmetic as k_motion_x (a
// direct sum starting every chunk, then add-the-entering / drop-the-leaving
// sample), with chunks of TCH = 17 outputs: an odd chunk stride puts the 32
// lanes of a warp on 32 distinct banks with no padding.  A value written
// near a row end is also written to the continued positions that map onto
// it, so each iteration needs two barriers.  Inactive pixels keep their q
// entry: it is the ratio of their last active iteration (Eq. 5).

__device__ __forceinline__ void put_cont(float *E, int x, float v, int W, int lo, int hi,
                                         int clamp) {
    // E holds extended coordinates [-lo, W + hi) at index e + lo.
    if (clamp) {
        if (x == 0)
            for (int i = 0; i < lo; ++i) E[i] = v;
        if (x == W - 1)
            for (int i = 0; i < hi; ++i) E[W + lo + i] = v;
    } else {
        if (x < lo) E[lo - 1 - x] = v;
        if (x >= W - hi) E[2 * W - 1 - x + lo] = v;
    }
}

// Exact-transpose adjoint along a row (a.transpose): q is zero outside the
// image, and an output s near a row end also receives, for each padded
// position e != s that the boundary map sends to s, z(e) = w * (sum of q over
// [e - A, e + B] inside the image).  Mirror: e = -1 - s (s < B) gives the
// left-end prefix sum of q over [0, B - 1 - s]; e = 2W - 1 - s (s >= W - A)
// the right-end suffix sum over [2W - 1 - s - A, W - 1]; both slide by one
// sample per output.  Clamp: the whole apron [-B, -1] folds onto s = 0, i.e.
// sum_k (B - k) q(k) over k < B, and [W, W - 1 + A] onto s = W - 1, i.e.
// sum_k (k - W + A + 1) q(k) over k >= W - A.  Qe[k + A] = q(k).  The fold
// sums are formed once per chunk at a row end, outside the output loop.
template <typename T, bool THIN, int TCH, bool TRANS>
__global__ void __launch_bounds__(256) k_motion_x_tb(IterArgs a, TBArgs tb, int tpr, int rpc,
                                                     int line_floats, int mask_bytes) {
    extern __shared__ float sm[];
    const int W = a.W, A = a.ax, B = a.bx, L = A + B + 1;
    const int g = threadIdx.x / tpr, t = threadIdx.x - g * tpr;
    const int y = blockIdx.x * rpc + g;
    const bool row_ok = y < a.H;
    float *Ue = sm + (size_t)g * 3 * line_floats;  // u over [-B, W + A) at e + B
    float *Qe = Ue + line_floats;                  // q over [-A, W + B) at e + A
    float *Fr = Qe + line_floats;                  // f over [0, W)
    uint8_t *Mk = reinterpret_cast<uint8_t *>(sm + (size_t)rpc * 3 * line_floats) + (size_t)g * mask_bytes;
    const float w = a.weight;
    const int edge = A > B ? A : B;  // chunks closer than this to a row end write continuations
    unsigned used = 0;

    if (row_ok) {
        const T *urow = (const T *)a.u_in + (long long)y * a.in_pitch;
        row_to_smem<4>(Ue, [B](int i) { return i + B; }, urow, W, t, tpr);
        row_to_smem<4>(Fr, [](int i) { return i; }, (const T *)a.f + (long long)y * a.f_pitch, W, t, tpr);
        gather_batched<4>(A + B, t, tpr,
            [&](int i) { return Stor<T>::ld(urow, bmap(i < B ? i - B : W + i - B, W, a.clamp)); },
            [&](int i, float v) { Ue[i < B ? i : W + i] = v; });
        for (int i = t; i < W + L - 1; i += tpr) Qe[i] = 0.f;  // stale ratio of a never-used pixel
        if (THIN)
            for (int x = t; x < W; x += tpr) Mk[x] = 1;
    }
    __syncthreads();
    for (int k = 0; k < tb.K; ++k) {
        const bool full = !THIN || (k % tb.P) == 0;
        const uint8_t *srow = (THIN && tb.sched && row_ok)
                                  ? tb.sched + (long long)k * tb.s_plane + (long long)y * tb.s_pitch
                                  : nullptr;
        if (row_ok) {  // q = f / (h (x) u) at the used pixels
            for (int x0 = t * TCH; x0 < W; x0 += tpr * TCH) {
                const bool near_end = x0 < edge || x0 + TCH > W - edge;
                const float *u = Ue + x0;
                float s = 0.f;
                for (int kk = 0; kk < L; ++kk) s += u[kk];
#pragma unroll
                for (int j = 0; j < TCH; ++j) {
                    const int x = x0 + j;
                    if (x < W) {
                        bool use = true;
                        if (THIN) use = srow ? srow[x] != 0 : (full || Mk[x] != 0);
                        if (use) {
                            const float q = rl_ratio(Fr[x], s * w);
                            Qe[x + A] = q;
                            if (near_end && !TRANS) put_cont(Qe, x, q, W, A, B, a.clamp);
                        }
                        if (j + 1 < TCH) s += u[j + L] - u[j];
                    }
                }
            }
        }
        __syncthreads();
        if (row_ok) {  // c = h* (x) q, u' = u c
            for (int x0 = t * TCH; x0 < W; x0 += tpr * TCH) {
                const bool near_end = x0 < edge || x0 + TCH > W - edge;
                const float *qq = Qe + x0;
                float s = 0.f;
                for (int kk = 0; kk < L; ++kk) s += qq[kk];
                // folds of the exact transpose at a row end (mirror: the sums
                // at this chunk's first folded outputs, then sliding)
                const bool tr = TRANS && near_end;
                float fl = 0.f, fr = 0.f;
                if (tr) {
                    if (a.clamp) {
                        if (x0 == 0)
                            for (int k = 0; k < B && k < W; ++k) fl += (float)(B - k) * Qe[k + A];
                        if (W - 1 < x0 + TCH)
                            for (int k = max(0, W - A); k < W; ++k) fr += (float)(k - W + A + 1) * Qe[k + A];
                    } else {
                        for (int k = 0; k <= B - 1 - x0; ++k) fl += Qe[k + A];
                        const int s0 = max(x0, W - A);
                        for (int k = 2 * W - 1 - s0 - A; k <= W - 1 && s0 < x0 + TCH; ++k) fr += Qe[k + A];
                    }
                }
#pragma unroll
                for (int j = 0; j < TCH; ++j) {
                    const int x = x0 + j;
                    if (x < W) {
                        const float u = Ue[x + B];
                        float c = s * w;
                        if (tr) {
                            if (a.clamp) {
                                if (x == 0) c += w * fl;
                                if (x == W - 1) c += w * fr;
                            } else {
                                if (x < B) {
                                    c += w * fl;
                                    fl -= Qe[B - 1 - x + A];
                                }
                                if (x >= W - A) {
                                    c += w * fr;
                                    if (x + 1 < W) fr += Qe[2 * W - 2 - x];
                                }
                            }
                        }
                        float un = u * c;
                        if (THIN) {
                            const bool use = srow ? srow[x] != 0 : (full || Mk[x] != 0);
                            used += use;
                            if (!use) un = u;
                            if (!srow && (tb.Q == 1 || full)) {
                                float d = 0.f;
                                if (use) d = a.relative ? (u > 0.f ? fabsf(c - 1.f) : 0.f) : fabsf(un - u);
                                Mk[x] = (uint8_t)(use && d >= a.tau);
                            }
                        }
                        if (tb.round) un = Stor<T>::round(un);
                        if (j + 1 < TCH) s += qq[j + L] - qq[j];
                        Ue[x + B] = un;
                        if (near_end) put_cont(Ue, x, un, W, B, A, a.clamp);
                    }
                }
            }
        }
        __syncthreads();
    }
    if (row_ok) {
        smem_to_row((T *)a.u_out + (long long)y * a.out_pitch, Ue, [B](int i) { return i + B; }, W, t, tpr);
        if (THIN && !tb.sched && a.mask_out)
            for (int x = t; x < W; x += tpr) a.mask_out[(long long)y * a.m_pitch + x] = Mk[x];
    }
    if (THIN && a.active_count) warp_count_add(a.active_count, used);
}

// Chunk width, threads per row and rows per CTA of the resident kernel.
// chunk = 0: the built-in table by row length; else 13, 17 or 33 (a tuned
// choice).
inline int tb_chunk(int W, int chunk = 0) {
    if (chunk == 13 || chunk == 17 || chunk == 33) return chunk;
    return W <= 13 * 256 ? 13 : (W <= 17 * 256 ? 17 : 33);
}
inline void tb_shape(int W, int chunk, int &tpr, int &rpc) {
    const int ch = tb_chunk(W, chunk);
    const int chunks = (W + ch - 1) / ch;
    tpr = ((chunks + 31) / 32) * 32;
    if (tpr > 256) tpr = 256;
    rpc = 256 / tpr;
}

template <typename T, bool THIN, int TCH>
cudaError_t launch_x_tb_c(const IterArgs &a, const TBArgs &tb, cudaStream_t s) {
    const int L = a.ax + a.bx + 1;
    int tpr, rpc;
    tb_shape(a.W, TCH, tpr, rpc);
    const int line_floats = ((a.W + L - 1) + 3) & ~3;
    const int mask_bytes = THIN ? (a.W + 15) & ~15 : 0;
    const size_t smem = (size_t)rpc * (3 * line_floats * sizeof(float) + mask_bytes);
    dim3 grid((a.H + rpc - 1) / rpc);
    if (a.transpose) {
        cudaError_t e = ensure_smem<k_motion_x_tb<T, THIN, TCH, true>>(smem);
        if (e != cudaSuccess) return e;
        k_motion_x_tb<T, THIN, TCH, true><<<grid, tpr * rpc, smem, s>>>(a, tb, tpr, rpc, line_floats, mask_bytes);
    } else {
        cudaError_t e = ensure_smem<k_motion_x_tb<T, THIN, TCH, false>>(smem);
        if (e != cudaSuccess) return e;
        k_motion_x_tb<T, THIN, TCH, false><<<grid, tpr * rpc, smem, s>>>(a, tb, tpr, rpc, line_floats, mask_bytes);
    }
    return cudaGetLastError();
}

template <typename T, bool THIN>
cudaError_t launch_x_tb_t(const IterArgs &a, const TBArgs &tb, cudaStream_t s) {
    switch (tb_chunk(a.W, tb.chunk)) {
    case 13: return launch_x_tb_c<T, THIN, 13>(a, tb, s);
    case 17: return launch_x_tb_c<T, THIN, 17>(a, tb, s);
    default: return launch_x_tb_c<T, THIN, 33>(a, tb, s);
    }
}

}  // namespace mtb
}  // namespace rl

#define RL_MOTION_TB_TU(NAME, T, THIN)                                                      \
    namespace rl {                                                                           \
    cudaError_t NAME(const IterArgs &a, const TBArgs &tb, cudaStream_t s) {                  \
        return mtb::launch_x_tb_t<T, THIN>(a, tb, s);                                        \
    }                                                                                        \
    }
