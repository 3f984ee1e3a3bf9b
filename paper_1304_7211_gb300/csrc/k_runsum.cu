// k_runsum.cu -- running-sum (sliding window) box filter kernels for linear
// motion blur along x or y, each fusing one whole RL iteration (Eq. 3):
//   v = h (x) u,  q = f / v,  c = h* (x) q,  u' = u c
// into a single pass over HBM (read f and u once, write u' once).
//
// Sec. 3 "Linear motion blur": along a scan-line the box of length M is a
// sliding window, O(N + M) per line instead of O(N M).  Here every thread
// slides its own window over a contiguous chunk of outputs: the first output
// of the chunk is summed directly, the rest by adding the sample entering the
// window and subtracting the one leaving it.  Chunks are short (16 or 32
// outputs), so the FP32 error of the running sum stays at a few ulps of the
// window sum (no long-row drift).
#include "rl_launch.h"
#include "k_motion_tb.cuh"

namespace rl {

namespace {

// Shared-memory index with one pad word every 32: keeps the 16-float chunks
// of consecutive lanes on distinct banks.
__device__ __forceinline__ int PI(int i) { return i + (i >> 5); }

constexpr int XCH = 16;     // outputs per thread chunk along x
constexpr int YCH_TS = 256; // output rows per CTA for the y kernel

__device__ __forceinline__ void warp_count_add(unsigned long long *ctr, unsigned cnt) {
    unsigned s = __reduce_add_sync(0xffffffffu, cnt);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(ctr, (unsigned long long)s);
}

// ---- motion along x -----------------------------------------------------------
// CTA = `rpc` rows, `tpr` threads per row.  Per row, shared memory holds the
// continued row of u over extended coordinates [-B, W + A) and the ratio q
// over [-A, W + B) (taps at offsets [-A, B], L = A + B + 1).
template <typename T, bool THIN>
__global__ void __launch_bounds__(256) k_motion_x(IterArgs a, int tpr, int rpc, int row_floats) {
    extern __shared__ float sm[];
    const int W = a.W, A = a.ax, B = a.bx, L = A + B + 1;
    const int g = threadIdx.x / tpr, t = threadIdx.x - g * tpr;
    const int y = blockIdx.x * rpc + g;
    const bool row_ok = y < a.H;
    float *Ue = sm + (size_t)g * 2 * row_floats;
    float *Qe = Ue + row_floats;
    const T *f = (const T *)a.f;
    const T *u_in = (const T *)a.u_in;
    T *u_out = (T *)a.u_out;
    const float w = a.weight;
    const long long mrow = (long long)y * a.m_pitch;
    const long long mirow = (long long)y * a.mi_pitch;
    unsigned used = 0;

    if (row_ok) {
        // interior of u and f with batched (vector) loads; the continued
        // ends of u (A + B samples) with mapped scalar loads
        const T *urow = u_in + (long long)y * a.in_pitch;
        row_to_smem<4>(Ue, [B](int i) { return PI(i + B); }, urow, W, t, tpr);
        row_to_smem<4>(Qe, [A](int i) { return PI(i + A); }, f + (long long)y * a.f_pitch, W, t, tpr);
        gather_batched<4>(A + B, t, tpr,
            [&](int i) { return Stor<T>::ld(urow, bmap(i < B ? i - B : W + i - B, W, a.clamp)); },
            [&](int i, float v) { Ue[PI(i < B ? i : W + i)] = v; });
    }
    __syncthreads();
    // forward: v(x) = w * sum_{e=x-B}^{x+A} u(m(e)) = w * sum_k Ue[x + k]
    if (row_ok) {
        for (int x0 = t * XCH; x0 < W; x0 += tpr * XCH) {
            float s = 0.f;
            for (int k = 0; k < L; ++k) s += Ue[PI(x0 + k)];
#pragma unroll
            for (int j = 0; j < XCH; ++j) {
                const int x = x0 + j;
                if (x < W) {
                    bool use = true;
                    if (THIN && !a.full) use = a.mask_in[mirow + x] != 0;
                    const float fx = Qe[PI(x + A)];
                    Qe[PI(x + A)] = use ? rl_ratio(fx, s * w) : a.rstale[mrow + x];
                    if (j + 1 < XCH && x + 1 < W) s += Ue[PI(x + L)] - Ue[PI(x)];
                }
            }
        }
    }
    __syncthreads();
    if (row_ok) {  // continue q beyond the row ends
        for (int i = t; i < A; i += tpr) Qe[PI(i)] = Qe[PI(bmap(i - A, W, a.clamp) + A)];
        for (int i = t; i < B; i += tpr) Qe[PI(W + A + i)] = Qe[PI(bmap(W + i, W, a.clamp) + A)];
    }
    __syncthreads();
    // adjoint: c(x) = w * sum_{e=x-A}^{x+B} q(m(e)) = w * sum_k Qe[x + k]
    if (row_ok) {
        for (int x0 = t * XCH; x0 < W; x0 += tpr * XCH) {
            float s = 0.f;
            for (int k = 0; k < L; ++k) s += Qe[PI(x0 + k)];
#pragma unroll
            for (int j = 0; j < XCH; ++j) {
                const int x = x0 + j;
                if (x < W) {
                    const float u = Ue[PI(x + B)];
                    const float c = s * w;
                    float un;
                    if (THIN) {
                        const bool use = a.full || a.mask_in[mirow + x] != 0;
                        used += use;
                        un = thin_update(a, mrow + x, use, u, c, Qe[PI(x + A)]);
                    } else {
                        un = u * c;
                    }
                    Ue[PI(x + B)] = un;
                    if (j + 1 < XCH && x + 1 < W) s += Qe[PI(x + L)] - Qe[PI(x)];
                }
            }
        }
    }
    __syncthreads();
    if (row_ok)
        smem_to_row(u_out + (long long)y * a.out_pitch, Ue, [B](int i) { return PI(i + B); }, W, t, tpr);
    if (THIN && a.active_count) warp_count_add(a.active_count, used);
}

// ---- motion along y -----------------------------------------------------------
// CTA = 32 columns (one per lane) x a segment of up to YCH_TS output rows.
// Shared memory [row][32]: u over extended rows [P0 - B, P1 + A) and q over
// [y0 - A, y1 + B), where P = [max(0, y0 - A), min(H, y1 + B)) are the image
// rows whose ratio the segment needs.  Each warp slides down a contiguous
// range of rows.
template <typename T, bool THIN>
__global__ void __launch_bounds__(256) k_motion_y(IterArgs a, int TS) {
    extern __shared__ float sm[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, NW = blockDim.x >> 5;
    const int W = a.W, H = a.H;
    const int x = blockIdx.x * 32 + lane;
    const bool col_ok = x < W;
    const int xs = col_ok ? x : W - 1;
    const int y0 = blockIdx.y * TS, y1 = min(y0 + TS, H);
    const int A = a.ay, B = a.by, L = A + B + 1;
    const int P0 = max(0, y0 - A), P1 = min(H, y1 + B);
    const int UL = P1 - P0 + L - 1;
    float *U = sm;
    float *Q = sm + (size_t)UL * 32;
    const T *f = (const T *)a.f;
    const T *u_in = (const T *)a.u_in;
    T *u_out = (T *)a.u_out;
    const float w = a.weight;
    unsigned used = 0;

    // each warp stages whole rows (lane = column), 8 rows in flight per thread
    gather_batched<8>(UL, wid, NW,
        [&](int r) { return Stor<T>::ld(u_in, (long long)bmap(P0 - B + r, H, a.clamp) * a.in_pitch + xs); },
        [&](int r, float v) { U[r * 32 + lane] = v; });
    gather_batched<8>(P1 - P0, wid, NW,
        [&](int r) { return Stor<T>::ld(f, (long long)(P0 + r) * a.f_pitch + xs); },
        [&](int r, float v) { Q[(P0 + r - y0 + A) * 32 + lane] = v; });
    __syncthreads();
    {  // forward over rows P: v(p) = w * sum_{e=p-B}^{p+A} u(m(e))
        const int n = P1 - P0, per = (n + NW - 1) / NW;
        const int r0 = P0 + wid * per, r1 = min(P1, r0 + per);
        if (r0 < r1) {
            float s = 0.f;
            for (int k = 0; k < L; ++k) s += U[(r0 - P0 + k) * 32 + lane];
            for (int p = r0; p < r1; ++p) {
                bool use = true;
                const long long mi = (long long)p * a.m_pitch + xs;
                if (THIN && !a.full) use = a.mask_in[(long long)p * a.mi_pitch + xs] != 0;
                float *qp = &Q[(p - y0 + A) * 32 + lane];
                *qp = use ? rl_ratio(*qp, s * w) : a.rstale[mi];
                if (p + 1 < r1) s += U[(p - P0 + L) * 32 + lane] - U[(p - P0) * 32 + lane];
            }
        }
    }
    __syncthreads();
    const int QL = y1 - y0 + L - 1;
    for (int r = wid; r < QL; r += NW) {
        const int e = y0 - A + r;
        if (e < 0 || e >= H) Q[r * 32 + lane] = Q[(bmap(e, H, a.clamp) - y0 + A) * 32 + lane];
    }
    __syncthreads();
    {  // adjoint over output rows: c(p) = w * sum_{e=p-A}^{p+B} q(m(e))
        const int n = y1 - y0, per = (n + NW - 1) / NW;
        const int r0 = y0 + wid * per, r1 = min(y1, r0 + per);
        if (r0 < r1) {
            float s = 0.f;
            for (int k = 0; k < L; ++k) s += Q[(r0 - y0 + k) * 32 + lane];
            for (int p = r0; p < r1; ++p) {
                const float u = U[(p - P0 + B) * 32 + lane];
                const float c = s * w;
                float un;
                if (THIN) {
                    const long long mi = (long long)p * a.m_pitch + xs;
                    const bool use = a.full || a.mask_in[(long long)p * a.mi_pitch + xs] != 0;
                    used += (use && col_ok);
                    if (col_ok) un = thin_update(a, mi, use, u, c, Q[(p - y0 + A) * 32 + lane]);
                    else un = u;
                } else {
                    un = u * c;
                }
                if (col_ok) Stor<T>::st(u_out, (long long)p * a.out_pitch + x, un);
                if (p + 1 < r1) s += Q[(p - y0 + L) * 32 + lane] - Q[(p - y0) * 32 + lane];
            }
        }
    }
    if (THIN && a.active_count) warp_count_add(a.active_count, used);
}

template <typename T, bool THIN>
cudaError_t launch_x_t(const IterArgs &a, cudaStream_t s) {
    const int L = a.ax + a.bx + 1;
    const int chunks = (a.W + XCH - 1) / XCH;
    int tpr = ((chunks + 31) / 32) * 32;
    if (tpr > 256) tpr = 256;
    const int rpc = 256 / tpr;
    const int n_ext = a.W + L - 1;
    const int row_floats = ((n_ext + (n_ext >> 5) + 1) + 3) & ~3;
    const size_t smem = (size_t)rpc * 2 * row_floats * sizeof(float);
    auto kern = k_motion_x<T, THIN>;
    cudaError_t e = ensure_smem<k_motion_x<T, THIN>>(smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.H + rpc - 1) / rpc);
    kern<<<grid, tpr * rpc, smem, s>>>(a, tpr, rpc, row_floats);
    return cudaGetLastError();
}

template <typename T, bool THIN>
cudaError_t launch_y_t(const IterArgs &a, cudaStream_t s) {
    const int L = a.ay + a.by + 1;
    const int TS = a.H < YCH_TS ? a.H : YCH_TS;
    const size_t smem = (size_t)((TS + 2 * (L - 1)) + (TS + L - 1)) * 32 * sizeof(float);
    auto kern = k_motion_y<T, THIN>;
    cudaError_t e = ensure_smem<k_motion_y<T, THIN>>(smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.W + 31) / 32, (a.H + TS - 1) / TS);
    kern<<<grid, 256, smem, s>>>(a, TS);
    return cudaGetLastError();
}

}  // namespace

size_t motion_x_tb_smem_bytes(int W, int L, bool thin, int chunk) {
    int tpr, rpc;
    mtb::tb_shape(W, chunk, tpr, rpc);
    const int line_floats = ((W + L - 1) + 3) & ~3;
    const int mask_bytes = thin ? (W + 15) & ~15 : 0;
    return (size_t)rpc * (3 * line_floats * sizeof(float) + mask_bytes);
}

bool motion_x_tb_fits(int W, int L, bool thin, int chunk) {
    return motion_x_tb_smem_bytes(W, L, thin, chunk) <= 200 * 1024;
}

cudaError_t launch_motion_x_tb(const IterArgs &a, const TBArgs &tb, int storage, bool thin,
                               cudaStream_t s) {
    switch (storage) {
    case ST_F32: return thin ? launch_motion_tb_f32_thin(a, tb, s) : launch_motion_tb_f32(a, tb, s);
    case ST_BF16: return thin ? launch_motion_tb_bf16_thin(a, tb, s) : launch_motion_tb_bf16(a, tb, s);
    case ST_F16: return thin ? launch_motion_tb_f16_thin(a, tb, s) : launch_motion_tb_f16(a, tb, s);
    }
    return cudaErrorInvalidValue;
}

size_t motion_x_smem_bytes(int W, int L) {
    const int n_ext = W + L - 1;
    const int row_floats = ((n_ext + (n_ext >> 5) + 1) + 3) & ~3;
    const int chunks = (W + XCH - 1) / XCH;
    int tpr = ((chunks + 31) / 32) * 32;
    if (tpr > 256) tpr = 256;
    return (size_t)(256 / tpr) * 2 * row_floats * sizeof(float);
}

bool motion_x_fits(int W, int L) { return motion_x_smem_bytes(W, L) <= 200 * 1024; }

cudaError_t launch_motion_x(const IterArgs &a, int storage, bool thin, cudaStream_t s) {
    switch (storage) {
    case ST_F32: return thin ? launch_x_t<float, true>(a, s) : launch_x_t<float, false>(a, s);
    case ST_BF16: return thin ? launch_x_t<__nv_bfloat16, true>(a, s) : launch_x_t<__nv_bfloat16, false>(a, s);
    case ST_F16: return thin ? launch_x_t<__half, true>(a, s) : launch_x_t<__half, false>(a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_motion_y(const IterArgs &a, int storage, bool thin, cudaStream_t s) {
    switch (storage) {
    case ST_F32: return thin ? launch_y_t<float, true>(a, s) : launch_y_t<float, false>(a, s);
    case ST_BF16: return thin ? launch_y_t<__nv_bfloat16, true>(a, s) : launch_y_t<__nv_bfloat16, false>(a, s);
    case ST_F16: return thin ? launch_y_t<__half, true>(a, s) : launch_y_t<__half, false>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace rl
