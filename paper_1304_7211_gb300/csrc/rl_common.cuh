// rl_common.cuh -- device-side building blocks shared by the RL kernels.
//
// Storage types, the boundary index map of Sec. 2, and the argument block of
// one fused RL iteration (Eq. 3, with the selective-convolution state of
// Eq. 4-5).  Every kernel computes in FP32 whatever the storage type.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace rl {

// ---- storage ---------------------------------------------------------------
template <typename T> struct Stor;
template <> struct Stor<float> {
    static __device__ __forceinline__ float ld(const float *p, long long i) { return __ldg(p + i); }
    static __device__ __forceinline__ float ldc(const float *p, long long i) { return p[i]; }
    static __device__ __forceinline__ void st(float *p, long long i, float v) { p[i] = v; }
    static __device__ __forceinline__ float round(float v) { return v; }
};
template <> struct Stor<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p, long long i) { return __bfloat162float(__ldg(p + i)); }
    static __device__ __forceinline__ float ldc(const __nv_bfloat16 *p, long long i) { return __bfloat162float(p[i]); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, long long i, float v) { p[i] = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ float round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
};
template <> struct Stor<__half> {
    static __device__ __forceinline__ float ld(const __half *p, long long i) { return __half2float(__ldg(p + i)); }
    static __device__ __forceinline__ float ldc(const __half *p, long long i) { return __half2float(p[i]); }
    static __device__ __forceinline__ void st(__half *p, long long i, float v) { p[i] = __float2half_rn(v); }
    static __device__ __forceinline__ float round(float v) { return __half2float(__float2half_rn(v)); }
};

// 16-byte vectors of a storage type: VEC elements per 16-byte load/store.
template <typename T> struct Vec16 { static constexpr int N = 16 / sizeof(T); };

template <typename T>
__device__ __forceinline__ void ld16(const T *p, float *out) {
    const uint4 r = __ldg(reinterpret_cast<const uint4 *>(p));
    if constexpr (sizeof(T) == 4) {
        out[0] = __uint_as_float(r.x); out[1] = __uint_as_float(r.y);
        out[2] = __uint_as_float(r.z); out[3] = __uint_as_float(r.w);
    } else {
        const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            T lo, hi;
            unsigned short a = (unsigned short)(w[k] & 0xffffu), b = (unsigned short)(w[k] >> 16);
            memcpy(&lo, &a, 2);
            memcpy(&hi, &b, 2);
            out[2 * k] = Stor<T>::ldc(&lo, 0);
            out[2 * k + 1] = Stor<T>::ldc(&hi, 0);
        }
    }
}

template <typename T>
__device__ __forceinline__ void st16(T *p, const float *in) {
    uint4 r;
    if constexpr (sizeof(T) == 4) {
        r.x = __float_as_uint(in[0]); r.y = __float_as_uint(in[1]);
        r.z = __float_as_uint(in[2]); r.w = __float_as_uint(in[3]);
    } else {
        unsigned w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            T lo, hi;
            Stor<T>::st(&lo, 0, in[2 * k]);
            Stor<T>::st(&hi, 0, in[2 * k + 1]);
            unsigned short a, b;
            memcpy(&a, &lo, 2);
            memcpy(&b, &hi, 2);
            w[k] = (unsigned)a | ((unsigned)b << 16);
        }
        r = make_uint4(w[0], w[1], w[2], w[3]);
    }
    *reinterpret_cast<uint4 *>(p) = r;
}

// Copy a contiguous run src[0, n) of a global row into shared memory,
// element i going to dst[didx(i)].  Each of the nt cooperating threads (index
// t) keeps BATCH independent loads in flight before it stores any; 16-byte
// vector loads are used when the run starts on a 16-byte boundary.
template <int BATCH, typename T, typename DI>
__device__ __forceinline__ void row_to_smem(float *dst, DI didx, const T *src, int n, int t, int nt) {
    constexpr int V = Vec16<T>::N;
    int done = 0;
    if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        const int nv = n / V;
        for (int base = t; base < nv; base += BATCH * nt) {
            float v[BATCH][V];
#pragma unroll
            for (int j = 0; j < BATCH; ++j) {
                const int i = base + j * nt;
                if (i < nv) ld16(src + (long long)i * V, v[j]);
            }
#pragma unroll
            for (int j = 0; j < BATCH; ++j) {
                const int i = base + j * nt;
                if (i < nv) {
#pragma unroll
                    for (int k = 0; k < V; ++k) dst[didx(i * V + k)] = v[j][k];
                }
            }
        }
        done = nv * V;
    }
    for (int base = done + t; base < n; base += BATCH * nt) {
        float v[BATCH];
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
            const int i = base + j * nt;
            if (i < n) v[j] = Stor<T>::ld(src, i);
        }
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
            const int i = base + j * nt;
            if (i < n) dst[didx(i)] = v[j];
        }
    }
}

// Store a shared-memory run src[sidx(i)], i in [0, n), to a contiguous global
// row dst[0, n), with 16-byte vector stores when dst is 16-byte aligned.
template <typename T, typename SI>
__device__ __forceinline__ void smem_to_row(T *dst, const float *src, SI sidx, int n, int t, int nt) {
    constexpr int V = Vec16<T>::N;
    int done = 0;
    if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
        const int nv = n / V;
        for (int i = t; i < nv; i += nt) {
            float v[V];
#pragma unroll
            for (int k = 0; k < V; ++k) v[k] = src[sidx(i * V + k)];
            st16(dst + (long long)i * V, v);
        }
        done = nv * V;
    }
    for (int i = done + t; i < n; i += nt) Stor<T>::st(dst, i, src[sidx(i)]);
}

// Gather n elements into shared memory through arbitrary index maps
// (ld(i) -> float, st(i, v)), BATCH loads in flight per thread.
template <int BATCH, typename LD, typename ST>
__device__ __forceinline__ void gather_batched(int n, int t, int nt, LD ld, ST st) {
    for (int base = t; base < n; base += BATCH * nt) {
        float v[BATCH];
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
            const int i = base + j * nt;
            if (i < n) v[j] = ld(i);
        }
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
            const int i = base + j * nt;
            if (i < n) st(i, v[j]);
        }
    }
}

// Asynchronous 4-byte global -> shared copy (completes at cp_async_wait_all).
__device__ __forceinline__ void cp_async4(float *smem_dst, const float *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// ---- boundary continuation (Sec. 2) ----------------------------------------
// clamp = closest image pixel; mirror = half-sample symmetric, 2n-periodic.
__device__ __forceinline__ int bmap(int e, int n, int clamp) {
    if (e >= 0 && e < n) return e;
    if (clamp) return e < 0 ? 0 : n - 1;
    int period = 2 * n;
    int r = e % period;
    if (r < 0) r += period;
    return r < n ? r : period - 1 - r;
}

// ---- one fused iteration ----------------------------------------------------
// The PSF support lies in offsets t in [-ax, bx] x [-ay, by]:
//   forward  v(p) = sum_t h(t) u(m(p - t))          (reads [p-b, p+a])
//   adjoint  c(p) = sum_t h(t) q(m(p + t))          (reads [p-a, p+b])
// i.e. the pad-flip reading of h* in Eq. 3 (same continuation m for both).
struct IterArgs {
    const void *f;
    const void *u_in;
    void *u_out;
    int W, H;
    long long f_pitch, in_pitch, out_pitch;  // elements
    int clamp;                               // 1 = clamp, 0 = mirror
    int ax, bx, ay, by;                      // PSF extents
    float weight;                            // uniform weight (RUNSUM, SPAN)
    const float *taps;                       // STENCIL: dense (ay+by+1) x (ax+bx+1)
    const int2 *spans;                       // SPAN: per PSF row j (ty = j - ay): [lo, hi] of tx
    // selective convolution (Eq. 4-5)
    const uint8_t *mask_in;                  // 1 = active; read when !full
    uint8_t *mask_out;                       // written when update_mask
    float *rstale;                           // f/v of the last active iteration
    long long mi_pitch;                      // pitch of mask_in
    long long m_pitch;                       // pitch of mask_out and rstale
    int full;                                // every pixel used this iteration
    int update_mask;                         // write mask_out
    int replay;                              // mask_in is a recorded schedule
    int relative;                            // |c-1| (1) or |u'-u| (0)
    float tau;                               // threshold (strict < -> inactive)
    unsigned long long *active_count;        // += used pixels (nullable)
    int *tile_flags;                         // per tile: any pixel active next (nullable)
    int tiles_x;                             // tiles per row of tile_flags
    int transpose;                           // adjoint = exact transpose A^T (STENCIL tiles)
    // Exact transpose on the two-half kernels: when fold_ct is set the band
    // kernel runs between the halves and writes A^T q at the pixels within
    // (fold_rx, fold_ry) of the border, which the adjoint half takes there.
    float *fold_ct;                          // pitch = q plane's
    const float *fold_taps;                  // the PSF: fold_kh x fold_kw, anchor (fold_ax, fold_ay)
    int fold_kw, fold_kh, fold_ax, fold_ay;
    int fold_rx, fold_ry;
    float *fold_z;                           // z on the apron, extended plane
    long long fold_zp;                       // its pitch: W + kw - 1
};

// Several iterations in one launch (kernels that keep their lines resident).
struct TBArgs {
    int K;                  // iterations
    int P;                  // reset period of selective convolution (full when k % P == 0)
    int Q;                  // mask update period: 1 or P
    const uint8_t *sched;   // replayed used-pixel masks, K planes (nullable)
    long long s_pitch;      // row pitch of a schedule plane (bytes)
    long long s_plane;      // bytes per schedule plane
    int round;              // round u to the storage type after every iteration
    int chunk;              // running-sum chunk width: 0 = built-in table, else 13 / 17 / 33
};

// Ratio f / v of Eq. 3 with q = 0 where the re-blurred value vanishes.
__device__ __forceinline__ float rl_ratio(float f, float v) { return v > 0.f ? f / v : 0.f; }

// Per-pixel selective-convolution bookkeeping at an output pixel p (Eq. 4-5).
// Returns u'(p).  `use` says whether p was used this iteration, q is its
// ratio (fresh when used).
__device__ __forceinline__ float thin_update(const IterArgs &a, long long mi, bool use, float u,
                                             float c, float q) {
    float un = use ? u * c : u;
    if (a.replay) {
        // the schedule decides; keep the ratio of every used pixel
        if (use) a.rstale[mi] = q;
    } else if (a.update_mask) {
        float d = 0.f;
        if (use) d = a.relative ? (u > 0.f ? fabsf(c - 1.f) : 0.f) : fabsf(un - u);
        bool keep = use && (d >= a.tau);
        a.mask_out[mi] = (uint8_t)keep;
        if (use && !keep) a.rstale[mi] = q;
    }
    return un;
}

__device__ __forceinline__ void count_active(unsigned long long *ctr, bool use) {
    unsigned b = __ballot_sync(0xffffffffu, use);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(ctr, (unsigned long long)__popc(b));
}

// Raise a kernel's dynamic shared-memory limit to the device's opt-in
// maximum less the kernel's static shared memory, once per kernel and device
// (the attribute persists in the context).
template <auto KERN>
inline cudaError_t ensure_smem(size_t bytes) {
    static unsigned long long done = 0;  // bit per device ordinal (< 64)
    if (bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (__atomic_load_n(&done, __ATOMIC_ACQUIRE) & bit) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa = {};
    e = cudaFuncGetAttributes(&fa, KERN);
    if (e != cudaSuccess) return e;
    const size_t room = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    if (bytes > room) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(KERN, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)room);
    if (e == cudaSuccess) __atomic_fetch_or(&done, bit, __ATOMIC_RELEASE);
    return e;
}

}  // namespace rl
