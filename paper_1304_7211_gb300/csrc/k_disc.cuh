// k_disc.cuh -- the register-blocked two-half RL iteration (Eq. 3): the
// generic box filter for the defocus disc (Sec. 3 "Defocus blur"), separable
// sliding sums for the square box and any uniform rectangle (Sec. 3
// "Rectangular blur"), and the direct stencil for taps within 4 pixels of
// the anchor; one output tile per CTA, a block operation policy for the
// convolution (DiscOp, BoxOp, RectOp, StencilOp).  The tile body serves both
// the single-image kernel and the batched (request, tile) kernel.
//
// Disc (DiscOp<R>): the disc of radius R (pixel-centre inclusion) is a stack
// of horizontal runs; PSF row ty covers tx in [-s(ty), s(ty)],
// s(ty) = floor(sqrt(R^2 - ty^2)).  After staging, one pass turns every
// staged row into its exclusive prefix sum in place (one thread per row; a
// row of at most 64 + 2 * 16 values keeps FP32 prefix differences accurate
// to a few ulps of the row sum).  Each thread owns a block of SY x SX
// outputs: for every input row the block touches it loads the prefix entries
// its runs end on -- a compile-time subset of its window -- and adds to each
// output row that uses this input row the run sum P[j + R + 1 + s] -
// P[j + R - s]: sliding the PSF only exchanges the run ends (Sec. 3), and
// with a prefix a run of any length costs one difference.  R is a template
// parameter, so every run end is a compile-time register index; the disc is
// symmetric, so the forward convolution and the adjoint (h* = h reflected)
// use the same table.  Stencil (StencilOp<K>): K x K taps in the kernel's
// parameter block, each a constant-bank FMA operand at a compile-time window
// offset.
//
// The iteration runs as two launches (forward + ratio into a q plane, then
// adjoint + update in place): the second 12 B/px of traffic is cheaper than
// recomputing the forward convolution over a 2R apron, and each launch
// stages a single halo'd array (more resident CTAs).  The q plane doubles as
// the stale ratio of Eq. 5: inactive pixels are simply not rewritten.  With
// the exact-transpose adjoint, a band kernel between the halves (k_fold.cu)
// supplies A^T q on the border band.
#pragma once

#include <algorithm>
#include <type_traits>

#include "rl_launch.h"

namespace rl {
namespace disc {

constexpr int SX = 8;  // outputs per thread along x
constexpr int SY = 4;  // outputs per thread along y
constexpr int TX = 64, TY = 64;  // output tile of one CTA (128 threads)
static_assert(TX == disc_tile() && TY == disc_tile(), "the host sizes tile arrays by disc_tile()");

// Shared-memory layout of a staged halo tile: rows of 4-float units, the
// halo rounded up to R4 = 4 ceil(R / 4) columns on each side so that every
// unit starts on a 16-byte boundary in the image too.  Unit u of a row is
// stored at u ^ ((u >> 3) & 1): the 8 lanes of a 16-byte load phase (block
// columns bx = 0..7 of one block row, reading unit 2 bx + t) then hit 8
// distinct bank quads for every t.
__device__ __forceinline__ int hunit(int u) { return u ^ ((u >> 3) & 1); }
__device__ __forceinline__ int hidx(int c) { return (hunit(c >> 2) << 2) | (c & 3); }
__host__ __device__ constexpr int round4(int r) { return (r + 3) & ~3; }

// Half-width of the disc's run in PSF row ty: largest s with s^2 + ty^2 <= R^2.
__host__ __device__ constexpr int run_half_width(int R, int ty) {
    int t2 = ty * ty, s = 0;
    while ((s + 1) * (s + 1) + t2 <= R * R) ++s;
    return s;
}

__device__ __forceinline__ void warp_count_add(unsigned long long *ctr, unsigned cnt) {
    unsigned s = __reduce_add_sync(0xffffffffu, cnt);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(ctr, (unsigned long long)s);
}

__device__ __forceinline__ void cp_async16(float *smem_dst, const float *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}

// Loads of data that other CTAs of the same grid write while it runs (the
// persistent kernel's u and q planes) must come from L2, the point of
// coherence: COH selects ld.global.cg for them.  Read-only data (f) and the
// two-launch kernels keep the cached / non-coherent loads.
template <bool COH, typename V>
__device__ __forceinline__ V gld(const V *p) {
    if constexpr (COH) return __ldcg(p);
    else return *p;
}
template <bool COH, typename T>
__device__ __forceinline__ float gld_elem(const T *p, long long i) {
    if constexpr (!COH) {
        return Stor<T>::ld(p, i);
    } else if constexpr (sizeof(T) == 4) {
        return __ldcg(reinterpret_cast<const float *>(p) + i);
    } else {
        const unsigned short b = __ldcg(reinterpret_cast<const unsigned short *>(p) + i);
        if constexpr (std::is_same<T, __half>::value) return __half2float(__ushort_as_half(b));
        else return __bfloat162float(__ushort_as_bfloat16(b));
    }
}

// Stage the halo tile: array row r, column c (r < nrows, c < 4 nu) is image
// pixel (y0 + r, xs + c), continued across the border (clamp or mirror).
// xs is a multiple of 4.  FP32 goes by asynchronous copies -- 16 bytes where
// the unit lies inside the image and the row is 16-byte aligned, else four
// 4-byte copies of the boundary-mapped pixels; the caller waits
// (cp_async_wait_all) before the barrier.  16-bit storage goes through
// registers, converted to FP32, several units in flight per thread.
template <typename T, int nrows, int nu, int pitch, bool COH = false, int NT = 128>
__device__ __forceinline__ void stage_halo(float *dst, int clamp, int W, int H, int y0, int xs, const T *src,
                                           long long sp, int tid) {
    constexpr int total = nrows * nu;
    if constexpr (sizeof(T) == 4) {
        const float *s = reinterpret_cast<const float *>(src);
        // Interior tile with 16-byte aligned rows: warp w copies rows w, w +
        // NT / 32, ..., lane l units l and l + 32 of each (nu <= 64), no
        // boundary map.
        static_assert(nu <= 64, "two units per lane");
        if (y0 >= 0 && y0 + nrows <= H && xs >= 0 && xs + 4 * nu <= W &&
            ((reinterpret_cast<uintptr_t>(s) | (uintptr_t)(sp * 4)) & 15) == 0) {
            const int lane = tid & 31, w = tid >> 5;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int u = lane + 32 * h;
                if (u < nu) {
                    const float *g = s + (long long)(y0 + w) * sp + xs + 4 * u;
                    float *d = dst + w * pitch + (hunit(u) << 2);
                    constexpr int NW = NT / 32;
#pragma unroll 4
                    for (int r = w; r < nrows; r += NW) {
                        cp_async16(d, g);
                        g += NW * sp;
                        d += NW * pitch;
                    }
                }
            }
            return;
        }
        for (int e = tid; e < total; e += NT) {
            const int r = e / nu, u = e - r * nu;
            const int yy = bmap(y0 + r, H, clamp);
            const float *srow = s + (long long)yy * sp;
            const int x = xs + 4 * u;
            float *d = dst + r * pitch + (hunit(u) << 2);
            if (x >= 0 && x + 4 <= W && (reinterpret_cast<uintptr_t>(srow) & 15) == 0) {
                cp_async16(d, srow + x);
            } else if constexpr (COH) {
#pragma unroll
                for (int k = 0; k < 4; ++k) d[k] = __ldcg(srow + bmap(x + k, W, clamp));
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) cp_async4(d + k, srow + bmap(x + k, W, clamp));
            }
        }
        return;
    }
    constexpr int B = 4;
    for (int e0 = tid; e0 < total; e0 += NT * B) {
        float v[B][4];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int e = e0 + NT * b;
            if (e < total) {
                const int r = e / nu, u = e - r * nu;
                const T *srow = src + (long long)bmap(y0 + r, H, clamp) * sp;
                const int x = xs + 4 * u;
                if (x >= 0 && x + 4 <= W && (reinterpret_cast<uintptr_t>(srow + x) & 7) == 0) {
                    // a whole unit inside the image: one 8-byte load of 4 values
                    const uint2 w2 = COH ? __ldcg(reinterpret_cast<const uint2 *>(srow + x))
                                         : __ldg(reinterpret_cast<const uint2 *>(srow + x));
                    const unsigned wv[2] = {w2.x, w2.y};
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const unsigned short lo = (unsigned short)(wv[k] & 0xffffu), hi = (unsigned short)(wv[k] >> 16);
                        if constexpr (std::is_same<T, __half>::value) {
                            v[b][2 * k] = __half2float(__ushort_as_half(lo));
                            v[b][2 * k + 1] = __half2float(__ushort_as_half(hi));
                        } else {
                            v[b][2 * k] = __bfloat162float(__ushort_as_bfloat16(lo));
                            v[b][2 * k + 1] = __bfloat162float(__ushort_as_bfloat16(hi));
                        }
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) v[b][k] = gld_elem<COH>(srow, bmap(x + k, W, clamp));
                }
            }
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int e = e0 + NT * b;
            if (e < total) {
                const int r = e / nu, u = e - r * nu;
                *reinterpret_cast<float4 *>(dst + r * pitch + (hunit(u) << 2)) =
                    make_float4(v[b][0], v[b][1], v[b][2], v[b][3]);
            }
        }
    }
}

// Geometry of the staged halo tile for a filter of radius R; XU spare units
// at the end of every row (the disc's row prefix has one more entry than
// the row has columns).
template <int R, int XU = 0, int TXg = TX, int TYg = TY>
struct Halo {
    static constexpr int R4 = round4(R);           // halo rounded up to whole units
    static constexpr int NU = (TXg + 2 * R4) / 4;  // units per row (even)
    static constexpr int HP = 4 * (NU + XU);       // row pitch in floats
    static constexpr int NR = TYg + 2 * R;         // staged rows
    static constexpr int NWU = (SX + 2 * R4) / 4;  // units in one block's window
    static constexpr int OFF = R4 - R;             // window column of offset -R
    static constexpr size_t bytes = (size_t)NR * HP * sizeof(float);
};

// The window of block column bx in one staged row: w[k], k < SX + 2R, is the
// input at offset k - R from the block's first column.  Whole units go as
// 16-byte loads; the partial units at the two ends load only the columns in
// use (8- or 4-byte loads: for a warp those take no more shared-memory
// wavefronts than one 16-byte load, and they keep no dead registers).
template <int R, int NW>
__device__ __forceinline__ void load_window_n(const float *row, int bx, float (&w)[NW]) {
    constexpr int OFF = round4(R) - R;      // window column of offset -R
    constexpr int NWU = (OFF + NW + 3) / 4;  // units the window touches
#pragma unroll
    for (int t = 0; t < NWU; ++t) {
        const float *p = row + (hunit(2 * bx + t) << 2);
        const int lo = OFF - 4 * t > 0 ? OFF - 4 * t : 0;
        const int hi = OFF + NW - 4 * t < 4 ? OFF + NW - 4 * t : 4;
        const int d = 4 * t - OFF;  // w index of unit column 0
        if (lo == 0 && hi == 4) {
            const float4 v = *reinterpret_cast<const float4 *>(p);
            w[d] = v.x; w[d + 1] = v.y; w[d + 2] = v.z; w[d + 3] = v.w;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (k < lo || k >= hi) continue;
                const bool pair_head = (k & 1) == 0 && k + 1 < hi;
                const bool pair_tail = (k & 1) == 1 && k - 1 >= lo;
                if (pair_head) {
                    const float2 v = *reinterpret_cast<const float2 *>(p + k);
                    w[d + k] = v.x;
                    w[d + k + 1] = v.y;
                } else if (!pair_tail) {
                    w[d + k] = p[k];
                }
            }
        }
    }
}

template <int R>
__device__ __forceinline__ void load_window(const float *row, int bx, float (&w)[SX + 2 * R]) {
    load_window_n<R, SX + 2 * R>(row, bx, w);
}

// Sum of the disc over the block's SY x SX outputs.  Input row m of the
// block is array row row0 + m; output row i uses it with ty = i + R - m
// (forward) -- the adjoint reads the mirrored offset, which has the same run.
// Packed pairs of FP32 values (one 64-bit register pair) and the paired add
// of sm_100+ (add.rn.f32x2: two IEEE round-to-nearest adds in one
// instruction, each bitwise equal to the scalar add).
__device__ __forceinline__ unsigned long long f2pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2unpack(unsigned long long v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ void f2add(unsigned long long &acc, unsigned long long d) {
    asm("add.rn.f32x2 %0, %0, %1;" : "+l"(acc) : "l"(d));
}

// Disc geometry: spare units at the end of every staged row hold the row
// prefix's last entry (at unit hunit(NU), which is NU or NU + 1): one spare
// unit, or three when hunit(NU) = NU + 1, so that the row pitch is an odd
// number of units and the prefix pass (one thread per row, all at the same
// unit) puts 8 consecutive rows on 8 distinct bank quads.  (Eight CTAs per
// SM, which the smaller pitch would allow up to R = 8 at a 64-register cap,
// measured slower.)
template <int R, int TXg = TX, int TYg = TY>
using DiscHalo = Halo<R, ((((TXg + 2 * round4(R)) / 4) >> 3) & 1) ? 3 : 1, TXg, TYg>;

// Exclusive prefix of every staged row, in place: logical column k of a row
// (0 <= k <= 4 NU, the last in the spare unit) becomes the sum of columns
// [0, k).  One thread per row, a unit at a time.
template <int R, int TXg, int TYg, int NT>
__device__ __forceinline__ void row_prefix(float *tile) {
    using G = DiscHalo<R, TXg, TYg>;
    static_assert(G::NR <= NT, "one thread per staged row");
    if (threadIdx.x < G::NR) {
        float *row = tile + threadIdx.x * G::HP;
        float acc = 0.f;
#pragma unroll
        for (int u = 0; u < G::NU; ++u) {
            float4 *p = reinterpret_cast<float4 *>(row + (hunit(u) << 2));
            const float4 v = *p;
            float4 o;
            o.x = acc;
            o.y = o.x + v.x;
            o.z = o.y + v.y;
            o.w = o.z + v.z;
            acc = o.w + v.w;
            *p = o;
        }
        row[hunit(G::NU) << 2] = acc;
    }
}

// Which prefix entries of its window a block reads in input row m: bit k of
// mask[m] is set when some output row i < SY uses row m (PSF row ty = i + R -
// m) and some output column j < SX has a run end at k, i.e. k = j + R - s or
// k = j + R + 1 + s with s = s(ty).  Rows near the top and bottom of the disc
// use short runs, so whole units of the window go unread there.
template <int R, int SYb>
struct DiscNeed {
    static constexpr int NP = SX + 2 * R + 1;
    static constexpr int NR = SYb + 2 * R;
    struct Table { unsigned long long mask[NR]; };
    static constexpr Table make() {
        Table t{};
        for (int m = 0; m < NR; ++m) {
            unsigned long long b = 0;
            for (int i = 0; i < SYb; ++i) {
                const int ty = i + R - m;
                if (ty < -R || ty > R) continue;
                const int s = run_half_width(R, ty);
                for (int j = 0; j < SX; ++j) b |= (1ull << (j + R - s)) | (1ull << (j + R + 1 + s));
            }
            t.mask[m] = b;
        }
        return t;
    }
};

// Load the prefix entries of input row m that the block reads (DiscNeed):
// per 16-byte unit of the window, the needed span only -- one 16-byte load
// when it is the whole unit, else 8- and 4-byte loads.  Entries left out are
// never read.
template <int R, int NW>
struct WinUnits {
    static constexpr int OFF = round4(R) - R;
    static constexpr int N = (OFF + NW + 3) / 4;  // units a window touches
};

// up[t] points at unit t of the block's window in its first input row; row m
// adds m * HP, a compile-time offset.
template <int R, int NW>
__device__ __forceinline__ void load_needed(const float *const (&up)[WinUnits<R, NW>::N], int roff,
                                            unsigned long long need, float (&w)[NW]) {
    constexpr int OFF = WinUnits<R, NW>::OFF;
    constexpr int NWU = WinUnits<R, NW>::N;
#pragma unroll
    for (int t = 0; t < NWU; ++t) {
        const float *p = up[t] + roff;
        const int d = 4 * t - OFF;  // w index of unit column 0
        int lo = 4, hi = 0;         // needed columns [lo, hi) of this unit
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = d + k;
            if (i >= 0 && i < NW && ((need >> i) & 1ull)) {
                lo = lo < k ? lo : k;
                hi = hi > k + 1 ? hi : k + 1;
            }
        }
        if (lo >= hi) continue;
        if (lo == 0 && hi == 4) {
            const float4 v = *reinterpret_cast<const float4 *>(p);
            w[d] = v.x; w[d + 1] = v.y; w[d + 2] = v.z; w[d + 3] = v.w;
            continue;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (k < lo || k >= hi) continue;
            const bool pair_head = (k & 1) == 0 && k + 1 < hi;
            const bool pair_tail = (k & 1) == 1 && k - 1 >= lo;
            if (pair_head) {
                const float2 v = *reinterpret_cast<const float2 *>(p + k);
                w[d + k] = v.x;
                w[d + k + 1] = v.y;
            } else if (!pair_tail) {
                w[d + k] = p[k];
            }
        }
    }
}

template <int R, int TXg, int TYg, int SYb>
__device__ __forceinline__ void disc_block(const float *tile, int row0, int bx, float (&out)[SYb][SX]) {
    using G = DiscHalo<R, TXg, TYg>;
    using N = DiscNeed<R, SYb>;
    constexpr int NP = N::NP;  // prefix entries in a block's window
    constexpr int NR = N::NR;
    constexpr typename N::Table need = N::make();  // folded: m is unrolled
    // accumulators of output columns (2h, 2h + 1) as packed pairs
    unsigned long long acc[SYb][SX / 2];
#pragma unroll
    for (int i = 0; i < SYb; ++i)
#pragma unroll
        for (int h = 0; h < SX / 2; ++h) acc[i][h] = 0ull;
    // unit pointers of the window in the first input row, computed once
    constexpr int NWU = WinUnits<R, NP>::N;
    const float *up[NWU];
#pragma unroll
    for (int t = 0; t < NWU; ++t) up[t] = tile + row0 * G::HP + (hunit(2 * bx + t) << 2);
    // P[k] is the row prefix at the block's window column k (column offset
    // k - R from its first output): the run [j - s, j + s] of output j sums
    // to P[j + R + 1 + s] - P[j + R - s].  The next input row's entries are
    // loaded while the current ones are used.
    float P[NP];
    load_needed<R, NP>(up, 0, need.mask[0], P);
#pragma unroll
    for (int m = 0; m < NR; ++m) {
        float Pn[NP];
        if (m + 1 < NR) load_needed<R, NP>(up, (m + 1) * G::HP, need.mask[m + 1], Pn);
#pragma unroll
        for (int i = 0; i < SYb; ++i) {
            const int ty = i + R - m;
            if (ty < -R || ty > R) continue;
            const int s = run_half_width(R, ty);
#pragma unroll
            for (int h = 0; h < SX / 2; ++h) {
                const int j = 2 * h;
                f2add(acc[i][h], f2pack(P[j + R + 1 + s] - P[j + R - s], P[j + R + 2 + s] - P[j + 1 + R - s]));
            }
        }
        if (m + 1 < NR) {
#pragma unroll
            for (int k = 0; k < NP; ++k)
                if ((need.mask[m + 1] >> k) & 1ull) P[k] = Pn[k];
        }
    }
#pragma unroll
    for (int i = 0; i < SYb; ++i)
#pragma unroll
        for (int h = 0; h < SX / 2; ++h) f2unpack(acc[i][h], out[i][2 * h], out[i][2 * h + 1]);
}

// Block operations of the generic half-iteration kernel.  kR is the halo
// radius, Geom the staged tile's geometry, kUniform says whether the result
// still has to be scaled by the uniform tap weight, Params travels in the
// kernel's parameter block.  An op with kPrepass runs prepass() over the
// staged tile (all threads, then a barrier) before the blocks, into
// kExtraFloats of shared memory after it.  kTX x kTY is the output tile of
// one CTA and kSY the rows of a thread's block (kSY x SX outputs); the ops
// without these members use the default 64 x 64 tile and 4-row blocks.
struct DefaultGeo {
    static constexpr int kTX = TX, kTY = TY, kSY = SY;
    static constexpr int kNT = 128;
    static constexpr bool kWide = false;
    static constexpr bool kDefaultTile = true;
    static constexpr int kMinBlocks = 0;  // 0: the register cap of the table below
};

// The disc on a TXg x 64 tile with SYb-row blocks.  Every form of the path
// uses the default (64, 4).  A (128, 8) form reads each staged row's prefix
// entries once for 8 output rows instead of 4 -- a third fewer shared-memory
// wavefronts per output -- but needs 126-166 registers, leaves 12-16 warps
// per SM and measured slower at every size and radius tried.
template <int R, int TXg = TX, int SYb = SY, int TYg = TY>
struct DiscOp {
    static constexpr int kR = R;
    static constexpr int kTX = TXg, kTY = TYg, kSY = SYb;
    static constexpr int kNT = TXg / SX * (TYg / SYb);  // one block per thread
    static constexpr bool kWide = TXg != TX;
    static constexpr bool kDefaultTile = TXg == TX && TYg == TY && SYb == SY;
    static constexpr int kMinBlocks = 0;
    using Geom = DiscHalo<R, TXg, TYg>;
    static constexpr bool kUniform = true;
    static constexpr bool kPrepass = true;
    static constexpr int kExtraFloats = 0;
    struct Params {};
    template <bool FWD>
    static __device__ __forceinline__ void prepass(float *tile, float *, const Params &) {
        row_prefix<R, TXg, TYg, kNT>(tile);
    }
    template <bool FWD>
    static __device__ __forceinline__ void block(const float *tile, int row0, int bx, float (&acc)[SYb][SX],
                                                 const Params &) {
        disc_block<R, TXg, TYg, SYb>(tile, row0, bx, acc);  // symmetric: forward = adjoint
    }
};

// Horizontal box sums of one staged row: h[j] = sum of the 2R + 1 window
// values centred on column j of the block (a sliding sum).
template <int R>
__device__ __forceinline__ void box_row(const float *row, int bx, float (&h)[SX]) {
    constexpr int NW = SX + 2 * R;
    float w[NW];
    load_window<R>(row, bx, w);
    float s = w[0];
#pragma unroll
    for (int k = 1; k <= 2 * R; ++k) s += w[k];
    h[0] = s;
#pragma unroll
    for (int j = 1; j < SX; ++j) {
        s += w[j + 2 * R] - w[j - 1];
        h[j] = s;
    }
}

// Uniform (2R + 1)^2 box: separable sums.  Output row i adds the box sums of
// input rows i..i + 2R.  Rows SY - 1..2R are common to all SY outputs and
// summed once; the 2 (SY - 1) edge rows go to the outputs that reach them.
template <int R>
__device__ __forceinline__ void box_block(const float *tile, int row0, int bx, float (&out)[SY][SX]) {
    using G = Halo<R>;
    static_assert(2 * R + 1 >= SY - 1, "the top and bottom edge rows must not overlap");
    const float *base = tile + row0 * G::HP;
    float c[SX];
    if constexpr (2 * R >= SY - 1) {
        box_row<R>(base + (SY - 1) * G::HP, bx, c);
    } else {  // no common row (R = 1)
#pragma unroll
        for (int j = 0; j < SX; ++j) c[j] = 0.f;
    }
#pragma unroll(R > 8 ? 2 : 1)  // two rows in flight where the register cap allows
    for (int m = SY; m <= 2 * R; ++m) {
        float h[SX];
        box_row<R>(base + m * G::HP, bx, h);
#pragma unroll
        for (int j = 0; j < SX; ++j) c[j] += h[j];
    }
#pragma unroll
    for (int i = 0; i < SY; ++i)
#pragma unroll
        for (int j = 0; j < SX; ++j) out[i][j] = c[j];
    // edge row e < SY - 1 reaches outputs 0..e; edge row 2R + e (e >= 1)
    // reaches outputs e..SY - 1
#pragma unroll
    for (int e = 0; e < SY - 1; ++e) {
        float h[SX];
        box_row<R>(base + e * G::HP, bx, h);
#pragma unroll
        for (int i = 0; i <= e; ++i)
#pragma unroll
            for (int j = 0; j < SX; ++j) out[i][j] += h[j];
        box_row<R>(base + (2 * R + 1 + e) * G::HP, bx, h);
#pragma unroll
        for (int i = e + 1; i < SY; ++i)
#pragma unroll
            for (int j = 0; j < SX; ++j) out[i][j] += h[j];
    }
}

// Uniform (2R + 1)^2 box (Sec. 3, rectangular blur).
template <int R>
struct BoxOp : DefaultGeo {
    static constexpr int kR = R;
    using Geom = Halo<R>;
    static constexpr bool kUniform = true;
    static constexpr bool kPrepass = false;
    static constexpr int kExtraFloats = 0;
    struct Params {};
    template <bool FWD>
    static __device__ __forceinline__ void block(const float *tile, int row0, int bx, float (&acc)[SY][SX],
                                                 const Params &) {
        box_block<R>(tile, row0, bx, acc);  // symmetric: forward = adjoint
    }
};

// Uniform rectangle of any size and anchor within the halo R (Sec. 3,
// rectangular blur: separable sliding sums), given at run time as the tap
// offsets [lox, hix] x [loy, hiy] about the anchor.  The prepass forms the
// vertical sums V(r, c) of every staged column for the tile's rows and
// writes them over the staged tile (all reads finish, in registers, before
// the first write); each block then slides the horizontal sums along V.
// Both passes cost O(1) per pixel whatever the rectangle's size, and the
// shared memory is the staged tile's alone.
template <int R>
struct RectOp : DefaultGeo {
    static constexpr int kR = R;
    using Geom = Halo<R>;
    static constexpr bool kUniform = true;
    static constexpr bool kPrepass = true;
    static constexpr int kExtraFloats = 0;
    using G = Halo<R>;
    // V row pitch: a multiple of 8, room for the column skew (one float per
    // 32 columns) and the row skew (2 ((r >> 2) & 3)), which together keep the
    // 32 lanes of a warp -- 8 columns 8 apart x 4 rows 4 apart -- on distinct
    // banks
    static constexpr int VP = (G::HP + (G::HP - 1) / 32 + 6 + 7) / 8 * 8;
    static_assert(TY * VP <= G::NR * G::HP, "V must fit over the staged tile");
    static constexpr int NG = TY / 16;                      // 16-row groups per column
    static constexpr int NI = (G::HP * NG + 127) / 128;     // (column, group) items per thread
    struct Params { int lox, hix, loy, hiy; };
    static __device__ __forceinline__ int vidx(int r, int c) { return r * VP + c + (c >> 5) + 2 * ((r >> 2) & 3); }
    // staged-tile index of logical column c of staged row m (16-byte units swizzled)
    static __device__ __forceinline__ int sidx(int m, int c) { return m * G::HP + (hunit(c >> 2) << 2) + (c & 3); }

    // V(r, c) = sum over d in [dlo, dhi] of staged row r + R + d, column c;
    // forward: v(p) = sum_t u(p - t), so d runs over -[loy, hiy]; adjoint:
    // c(p) = sum_t q(p + t).  A column's sum slides down 16 rows, then
    // restarts (bounded FP32 drift).
    template <bool FWD>
    static __device__ __forceinline__ void prepass(float *tile, float *, const Params &p) {
        const int dlo = FWD ? -p.hiy : p.loy, dhi = FWD ? -p.loy : p.hiy;
        float v[NI][16];
#pragma unroll
        for (int k = 0; k < NI; ++k) {
            const int it = threadIdx.x + 128 * k;
            if (it < G::HP * NG) {
                const int c = it % G::HP, r0 = it / G::HP * 16;
                float s = 0.f;
                for (int d = dlo; d <= dhi; ++d) s += tile[sidx(r0 + R + d, c)];
                v[k][0] = s;
#pragma unroll
                for (int r = 1; r < 16; ++r) {
                    s += tile[sidx(r0 + r + R + dhi, c)] - tile[sidx(r0 + r - 1 + R + dlo, c)];
                    v[k][r] = s;
                }
            }
        }
        __syncthreads();  // every staged value read: V may overwrite the tile
#pragma unroll
        for (int k = 0; k < NI; ++k) {
            const int it = threadIdx.x + 128 * k;
            if (it < G::HP * NG) {
                const int c = it % G::HP, r0 = it / G::HP * 16;
#pragma unroll
                for (int r = 0; r < 16; ++r) tile[vidx(r0 + r, c)] = v[k][r];
            }
        }
    }

    template <bool FWD>
    static __device__ __forceinline__ void block(const float *tile, int row0, int bx, float (&acc)[SY][SX],
                                                 const Params &p) {
        const float *V = tile;  // the prepass wrote V over the staged tile
        const int elo = FWD ? -p.hix : p.lox, ehi = FWD ? -p.lox : p.hix;
        const int c0 = bx * SX + G::R4 + elo;  // V column of output 0's first term
#pragma unroll
        for (int i = 0; i < SY; ++i) {
            const int r = row0 + i;
            float s = 0.f;
            for (int c = c0; c <= c0 + ehi - elo; ++c) s += V[vidx(r, c)];
            acc[i][0] = s;
#pragma unroll
            for (int j = 1; j < SX; ++j) {
                s += V[vidx(r, c0 + j + ehi - elo)] - V[vidx(r, c0 + j - 1)];
                acc[i][j] = s;
            }
        }
    }
};

// Uniform rectangle by a summed-area table (Sec. 3, rectangular blur: the
// 2D cumulated sums, four lookups per output whatever the rectangle's size).
// An FP32 table over a staged tile reaches thousands of times a pixel value,
// so a small rectangle's sum -- a difference of four entries -- would lose
// about ten bits.  The table is built instead in 64-bit fixed point: every
// staged value is scaled by a power of two 2^e chosen per tile (the largest
// with max|v| 2^e (rows x columns) < 2^62) and rounded to an integer, after
// which every prefix sum and every box sum is exact; the only roundings are
// that conversion (2^-e absolute) and the final conversion back to FP32.
template <int R>
struct SatOp : DefaultGeo {
    static constexpr int kR = R;
    using Geom = Halo<R>;
    using G = Geom;
    static constexpr bool kUniform = true;
    static constexpr bool kPrepass = true;
    static constexpr int NC = 4 * G::NU;  // logical staged columns
    static constexpr int SR = G::NR + 1, SC = NC + 1;
    // table pitch (in 64-bit entries): room for one entry of skew per 8
    // columns, and = 2 (mod 4) so that the rows 4 apart of a 16-lane phase
    // land on complementary banks
    static constexpr int SCP = ((SC + SC / 8 + 1) + 3) / 4 * 4 + 2;
    static constexpr int kExtraFloats = 2 * (SR * SCP + 2);  // the table, then the scale
    // the table (61 KB at R = 8, 89 KB at R = 16) leaves room for two CTAs
    // per SM, one at R = 16: no point capping registers for more
    static constexpr int kMinBlocks = R > 8 ? 1 : 2;
    struct Params { int lox, hix, loy, hiy; };
    static __device__ __forceinline__ int sidx(int m, int c) { return m * G::HP + (hunit(c >> 2) << 2) + (c & 3); }
    static __device__ __forceinline__ int tidx(int r, int c) { return r * SCP + c + (c >> 3); }

    template <bool FWD>
    static __device__ __forceinline__ void prepass(float *tile, float *extra, const Params &) {
        long long *S = reinterpret_cast<long long *>(extra);
        float *scale = reinterpret_cast<float *>(S + SR * SCP);
        __shared__ float wmax[4];
        // the largest magnitude in the staged tile
        float m = 0.f;
        for (int e = threadIdx.x; e < G::NR * NC; e += 128) m = fmaxf(m, fabsf(tile[sidx(e / NC, e % NC)]));
#pragma unroll
        for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            const float mx = fmaxf(fmaxf(wmax[0], wmax[1]), fmaxf(wmax[2], wmax[3]));
            // max |v| 2^e G::NR NC < 2^62
            int e = 40;
            if (mx > 0.f) {
                int ex;
                frexpf(mx * (float)(G::NR * NC), &ex);  // 2^(ex - 1) <= mx NR NC < 2^ex
                e = min(40, 62 - ex);
            }
            scale[0] = ldexpf(1.f, e);
            scale[1] = ldexpf(1.f, -e);
        }
        __syncthreads();
        const float up = scale[0];
        // row prefix sums, one thread per staged row; row 0 and column 0 are 0
        if (threadIdx.x < G::NR) {
            const int r = threadIdx.x;
            long long acc = 0;
            S[tidx(r + 1, 0)] = 0;
            for (int c = 0; c < NC; ++c) {
                acc += __float2ll_rn(tile[sidx(r, c)] * up);
                S[tidx(r + 1, c + 1)] = acc;
            }
        }
        for (int c = threadIdx.x; c < SC; c += 128) S[tidx(0, c)] = 0;
        __syncthreads();
        // then down the columns, one thread per column
        for (int c = threadIdx.x; c < SC; c += 128) {
            long long acc = 0;
            for (int r = 1; r < SR; ++r) {
                acc += S[tidx(r, c)];
                S[tidx(r, c)] = acc;
            }
        }
    }

    // forward: v(p) = sum_t u(p - t), rows p.y - hiy .. p.y - loy and columns
    // p.x - hix .. p.x - lox; adjoint: c(p) = sum_t q(p + t)
    template <bool FWD>
    static __device__ __forceinline__ void block(const float *tile, int row0, int bx, float (&acc)[SY][SX],
                                                 const Params &p) {
        const long long *S = reinterpret_cast<const long long *>(tile + G::NR * G::HP);
        const float down = reinterpret_cast<const float *>(S + SR * SCP)[1];
        const int ylo = FWD ? -p.hiy : p.loy, yhi = FWD ? -p.loy : p.hiy;
        const int xlo = FWD ? -p.hix : p.lox, xhi = FWD ? -p.lox : p.hix;
#pragma unroll
        for (int i = 0; i < SY; ++i) {
            const int r = row0 + i + R;  // staged row of the output
            const int a0 = r + ylo, a1 = r + yhi + 1;
#pragma unroll
            for (int j = 0; j < SX; ++j) {
                const int c = bx * SX + j + G::R4;  // staged column of the output
                const int b0 = c + xlo, b1 = c + xhi + 1;
                const long long sum = S[tidx(a1, b1)] - S[tidx(a0, b1)] - S[tidx(a1, b0)] + S[tidx(a0, b0)];
                acc[i][j] = __ll2float_rn(sum) * down;
            }
        }
    }
};

// Dense K x K taps centred on the origin (naive spatial convolution / list
// filter of Sec. 3 and 5): every tap is a compile-time offset into the
// register window and a constant-bank operand of its FMA.
template <int K>
struct StencilOp : DefaultGeo {
    static constexpr int kR = K / 2;
    using Geom = Halo<K / 2>;
    static constexpr bool kUniform = false;
    static constexpr bool kPrepass = false;
    static constexpr int kExtraFloats = 0;
    struct Params { float w[K * K]; };  // w[(ty + R) * K + (tx + R)] = h(tx, ty)
    template <bool FWD>
    static __device__ __forceinline__ void block(const float *tile, int row0, int bx, float (&acc)[SY][SX],
                                                 const Params &p) {
        using G = Halo<K / 2>;
        constexpr int R = K / 2;
#pragma unroll
        for (int i = 0; i < SY; ++i)
#pragma unroll
            for (int j = 0; j < SX; ++j) acc[i][j] = 0.f;
        constexpr int NW = SX + 2 * R, NR = SY + 2 * R;
        const float *base = tile + row0 * G::HP;
        // next input row's window loaded while the current one is used
        float win[NW];
        load_window<R>(base, bx, win);
#pragma unroll
        for (int m = 0; m < NR; ++m) {
            float wn[NW];
            if (m + 1 < NR) load_window<R>(base + (m + 1) * G::HP, bx, wn);
#pragma unroll
            for (int i = 0; i < SY; ++i) {
                // forward: v(p) = sum_t h(t) u(p - t); adjoint: c(p) = sum_t h(t) q(p + t)
                const int ty = FWD ? i + R - m : m - i - R;
                if (ty < -R || ty > R) continue;
#pragma unroll
                for (int tx = -R; tx <= R; ++tx) {
                    const float wv = p.w[(ty + R) * K + (tx + R)];
#pragma unroll
                    for (int j = 0; j < SX; ++j)
                        acc[i][j] = fmaf(wv, win[FWD ? j + R - tx : j + R + tx], acc[i][j]);
                }
            }
            if (m + 1 < NR) {
#pragma unroll
                for (int k = 0; k < NW; ++k) win[k] = wn[k];
            }
        }
    }
};

// One thread's row segment of SX = 8 pixels in the epilogue: all loads of
// the segment are issued before any is used (one memory round trip per row,
// not per pixel) and go out as 16-byte accesses when the segment is whole
// and aligned, else as n scalars.
template <typename T, bool COH = false>
__device__ __forceinline__ void ld_seg(const T *p, int n, float (&v)[SX]) {
    if (n == SX && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        if constexpr (sizeof(T) == 4) {
            const float4 a = gld<COH>(reinterpret_cast<const float4 *>(p));
            const float4 b = gld<COH>(reinterpret_cast<const float4 *>(p) + 1);
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        } else {
            const uint4 r = gld<COH>(reinterpret_cast<const uint4 *>(p));
            const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const unsigned short lo = (unsigned short)(w[k] & 0xffffu), hi = (unsigned short)(w[k] >> 16);
                if constexpr (std::is_same<T, __half>::value) {
                    v[2 * k] = __half2float(__ushort_as_half(lo));
                    v[2 * k + 1] = __half2float(__ushort_as_half(hi));
                } else {
                    v[2 * k] = __bfloat162float(__ushort_as_bfloat16(lo));
                    v[2 * k + 1] = __bfloat162float(__ushort_as_bfloat16(hi));
                }
            }
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < SX; ++j) v[j] = j < n ? gld_elem<COH>(p, j) : 0.f;
}

template <typename T>
__device__ __forceinline__ void st_seg(T *p, int n, const float (&v)[SX]) {
    if (n == SX && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        if constexpr (sizeof(T) == 4) {
            reinterpret_cast<float4 *>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
            reinterpret_cast<float4 *>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
        } else {
            unsigned w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                unsigned short lo, hi;
                if constexpr (std::is_same<T, __half>::value) {
                    lo = __half_as_ushort(__float2half_rn(v[2 * k]));
                    hi = __half_as_ushort(__float2half_rn(v[2 * k + 1]));
                } else {
                    lo = __bfloat16_as_ushort(__float2bfloat16_rn(v[2 * k]));
                    hi = __bfloat16_as_ushort(__float2bfloat16_rn(v[2 * k + 1]));
                }
                w[k] = (unsigned)lo | (unsigned)hi << 16;
            }
            *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < SX; ++j)
        if (j < n) Stor<T>::st(p, j, v[j]);
}

// Eight bytes of a mask row segment (byte j = pixel j, non-zero = active) as
// one 8-byte access when whole and aligned, else the first n bytes.
template <bool COH = false>
__device__ __forceinline__ unsigned long long ld_mask8(const uint8_t *p, int n) {
    if (n == SX && (reinterpret_cast<uintptr_t>(p) & 7) == 0)
        return gld<COH>(reinterpret_cast<const unsigned long long *>(p));
    unsigned long long v = 0;
#pragma unroll
    for (int j = 0; j < SX; ++j)
        if (j < n) v |= (unsigned long long)gld<COH>(p + j) << (8 * j);
    return v;
}

__device__ __forceinline__ void st_mask8(uint8_t *p, int n, unsigned long long v) {
    if (n == SX && (reinterpret_cast<uintptr_t>(p) & 7) == 0) {
        *reinterpret_cast<unsigned long long *>(p) = v;
        return;
    }
#pragma unroll
    for (int j = 0; j < SX; ++j)
        if (j < n) p[j] = (uint8_t)(v >> (8 * j));
}

// One half of an RL iteration for a TX x TY output tile (128 threads, one
// SY x SX block each).  FWD: v = h (x) u and q = f / v on the tile, written
// to the q plane (inactive pixels keep their q: it is the ratio of their last
// active iteration, Eq. 5).  !FWD: c = h* (x) q and u' = u c with the
// selective-convolution bookkeeping.  The input plane (u or q) is staged with
// a 2R halo continued across the image border.

// Seven resident CTAs per SM (<= 72 registers) while the staged halo allows
// it; the selective-convolution variant needs more registers.
template <int R, bool THIN>
constexpr int min_blocks() { return disc_min_blocks(R, THIN); }
// A wide disc tile (8 x 8 blocks, 64 accumulators per thread) fits four
// CTAs per SM up to R = 8 (its staged tile is 50 KB), three beyond.
template <typename Op, bool THIN>
constexpr int op_min_blocks() {
    // the register cap of the 128-thread tile, for any number of threads
    if constexpr (Op::kWide) return Op::kR > 8 ? 3 : 4;
    else if constexpr (Op::kDefaultTile && Op::kMinBlocks > 0) return Op::kMinBlocks;
    else return min_blocks<Op::kR, THIN>() * 128 / Op::kNT;
}

// One output tile (tbx, tby) of a half-iteration (Op::kTX x Op::kTY, blocks
// of Op::kSY x SX), run by the whole CTA; the kernels below call it once per
// CTA or per work item.
template <typename T, bool THIN, typename Op, bool FWD, bool COH = false>
__device__ __forceinline__ void half_tile(const IterArgs &a, const typename Op::Params &prm, float *qplane,
                                          long long q_pitch, int tbx, int tby, int full, int update_mask) {
    constexpr int R = Op::kR;
    constexpr int GTX = Op::kTX, GTY = Op::kTY, GSY = Op::kSY;
    constexpr int NBX = GTX / SX;  // block columns of the tile
    constexpr int NT = Op::kNT;    // threads of the CTA
    static_assert(NBX % 8 == 0 && (GTY / GSY) % 4 == 0, "a warp covers 8 x 4 blocks");
    static_assert(NBX * (GTY / GSY) == NT && NT % 32 == 0, "one block per thread");
    static_assert(!THIN || Op::kDefaultTile, "selective convolution uses the default tile (tile flags)");
    using G = typename Op::Geom;
    extern __shared__ float sm[];
    const int x0 = tbx * GTX, y0 = tby * GTY;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned used = 0;
    bool tile_any = false;  // a pixel of this thread's blocks stays active
    // Selective convolution at tile granularity: a tile none of whose pixels
    // is active does nothing (u stays, q keeps the stale ratios).
    int *tflag = (THIN && a.tile_flags) ? a.tile_flags + tby * a.tiles_x + tbx : nullptr;
    if (tflag && !full && gld<COH>(tflag) == 0) return;
    if (FWD)
        stage_halo<T, G::NR, G::NU, G::HP, COH, NT>(sm, a.clamp, a.W, a.H, y0 - R, x0 - G::R4, (const T *)a.u_in, a.in_pitch,
                                    threadIdx.x);
    else
        stage_halo<float, G::NR, G::NU, G::HP, COH, NT>(sm, a.clamp, a.W, a.H, y0 - R, x0 - G::R4, qplane, q_pitch,
                                        threadIdx.x);
    {
        // The epilogue reads f (forward) or u (adjoint) at the tile's pixels:
        // start moving those rows into L2 now, while the halo lands and the
        // blocks are summed.  Entry e covers 128 bytes of tile row e / L.
        constexpr int L = (GTX * (int)sizeof(T) + 127) / 128;  // 128-byte lines per tile row
#pragma unroll
        for (int e = threadIdx.x; e < GTY * L; e += NT) {
            const int y = y0 + e / L, x = x0 + (e % L) * (128 / (int)sizeof(T));
            if (y < a.H && x < a.W) {
                const T *p = FWD ? (const T *)a.f + (long long)y * a.f_pitch + x
                                 : (const T *)a.u_in + (long long)y * a.in_pitch + x;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
            }
        }
    }
    // Natural block of this thread: a warp covers 8 (x) x 4 (y) blocks -- the
    // 8 lanes of a 16-byte load phase share a block row -- and the warps tile
    // the NBX x (GTY / GSY) blocks row group by row group.
    const int nbx = (lane & 7) + 8 * (wid % (NBX / 8)), nby = wid / (NBX / 8) * 4 + (lane >> 3);
    // Selective convolution: is any pixel of this thread's block used this
    // iteration?  The mask loads go out now, while the halo lands.
    // The mask words are kept in shared memory (4 KB after the staged tile
    // and the op's extra floats) for the epilogue of this block: in
    // registers they would spill across the block sums.
    bool blk_any = false;
    unsigned long long *bmask = reinterpret_cast<unsigned long long *>(sm + G::NR * G::HP + Op::kExtraFloats);
    if (THIN && !full) {
#pragma unroll
        for (int i = 0; i < GSY; ++i) {
            const int y = y0 + nby * GSY + i, x = x0 + nbx * SX;
            unsigned long long mw = 0ull;
            if (y < a.H && x < a.W) mw = ld_mask8<COH>(a.mask_in + (long long)y * a.mi_pitch + x, min(SX, a.W - x));
            bmask[i * NT + threadIdx.x] = mw;
            blk_any |= mw != 0ull;
        }
    }
    cp_async_wait_all();
    __syncthreads();
    if constexpr (Op::kPrepass) {
        Op::template prepass<FWD>(sm, sm + G::NR * G::HP, prm);
        __syncthreads();
    }
    // Selective convolution: compact the blocks with at least one pixel used
    // this iteration (warp ballot + prefix over the warps) and convolve only
    // those; warps left without blocks retire early.
    int n_active = GTX / SX * GTY / GSY;
    __shared__ int blist[GTX / SX * GTY / GSY];
    __shared__ int wcount[4];
    bool compact = false;  // a block list is used (some block has no used pixel)
    if (THIN && !full) {
        const bool any = blk_any;
        const unsigned bal = __ballot_sync(0xffffffffu, any);
        if (lane == 0) wcount[wid] = __popc(bal);
        __syncthreads();
        int off = 0;
        for (int k = 0; k < wid; ++k) off += wcount[k];
        n_active = wcount[0] + wcount[1] + wcount[2] + wcount[3];
        // every block used (the usual case): keep the natural layout
        compact = n_active < NT;
        if (compact) {
            if (any) blist[off + __popc(bal & ((1u << lane) - 1u))] = nby * (GTX / SX) + nbx;
            __syncthreads();
        }
    }
#pragma unroll 1
    for (int e = threadIdx.x; e < n_active; e += NT) {
        int bx = nbx, by = nby;
        if (THIN && compact) {
            const int b = blist[e];
            bx = b % (GTX / SX);
            by = b / (GTX / SX);
        }
        const int xb = x0 + bx * SX, yb = y0 + by * GSY;
        float acc[GSY][SX];
        Op::template block<FWD>(sm, by * GSY, bx, acc, prm);
        // exact transpose: band pixels of border tiles take A^T q from the band plane
        const bool band = !FWD && a.fold_ct &&
                          (x0 < a.fold_rx || x0 + GTX > a.W - a.fold_rx || y0 < a.fold_ry || y0 + GTY > a.H - a.fold_ry);
        if (band) {
#pragma unroll
            for (int i = 0; i < GSY; ++i) {
                const int y = yb + i;
#pragma unroll
                for (int j = 0; j < SX; ++j) {
                    const int x = xb + j;
                    if (y < a.H && x < a.W &&
                        (x < a.fold_rx || x >= a.W - a.fold_rx || y < a.fold_ry || y >= a.H - a.fold_ry)) {
                        const float ct = a.fold_ct[(long long)y * q_pitch + x];
                        acc[i][j] = Op::kUniform ? ct / a.weight : ct;
                    }
                }
            }
        }
        if (!THIN) {
            const int n = min(SX, a.W - xb);
#pragma unroll
            for (int i = 0; i < GSY; ++i) {
                const int y = yb + i;
                if (y >= a.H || n <= 0) break;
                float e[SX], o[SX];
                if (FWD) {
                    ld_seg<T>((const T *)a.f + (long long)y * a.f_pitch + xb, n, e);
#pragma unroll
                    for (int j = 0; j < SX; ++j)
                        o[j] = rl_ratio(e[j], Op::kUniform ? acc[i][j] * a.weight : acc[i][j]);
                    st_seg<float>(qplane + (long long)y * q_pitch + xb, n, o);
                } else {
                    ld_seg<T, COH>((const T *)a.u_in + (long long)y * a.in_pitch + xb, n, e);
#pragma unroll
                    for (int j = 0; j < SX; ++j)
                        o[j] = e[j] * (Op::kUniform ? acc[i][j] * a.weight : acc[i][j]);
                    st_seg<T>((T *)a.u_out + (long long)y * a.out_pitch + xb, n, o);
                }
            }
            continue;
        }
        // selective convolution (Eq. 4-5), one row segment of SX pixels at a
        // time: mask bytes as one 8-byte access, f / u and u' as 16-byte ones.
        // The segment's mask is cut to its n pixels first, so every pixel
        // step below is branch-free (selects and predicated stores); the
        // arguments it needs are read once, into registers.
        const int n = min(SX, a.W - xb);
        const float w = a.weight, tau = a.tau;
        const bool rel = a.relative != 0;
        const bool write_mask = update_mask && !a.replay;
        const long long mip = a.mi_pitch;
        const uint8_t *mrow = full ? nullptr : a.mask_in + (long long)yb * mip + xb;
        const unsigned long long ones = 0x0101010101010101ull;
        const unsigned long long valid = n >= SX ? ~0ull : (n > 0 ? (1ull << (8 * n)) - 1ull : 0ull);
#pragma unroll
        for (int i = 0; i < GSY; ++i) {
            const int y = yb + i;
            if (y >= a.H || n <= 0) break;
            // the block's own mask words were loaded with the halo, unless the
            // block list gave this thread another block
            const unsigned long long m =
                (full ? ones : (compact ? ld_mask8<COH>(mrow + i * mip, n) : bmask[i * NT + threadIdx.x])) & valid;
            if (FWD) {
                if (m == 0) continue;  // no pixel of the segment used: q keeps its stale ratios
                float e[SX], o[SX];
                ld_seg<T>((const T *)a.f + (long long)y * a.f_pitch + xb, n, e);
#pragma unroll
                for (int j = 0; j < SX; ++j) o[j] = rl_ratio(e[j], Op::kUniform ? acc[i][j] * w : acc[i][j]);
                float *qrow = qplane + (long long)y * q_pitch + xb;
                if (m == ones) {  // every pixel used (then n == SX)
                    st_seg<float>(qrow, SX, o);
                } else {
#pragma unroll
                    for (int j = 0; j < SX; ++j)
                        if ((m >> (8 * j)) & 0xff) qrow[j] = o[j];
                }
            } else {
                float uv[SX], o[SX];
                ld_seg<T, COH>((const T *)a.u_in + (long long)y * a.in_pitch + xb, n, uv);
                unsigned long long mo = 0;
#pragma unroll
                for (int j = 0; j < SX; ++j) {
                    const float u = uv[j];
                    const float c = Op::kUniform ? acc[i][j] * w : acc[i][j];
                    const bool use = ((m >> (8 * j)) & 0xff) != 0;
                    const float un = use ? u * c : u;
                    o[j] = un;
                    used += use;
                    const float d = rel ? (u > 0.f ? fabsf(c - 1.f) : 0.f) : fabsf(un - u);
                    mo |= (unsigned long long)(use && d >= tau) << (8 * j);
                }
                st_seg<T>((T *)a.u_out + (long long)y * a.out_pitch + xb, n, o);
                if (write_mask) {
                    st_mask8(a.mask_out + (long long)y * a.m_pitch + xb, n, mo);
                    tile_any |= mo != 0;
                }
            }
        }
    }
    if (!FWD && THIN) {
        if (a.active_count) warp_count_add(a.active_count, used);
        if (tflag && update_mask) {
            // does any pixel of the tile stay active for the next iteration?
            // (blocks not processed had no active pixel and keep mask 0)
            const int cnt = __syncthreads_count(tile_any);
            if (threadIdx.x == 0) *tflag = cnt;
        }
    }
}

template <typename T, bool THIN, typename Op, bool FWD>
__global__ void __launch_bounds__(Op::kNT, op_min_blocks<Op, THIN>())
    k_disc_half(const __grid_constant__ IterArgs a, const __grid_constant__ typename Op::Params prm, float *qplane,
                long long q_pitch) {
    // Programmatic dependent launch: this grid may start while the previous
    // kernel of the stream drains; every read of its output (u, q, the tile
    // flags) comes after this wait, and the next grid may launch as soon as
    // every CTA of this one has started.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" :::);
    half_tile<T, THIN, Op, FWD>(a, prm, qplane, q_pitch, blockIdx.x, blockIdx.y, a.full, a.update_mask);
}

// Batched (request, tile) form: CTA b runs tile items[b].y of job items[b].x,
// with the job's arguments for the first iteration (phase 0) or the later
// ones (phase 1).  Jobs of one launch share the block operation; FP32
// storage, no thinning.
template <typename Op, bool FWD>
__global__ void __launch_bounds__(Op::kNT, op_min_blocks<Op, false>())
    k_disc_half_tiles(const TileJob *jobs, const int2 *items, int phase,
                      const __grid_constant__ typename Op::Params prm) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" :::);
    const int2 it = items[blockIdx.x];
    const TileJob &job = jobs[it.x];
    const IterArgs &a = job.a[phase];
    const int tiles_x = (a.W + Op::kTX - 1) / Op::kTX;
    half_tile<float, false, Op, FWD>(a, prm, job.qplane, job.q_pitch, it.y % tiles_x, it.y / tiles_x, 1, 0);
}

// Dynamic shared memory of the tile body: the staged tile, the op's extra
// floats and, with selective convolution, one 8-byte mask word per block row.
template <typename Op, bool THIN>
constexpr size_t tile_smem() {
    return Op::Geom::bytes + Op::kExtraFloats * sizeof(float) +
           (THIN ? (size_t)Op::kSY * Op::kNT * sizeof(unsigned long long) : 0);
}

// ---- persistent form --------------------------------------------------------
__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until *w >= need (a neighbour tile has finished the previous half).
// Gives up when another CTA reported an error or after wait_ns, which it
// reports; returns whether the wait succeeded.
__device__ __forceinline__ bool wait_tile(const int *w, int need, int *status, unsigned long long wait_ns) {
    if (ld_acquire_gpu(w) >= need) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        __nanosleep(64);
        if (ld_acquire_gpu(w) >= need) return true;
        if (*(volatile int *)status != 0) return false;
        if (global_ns() - t0 > wait_ns) {
            atomicCAS(status, 0, 1);
            return false;
        }
    }
}

template <typename T, typename Op, bool THIN>
__global__ void __launch_bounds__(Op::kNT, op_min_blocks<Op, THIN>())
    k_disc_persist(const __grid_constant__ PersistArgs p, const __grid_constant__ typename Op::Params prm) {
    __shared__ int s_item;
    const int n_tiles = p.tiles_x * p.tiles_y;
    const int n_items = 2 * p.K * n_tiles;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(p.ticket, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= n_items) break;
        const int hk = item / n_tiles;  // half index: 2 k (forward) or 2 k + 1 (adjoint)
        const int t = item - hk * n_tiles;
        const int tbx = t % p.tiles_x, tby = t / p.tiles_x;
        // the previous half must be complete on the tile and its 8 neighbours
        // (halo <= 16 < 64 pixels): threads 0..8 wait for one tile each
        bool ok = true;
        if (hk > 0 && threadIdx.x < 9) {
            const int nx = tbx + (int)threadIdx.x % 3 - 1, ny = tby + (int)threadIdx.x / 3 - 1;
            if (nx >= 0 && nx < p.tiles_x && ny >= 0 && ny < p.tiles_y)
                ok = wait_tile(p.progress + ny * p.tiles_x + nx, hk, p.status, p.wait_ns);
        }
        if (!__syncthreads_and(ok)) break;
        const int k = hk >> 1;
        const IterArgs &a = p.a[(k > 0) + 2 * (k == p.K - 1)];
        // selective convolution: every pixel used when k % P == 0; the mask
        // is rewritten every iteration (Q = 1) or on those only (Q = P)
        const int full = !THIN || k % p.thin_p == 0;
        const int update_mask = THIN && (p.thin_q == 1 || full);
        if ((hk & 1) == 0)
            half_tile<T, THIN, Op, true, true>(a, prm, p.qplane, p.q_pitch, tbx, tby, full, update_mask);
        else
            half_tile<T, THIN, Op, false, true>(a, prm, p.qplane, p.q_pitch, tbx, tby, full, update_mask);
        // every store of the tile is issued; publish them, then the progress
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            st_release_gpu(p.progress + t, hk + 1);
        }
    }
}

// Batched persistent form: the half-step of a ticket by binary search over
// the half-steps' first tickets, then the same wait / tile body / publish as
// the one-image kernel, with the job's arguments from the table.
template <typename Op>
__global__ void __launch_bounds__(Op::kNT, op_min_blocks<Op, false>())
    k_tiles_persist(const __grid_constant__ TilesPersistArgs p, const __grid_constant__ typename Op::Params prm) {
    __shared__ int s_item;
    const int total = p.start[p.n_halves];
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(p.ticket, 1u);
        __syncthreads();
        const int tk = s_item;
        if (tk >= total) break;
        int lo = 0, hi = p.n_halves - 1;  // last half-step whose start <= tk
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.start[mid] <= tk) lo = mid;
            else hi = mid - 1;
        }
        const int hk = lo, idx = tk - p.start[hk];
        const int2 it = p.items[idx];
        const TileJob &job = p.jobs[it.x];
        const IterArgs &a = job.a[hk >= 2 ? 1 : 0];
        const int tx = p.tiles_x[it.x], ty = (a.H + Op::kTY - 1) / Op::kTY;
        const int tbx = it.y % tx, tby = it.y / tx;
        bool ok = true;
        if (hk > 0 && threadIdx.x < 9) {
            const int nx = tbx + (int)threadIdx.x % 3 - 1, ny = tby + (int)threadIdx.x / 3 - 1;
            if (nx >= 0 && nx < tx && ny >= 0 && ny < ty)
                ok = wait_tile(p.progress + p.first[it.x] + ny * tx + nx, hk, p.status, p.wait_ns);
        }
        if (!__syncthreads_and(ok)) break;
        if ((hk & 1) == 0)
            half_tile<float, false, Op, true, true>(a, prm, job.qplane, job.q_pitch, tbx, tby, 1, 0);
        else
            half_tile<float, false, Op, false, true>(a, prm, job.qplane, job.q_pitch, tbx, tby, 1, 0);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            st_release_gpu(p.progress + idx, hk + 1);
        }
    }
}

template <typename Op>
cudaError_t launch_tiles_persist_t(const TilesPersistArgs &p, const typename Op::Params &prm, cudaStream_t s) {
    constexpr size_t smem = Op::Geom::bytes + Op::kExtraFloats * sizeof(float);
    cudaError_t e = ensure_smem<k_tiles_persist<Op>>(smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tiles_persist<Op>, Op::kNT, smem)) != cudaSuccess)
        return e;
    if (occ < 1) return cudaErrorNotSupported;
    const long long grid = std::min<long long>((long long)occ * sms, (long long)p.n_items0);
    if (grid < 1) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(Op::kNT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_tiles_persist<Op>, p, prm);
}

template <typename Op, typename T, bool THIN>
cudaError_t launch_persist_t(PersistArgs p, const typename Op::Params &prm, cudaStream_t s) {
    constexpr size_t smem = tile_smem<Op, THIN>();
    // tiles of this op (the host sized progress for 64 x 64 tiles, at least as many)
    p.tiles_x = (p.a[0].W + Op::kTX - 1) / Op::kTX;
    p.tiles_y = (p.a[0].H + Op::kTY - 1) / Op::kTY;
    cudaError_t e = ensure_smem<k_disc_persist<T, Op, THIN>>(smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_disc_persist<T, Op, THIN>, Op::kNT, smem)) !=
        cudaSuccess)
        return e;
    if (occ < 1) return cudaErrorNotSupported;
    if (p.ctas_per_sm > 0 && p.ctas_per_sm < occ) occ = p.ctas_per_sm;
    // no more CTAs than tiles: a half has one item per tile, so extra CTAs
    // would only wait -- and a small image then leaves the other SMs to the
    // other streams of a batch
    const long long grid = std::min<long long>((long long)occ * sms, (long long)p.tiles_x * p.tiles_y);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(Op::kNT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: waits between them cannot deadlock
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_disc_persist<T, Op, THIN>, p, prm);
}

template <typename Op>
cudaError_t launch_persist(const PersistArgs &p, const typename Op::Params &prm, int storage, cudaStream_t s) {
    const bool thin = p.thin_p > 0;
    switch (storage) {
    case ST_F32: return thin ? launch_persist_t<Op, float, true>(p, prm, s) : launch_persist_t<Op, float, false>(p, prm, s);
    case ST_BF16: return thin ? launch_persist_t<Op, __nv_bfloat16, true>(p, prm, s)
                              : launch_persist_t<Op, __nv_bfloat16, false>(p, prm, s);
    case ST_F16: return thin ? launch_persist_t<Op, __half, true>(p, prm, s) : launch_persist_t<Op, __half, false>(p, prm, s);
    }
    return cudaErrorInvalidValue;
}

template <typename Op, typename T, bool THIN>
cudaError_t launch_one(const IterArgs &a, const typename Op::Params &prm, float *qplane,
                       long long q_pitch, cudaStream_t s) {
    constexpr size_t smem = tile_smem<Op, THIN>();
    cudaError_t e = ensure_smem<k_disc_half<T, THIN, Op, true>>(smem);
    if (e == cudaSuccess) e = ensure_smem<k_disc_half<T, THIN, Op, false>>(smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((a.W + Op::kTX - 1) / Op::kTX, (a.H + Op::kTY - 1) / Op::kTY);
    cfg.blockDim = dim3(Op::kNT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_disc_half<T, THIN, Op, true>, a, prm, qplane, q_pitch);
    if (e == cudaSuccess && a.fold_ct) e = launch_fold_band(a, qplane, q_pitch, s);
    if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, k_disc_half<T, THIN, Op, false>, a, prm, qplane, q_pitch);
    return e;
}

// One forward and one adjoint launch of the batched form over n_items items.
template <typename Op>
cudaError_t launch_op_tiles(const TileJob *jobs, const int2 *items, int n_items, int phase,
                            const typename Op::Params &prm, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    constexpr size_t smem = Op::Geom::bytes + Op::kExtraFloats * sizeof(float);
    cudaError_t e = ensure_smem<k_disc_half_tiles<Op, true>>(smem);
    if (e == cudaSuccess) e = ensure_smem<k_disc_half_tiles<Op, false>>(smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n_items);
    cfg.blockDim = dim3(Op::kNT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_disc_half_tiles<Op, true>, jobs, items, phase, prm);
    if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, k_disc_half_tiles<Op, false>, jobs, items, phase, prm);
    return e;
}

template <typename Op, bool THIN>
cudaError_t launch_op_t(const IterArgs &a, const typename Op::Params &prm, int storage, float *qplane,
                        long long q_pitch, cudaStream_t s) {
    switch (storage) {
    case ST_F32: return launch_one<Op, float, THIN>(a, prm, qplane, q_pitch, s);
    case ST_BF16: return launch_one<Op, __nv_bfloat16, THIN>(a, prm, qplane, q_pitch, s);
    case ST_F16: return launch_one<Op, __half, THIN>(a, prm, qplane, q_pitch, s);
    }
    return cudaErrorInvalidValue;
}

template <typename Op>
cudaError_t launch_op(const IterArgs &a, const typename Op::Params &prm, int storage, bool thin,
                      float *qplane, long long q_pitch, cudaStream_t s) {
    return thin ? launch_op_t<Op, true>(a, prm, storage, qplane, q_pitch, s)
                : launch_op_t<Op, false>(a, prm, storage, qplane, q_pitch, s);
}


}  // namespace disc
}  // namespace rl

// One translation unit per radius / stencil size keeps each compile short and
// lets them run in parallel.
#define RL_DISC_RADIUS_TU(R)                                                                 \
    namespace rl {                                                                           \
    cudaError_t launch_disc_r##R(const IterArgs &a, int storage, bool thin, float *qplane,   \
                                 long long q_pitch, cudaStream_t s) {                        \
        return disc::launch_op<disc::DiscOp<R>>(a, {}, storage, thin, qplane, q_pitch, s);  \
    }                                                                                        \
    cudaError_t launch_disc_tiles_r##R(const TileJob *jobs, const int2 *items, int n_items,  \
                                       int phase, cudaStream_t s) {                          \
        return disc::launch_op_tiles<disc::DiscOp<R>>(jobs, items, n_items, phase, {}, s);   \
    }                                                                                        \
    cudaError_t launch_disc_tiles_persist_r##R(const TilesPersistArgs &p, cudaStream_t s) {  \
        return disc::launch_tiles_persist_t<disc::DiscOp<R>>(p, {}, s);                      \
    }                                                                                        \
    cudaError_t launch_disc_persist_r##R(const PersistArgs &p, int storage, cudaStream_t s) { \
        return disc::launch_persist<disc::DiscOp<R>>(p, {}, storage, s);                     \
    }                                                                                        \
    }

#define RL_BOX_TU(R)                                                                         \
    namespace rl {                                                                           \
    cudaError_t launch_box_r##R(const IterArgs &a, int storage, bool thin, float *qplane,    \
                                long long q_pitch, cudaStream_t s) {                         \
        return disc::launch_op<disc::BoxOp<R>>(a, {}, storage, thin, qplane, q_pitch, s);   \
    }                                                                                        \
    cudaError_t launch_box_tiles_r##R(const TileJob *jobs, const int2 *items, int n_items,   \
                                      int phase, cudaStream_t s) {                           \
        return disc::launch_op_tiles<disc::BoxOp<R>>(jobs, items, n_items, phase, {}, s);    \
    }                                                                                        \
    cudaError_t launch_box_tiles_persist_r##R(const TilesPersistArgs &p, cudaStream_t s) {   \
        return disc::launch_tiles_persist_t<disc::BoxOp<R>>(p, {}, s);                       \
    }                                                                                        \
    }

#define RL_RECT_TU(R)                                                                        \
    namespace rl {                                                                           \
    cudaError_t launch_rect_r##R(const IterArgs &a, int lox, int hix, int loy, int hiy,      \
                                 int storage, bool thin, float *qplane, long long q_pitch,   \
                                 cudaStream_t s) {                                           \
        return disc::launch_op<disc::RectOp<R>>(a, {lox, hix, loy, hiy}, storage, thin,      \
                                                qplane, q_pitch, s);                         \
    }                                                                                        \
    }

#define RL_SAT_TU(R)                                                                         \
    namespace rl {                                                                           \
    cudaError_t launch_sat_r##R(const IterArgs &a, int lox, int hix, int loy, int hiy,       \
                                int storage, float *qplane, long long q_pitch,               \
                                cudaStream_t s) {                                            \
        return disc::launch_op_t<disc::SatOp<R>, false>(a, {lox, hix, loy, hiy}, storage,    \
                                                        qplane, q_pitch, s);                 \
    }                                                                                        \
    }

#define RL_STENCIL_TU(K)                                                                     \
    namespace rl {                                                                           \
    cudaError_t launch_stencil_k##K(const IterArgs &a, const float *taps, int storage,       \
                                    bool thin, float *qplane, long long q_pitch,             \
                                    cudaStream_t s) {                                        \
        disc::StencilOp<K>::Params p;                                                        \
        for (int i = 0; i < K * K; ++i) p.w[i] = taps[i];                                    \
        return disc::launch_op<disc::StencilOp<K>>(a, p, storage, thin, qplane, q_pitch, s); \
    }                                                                                        \
    }
