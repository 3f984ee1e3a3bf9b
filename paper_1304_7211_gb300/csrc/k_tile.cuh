// k_tile.cuh -- 2D tile kernels for general PSFs, each fusing one whole RL
// iteration (Eq. 3) into one pass over HBM.
//
//   TILE_SPAN     uniform PSF given by one contiguous run of taps per PSF row
//                 (disc, motion, rectangles): every row contributes a span sum
//                 that each thread slides along its chunk of outputs -- the
//                 "generic box filter" of Sec. 3 ("Defocus blur"): moving one
//                 pixel right adds the pixel entering each row's run and drops
//                 the one leaving it (2 M_y operations per pixel).
//   TILE_STENCIL  direct summation over the non-zero taps ("naive spatial
//                 convolution" / "list filter", Sec. 3 "Sparse blur").
//
// A CTA owns a TX x TY output tile.  It stages u over the extended region the
// forward convolution needs, computes q = f / (h (x) u) on the image pixels P
// whose ratio the tile's adjoint convolution reads, continues q beyond the
// image borders by the boundary map, then computes c = h* (x) q and
// u' = u c on the tile.  Only the tile's own outputs are written.
#pragma once

#include "rl_launch.h"

namespace rl {

namespace tile {

constexpr int CHX = 16;   // outputs per thread chunk along x
constexpr int NT = 256;   // threads per CTA

__device__ __forceinline__ void warp_count_add(unsigned long long *ctr, unsigned cnt) {
    unsigned s = __reduce_add_sync(0xffffffffu, cnt);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(ctr, (unsigned long long)s);
}

struct Geo {
    int x0, y0, x1, y1;        // tile outputs [x0,x1) x [y0,y1)
    int qx0, qy0, QW, QH, QP;  // q region (extended coords) and its smem pitch
    int px0, px1, py0, py1;    // image pixels whose ratio is computed
    int ux0, uy0, UW, UH, UP;  // u region (extended coords) and its smem pitch
};

// Image range whose ratio a q region [lo, hi) needs: the region clipped to
// the image plus the image pixels its out-of-image part maps to.  Valid when
// the PSF extents are smaller than n (one reflection at most).
__device__ __forceinline__ void p_range(int lo, int hi, int n, int clamp, int &p0, int &p1) {
    int a = lo, b = hi;
    if (hi > n) a = min(a, clamp ? n - 1 : 2 * n - hi);
    if (lo < 0) b = max(b, clamp ? 1 : -lo);
    p0 = max(0, a);
    p1 = min(n, b);
}

// Exact-transpose adjoint (A^T): the q region is the adjoint's reach
// [lo - a_, hi + b_) plus, for outputs that receive folded contributions, the
// image pixels those contributions read: [0, b_) at the low end and
// [n - a_, n) at the high end.  P is its part inside the image; q is zero
// outside the image.
__device__ __forceinline__ void t_range(int lo, int hi, int n, int ext_lo, int ext_hi, int clamp, int &q0,
                                        int &q1) {
    q0 = lo - ext_lo;
    q1 = hi + ext_hi;
    if (lo < (clamp ? 1 : ext_hi)) q0 = min(q0, 0);      // outputs with a low-end fold
    if (hi > (clamp ? n - 1 : n - ext_lo)) q1 = max(q1, n);  // outputs with a high-end fold
}

__device__ __forceinline__ Geo make_geo(const IterArgs &a, int TX, int TY) {
    Geo g;
    g.x0 = blockIdx.x * TX;
    g.y0 = blockIdx.y * TY;
    g.x1 = min(g.x0 + TX, a.W);
    g.y1 = min(g.y0 + TY, a.H);
    if (a.transpose) {
        int qx1, qy1;
        t_range(g.x0, g.x1, a.W, a.ax, a.bx, a.clamp, g.qx0, qx1);
        t_range(g.y0, g.y1, a.H, a.ay, a.by, a.clamp, g.qy0, qy1);
        g.px0 = max(0, g.qx0);
        g.px1 = min(a.W, qx1);
        g.py0 = max(0, g.qy0);
        g.py1 = min(a.H, qy1);
        g.QW = qx1 - g.qx0;
        g.QH = qy1 - g.qy0;
        g.QP = g.QW | 1;
        g.ux0 = g.px0 - a.bx;
        g.uy0 = g.py0 - a.by;
        g.UW = g.px1 - g.px0 + a.ax + a.bx;
        g.UH = g.py1 - g.py0 + a.ay + a.by;
        g.UP = g.UW | 1;
        return g;
    }
    // q region read by the adjoint: [x0 - ax, x1 + bx) x [y0 - ay, y1 + by);
    // the array also covers P, which can reach past it for off-centre anchors.
    p_range(g.x0 - a.ax, g.x1 + a.bx, a.W, a.clamp, g.px0, g.px1);
    p_range(g.y0 - a.ay, g.y1 + a.by, a.H, a.clamp, g.py0, g.py1);
    g.qx0 = min(g.x0 - a.ax, g.px0);
    g.qy0 = min(g.y0 - a.ay, g.py0);
    g.QW = max(g.x1 + a.bx, g.px1) - g.qx0;
    g.QH = max(g.y1 + a.by, g.py1) - g.qy0;
    g.QP = g.QW | 1;
    g.ux0 = g.px0 - a.bx;
    g.uy0 = g.py0 - a.by;
    g.UW = g.px1 - g.px0 + a.ax + a.bx;
    g.UH = g.py1 - g.py0 + a.ay + a.by;
    g.UP = g.UW | 1;
    return g;
}

// Forward convolution for a chunk of CHX outputs starting at image pixel
// (px, py): acc[j] = v(px + j, py) for j < n.
template <int MODE>
__device__ __forceinline__ void fwd_chunk(const IterArgs &a, const Geo &g, const float *U,
                                          const int2 *spans, const float *taps, int px, int py,
                                          int n, float *acc) {
#pragma unroll
    for (int j = 0; j < CHX; ++j) acc[j] = 0.f;
    const int kw = a.ax + a.bx + 1;
    for (int jr = 0; jr <= a.ay + a.by; ++jr) {
        const int ty = jr - a.ay;
        const float *row = U + (py - ty - g.uy0) * g.UP - g.ux0;  // row[x'] = u(x', py - ty)
        if (MODE == TILE_SPAN) {
            const int2 sp = spans[jr];
            if (sp.x > sp.y) continue;
            // window over x' in [px + j - hi, px + j - lo]
            float s = 0.f;
            for (int xx = px - sp.y; xx <= px - sp.x; ++xx) s += row[xx];
            acc[0] += s;
#pragma unroll
            for (int j = 1; j < CHX; ++j) {
                if (j < n) {
                    s += row[px + j - sp.x] - row[px + j - 1 - sp.y];
                    acc[j] += s;
                }
            }
        } else {
            const float *trow = taps + jr * kw;
            for (int i = 0; i < kw; ++i) {
                const float wt = trow[i];
                if (wt == 0.f) continue;
                const int tx = i - a.ax;
#pragma unroll
                for (int j = 0; j < CHX; ++j)
                    if (j < n) acc[j] = fmaf(wt, row[px + j - tx], acc[j]);
            }
        }
    }
    if (MODE == TILE_SPAN) {
#pragma unroll
        for (int j = 0; j < CHX; ++j) acc[j] *= a.weight;
    }
}

// Adjoint (pad-flip) convolution for a chunk: acc[j] = c(px + j, py),
// c(p) = sum_t h(t) q(m(p + t)) read from the continued q tile.
template <int MODE>
__device__ __forceinline__ void adj_chunk(const IterArgs &a, const Geo &g, const float *Q,
                                          const int2 *spans, const float *taps, int px, int py,
                                          int n, float *acc) {
#pragma unroll
    for (int j = 0; j < CHX; ++j) acc[j] = 0.f;
    const int kw = a.ax + a.bx + 1;
    for (int jr = 0; jr <= a.ay + a.by; ++jr) {
        const int ty = jr - a.ay;
        const float *row = Q + (py + ty - g.qy0) * g.QP - g.qx0;  // row[x'] = q(x', py + ty)
        if (MODE == TILE_SPAN) {
            const int2 sp = spans[jr];
            if (sp.x > sp.y) continue;
            float s = 0.f;
            for (int xx = px + sp.x; xx <= px + sp.y; ++xx) s += row[xx];
            acc[0] += s;
#pragma unroll
            for (int j = 1; j < CHX; ++j) {
                if (j < n) {
                    s += row[px + j + sp.y] - row[px + j - 1 + sp.x];
                    acc[j] += s;
                }
            }
        } else {
            const float *trow = taps + jr * kw;
            for (int i = 0; i < kw; ++i) {
                const float wt = trow[i];
                if (wt == 0.f) continue;
                const int tx = i - a.ax;
#pragma unroll
                for (int j = 0; j < CHX; ++j)
                    if (j < n) acc[j] = fmaf(wt, row[px + j + tx], acc[j]);
            }
        }
    }
    if (MODE == TILE_SPAN) {
#pragma unroll
        for (int j = 0; j < CHX; ++j) acc[j] *= a.weight;
    }
}

// Exact-transpose adjoint at image pixel s: (A^T q)(s) is the sum, over the
// padded positions e with m(e) = s, of z(e) = sum_t h(t) q0(e + t) (q0 = q in
// the image, 0 outside).  adj_chunk on the zero-filled q tile gives the
// e = s term; fold_sum adds the others.  Along one axis of length n, z(e)
// can be non-zero only for e in [-b_, n - 1 + a_]; the positions other than
// s that map to s there are, for the mirror, -1 - s and 2n - 1 - s, and for
// clamp, [-b_, -1] (s = 0) and [n, n - 1 + a_] (s = n - 1).
__device__ __forceinline__ int fold_ranges(int s, int n, int ext_lo, int ext_hi, int clamp, int (&r)[2][2]) {
    int k = 0;
    if (clamp) {
        if (s == 0 && ext_hi >= 1) { r[k][0] = -ext_hi; r[k][1] = -1; ++k; }
        if (s == n - 1 && ext_lo >= 1) { r[k][0] = n; r[k][1] = n - 1 + ext_lo; ++k; }
    } else {
        if (-1 - s >= -ext_hi) { r[k][0] = r[k][1] = -1 - s; ++k; }
        if (2 * n - 1 - s <= n - 1 + ext_lo) { r[k][0] = r[k][1] = 2 * n - 1 - s; ++k; }
    }
    return k;
}

__device__ __forceinline__ float zval(const IterArgs &a, const Geo &g, const float *Q, const float *taps, int ex,
                                      int ey) {
    const int kw = a.ax + a.bx + 1;
    float z = 0.f;
    for (int jr = 0; jr <= a.ay + a.by; ++jr) {
        const int y = ey + jr - a.ay;
        if (y < 0 || y >= a.H) continue;
        const float *row = Q + (y - g.qy0) * g.QP - g.qx0;
        for (int i = 0; i < kw; ++i) {
            const int x = ex + i - a.ax;
            const float wt = taps[jr * kw + i];
            if (x >= 0 && x < a.W && wt != 0.f) z = fmaf(wt, row[x], z);
        }
    }
    return z;
}

static __device__ float fold_sum(const IterArgs &a, const Geo &g, const float *Q, const float *taps, int sx, int sy) {
    int rx[2][2], ry[2][2];
    // x positions of z: [-bx, W - 1 + ax]; y: [-by, H - 1 + ay]
    const int nx = fold_ranges(sx, a.W, a.ax, a.bx, a.clamp, rx);
    const int ny = fold_ranges(sy, a.H, a.ay, a.by, a.clamp, ry);
    if (nx == 0 && ny == 0) return 0.f;
    float acc = 0.f;
    for (int ix = -1; ix < nx; ++ix) {
        const int xlo = ix < 0 ? sx : rx[ix][0], xhi = ix < 0 ? sx : rx[ix][1];
        for (int iy = -1; iy < ny; ++iy) {
            if (ix < 0 && iy < 0) continue;  // e = s: the main term
            const int ylo = iy < 0 ? sy : ry[iy][0], yhi = iy < 0 ? sy : ry[iy][1];
            for (int ex = xlo; ex <= xhi; ++ex)
                for (int ey = ylo; ey <= yhi; ++ey) acc += zval(a, g, Q, taps, ex, ey);
        }
    }
    return acc;
}

template <typename T, bool THIN, int MODE>
__global__ void __launch_bounds__(NT) k_tile(IterArgs a, int TX, int TY, int psf_floats) {
    extern __shared__ float sm[];
    const Geo g = make_geo(a, TX, TY);
    const int kh = a.ay + a.by + 1, kw = a.ax + a.bx + 1;
    float *psf = sm;
    float *U = sm + psf_floats;
    float *Q = U + g.UH * g.UP;
    const int2 *spans = reinterpret_cast<const int2 *>(psf);
    const float *taps = psf;
    const T *f = (const T *)a.f;
    const T *u_in = (const T *)a.u_in;
    T *u_out = (T *)a.u_out;
    unsigned used = 0;

    // PSF table
    if (MODE == TILE_SPAN) {
        int *dst = reinterpret_cast<int *>(psf);
        const int *src = reinterpret_cast<const int *>(a.spans);
        for (int i = threadIdx.x; i < 2 * kh; i += NT) dst[i] = src[i];
    } else {
        for (int i = threadIdx.x; i < kh * kw; i += NT) psf[i] = a.taps[i];
    }
    // u over the extended region, continued at the borders, and f on P
    // (staged where q will be written); 8 loads in flight per thread
    gather_batched<8>(g.UH * g.UW, threadIdx.x, NT,
        [&](int i) {
            const int r = i / g.UW, c = i - r * g.UW;
            const int yy = bmap(g.uy0 + r, a.H, a.clamp), xx = bmap(g.ux0 + c, a.W, a.clamp);
            return Stor<T>::ld(u_in, (long long)yy * a.in_pitch + xx);
        },
        [&](int i, float v) {
            const int r = i / g.UW, c = i - r * g.UW;
            U[r * g.UP + c] = v;
        });
    const int PW = g.px1 - g.px0, PH = g.py1 - g.py0;
    gather_batched<8>(PH * PW, threadIdx.x, NT,
        [&](int i) {
            const int r = i / PW, c = i - r * PW;
            return Stor<T>::ld(f, (long long)(g.py0 + r) * a.f_pitch + g.px0 + c);
        },
        [&](int i, float v) {
            const int r = i / PW, c = i - r * PW;
            Q[(g.py0 + r - g.qy0) * g.QP + (g.px0 + c - g.qx0)] = v;
        });
    __syncthreads();

    // q = f / (h (x) u) on P.  Item = (row, chunk); consecutive lanes take
    // consecutive rows so that their shared-memory rows fall on distinct banks.
    {
        const int nch = (PW + CHX - 1) / CHX;
        for (int it = threadIdx.x; it < PH * nch; it += NT) {
            const int r = it % PH, ch = it / PH;
            const int py = g.py0 + r, px = g.px0 + ch * CHX;
            const int n = min(CHX, g.px1 - px);
            float v[CHX];
            fwd_chunk<MODE>(a, g, U, spans, taps, px, py, n, v);
            float *qrow = Q + (py - g.qy0) * g.QP + (px - g.qx0);
#pragma unroll
            for (int j = 0; j < CHX; ++j) {
                if (j < n) {
                    bool use = true;
                    const long long mi = (long long)py * a.m_pitch + px + j;
                    if (THIN && !a.full) use = a.mask_in[(long long)py * a.mi_pitch + px + j] != 0;
                    qrow[j] = use ? rl_ratio(qrow[j], v[j]) : a.rstale[mi];
                }
            }
        }
    }
    __syncthreads();
    // continue q beyond the image borders (pad-flip adjoint), or zero it there
    // (exact transpose: the folded contributions are added per output below)
    if (g.qx0 < 0 || g.qy0 < 0 || g.qx0 + g.QW > a.W || g.qy0 + g.QH > a.H) {
        for (int i = threadIdx.x; i < g.QH * g.QW; i += NT) {
            const int r = i / g.QW, c = i - r * g.QW;
            const int ey = g.qy0 + r, ex = g.qx0 + c;
            if (ey < 0 || ey >= a.H || ex < 0 || ex >= a.W) {
                if (a.transpose) {
                    Q[r * g.QP + c] = 0.f;
                } else {
                    const int sy = bmap(ey, a.H, a.clamp), sx = bmap(ex, a.W, a.clamp);
                    Q[r * g.QP + c] = Q[(sy - g.qy0) * g.QP + (sx - g.qx0)];
                }
            }
        }
        __syncthreads();
    }
    // c = h* (x) q and u' = u c on the tile; u' replaces u in shared memory
    {
        const int TWd = g.x1 - g.x0, THd = g.y1 - g.y0;
        const int nch = (TWd + CHX - 1) / CHX;
        for (int it = threadIdx.x; it < THd * nch; it += NT) {
            const int r = it % THd, ch = it / THd;
            const int py = g.y0 + r, px = g.x0 + ch * CHX;
            const int n = min(CHX, g.x1 - px);
            float c[CHX];
            adj_chunk<MODE>(a, g, Q, spans, taps, px, py, n, c);
            if (MODE == TILE_STENCIL && a.transpose) {
                // outputs near the border receive the folded contributions
                const bool ybord = py < a.by || py >= a.H - a.ay || (a.clamp && (py == 0 || py == a.H - 1));
                const bool xbord = px < a.bx || px + n > a.W - a.ax || (a.clamp && (px == 0 || px + n == a.W));
                if (ybord || xbord) {
#pragma unroll
                    for (int j = 0; j < CHX; ++j)
                        if (j < n) c[j] += fold_sum(a, g, Q, taps, px + j, py);
                }
            }
            float *urow = U + (py - g.uy0) * g.UP + (px - g.ux0);
            const float *qrow = Q + (py - g.qy0) * g.QP + (px - g.qx0);
#pragma unroll
            for (int j = 0; j < CHX; ++j) {
                if (j < n) {
                    const float u = urow[j];
                    float un;
                    if (THIN) {
                        const long long mi = (long long)py * a.m_pitch + px + j;
                        const bool use = a.full || a.mask_in[(long long)py * a.mi_pitch + px + j] != 0;
                        used += use;
                        un = thin_update(a, mi, use, u, c[j], qrow[j]);
                    } else {
                        un = u * c[j];
                    }
                    urow[j] = un;
                }
            }
        }
    }
    __syncthreads();
    {
        // one warp per output row, 16-byte stores where the row allows
        const int TWd = g.x1 - g.x0, THd = g.y1 - g.y0;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int r = wid; r < THd; r += NT / 32) {
            const float *src = U + (g.y0 + r - g.uy0) * g.UP + (g.x0 - g.ux0);
            smem_to_row(u_out + (long long)(g.y0 + r) * a.out_pitch + g.x0, src,
                        [](int i) { return i; }, TWd, lane, 32);
        }
    }
    if (THIN && a.active_count) warp_count_add(a.active_count, used);
}

inline size_t tile_smem_bytes(const IterArgs &a, TileShape ts, int mode, int *psf_floats) {
    const int kh = a.ay + a.by + 1, kw = a.ax + a.bx + 1;
    int pf = mode == TILE_SPAN ? 2 * kh : kh * kw;
    pf = (pf + 3) & ~3;
    const int ex = a.ax + a.bx, ey = a.ay + a.by;
    // P spans at most tile + ex per axis, so u needs tile + 2 ex; the q array
    // (q region united with P) is bounded by tile + 2 ex as well.  With the
    // exact transpose, P is the q region inside the image, which can reach
    // tile + 2 max(a_, b_) where fold sources widen it: u then needs up to
    // tile + 3 ex.
    const int uf = a.transpose ? 3 : 2;
    const int UW = ts.tx + uf * ex, UH = ts.ty + uf * ey;
    const int QW = ts.tx + 2 * ex, QH = ts.ty + 2 * ey;
    *psf_floats = pf;
    return (size_t)(pf + UH * (UW | 1) + QH * (QW | 1)) * sizeof(float);
}

template <typename T, bool THIN, int MODE>
cudaError_t launch_t(const IterArgs &a, TileShape ts, cudaStream_t s) {
    int pf = 0;
    const size_t smem = tile_smem_bytes(a, ts, MODE, &pf);
    auto kern = k_tile<T, THIN, MODE>;
    cudaError_t e = ensure_smem<k_tile<T, THIN, MODE>>(smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.W + ts.tx - 1) / ts.tx, (a.H + ts.ty - 1) / ts.ty);
    kern<<<grid, NT, smem, s>>>(a, ts.tx, ts.ty, pf);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tt(const IterArgs &a, bool thin, int mode, TileShape ts, cudaStream_t s) {
    if (mode == TILE_SPAN)
        return thin ? launch_t<T, true, TILE_SPAN>(a, ts, s) : launch_t<T, false, TILE_SPAN>(a, ts, s);
    return thin ? launch_t<T, true, TILE_STENCIL>(a, ts, s) : launch_t<T, false, TILE_STENCIL>(a, ts, s);
}

}  // namespace tile
}  // namespace rl

// One translation unit per storage type (compiled in parallel).
#define RL_TILE_TU(NAME, T)                                                                   \
    namespace rl {                                                                            \
    cudaError_t NAME(const IterArgs &a, bool thin, int mode, TileShape ts, cudaStream_t s) {  \
        return tile::launch_tt<T>(a, thin, mode, ts, s);                                      \
    }                                                                                         \
    }
