// k_fold.cu -- exact-transpose adjoint on the border band, for the two-half
// kernels (disc, register-blocked stencil).
//
// The adjoint half computes the pad-flip sum c(p) = sum_t h(t) q(m(p + t)).
// Away from the border that is (A^T q)(p); within the PSF's reach of the
// border it is not, unless the PSF is symmetric in each axis under the
// mirror.  Between the halves two small kernels write, for every pixel s of
// that band, (A^T q)(s) = sum over the padded positions e with m(e) = s of
// z(e) = sum_t h(t) q0(e + t) (q0 = q in the image, 0 outside), from the full
// q plane the forward half left: the first computes z once on the apron
// (the padded positions outside the image where z can be non-zero) into an
// extended plane, the second z(s) on the band plus the apron values that
// fold onto s -- one per axis for the mirror, the whole apron side for clamp.
// The adjoint half takes the result on the band.
#include "k_tile.cuh"

namespace rl {
namespace {

// The PSF's non-zero taps as (tx, ty, weight), in row-major order.
struct Tap {
    int tx, ty;
    float w;
};

constexpr int kFoldThreads = 128;
constexpr int kMaxTaps = 33 * 33;  // the largest disc (radius 16)

// Compact the non-zero taps into shared memory, in order (ballot + prefix
// over the warps; deterministic).  Every thread of the CTA must call it.
__device__ int compact_taps(const IterArgs &a, Tap *taps, int *wbase) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nt_all = a.fold_kw * a.fold_kh;
    int nt = 0;
    for (int base = 0; base < nt_all; base += kFoldThreads) {
        const int k = base + tid;
        const float w = k < nt_all ? a.fold_taps[k] : 0.f;
        const bool nz = w != 0.f;
        const unsigned bal = __ballot_sync(0xffffffffu, nz);
        if (lane == 0) wbase[wid] = __popc(bal);
        __syncthreads();
        int off = nt;
        for (int v = 0; v < wid; ++v) off += wbase[v];
        if (nz) {
            const int jr = k / a.fold_kw, i = k - jr * a.fold_kw;
            taps[off + __popc(bal & ((1u << lane) - 1u))] = Tap{i - a.fold_ax, jr - a.fold_ay, w};
        }
        for (int v = 0; v < kFoldThreads / 32; ++v) nt += wbase[v];
        __syncthreads();
    }
    return nt;
}

__device__ __forceinline__ float zq(const Tap *taps, int nt, const float *q, long long qp, int W, int H, int ex,
                                    int ey) {
    float z0 = 0.f, z1 = 0.f;
    int k = 0;
    for (; k + 1 < nt; k += 2) {  // two chains, loads in flight
        const int x0 = ex + taps[k].tx, y0 = ey + taps[k].ty;
        const int x1 = ex + taps[k + 1].tx, y1 = ey + taps[k + 1].ty;
        if (x0 >= 0 && x0 < W && y0 >= 0 && y0 < H) z0 = fmaf(taps[k].w, q[(long long)y0 * qp + x0], z0);
        if (x1 >= 0 && x1 < W && y1 >= 0 && y1 < H) z1 = fmaf(taps[k + 1].w, q[(long long)y1 * qp + x1], z1);
    }
    if (k < nt) {
        const int x0 = ex + taps[k].tx, y0 = ey + taps[k].ty;
        if (x0 >= 0 && x0 < W && y0 >= 0 && y0 < H) z0 = fmaf(taps[k].w, q[(long long)y0 * qp + x0], z0);
    }
    return z0 + z1;
}

// Item i of a frame: the top t rows and bottom b rows of a w x h region in
// full, then the l leftmost and r rightmost positions of the rows between;
// the whole region when those cover it.  (x, y) relative to the region.
__device__ __forceinline__ bool frame_item(long long i, int w, int h, int l, int r, int t, int b, int &x, int &y) {
    if (t + b >= h || l + r >= w) {
        if (i >= (long long)w * h) return false;
        y = (int)(i / w);
        x = (int)(i - (long long)y * w);
        return true;
    }
    const long long top = (long long)t * w, bot = (long long)b * w;
    if (i < top) {
        y = (int)(i / w);
        x = (int)(i - (long long)y * w);
        return true;
    }
    i -= top;
    if (i < bot) {
        y = h - b + (int)(i / w);
        x = (int)(i - (long long)(y - (h - b)) * w);
        return true;
    }
    i -= bot;
    const int per = l + r;
    if (i >= (long long)(h - t - b) * per) return false;
    y = t + (int)(i / per);
    const int k = (int)(i - (long long)(y - t) * per);
    x = k < l ? k : w - per + k;
    return true;
}

__host__ __device__ __forceinline__ long long frame_size(int w, int h, int l, int r, int t, int b) {
    if (t + b >= h || l + r >= w) return (long long)w * h;
    return (long long)(t + b) * w + (long long)(h - t - b) * (l + r);
}

// z on the apron: the extended region [-bx, W - 1 + ax] x [-by, H - 1 + ay]
// minus the image, into the extended plane (index (e_y + by) * ep + e_x + bx).
__global__ void __launch_bounds__(kFoldThreads) k_fold_apron(IterArgs a, const float *q, long long qp, float *zp,
                                                             long long ep) {
    __shared__ Tap taps[kMaxTaps];
    __shared__ int wbase[kFoldThreads / 32];
    const int nt = compact_taps(a, taps, wbase);
    const int bx = a.fold_kw - 1 - a.fold_ax, by = a.fold_kh - 1 - a.fold_ay;
    const int EW = a.W + a.fold_ax + bx, EH = a.H + a.fold_ay + by;
    int x, y;
    if (!frame_item((long long)blockIdx.x * kFoldThreads + threadIdx.x, EW, EH, bx, a.fold_ax, by, a.fold_ay, x,
                    y))
        return;
    zp[(long long)y * ep + x] = zq(taps, nt, q, qp, a.W, a.H, x - bx, y - by);
}

// (A^T q)(s) on the band: z(s) plus the apron values of the other positions
// the boundary map sends to s.
__global__ void __launch_bounds__(kFoldThreads) k_fold_band(IterArgs a, const float *q, long long qp,
                                                            const float *zp, long long ep) {
    __shared__ Tap taps[kMaxTaps];
    __shared__ int wbase[kFoldThreads / 32];
    const int nt = compact_taps(a, taps, wbase);
    int x, y;
    if (!frame_item((long long)blockIdx.x * kFoldThreads + threadIdx.x, a.W, a.H, a.fold_rx, a.fold_rx, a.fold_ry,
                    a.fold_ry, x, y))
        return;
    const int bx = a.fold_kw - 1 - a.fold_ax, by = a.fold_kh - 1 - a.fold_ay;
    int rxr[2][2], ryr[2][2];
    const int nx = tile::fold_ranges(x, a.W, a.fold_ax, bx, a.clamp, rxr);
    const int ny = tile::fold_ranges(y, a.H, a.fold_ay, by, a.clamp, ryr);
    float acc = zq(taps, nt, q, qp, a.W, a.H, x, y);
    for (int ix = -1; ix < nx; ++ix) {
        const int xlo = ix < 0 ? x : rxr[ix][0], xhi = ix < 0 ? x : rxr[ix][1];
        for (int iy = -1; iy < ny; ++iy) {
            if (ix < 0 && iy < 0) continue;  // e = s: z(s) above
            const int ylo = iy < 0 ? y : ryr[iy][0], yhi = iy < 0 ? y : ryr[iy][1];
            for (int ey = ylo; ey <= yhi; ++ey)
                for (int ex = xlo; ex <= xhi; ++ex) acc += zp[(long long)(ey + by) * ep + ex + bx];
        }
    }
    a.fold_ct[(long long)y * qp + x] = acc;
}

}  // namespace

cudaError_t launch_fold_band(const IterArgs &a, const float *qplane, long long q_pitch, cudaStream_t s) {
    if (a.fold_kw * a.fold_kh > kMaxTaps) return cudaErrorInvalidValue;
    const int bx = a.fold_kw - 1 - a.fold_ax, by = a.fold_kh - 1 - a.fold_ay;
    const int EW = a.W + a.fold_ax + bx, EH = a.H + a.fold_ay + by;
    const long long na = frame_size(EW, EH, bx, a.fold_ax, by, a.fold_ay);
    if (na > 0 && !(bx == 0 && a.fold_ax == 0 && by == 0 && a.fold_ay == 0)) {
        k_fold_apron<<<(unsigned)((na + kFoldThreads - 1) / kFoldThreads), kFoldThreads, 0, s>>>(
            a, qplane, q_pitch, a.fold_z, a.fold_zp);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const long long nb = frame_size(a.W, a.H, a.fold_rx, a.fold_rx, a.fold_ry, a.fold_ry);
    if (nb == 0) return cudaSuccess;
    k_fold_band<<<(unsigned)((nb + kFoldThreads - 1) / kFoldThreads), kFoldThreads, 0, s>>>(
        a, qplane, q_pitch, a.fold_z, a.fold_zp);
    return cudaGetLastError();
}

}  // namespace rl
