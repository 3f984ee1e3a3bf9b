// k_fold.cu -- exact-transpose adjoint on the border band, for the two-half
// kernels (disc, register-blocked stencil).
//
// The adjoint half computes the pad-flip sum c(p) = sum_t h(t) q(m(p + t)).
// Away from the border that is (A^T q)(p); within the PSF's reach of the
// border it is not, unless the PSF is symmetric in each axis under the
// mirror.  Between the halves this kernel writes, for every pixel s of that
// band, (A^T q)(s) = sum over the padded positions e with m(e) = s of
// z(e) = sum_t h(t) q0(e + t) (q0 = q in the image, 0 outside), reading the
// full q plane the forward half left; the adjoint half takes it there.
#include "k_tile.cuh"

namespace rl {
namespace {

// The PSF's non-zero taps as (tx, ty, weight), in row-major order.
struct Tap {
    int tx, ty;
    float w;
};

__device__ __forceinline__ float zq(const Tap *taps, int nt, const float *q, long long qp, int W, int H, int ex,
                                    int ey) {
    float z = 0.f;
    for (int k = 0; k < nt; ++k) {
        const int x = ex + taps[k].tx, y = ey + taps[k].ty;
        if (x >= 0 && x < W && y >= 0 && y < H) z = fmaf(taps[k].w, q[(long long)y * qp + x], z);
    }
    return z;
}

// Band pixel i (one per thread): the top fold_ry rows, the bottom fold_ry
// rows, then the fold_rx pixels at each end of the rows between; the whole
// image when the bands cover it.
__device__ __forceinline__ bool band_pixel(long long i, int W, int H, int rx, int ry, int &x, int &y) {
    if (2 * ry >= H || 2 * rx >= W) {
        if (i >= (long long)W * H) return false;
        y = (int)(i / W);
        x = (int)(i - (long long)y * W);
        return true;
    }
    const long long rows = (long long)ry * W;
    if (i < rows) {
        y = (int)(i / W);
        x = (int)(i - (long long)y * W);
        return true;
    }
    i -= rows;
    if (i < rows) {
        y = H - ry + (int)(i / W);
        x = (int)(i - (long long)(y - (H - ry)) * W);
        return true;
    }
    i -= rows;
    const int per = 2 * rx;
    if (i >= (long long)(H - 2 * ry) * per) return false;
    y = ry + (int)(i / per);
    const int k = (int)(i - (long long)(y - ry) * per);
    x = k < rx ? k : W - per + k;
    return true;
}

constexpr int kFoldThreads = 128;
constexpr int kMaxTaps = 33 * 33;  // the largest disc (radius 16)

__global__ void __launch_bounds__(kFoldThreads) k_fold_band(IterArgs a, const float *q, long long qp, int nt_all) {
    __shared__ Tap taps[kMaxTaps];
    __shared__ int wbase[kFoldThreads / 32 + 1];
    __shared__ int ntaps;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // compact the non-zero taps, in order (ballot + prefix over the warps)
    if (tid == 0) ntaps = 0;
    __syncthreads();
    for (int base = 0; base < nt_all; base += kFoldThreads) {
        const int k = base + tid;
        const float w = k < nt_all ? a.fold_taps[k] : 0.f;
        const bool nz = w != 0.f;
        const unsigned bal = __ballot_sync(0xffffffffu, nz);
        if (lane == 0) wbase[wid] = __popc(bal);
        __syncthreads();
        if (tid == 0) {
            int acc = ntaps;
            for (int v = 0; v < kFoldThreads / 32; ++v) {
                const int c = wbase[v];
                wbase[v] = acc;
                acc += c;
            }
            wbase[kFoldThreads / 32] = acc;
        }
        __syncthreads();
        if (nz) {
            const int pos = wbase[wid] + __popc(bal & ((1u << lane) - 1u));
            const int jr = k / a.fold_kw, i = k - jr * a.fold_kw;
            taps[pos] = Tap{i - a.fold_ax, jr - a.fold_ay, w};
        }
        __syncthreads();
        if (tid == 0) ntaps = wbase[kFoldThreads / 32];
        __syncthreads();
    }
    const int nt = ntaps;
    int x, y;
    if (!band_pixel((long long)blockIdx.x * kFoldThreads + tid, a.W, a.H, a.fold_rx, a.fold_ry, x, y)) return;
    // (A^T q)(s) = sum over the padded positions e with m(e) = s of z(e);
    // z(e) can be non-zero for e in [-b, n - 1 + a] per axis
    const int bxe = a.fold_kw - 1 - a.fold_ax, bye = a.fold_kh - 1 - a.fold_ay;
    int rxr[2][2], ryr[2][2];
    const int nx = tile::fold_ranges(x, a.W, a.fold_ax, bxe, a.clamp, rxr);
    const int ny = tile::fold_ranges(y, a.H, a.fold_ay, bye, a.clamp, ryr);
    float acc = 0.f;
    for (int ix = -1; ix < nx; ++ix) {
        const int xlo = ix < 0 ? x : rxr[ix][0], xhi = ix < 0 ? x : rxr[ix][1];
        for (int iy = -1; iy < ny; ++iy) {
            const int ylo = iy < 0 ? y : ryr[iy][0], yhi = iy < 0 ? y : ryr[iy][1];
            for (int ex = xlo; ex <= xhi; ++ex)
                for (int ey = ylo; ey <= yhi; ++ey) acc += zq(taps, nt, q, qp, a.W, a.H, ex, ey);
        }
    }
    a.fold_ct[(long long)y * qp + x] = acc;
}

}  // namespace

cudaError_t launch_fold_band(const IterArgs &a, const float *qplane, long long q_pitch, cudaStream_t s) {
    const int nt = a.fold_kw * a.fold_kh;
    if (nt > kMaxTaps) return cudaErrorInvalidValue;
    const long long rows = 2ll * a.fold_ry * a.W, ends = 2ll * a.fold_rx * (a.H - 2 * a.fold_ry);
    const long long n = (2 * a.fold_ry >= a.H || 2 * a.fold_rx >= a.W) ? (long long)a.W * a.H : rows + ends;
    if (n == 0) return cudaSuccess;
    k_fold_band<<<(unsigned)((n + kFoldThreads - 1) / kFoldThreads), kFoldThreads, 0, s>>>(a, qplane, q_pitch, nt);
    return cudaGetLastError();
}

}  // namespace rl
