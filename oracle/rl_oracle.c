/*
 * rl_oracle.c -- plain, slow, FP64 CPU reference for non-blind Richardson-Lucy
 * deconvolution (Welk & Erler, "Algorithmic Optimisations for Iterative
 * Deconvolution Methods").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  It shares no code, header,
 * table or constant with the CUDA library; neither side includes the other.
 *
 * Everything is written out from the definitions, by direct summation over the
 * PSF support, in double precision, in a fixed loop order (PSF row dy outer,
 * PSF column dx inner), so that a reader can check it against the paper:
 *
 *   Eq. 3 (Sec. 2)   u^{k+1} = ( h* (x) ( f / (u^k (x) h) ) ) . u^k,  u^0 = f,
 *                    h* = h reflected about the origin.
 *   Sec. 2 "Boundary treatment": every missing pixel is replaced by a pixel of
 *                    the image (closest pixel = clamp); the half-sample mirror
 *                    continuation is the second supported rule.
 *   Eq. 4-5 (Sec. 4) selective convolution ("thinning"): inactive pixels keep
 *                    the v of their last active iteration and do not change;
 *                    all pixels are set active again every P (=10) iterations.
 *
 * Conventions.
 *   Images are row-major, index y*W + x, no padding.
 *   A PSF is a dense kh x kw array h[j*kw + i] whose entry (i, j) sits at the
 *   offset t = (i - ax, j - ay) from the origin (anchor (ax, ay)).
 *   Forward operator A (convolution):   v(p) = sum_t h(t) u(m(p - t)).
 *   Pad-flip adjoint B (Eq. 3 read literally: convolution with h*, same
 *   boundary continuation):             c(p) = sum_t h(t) q(m(p + t)).
 *   Exact transpose A^T (scatter form): c(m(p - t)) += h(t) q(p).
 *   m is the boundary index map applied per axis.
 *
 * Parity status: every function here is pinned by the non-GPU tests (brute
 * force on tiny images, scipy.ndimage library routines, closed forms and
 * invariants); none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MIRROR 0 /* half-sample symmetric: ... c b a | a b c ... */
#define ORC_CLAMP 1  /* closest image pixel (Sec. 2)                  */

#define ORC_ADJ_PADFLIP 0
#define ORC_ADJ_TRANSPOSE 1

/* Boundary index map for one axis of length n (Sec. 2).  Mirror is the
 * 2n-periodic even extension, so any offset is valid. */
long orc_map(long e, long n, int boundary)
{
    if (boundary == ORC_CLAMP) {
        if (e < 0) return 0;
        if (e >= n) return n - 1;
        return e;
    }
    long period = 2 * n;
    long r = e % period;
    if (r < 0) r += period;
    return r < n ? r : period - 1 - r;
}

/* ---- PSF construction (Sec. 3, Fig. 1) -------------------------------- */

/* Rescale taps to unit sum.  Returns 0 on success, -1 if a tap is negative or
 * not finite or if the sum is not positive. */
int orc_psf_normalize(double *h, int n)
{
    double s = 0.0;
    for (int k = 0; k < n; ++k) {
        if (!isfinite(h[k]) || h[k] < 0.0) return -1;
        s += h[k];
    }
    if (!(s > 0.0) || !isfinite(s)) return -1;
    for (int k = 0; k < n; ++k) h[k] /= s;
    return 0;
}

/* Linear motion blur of `length` pixels along axis 0 (x, scan-lines,
 * Fig. 1a) or axis 1 (y).  Uniform taps, anchor at index length/2, so the
 * support runs over offsets [-(length/2), length-1-length/2].  `h` holds
 * `length` doubles. */
int orc_psf_motion(int length, int axis, double *h, int *kw, int *kh, int *ax,
                   int *ay)
{
    if (length < 1 || (axis != 0 && axis != 1)) return -1;
    for (int k = 0; k < length; ++k) h[k] = 1.0 / (double)length;
    if (axis == 0) {
        *kw = length; *kh = 1; *ax = length / 2; *ay = 0;
    } else {
        *kw = 1; *kh = length; *ax = 0; *ay = length / 2;
    }
    return 0;
}

/* Defocus (pillbox) PSF of radius r sampled by pixel-centre inclusion
 * (Sec. 3 "Defocus blur", Fig. 1c): support dx^2 + dy^2 <= r^2, uniform
 * weight 1/count.  `h` holds (2r+1)^2 doubles.  Returns the support size. */
int orc_psf_disc(int r, double *h, int *kw, int *kh, int *ax, int *ay)
{
    if (r < 0) return -1;
    int n = 2 * r + 1, count = 0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            long dx = i - r, dy = j - r;
            int in = dx * dx + dy * dy <= (long)r * r;
            h[j * n + i] = in ? 1.0 : 0.0;
            count += in;
        }
    for (int k = 0; k < n * n; ++k) h[k] /= (double)count;
    *kw = n; *kh = n; *ax = r; *ay = r;
    return count;
}

/* ---- Convolution operators (Sec. 3; naive spatial convolution of Sec. 5) - */

/* v = A u : v(x,y) = sum_j sum_i h[j][i] u(m(x-(i-ax)), m(y-(j-ay))). */
void orc_conv(const double *u, double *v, int W, int H, const double *h,
              int kw, int kh, int ax, int ay, int boundary)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double acc = 0.0;
            for (int j = 0; j < kh; ++j) {
                long yy = orc_map((long)y - (j - ay), H, boundary);
                for (int i = 0; i < kw; ++i) {
                    double w = h[j * kw + i];
                    if (w == 0.0) continue;
                    long xx = orc_map((long)x - (i - ax), W, boundary);
                    acc += w * u[yy * W + xx];
                }
            }
            v[(long)y * W + x] = acc;
        }
}

/* c = B q : convolution with the reflected PSF h*(t) = h(-t) under the same
 * boundary continuation: c(x,y) = sum_j sum_i h[j][i] q(m(x+(i-ax)), m(y+(j-ay))). */
void orc_conv_padflip(const double *q, double *c, int W, int H, const double *h,
                      int kw, int kh, int ax, int ay, int boundary)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double acc = 0.0;
            for (int j = 0; j < kh; ++j) {
                long yy = orc_map((long)y + (j - ay), H, boundary);
                for (int i = 0; i < kw; ++i) {
                    double w = h[j * kw + i];
                    if (w == 0.0) continue;
                    long xx = orc_map((long)x + (i - ax), W, boundary);
                    acc += w * q[yy * W + xx];
                }
            }
            c[(long)y * W + x] = acc;
        }
}

/* c = A^T q by scattering every product of A back onto the pixel it was read
 * from.  Serial: it is only used on small images. */
void orc_conv_transpose(const double *q, double *c, int W, int H,
                        const double *h, int kw, int kh, int ax, int ay,
                        int boundary)
{
    memset(c, 0, sizeof(double) * (size_t)W * (size_t)H);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double qv = q[(long)y * W + x];
            for (int j = 0; j < kh; ++j) {
                long yy = orc_map((long)y - (j - ay), H, boundary);
                for (int i = 0; i < kw; ++i) {
                    double w = h[j * kw + i];
                    if (w == 0.0) continue;
                    long xx = orc_map((long)x - (i - ax), W, boundary);
                    c[yy * W + xx] += w * qv;
                }
            }
        }
}

/* ---- Richardson-Lucy with optional selective convolution --------------- */

/*
 * Runs K iterations of Eq. 3 starting from u0 (u0 == NULL means u^0 = f) and
 * writes u^K to u_out.
 *
 * Thinning (Eq. 4-5), enabled by thin != 0:
 *   iteration k is "full" when k mod P == 0; then every pixel is used.
 *   Otherwise pixel p is used iff its mask bit M(p) is set.
 *   Used pixel:   v = (A u)(p), q = f/v (0 where v == 0), r_stale(p) = q.
 *   Unused pixel: q = r_stale(p) (the v of its last active iteration),
 *                 u'(p) = u(p).
 *   Used pixel:   c = (adjoint q)(p), u'(p) = u(p) c.
 *   Change d(p) = relative ? (u(p) > 0 ? |c - 1| : 0) : |u'(p) - u(p)|,
 *   d = 0 for unused pixels.  A pixel whose change is below tau (strict <)
 *   becomes inactive:
 *     Q == 1 (Sec. 4, checked every iteration):  M(p) = used(p) && d >= tau;
 *     Q == P (mask recomputed on full iterations only): on a full iteration
 *            M(p) = d >= tau, otherwise M is left unchanged.
 * mask_trace (nullable, K*W*H bytes) receives used(p) for every iteration.
 * active (nullable) receives the number of used pixel-iterations.
 * Returns 0 on success, -1 on bad arguments.
 */
int orc_rl(const double *f, const double *u0, double *u_out, int W, int H,
           const double *h, int kw, int kh, int ax, int ay, int boundary,
           int adjoint, int K, int thin, double tau, int relative, int P,
           int Q, uint8_t *mask_trace, long long *active)
{
    if (W < 1 || H < 1 || K < 0 || kw < 1 || kh < 1) return -1;
    if (thin && (P < 1 || (Q != 1 && Q != P))) return -1;
    size_t n = (size_t)W * (size_t)H;
    double *u = u_out;
    double *v = malloc(sizeof(double) * n);
    double *q = malloc(sizeof(double) * n);
    double *rs = malloc(sizeof(double) * n);
    double *c = malloc(sizeof(double) * n);
    uint8_t *M = malloc(n);
    if (!v || !q || !rs || !c || !M) {
        free(v); free(q); free(rs); free(c); free(M);
        return -1;
    }
    if (u != (u0 ? u0 : f)) memcpy(u, u0 ? u0 : f, sizeof(double) * n);
    memset(rs, 0, sizeof(double) * n);
    memset(M, 1, n);
    long long act = 0;

    for (int k = 0; k < K; ++k) {
        int full = !thin || (k % P == 0);
        /* v = A u at used pixels (computed everywhere, read only where used) */
        orc_conv(u, v, W, H, h, kw, kh, ax, ay, boundary);
        for (size_t p = 0; p < n; ++p) {
            int use = full || M[p];
            if (use) {
                q[p] = v[p] > 0.0 ? f[p] / v[p] : 0.0;
                rs[p] = q[p];
            } else {
                q[p] = rs[p];
            }
        }
        if (adjoint == ORC_ADJ_TRANSPOSE)
            orc_conv_transpose(q, c, W, H, h, kw, kh, ax, ay, boundary);
        else
            orc_conv_padflip(q, c, W, H, h, kw, kh, ax, ay, boundary);
        for (size_t p = 0; p < n; ++p) {
            int use = full || M[p];
            if (mask_trace) mask_trace[(size_t)k * n + p] = (uint8_t)use;
            act += use;
            double un = use ? u[p] * c[p] : u[p];
            if (thin) {
                double d = 0.0;
                if (use) d = relative ? (u[p] > 0.0 ? fabs(c[p] - 1.0) : 0.0)
                                      : fabs(un - u[p]);
                if (Q == 1)
                    M[p] = (uint8_t)(use && d >= tau);
                else if (full)
                    M[p] = (uint8_t)(d >= tau);
            }
            u[p] = un;
        }
    }
    if (active) *active = act;
    free(v); free(q); free(rs); free(c); free(M);
    return 0;
}
