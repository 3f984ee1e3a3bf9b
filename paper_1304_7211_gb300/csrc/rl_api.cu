// rl_api.cu -- host runtime and C ABI of the RL library (declared in
// include/rl.h).
//
// The runtime plans a PSF (dense taps, extents, per-row span table of Sec. 3's
// generic box filter), owns the scratch device memory (ping-pong u buffers,
// the selective-convolution mask and stale-ratio planes, host staging
// buffers) and drives the fused iteration kernels on the context stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/rl.h"
#include "rl_launch.h"

using rl::IterArgs;

struct rl_ctx {
    int device = 0;
    int sms = 0;  // multiprocessors of the device
    cudaStream_t stream = nullptr;
    int storage = RL_STORAGE_F32;
    int boundary = RL_BOUNDARY_MIRROR;
    int path_pref = RL_PATH_AUTO;
    int flags = 0;
    int launches = 0;  // kernel launches issued by the current rl_iterate call
    std::string err;

    // PSF plan
    bool has_psf = false;
    int kind = 0, axis = 0, disc_radius = 0;
    int kw = 0, kh = 0, ax = 0, ay = 0;  // dense layout; bx = kw-1-ax, by = kh-1-ay
    std::vector<float> taps;             // normalised, row-major kh x kw
    std::vector<float> sq_taps;          // taps embedded in a centred K x K square (K <= 9), or empty
    int sq_k = 0;
    int box_radius = 0;                  // uniform centred (2R + 1)^2 square, R <= 16, else 0
    bool rect = false;                   // uniform rectangle of taps reaching <= 16 from the anchor
    int rect_lox = 0, rect_hix = 0, rect_loy = 0, rect_hiy = 0;  // its tap offsets
    bool uniform = false;                // one contiguous run of equal taps per row
    bool axis_sym = false;               // h(tx, ty) = h(-tx, ty) = h(tx, -ty)
    std::vector<int2> spans;             // per row j: [lo, hi] offsets (lo > hi = empty)
    float weight = 0.f;                  // the common tap value when uniform
    float *d_taps = nullptr;
    int2 *d_spans = nullptr;
    size_t taps_cap = 0, spans_cap = 0;
    // pinned staging of taps + spans: a ring, so that a new upload waits only
    // for the one kPsfRing uploads back, not for the work queued since
    static constexpr int kPsfRing = 4;
    char *h_psf[kPsfRing] = {};
    size_t h_psf_cap[kPsfRing] = {};
    cudaEvent_t ev_psf[kPsfRing] = {};
    int psf_slot = 0;
    // The legacy / per-thread default stream cannot be captured into a CUDA
    // graph: for a context created on it, rl_iterate runs on this internal
    // non-blocking stream, fenced by events to the caller's stream.
    cudaStream_t own = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    double *d_flux = nullptr;     // flux_blocks() partials + 2 results
    // cached CUDA graph of one segment of iterations (see run_segments)
    cudaGraphExec_t gexec = nullptr;
    unsigned char gkey[sizeof(rl::IterArgs) + 4 * sizeof(int)] = {};

    // scratch
    void *ubuf[2] = {nullptr, nullptr};
    size_t ubuf_bytes = 0;
    uint8_t *mask[2] = {nullptr, nullptr};
    float *rstale = nullptr;
    size_t thin_px = 0;
    float *qplane = nullptr;  // ratio plane of the two-launch disc path
    float *ctplane = nullptr; // exact-transpose band of the two-launch path
    size_t ct_bytes = 0;
    float *zplane = nullptr;  // its apron values (extended plane)
    size_t z_bytes = 0;
    size_t q_px = 0;
    int *tflags = nullptr;    // per-tile activity of the disc path
    size_t tflags_n = 0;
    // persistent disc kernel: per-tile progress, work ticket and status word
    int *pscratch = nullptr;
    size_t pscratch_bytes = 0;
    const int *pstatus = nullptr;  // status word of the last persistent launch, or NULL
    int *status_sink = nullptr;    // pinned host word each persistent launch's status is copied to
    // autotuner: the choice in effect for the current call at its tunable
    // site (-1 = the built-in rule), and its scratch output
    int tune_choice = -1;
    void *tunebuf = nullptr;
    size_t tunebuf_bytes = 0;
    void *tbuf[2] = {nullptr, nullptr};  // transposed f and u (motion along y)
    size_t tbuf_bytes = 0;
    void *tsched = nullptr;              // transposed schedule / mask bytes
    size_t tsched_bytes = 0;
    unsigned long long *d_counter = nullptr;
    void *stage[3] = {nullptr, nullptr, nullptr};
    size_t stage_bytes[3] = {0, 0, 0};
    void *sched = nullptr;  // device copy of a host replay schedule
    size_t sched_bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // mask left by the last thinned call (rl_get_mask)
    const uint8_t *last_mask = nullptr;
    int last_W = 0, last_H = 0;
    long long last_mp = 0;
};

namespace {

thread_local std::string g_create_error;

size_t elem_size(int storage) { return storage == RL_STORAGE_F32 ? 4 : 2; }

rl_status fail(rl_ctx *c, rl_status st, const std::string &msg) {
    if (c) c->err = msg;
    return st;
}

rl_status cuda_fail(rl_ctx *c, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    (void)cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? RL_ERR_OOM : RL_ERR_CUDA, m);
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Fault injection for tests: when set to n > 0, the n-th scratch allocation
// from then on fails as if the device were out of memory.
std::atomic<int> g_fail_alloc{0};

// Test hooks: CTAs per SM of every persistent disc launch (0 = the rule),
// and the bound of its neighbour waits in ns (0 = 2 s).
std::atomic<int> g_test_persist_ctas{0};
std::atomic<unsigned long long> g_test_wait_ns{0};

// Every scratch allocation of rl_iterate: stream-ordered on the context
// stream (no device-wide synchronisation, unlike cudaMalloc / cudaFree).
rl_status salloc(rl_ctx *ctx, void **p, size_t bytes, const char *what) {
    int n = g_fail_alloc.load();
    while (n > 0 && !g_fail_alloc.compare_exchange_weak(n, n - 1)) {
    }
    if (n == 1) return fail(ctx, RL_ERR_OOM, std::string(what) + ": injected allocation failure");
    CK(cudaMallocAsync(p, bytes, ctx->stream), what);
    return RL_OK;
}

#define SALLOC(pp, bytes, what)                                   \
    do {                                                          \
        rl_status st_ = salloc(ctx, (void **)(pp), (bytes), what); \
        if (st_ != RL_OK) return st_;                             \
    } while (0)

// Scratch growth in stream order on the context stream: the old buffer is
// released after the work already queued there, and no other stream (of a
// batch, say) is waited on, as cudaFree would.
rl_status grow(rl_ctx *ctx, void **p, size_t *have, size_t need, const char *what) {
    if (*have >= need && *p) return RL_OK;
    if (*p) cudaFreeAsync(*p, ctx->stream);
    *p = nullptr;
    *have = 0;
    SALLOC(p, need, what);
    *have = need;
    return RL_OK;
}

void sfree(rl_ctx *ctx, void *p) {
    if (p) cudaFreeAsync(p, ctx->stream);
}

// No C++ exception crosses the C ABI: a host allocation failure inside an
// entry point (std::vector / std::string growth) becomes RL_ERR_OOM,
// anything else RL_ERR_STATE, with the context's message set if it can be.
template <typename F>
rl_status abi_guard(rl_ctx *ctx, F &&fn) noexcept {
    try {
        return fn();
    } catch (const std::bad_alloc &) {
        try {
            if (ctx) ctx->err = "out of host memory";
        } catch (...) {
        }
        return RL_ERR_OOM;
    } catch (...) {
        try {
            if (ctx) ctx->err = "internal error";
        } catch (...) {
        }
        return RL_ERR_STATE;
    }
}

}  // namespace

extern "C" {

const char *rl_version(void) { return "rl-gb300 0.1 sm_103a"; }

const char *rl_last_error(const rl_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

static rl_status create_impl(const rl_config *cfg, rl_ctx **out) {
    g_create_error.clear();
    if (!out) {
        g_create_error = "rl_create: out is NULL";
        return RL_ERR_INVALID_ARG;
    }
    *out = nullptr;
    rl_config c = {0, nullptr, RL_STORAGE_F32, RL_BOUNDARY_MIRROR, RL_PATH_AUTO, 0};
    if (cfg) c = *cfg;
    if (c.storage < RL_STORAGE_F32 || c.storage > RL_STORAGE_F16 ||
        (c.boundary != RL_BOUNDARY_MIRROR && c.boundary != RL_BOUNDARY_CLAMP) ||
        c.path < RL_PATH_AUTO || c.path > RL_PATH_SAT) {
        g_create_error = "rl_create: unknown storage, boundary or path value";
        return RL_ERR_INVALID_ARG;
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || c.device < 0 || c.device >= ndev) {
        (void)cudaGetLastError();
        g_create_error = "rl_create: no such CUDA device";
        return e == cudaSuccess ? RL_ERR_INVALID_ARG : RL_ERR_CUDA;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, c.device) != cudaSuccess) {
        g_create_error = "rl_create: cudaGetDeviceProperties failed";
        return RL_ERR_CUDA;
    }
    if (prop.major != 10 || prop.minor != 3) {
        char buf[160];
        snprintf(buf, sizeof buf, "rl_create: device %d is sm_%d%d; this library is built for sm_103a",
                 c.device, prop.major, prop.minor);
        g_create_error = buf;
        return RL_ERR_UNSUPPORTED;
    }
    rl_ctx *ctx = new (std::nothrow) rl_ctx;
    if (!ctx) {
        g_create_error = "rl_create: out of host memory";
        return RL_ERR_OOM;
    }
    ctx->device = c.device;
    ctx->sms = prop.multiProcessorCount;
    ctx->stream = (cudaStream_t)c.stream;
    ctx->storage = c.storage;
    ctx->boundary = c.boundary;
    ctx->path_pref = c.path;
    ctx->flags = c.flags;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    e = cudaMalloc(&ctx->d_counter, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_flux, (rl::flux_blocks() + 2) * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
    for (int i = 0; i < rl_ctx::kPsfRing && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&ctx->ev_psf[i], cudaEventDisableTiming);
    if (e == cudaSuccess && (ctx->stream == nullptr || ctx->stream == cudaStreamLegacy ||
                             ctx->stream == cudaStreamPerThread)) {
        e = cudaStreamCreateWithFlags(&ctx->own, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming);
    }
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        g_create_error = std::string("rl_create: ") + cudaGetErrorString(e);
        (void)cudaGetLastError();
        rl_destroy(ctx);
        return RL_ERR_CUDA;
    }
    *out = ctx;
    return RL_OK;
}

static rl_status destroy_impl(rl_ctx *ctx) {
    if (!ctx) return RL_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    // Scratch comes from the stream-ordered pool: let the work queued on the
    // context's streams finish before any of it is released.
    if (ctx->own) cudaStreamSynchronize(ctx->own);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->d_taps);
    cudaFree(ctx->d_spans);
    cudaFree(ctx->ubuf[0]);
    cudaFree(ctx->ubuf[1]);
    cudaFree(ctx->mask[0]);
    cudaFree(ctx->mask[1]);
    cudaFree(ctx->rstale);
    cudaFree(ctx->qplane);
    cudaFree(ctx->ctplane);
    cudaFree(ctx->zplane);
    cudaFree(ctx->tflags);
    cudaFree(ctx->pscratch);
    cudaFree(ctx->tunebuf);
    cudaFree(ctx->tbuf[0]);
    cudaFree(ctx->tbuf[1]);
    cudaFree(ctx->tsched);
    cudaFree(ctx->d_counter);
    cudaFree(ctx->d_flux);
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    for (int i = 0; i < 3; ++i) cudaFree(ctx->stage[i]);
    cudaFree(ctx->sched);
    for (int i = 0; i < rl_ctx::kPsfRing; ++i) {
        if (ctx->ev_psf[i]) {
            cudaEventSynchronize(ctx->ev_psf[i]);
            cudaEventDestroy(ctx->ev_psf[i]);
        }
        if (ctx->h_psf[i]) cudaFreeHost(ctx->h_psf[i]);
    }
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->own) {
        cudaStreamSynchronize(ctx->own);
        cudaStreamDestroy(ctx->own);
    }
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    cudaSetDevice(prev);
    delete ctx;
    return RL_OK;
}

static rl_status set_psf_impl(rl_ctx *ctx, const rl_psf_desc *d) {
    if (!ctx) return RL_ERR_INVALID_ARG;
    if (!d) return fail(ctx, RL_ERR_INVALID_ARG, "rl_set_psf: descriptor is NULL");
    std::vector<double> t;
    int kw = 0, kh = 0, ax = 0, ay = 0;
    if (d->kind == RL_PSF_MOTION) {
        if (d->length < 1 || (d->axis != 0 && d->axis != 1))
            return fail(ctx, RL_ERR_INVALID_ARG, "rl_set_psf: motion needs length >= 1 and axis 0 or 1");
        if (d->length > 65536) return fail(ctx, RL_ERR_INVALID_ARG, "rl_set_psf: motion length too large");
        t.assign(d->length, 1.0);
        kw = d->axis == 0 ? d->length : 1;
        kh = d->axis == 0 ? 1 : d->length;
        ax = kw / 2;
        ay = kh / 2;
    } else if (d->kind == RL_PSF_DISC) {
        if (d->radius < 0 || d->radius > 127)
            return fail(ctx, RL_ERR_INVALID_ARG, "rl_set_psf: disc radius must be in [0, 127]");
        const int r = d->radius;
        kw = kh = 2 * r + 1;
        ax = ay = r;
        t.assign((size_t)kw * kh, 0.0);
        for (int j = 0; j < kh; ++j)
            for (int i = 0; i < kw; ++i) {
                const long dx = i - r, dy = j - r;
                t[(size_t)j * kw + i] = (dx * dx + dy * dy <= (long)r * r) ? 1.0 : 0.0;
            }
    } else if (d->kind == RL_PSF_DENSE) {
        if (!d->taps || d->kw < 1 || d->kh < 1 || (long long)d->kw * d->kh > 65536)
            return fail(ctx, RL_ERR_INVALID_ARG, "rl_set_psf: dense taps need kw, kh >= 1, kw*kh <= 65536 and a taps array");
        kw = d->kw;
        kh = d->kh;
        ax = d->anchor_x < 0 ? kw / 2 : d->anchor_x;
        ay = d->anchor_y < 0 ? kh / 2 : d->anchor_y;
        if (ax >= kw || ay >= kh)
            return fail(ctx, RL_ERR_INVALID_ARG, "rl_set_psf: anchor outside the tap array");
        t.resize((size_t)kw * kh);
        for (size_t k = 0; k < t.size(); ++k) t[k] = d->taps[k];
    } else {
        return fail(ctx, RL_ERR_INVALID_ARG, "rl_set_psf: unknown PSF kind");
    }
    double sum = 0.0;
    for (double v : t) {
        if (!std::isfinite(v) || v < 0.0)
            return fail(ctx, RL_ERR_INVALID_ARG, "rl_set_psf: taps must be finite and >= 0");
        sum += v;
    }
    if (!(sum > 0.0) || !std::isfinite(sum))
        return fail(ctx, RL_ERR_INVALID_ARG, "rl_set_psf: taps must have a positive sum");

    // Span table (Sec. 3, generic box filter): uniform taps with one
    // contiguous run per row.
    bool uniform = true;
    double common = -1.0;
    std::vector<int2> spans(kh);
    for (int j = 0; j < kh; ++j) {
        int first = -1, last = -1;
        for (int i = 0; i < kw; ++i) {
            const double v = t[(size_t)j * kw + i];
            if (v != 0.0) {
                if (first < 0) first = i;
                else if (last != i - 1) uniform = false;
                last = i;
                if (common < 0.0) common = v;
                else if (v != common) uniform = false;
            }
        }
        spans[j] = first < 0 ? make_int2(1, 0) : make_int2(first - ax, last - ax);
    }
    const int want = ctx->path_pref;
    if (want == RL_PATH_RUNSUM && d->kind != RL_PSF_MOTION)
        return fail(ctx, RL_ERR_UNSUPPORTED, "rl_set_psf: the running-sum path needs a motion PSF");
    if (want == RL_PATH_SPAN && !uniform)
        return fail(ctx, RL_ERR_UNSUPPORTED,
                    "rl_set_psf: the span path needs equal taps in one contiguous run per row");

    std::vector<float> tf(t.size());
    for (size_t k = 0; k < t.size(); ++k) tf[k] = (float)(t[k] / sum);
    // Symmetric in each axis about the anchor: then the pad-flip adjoint under
    // the mirror boundary is the exact transpose.
    bool axis_sym = ax == kw - 1 - ax && ay == kh - 1 - ay;
    for (int j = 0; j < kh && axis_sym; ++j)
        for (int i = 0; i < kw && axis_sym; ++i) {
            const double v = t[(size_t)j * kw + i];
            axis_sym = v == t[(size_t)j * kw + (kw - 1 - i)] && v == t[(size_t)(kh - 1 - j) * kw + i];
        }

    // Stream-ordered upload through a ring of pinned staging buffers; device
    // buffers only grow, and grow in stream order (cudaFreeAsync /
    // cudaMallocAsync on the context stream), so changing the PSF between
    // calls neither synchronises the device nor waits for queued work (which
    // keeps the old taps).
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    const size_t tb = tf.size() * sizeof(float), sb = spans.size() * sizeof(int2);
    cudaError_t e = cudaSuccess;
    if (ctx->taps_cap < tb) {
        if (ctx->d_taps) cudaFreeAsync(ctx->d_taps, ctx->stream);
        ctx->d_taps = nullptr;
        ctx->taps_cap = 0;
        e = cudaMallocAsync((void **)&ctx->d_taps, tb, ctx->stream);
        if (e == cudaSuccess) ctx->taps_cap = tb;
    }
    if (e == cudaSuccess && ctx->spans_cap < sb) {
        if (ctx->d_spans) cudaFreeAsync(ctx->d_spans, ctx->stream);
        ctx->d_spans = nullptr;
        ctx->spans_cap = 0;
        e = cudaMallocAsync((void **)&ctx->d_spans, sb, ctx->stream);
        if (e == cudaSuccess) ctx->spans_cap = sb;
    }
    const int rs = ctx->psf_slot;
    ctx->psf_slot = (rs + 1) % rl_ctx::kPsfRing;
    if (e == cudaSuccess) e = cudaEventSynchronize(ctx->ev_psf[rs]);  // this staging buffer free again
    if (e == cudaSuccess && ctx->h_psf_cap[rs] < tb + sb) {
        if (ctx->h_psf[rs]) cudaFreeHost(ctx->h_psf[rs]);
        ctx->h_psf[rs] = nullptr;
        ctx->h_psf_cap[rs] = 0;
        e = cudaMallocHost((void **)&ctx->h_psf[rs], tb + sb);
        if (e == cudaSuccess) ctx->h_psf_cap[rs] = tb + sb;
    }
    if (e == cudaSuccess) {
        memcpy(ctx->h_psf[rs], tf.data(), tb);
        memcpy(ctx->h_psf[rs] + tb, spans.data(), sb);
        e = cudaMemcpyAsync(ctx->d_taps, ctx->h_psf[rs], tb, cudaMemcpyHostToDevice, ctx->stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->d_spans, ctx->h_psf[rs] + tb, sb, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_psf[rs], ctx->stream);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        ctx->has_psf = false;
        return cuda_fail(ctx, e, "rl_set_psf: upload");
    }

    ctx->kind = d->kind;
    ctx->axis = d->kind == RL_PSF_MOTION ? d->axis : 0;
    ctx->disc_radius = d->kind == RL_PSF_DISC ? d->radius : 0;
    ctx->kw = kw;
    ctx->kh = kh;
    ctx->ax = ax;
    ctx->ay = ay;
    ctx->taps = tf;
    ctx->uniform = uniform;
    ctx->axis_sym = axis_sym;
    // Taps within 4 pixels of the anchor on every side: the centred square
    // K = 2 max(extents) + 1 with zeros around them, for the register-blocked
    // stencil (a stencil over the square computes the same convolution).
    {
        const int r = std::max(std::max(ax, kw - 1 - ax), std::max(ay, kh - 1 - ay));
        ctx->sq_taps.clear();
        ctx->sq_k = 0;
        if (r <= 4) {
            const int rr = std::max(r, 1), K = 2 * rr + 1;
            ctx->sq_taps.assign((size_t)K * K, 0.f);
            for (int j = 0; j < kh; ++j)
                for (int i = 0; i < kw; ++i)
                    ctx->sq_taps[(size_t)(j - ay + rr) * K + (i - ax + rr)] = tf[(size_t)j * kw + i];
            ctx->sq_k = K;
        }
    }
    // A uniform centred odd square: the register-blocked box (separable sums).
    ctx->box_radius = 0;
    if (uniform && kw == kh && (kw & 1) && ax == kw / 2 && ay == kh / 2 && kw / 2 >= 1 &&
        kw / 2 <= rl::kDiscMaxRadius) {
        bool full = true;
        for (int j = 0; j < kh && full; ++j) full = spans[j].x == -ax && spans[j].y == kw - 1 - ax;
        if (full) ctx->box_radius = kw / 2;
    }
    // A uniform rectangle: the non-empty PSF rows are contiguous and share
    // one span (register-blocked separable sums, any anchor).
    ctx->rect = false;
    if (uniform) {
        int jlo = -1, jhi = -1;
        bool same = true;
        for (int j = 0; j < kh; ++j) {
            if (spans[j].x > spans[j].y) continue;
            if (jlo < 0) jlo = j;
            else same = same && jhi == j - 1 && spans[j].x == spans[jlo].x && spans[j].y == spans[jlo].y;
            jhi = j;
        }
        if (jlo >= 0 && same) {
            const int lox = spans[jlo].x, hix = spans[jlo].y, loy = jlo - ay, hiy = jhi - ay;
            const int reach = std::max(std::max(std::abs(lox), std::abs(hix)), std::max(std::abs(loy), std::abs(hiy)));
            if (reach <= rl::kRectMaxReach) {
                ctx->rect = true;
                ctx->rect_lox = lox;
                ctx->rect_hix = hix;
                ctx->rect_loy = loy;
                ctx->rect_hiy = hiy;
            }
        }
    }
    ctx->spans = spans;
    ctx->weight = uniform ? (float)(common / sum) : 0.f;
    ctx->has_psf = true;
    // a cached graph may carry the old taps in its kernel parameters
    if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    ctx->err.clear();
    return RL_OK;
}

}  // extern "C"

namespace {

// Exact-transpose adjoint requested where it differs from the pad-flip one.
bool needs_fold(const rl_ctx *ctx) {
    return (ctx->flags & RL_FLAG_ADJOINT_TRANSPOSE) &&
           !(ctx->boundary == RL_BOUNDARY_MIRROR && ctx->axis_sym);
}

int choose_path(const rl_ctx *ctx, int W) {
    const int L = ctx->kind == RL_PSF_MOTION ? (ctx->axis == 0 ? ctx->kw : ctx->kh) : 0;
    // The exact transpose folds in the disc, box and register-stencil halves
    // (a band kernel between them), in the resident motion rows (run_device)
    // and in the generic stencil tiles, not in the span tiles.
    if (needs_fold(ctx)) {
        if (ctx->kind == RL_PSF_DISC && ctx->disc_radius >= 1 && ctx->disc_radius <= rl::kDiscMaxRadius)
            return RL_PATH_SPAN;
        if (ctx->box_radius || (ctx->kind == RL_PSF_DENSE && ctx->rect)) return RL_PATH_SPAN;
        return RL_PATH_STENCIL;
    }
    int p = ctx->path_pref;
    if (p == RL_PATH_AUTO) {
        if (ctx->kind == RL_PSF_MOTION) p = RL_PATH_RUNSUM;
        else if (ctx->kind == RL_PSF_DISC) p = RL_PATH_SPAN;
        // a uniform centred square: the box kernel beats the stencil's taps
        // at every size; another uniform rectangle: the rectangle kernel,
        // except within 2 pixels of the anchor, where the register stencil
        // (K <= 5) is as fast as its shared-memory passes
        else if (ctx->box_radius) p = RL_PATH_SPAN;
        else if (ctx->rect && !(ctx->sq_k && ctx->sq_k <= 5)) p = RL_PATH_SPAN;
        // dense taps within 4 pixels of the anchor: the register-blocked
        // stencil beats span sums (every tap a register operand)
        else if (ctx->sq_k) p = RL_PATH_STENCIL;
        else if (ctx->uniform) p = RL_PATH_SPAN;
        else p = RL_PATH_STENCIL;
    }
    // Rows too long for shared memory fall back to the span tile kernel.
    if (p == RL_PATH_RUNSUM && ctx->axis == 0 && !rl::motion_x_fits(W, L)) p = RL_PATH_SPAN;
    return p;
}

// Issue iterations [k0, k1) through a CUDA graph of G consecutive iterations
// replayed (k1 - k0) / G times; `issue(k)` enqueues iteration k on the
// context stream and must give the same launches for k and k + G.  The
// instantiated graph is cached on the context, keyed by the arguments of its
// first iteration, so repeating an identical call skips the capture.  Returns
// the first iteration not issued.
template <typename ISSUE, typename KEYARGS>
rl_status run_segments(rl_ctx *ctx, int k0, int k1, int G, int extra_key, ISSUE issue,
                       KEYARGS key_args, int *k_next) {
    *k_next = k0;
    const int nseg = G > 0 ? (k1 - k0) / G : 0;
    if (!ctx->stream || nseg < 2) return RL_OK;
    unsigned char key[sizeof ctx->gkey];
    memset(key, 0, sizeof key);
    const IterArgs ka = key_args(k0);
    memcpy(key, &ka, sizeof ka);
    const int meta[4] = {G, extra_key, ctx->storage, ctx->disc_radius};
    memcpy(key + sizeof ka, meta, sizeof meta);
    if (!ctx->gexec || memcmp(key, ctx->gkey, sizeof key) != 0) {
        if (ctx->gexec) {
            cudaGraphExecDestroy(ctx->gexec);
            ctx->gexec = nullptr;
        }
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "rl_iterate: capture");
        rl_status st = RL_OK;
        const int launches = ctx->launches;
        for (int k = k0; k < k0 + G && st == RL_OK; ++k) st = issue(k);
        ctx->launches = launches;
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
        if (st != RL_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "rl_iterate: capture");
        const cudaError_t ei = cudaGraphInstantiate(&ctx->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            ctx->gexec = nullptr;
            return cuda_fail(ctx, ei, "rl_iterate: graph instantiate");
        }
        memcpy(ctx->gkey, key, sizeof key);
    }
    for (int s = 0; s < nseg; ++s)
        CK(cudaGraphLaunch(ctx->gexec, ctx->stream), "rl_iterate: graph launch");
    *k_next = k0 + nseg * G;
    return RL_OK;
}

// All K iterations of the running-sum path in one launch of the row-resident
// kernel.  Motion along y runs on the transposed image (transposed f, start,
// schedule in; transposed result and mask out).
rl_status run_resident(rl_ctx *ctx, const void *f, const void *start, void *u_out, int W, int H,
                       long long pitch, int K, const rl_thinning *thin, size_t plane, long long sp) {
    const size_t es = elem_size(ctx->storage);
    IterArgs a;
    memset(&a, 0, sizeof a);
    a.clamp = ctx->boundary == RL_BOUNDARY_CLAMP;
    a.weight = ctx->weight;
    a.transpose = needs_fold(ctx);
    rl::TBArgs tb;
    memset(&tb, 0, sizeof tb);
    tb.K = K;
    tb.round = ctx->storage != RL_STORAGE_F32;
    tb.chunk = ctx->tune_choice > 0 ? ctx->tune_choice : 0;
    const bool ydir = ctx->axis == 1;
    const int Wt = ydir ? H : W, Ht = ydir ? W : H;   // the problem the kernel sees
    const long long tp = ((long long)Wt + 63) / 64 * 64;
    if (thin) {
        tb.P = thin->reset_period;
        tb.Q = thin->update_period;
        a.relative = thin->relative != 0;
        a.tau = thin->threshold;
        a.active_count = ctx->d_counter;
        a.mask_out = ydir ? nullptr : ctx->mask[0];
        a.m_pitch = sp;
    }
    const uint8_t *sched = nullptr;
    if (thin && thin->schedule) {
        const size_t bytes = (size_t)W * H * K;
        if (is_device_ptr(thin->schedule)) {
            sched = thin->schedule;
        } else {
            rl_status st = grow(ctx, &ctx->sched, &ctx->sched_bytes, bytes, "rl_iterate: schedule");
            if (st != RL_OK) return st;
            CK(cudaMemcpyAsync(ctx->sched, thin->schedule, bytes, cudaMemcpyHostToDevice, ctx->stream),
               "rl_iterate: schedule upload");
            sched = (const uint8_t *)ctx->sched;
        }
    }
    if (!ydir) {
        a.f = f;
        a.u_in = start;
        a.u_out = u_out;
        a.W = W;
        a.H = H;
        a.f_pitch = a.in_pitch = a.out_pitch = pitch;
        a.ax = ctx->ax;
        a.bx = ctx->kw - 1 - ctx->ax;
        if (sched) {
            tb.sched = sched;
            tb.s_pitch = W;
            tb.s_plane = (long long)W * H;
        }
        cudaError_t e = rl::launch_motion_x_tb(a, tb, ctx->storage, thin != nullptr, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "rl_iterate: kernel launch");
        ctx->launches += 1;
    } else {
        const size_t tbytes = (size_t)Ht * tp * es;
        if (ctx->tbuf_bytes < tbytes) {
            sfree(ctx, ctx->tbuf[0]);
            sfree(ctx, ctx->tbuf[1]);
            ctx->tbuf[0] = ctx->tbuf[1] = nullptr;
            ctx->tbuf_bytes = 0;
            SALLOC(&ctx->tbuf[0], tbytes, "rl_iterate: transposed f");
            SALLOC(&ctx->tbuf[1], tbytes, "rl_iterate: transposed u");
            ctx->tbuf_bytes = tbytes;
        }
        CK(rl::launch_transpose(f, pitch, 0, ctx->tbuf[0], tp, 0, W, H, 1, (int)es, ctx->stream),
           "rl_iterate: transpose f");
        CK(rl::launch_transpose(start, pitch, 0, ctx->tbuf[1], tp, 0, W, H, 1, (int)es, ctx->stream),
           "rl_iterate: transpose u0");
        ctx->launches += 2;
        a.f = ctx->tbuf[0];
        a.u_in = ctx->tbuf[1];
        a.u_out = ctx->tbuf[1];
        a.W = Wt;
        a.H = Ht;
        a.f_pitch = a.in_pitch = a.out_pitch = tp;
        a.ax = ctx->ay;
        a.bx = ctx->kh - 1 - ctx->ay;
        const size_t sbytes = thin ? (size_t)Ht * tp * (sched ? (size_t)K : 1) : 0;
        if (thin) {
            rl_status st = grow(ctx, &ctx->tsched, &ctx->tsched_bytes, sbytes, "rl_iterate: transposed mask");
            if (st != RL_OK) return st;
        }
        if (sched) {
            CK(rl::launch_transpose(sched, W, (long long)W * H, ctx->tsched, tp, (long long)Ht * tp, W, H,
                                    K, 1, ctx->stream),
               "rl_iterate: transpose schedule");
            ctx->launches += 1;
            tb.sched = (const uint8_t *)ctx->tsched;
            tb.s_pitch = tp;
            tb.s_plane = (long long)Ht * tp;
        } else if (thin) {
            a.mask_out = (uint8_t *)ctx->tsched;
            a.m_pitch = tp;
        }
        cudaError_t e = rl::launch_motion_x_tb(a, tb, ctx->storage, thin != nullptr, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "rl_iterate: kernel launch");
        CK(rl::launch_transpose(ctx->tbuf[1], tp, 0, u_out, pitch, 0, Wt, Ht, 1, (int)es, ctx->stream),
           "rl_iterate: transpose back");
        ctx->launches += 2;
        if (thin && !sched) {
            CK(rl::launch_transpose(ctx->tsched, tp, 0, ctx->mask[0], sp, 0, Wt, Ht, 1, 1, ctx->stream),
               "rl_iterate: transpose mask");
            ctx->launches += 1;
        }
    }
    if (thin && !sched) {
        ctx->last_mask = ctx->mask[0];
        ctx->last_W = W;
        ctx->last_H = H;
        ctx->last_mp = sp;
    }
    (void)plane;
    return RL_OK;
}

// Block operations of the two-half kernels.
enum HalfOp { OP_DISC = 0, OP_BOX = 1, OP_STENCIL = 2, OP_RECT = 3, OP_SAT = 4 };

// Disc / box / register-stencil path: two launches per iteration (forward +
// ratio, adjoint + update).  The adjoint half reads u only at its own pixels,
// so u and the mask are updated in place in one working buffer; with
// thinning, tiles with no active pixel skip both launches.
rl_status run_disc(rl_ctx *ctx, const void *f, const void *start, void *u_out, int W, int H,
                   long long pitch, int K, const rl_thinning *thin, long long sp, int op) {
    const int R = op == OP_STENCIL ? ctx->sq_k / 2
                  : op == OP_BOX   ? ctx->box_radius
                  : (op == OP_RECT || op == OP_SAT) ? rl::rect_halo(std::max(std::max(std::abs(ctx->rect_lox), std::abs(ctx->rect_hix)),
                                                            std::max(std::abs(ctx->rect_loy), std::abs(ctx->rect_hiy))))
                                   : ctx->disc_radius;
    const size_t es = elem_size(ctx->storage);
    const size_t plane = (size_t)sp * H;
    if (ctx->ubuf_bytes < plane * es) {
        sfree(ctx, ctx->ubuf[0]);
        sfree(ctx, ctx->ubuf[1]);
        ctx->ubuf[0] = ctx->ubuf[1] = nullptr;
        ctx->ubuf_bytes = 0;
        SALLOC(&ctx->ubuf[0], plane * es, "rl_iterate: scratch u");
        SALLOC(&ctx->ubuf[1], plane * es, "rl_iterate: scratch u");
        ctx->ubuf_bytes = plane * es;
    }
    IterArgs a;
    memset(&a, 0, sizeof a);
    a.f = f;
    a.W = W;
    a.H = H;
    a.f_pitch = pitch;
    a.clamp = ctx->boundary == RL_BOUNDARY_CLAMP;
    a.ax = a.bx = a.ay = a.by = R;
    a.weight = ctx->weight;
    a.m_pitch = a.mi_pitch = sp;
    if (needs_fold(ctx)) {
        // exact transpose: A^T q on the border band, written between the halves
        rl_status st = grow(ctx, (void **)&ctx->ctplane, &ctx->ct_bytes, (size_t)sp * H * sizeof(float),
                            "rl_iterate: transpose band");
        if (st != RL_OK) return st;
        a.fold_ct = ctx->ctplane;
        a.fold_taps = ctx->d_taps;
        a.fold_kw = ctx->kw;
        a.fold_kh = ctx->kh;
        a.fold_ax = ctx->ax;
        a.fold_ay = ctx->ay;
        a.fold_rx = std::max(ctx->ax, ctx->kw - 1 - ctx->ax);
        a.fold_ry = std::max(ctx->ay, ctx->kh - 1 - ctx->ay);
        a.fold_zp = (long long)W + ctx->kw - 1;
        st = grow(ctx, (void **)&ctx->zplane, &ctx->z_bytes,
                  (size_t)a.fold_zp * (H + ctx->kh - 1) * sizeof(float), "rl_iterate: transpose apron");
        if (st != RL_OK) return st;
        a.fold_z = ctx->zplane;
    }
    const uint8_t *sched = nullptr;
    if (thin) {
        a.relative = thin->relative != 0;
        a.tau = thin->threshold;
        a.active_count = ctx->d_counter;
        a.mask_in = ctx->mask[0];
        a.mask_out = ctx->mask[0];
        if (thin->schedule) {
            const size_t bytes = (size_t)W * H * K;
            if (is_device_ptr(thin->schedule)) {
                sched = thin->schedule;
            } else {
                rl_status st = grow(ctx, &ctx->sched, &ctx->sched_bytes, bytes, "rl_iterate: schedule");
                if (st != RL_OK) return st;
                CK(cudaMemcpyAsync(ctx->sched, thin->schedule, bytes, cudaMemcpyHostToDevice, ctx->stream),
                   "rl_iterate: schedule upload");
                sched = (const uint8_t *)ctx->sched;
            }
        } else {
            const int tx = (W + 63) / 64, ty = (H + 63) / 64;
            const size_t n = (size_t)tx * ty;
            if (ctx->tflags_n < n) {
                sfree(ctx, ctx->tflags);
                ctx->tflags = nullptr;
                ctx->tflags_n = 0;
                SALLOC((void **)&ctx->tflags, n * sizeof(int), "rl_iterate: tile flags");
                ctx->tflags_n = n;
            }
            a.tile_flags = ctx->tflags;
            a.tiles_x = tx;
        }
    }
    void *work = ctx->ubuf[0];
    ctx->pstatus = nullptr;
    auto args_for = [&](int k) {
        IterArgs b = a;
        const bool last = k == K - 1;
        b.u_in = k == 0 ? start : work;
        b.in_pitch = k == 0 ? pitch : sp;
        // without thinning the last iteration writes the caller's buffer
        const bool direct = last && !thin;
        b.u_out = direct ? u_out : work;
        b.out_pitch = direct ? pitch : sp;
        if (sched) {
            b.replay = 1;
            b.full = 0;
            b.update_mask = 0;
            b.mask_in = sched + (size_t)k * W * H;
            b.mi_pitch = W;
        } else if (thin) {
            b.full = (k % thin->reset_period) == 0;
            b.update_mask = thin->update_period == 1 || b.full;
        }
        return b;
    };
    auto issue = [&](int k) -> rl_status {
        const IterArgs b = args_for(k);
        cudaError_t e =
            op == OP_STENCIL ? rl::launch_stencil(b, ctx->sq_taps.data(), ctx->sq_k, ctx->storage, thin != nullptr,
                                                  ctx->qplane, sp, ctx->stream)
            : op == OP_BOX   ? rl::launch_box(b, ctx->storage, thin != nullptr, R, ctx->qplane, sp, ctx->stream)
            : op == OP_SAT   ? rl::launch_sat(b, ctx->rect_lox, ctx->rect_hix, ctx->rect_loy, ctx->rect_hiy,
                                              ctx->storage, ctx->qplane, sp, ctx->stream)
            : op == OP_RECT  ? rl::launch_rect(b, ctx->rect_lox, ctx->rect_hix, ctx->rect_loy, ctx->rect_hiy,
                                               ctx->storage, thin != nullptr, ctx->qplane, sp, ctx->stream)
                             : rl::launch_disc(b, ctx->storage, thin != nullptr, R, ctx->qplane, sp, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "rl_iterate: kernel launch");
        ctx->launches += 2;
        return RL_OK;
    };
    // Disc: every iteration in one persistent launch (tiles advance as their
    // neighbourhood allows, no barrier between the halves) when the image has
    // enough tiles for the overlap to pay; the grid then holds about two
    // tiles per CTA (rl::disc_persist_ctas).  Measured (us/it, GB300): disc
    // r = 8 at 2048^2 38.4 two launches, 35.6 persistent with 3 CTAs per SM,
    // 41.5 with every resident CTA; r = 12 at 4096^2 137 against 127.  Below
    // about 6 tiles per SM (1024^2 and 1448^2 at r <= 8) the two launches
    // are faster, and so they are for plain 16-bit storage at 2048^2 (42.0
    // against 44.1), where the old margin of 1.25 tiles per resident CTA
    // slot stays.
    const int tx = (W + rl::disc_tile() - 1) / rl::disc_tile();
    const int ty = (H + rl::disc_persist_tile_h() - 1) / rl::disc_persist_tile_h();  // persistent tiles
    const long long tiles = (long long)tx * ty;
    const long long slots = (long long)ctx->sms * rl::disc_min_blocks(R, false);
    const bool narrow = ctx->storage != RL_STORAGE_F32 && !thin;
    // a tuned choice (0 = two launches, c >= 1 = persistent with c CTAs per
    // SM) overrides the rule
    const bool persist_pays = ctx->tune_choice >= 0 ? ctx->tune_choice >= 1
                              : narrow              ? 4LL * tiles >= 5LL * slots
                                                    : tiles >= 6LL * ctx->sms;
    // RL_FLAG_PERSISTENT asks for the persistent form; a batch slot's
    // contexts ask for it on plain solves only (thinned ones keep the rule:
    // measured on the served workload at 200 requests/s, 110 against 93
    // Gpx-it/s and a median latency of 60 against 330 ms)
    const bool forced = (ctx->flags & RL_FLAG_PERSISTENT) && ctx->tune_choice < 0 &&
                        !(thin && (ctx->flags & rl::kFlagBatchSlot));
    if (op == OP_DISC && !sched && !a.fold_ct && !(ctx->flags & RL_FLAG_PER_ITERATION) &&
        (persist_pays || forced)) {
        const size_t n = (size_t)tx * ty + 2;  // progress per tile, ticket, status
        rl_status st = grow(ctx, (void **)&ctx->pscratch, &ctx->pscratch_bytes, n * sizeof(int),
                            "rl_iterate: tile progress");
        if (st != RL_OK) return st;
        CK(cudaMemsetAsync(ctx->pscratch, 0, n * sizeof(int), ctx->stream), "rl_iterate: tile progress");
        rl::PersistArgs pa;
        memset(&pa, 0, sizeof pa);
        pa.a[0] = args_for(0);
        pa.a[1] = args_for(K > 2 ? 1 : 0);
        pa.a[2] = args_for(0);
        pa.a[3] = args_for(K - 1);
        pa.qplane = ctx->qplane;
        pa.q_pitch = sp;
        pa.K = K;
        pa.tiles_x = tx;
        pa.tiles_y = ty;
        pa.progress = ctx->pscratch;
        pa.ticket = (unsigned *)(ctx->pscratch + tx * ty);
        pa.status = ctx->pscratch + tx * ty + 1;
        const unsigned long long test_wait = g_test_wait_ns.load();
        pa.wait_ns = test_wait > 0 ? test_wait : 2000000000ull;  // 2 s for one neighbour tile: only a fault gets near it
        const int test_ctas = g_test_persist_ctas.load();
        pa.ctas_per_sm = test_ctas > 0               ? test_ctas
                         : ctx->tune_choice >= 1 ? ctx->tune_choice
                                                 : rl::disc_persist_ctas(tiles, ctx->sms);
        if (thin) {  // the mask and the u plane are updated in place; u_out is written after
            pa.thin_p = thin->reset_period;
            pa.thin_q = thin->update_period;
        }
        const cudaError_t e = rl::launch_disc_persist(pa, ctx->storage, R, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "rl_iterate: persistent launch");
        ctx->pstatus = pa.status;
        if (ctx->status_sink)  // in stream order, so it holds this launch's outcome once the stream passes it
            CK(cudaMemcpyAsync(ctx->status_sink, pa.status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
               "rl_iterate: status");
        ctx->launches += 1;
        if (thin) {
            CK(cudaMemcpy2DAsync(u_out, pitch * es, work, sp * es, W * es, H, cudaMemcpyDeviceToDevice,
                                 ctx->stream),
               "rl_iterate: copy out");
            ctx->last_mask = ctx->mask[0];
            ctx->last_W = W;
            ctx->last_H = H;
            ctx->last_mp = sp;
        }
        return RL_OK;
    }
    // iteration 0 reads the start image; the middle iterations repeat with
    // period G (in place; thinning epochs of reset_period) and are replayed
    // from a CUDA graph; the last one (no thinning) writes the caller's buffer
    int k = 0;
    rl_status st = issue(k++);
    if (st != RL_OK) return st;
    if (!sched && K > 1) {
        const int G = thin ? thin->reset_period : 10;
        const int kend = thin ? K : K - 1;
        int kn = k;
        st = run_segments(ctx, 1, kend, G >= 2 && G <= 64 ? G : 0, (thin ? 1 : 0) | op << 1 | R << 3, issue,
                          args_for, &kn);
        if (st != RL_OK) return st;
        ctx->launches += (kn - k) * 2;
        k = kn;
    }
    for (; k < K; ++k) {
        st = issue(k);
        if (st != RL_OK) return st;
    }
    if (thin) {
        CK(cudaMemcpy2DAsync(u_out, pitch * es, work, sp * es, W * es, H, cudaMemcpyDeviceToDevice,
                             ctx->stream),
           "rl_iterate: copy out");
        if (!sched) {
            ctx->last_mask = ctx->mask[0];
            ctx->last_W = W;
            ctx->last_H = H;
            ctx->last_mp = sp;
        }
    }
    return RL_OK;
}

rl_status run_device(rl_ctx *ctx, const void *f, const void *u0, void *u_out, int W, int H,
                     long long pitch, int K, const rl_thinning *thin, int *path_out) {
    const size_t es = elem_size(ctx->storage);
    const int path = choose_path(ctx, W);
    *path_out = path;
    const void *start = u0 ? u0 : f;
    if (K == 0) {
        if (u_out != start)
            CK(cudaMemcpy2DAsync(u_out, pitch * es, start, pitch * es, W * es, H,
                                 cudaMemcpyDeviceToDevice, ctx->stream),
               "rl_iterate: copy");
        return RL_OK;
    }
    const long long sp = ((long long)W + 63) / 64 * 64;  // scratch pitch (elements)
    const size_t plane = (size_t)sp * H;
    if (thin) {
        if (ctx->thin_px < plane) {
            for (int i = 0; i < 2; ++i) {
                sfree(ctx, ctx->mask[i]);
                ctx->mask[i] = nullptr;
            }
            sfree(ctx, ctx->rstale);
            ctx->rstale = nullptr;
            ctx->thin_px = 0;
            ctx->last_mask = nullptr;
            SALLOC((void **)&ctx->mask[0], plane, "rl_iterate: mask");
            SALLOC((void **)&ctx->mask[1], plane, "rl_iterate: mask");
            SALLOC((void **)&ctx->rstale, plane * sizeof(float), "rl_iterate: stale ratio");
            ctx->thin_px = plane;
        }
        CK(cudaMemsetAsync(ctx->d_counter, 0, sizeof(unsigned long long), ctx->stream),
           "rl_iterate: counter");
        // the stale ratio of a pixel that was never used is 0
        CK(cudaMemsetAsync(ctx->rstale, 0, plane * sizeof(float), ctx->stream), "rl_iterate: stale ratio");
    }
    // Exact transpose of a motion PSF: the resident rows fold it along the
    // row (every other path for it is the stencil tiles).
    if (needs_fold(ctx) && ctx->kind == RL_PSF_MOTION && !(ctx->flags & RL_FLAG_PER_ITERATION)) {
        const int L = ctx->axis == 0 ? ctx->kw : ctx->kh;
        const int line = ctx->axis == 0 ? W : H;
        if (rl::motion_x_tb_fits(line, L, thin != nullptr, ctx->tune_choice > 0 ? ctx->tune_choice : 0)) {
            *path_out = RL_PATH_RUNSUM;
            return run_resident(ctx, f, start, u_out, W, H, pitch, K, thin, plane, sp);
        }
    }
    // Running sum with whole lines resident for all iterations: one launch.
    if (path == RL_PATH_RUNSUM && !(ctx->flags & RL_FLAG_PER_ITERATION)) {
        const int L = ctx->axis == 0 ? ctx->kw : ctx->kh;
        const int line = ctx->axis == 0 ? W : H;
        if (rl::motion_x_tb_fits(line, L, thin != nullptr, ctx->tune_choice > 0 ? ctx->tune_choice : 0))
            return run_resident(ctx, f, start, u_out, W, H, pitch, K, thin, plane, sp);
    }
    if ((K > 1 || u_out == start) && ctx->ubuf_bytes < plane * es) {
        sfree(ctx, ctx->ubuf[0]);
        sfree(ctx, ctx->ubuf[1]);
        ctx->ubuf[0] = ctx->ubuf[1] = nullptr;
        ctx->ubuf_bytes = 0;
        SALLOC(&ctx->ubuf[0], plane * es, "rl_iterate: scratch u");
        SALLOC(&ctx->ubuf[1], plane * es, "rl_iterate: scratch u");
        ctx->ubuf_bytes = plane * es;
    }
    // the register-blocked two-half kernels: the disc; a uniform centred
    // square (box); another uniform rectangle given as dense taps (rect);
    // taps within 4 pixels of the anchor (stencil)
    int op = -1;
    if (path == RL_PATH_SPAN && ctx->kind == RL_PSF_DISC && ctx->disc_radius >= 1 &&
        ctx->disc_radius <= rl::kDiscMaxRadius)
        op = OP_DISC;
    else if (path == RL_PATH_SPAN && ctx->box_radius)
        op = OP_BOX;
    else if (path == RL_PATH_SPAN && ctx->kind == RL_PSF_DENSE && ctx->rect)
        op = OP_RECT;
    else if (path == RL_PATH_STENCIL && ctx->sq_k)
        op = OP_STENCIL;
    else if (path == RL_PATH_SAT) {
        if (!ctx->rect) return fail(ctx, RL_ERR_UNSUPPORTED, "rl_iterate: the SAT path takes uniform rectangles only");
        if (thin) return fail(ctx, RL_ERR_UNSUPPORTED, "rl_iterate: the SAT path has no selective convolution");
        op = OP_SAT;
    }
    if (op >= 0) {
        if (ctx->q_px < plane) {
            sfree(ctx, ctx->qplane);
            ctx->qplane = nullptr;
            ctx->q_px = 0;
            SALLOC((void **)&ctx->qplane, plane * sizeof(float), "rl_iterate: ratio plane");
            ctx->q_px = plane;
        }
        if (thin) CK(cudaMemsetAsync(ctx->qplane, 0, plane * sizeof(float), ctx->stream), "rl_iterate: ratio plane");
        return run_disc(ctx, f, start, u_out, W, H, pitch, K, thin, sp, op);
    }

    IterArgs a;
    memset(&a, 0, sizeof a);
    a.f = f;
    a.W = W;
    a.H = H;
    a.f_pitch = pitch;
    a.clamp = ctx->boundary == RL_BOUNDARY_CLAMP;
    a.ax = ctx->ax;
    a.bx = ctx->kw - 1 - ctx->ax;
    a.ay = ctx->ay;
    a.by = ctx->kh - 1 - ctx->ay;
    a.weight = ctx->weight;
    a.taps = ctx->d_taps;
    a.spans = ctx->d_spans;
    a.m_pitch = sp;
    a.mi_pitch = sp;
    a.rstale = ctx->rstale;
    a.transpose = needs_fold(ctx);
    const uint8_t *sched = nullptr;
    if (thin && thin->schedule) {
        const size_t bytes = (size_t)W * H * K;
        if (is_device_ptr(thin->schedule)) {
            sched = thin->schedule;
        } else {
            rl_status st = grow(ctx, &ctx->sched, &ctx->sched_bytes, bytes, "rl_iterate: schedule");
            if (st != RL_OK) return st;
            CK(cudaMemcpyAsync(ctx->sched, thin->schedule, bytes, cudaMemcpyHostToDevice, ctx->stream),
               "rl_iterate: schedule upload");
            sched = (const uint8_t *)ctx->sched;
        }
    }
    a.active_count = thin ? ctx->d_counter : nullptr;
    if (thin) {
        a.relative = thin->relative != 0;
        a.tau = thin->threshold;
    }
    // a tuned tile shape (tx << 16 | ty) overrides the table
    const rl::TileShape ts = ctx->tune_choice > 0
                                 ? rl::TileShape{ctx->tune_choice >> 16, ctx->tune_choice & 0xffff}
                                 : rl::tile_shape_for(a.ax, a.bx, a.ay, a.by);
    int cur = 0;  // mask plane holding the current mask
    auto args_for = [&](int k) {
        IterArgs b = a;
        const bool last = k == K - 1;
        b.u_in = k == 0 ? start : ctx->ubuf[(k - 1) & 1];
        b.in_pitch = k == 0 ? pitch : sp;
        const bool direct = last && !(k == 0 && u_out == start);
        b.u_out = direct ? u_out : ctx->ubuf[k & 1];
        b.out_pitch = direct ? pitch : sp;
        if (sched) {
            b.replay = 1;
            b.full = 0;
            b.update_mask = 0;
            b.mask_in = sched + (size_t)k * W * H;
            b.mi_pitch = W;
            b.mask_out = ctx->mask[cur];
        } else if (thin) {
            b.full = (k % thin->reset_period) == 0;
            b.update_mask = thin->update_period == 1 || b.full;
            b.mask_in = ctx->mask[cur];
            b.mask_out = ctx->mask[cur ^ 1];
        }
        return b;
    };
    auto issue = [&](int k) -> rl_status {
        const IterArgs b = args_for(k);
        cudaError_t e;
        if (path == RL_PATH_RUNSUM)
            e = ctx->axis == 0 ? rl::launch_motion_x(b, ctx->storage, thin != nullptr, ctx->stream)
                               : rl::launch_motion_y(b, ctx->storage, thin != nullptr, ctx->stream);
        else
            e = rl::launch_tile(b, ctx->storage, thin != nullptr,
                                path == RL_PATH_SPAN ? rl::TILE_SPAN : rl::TILE_STENCIL, ts, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "rl_iterate: kernel launch");
        ctx->launches += 1;
        if (thin && b.update_mask) cur ^= 1;
        return RL_OK;
    };
    int k = 0;
    rl_status st = issue(k++);
    if (st != RL_OK) return st;
    if (!thin && K > 2) {
        // plain RL: iterations 1 .. K-2 alternate the two scratch buffers,
        // so a segment of 10 repeats; replay it from a CUDA graph
        int kn = k;
        st = run_segments(ctx, 1, K - 1, 10, (2 + path) | (ts.tx << 4) | (ts.ty << 16), issue, args_for, &kn);
        if (st != RL_OK) return st;
        ctx->launches += kn - k;
        k = kn;
    }
    for (; k < K; ++k) {
        st = issue(k);
        if (st != RL_OK) return st;
    }
    if (thin && !sched) {
        ctx->last_mask = ctx->mask[cur];
        ctx->last_W = W;
        ctx->last_H = H;
        ctx->last_mp = sp;
    }
    {
        const IterArgs b = args_for(K - 1);
        if (b.u_out != u_out)
            CK(cudaMemcpy2DAsync(u_out, pitch * es, b.u_out, sp * es, W * es, H,
                                 cudaMemcpyDeviceToDevice, ctx->stream),
               "rl_iterate: copy out");
    }
    return RL_OK;
}


// ---- autotuner -------------------------------------------------------------
// The tunable site of a call, its candidates and its cache key.  Only choices
// that leave the arithmetic of every pixel unchanged, or change it by FP32
// rounding alone, are tuned: the disc path's launch form (bit-identical), the
// running-sum chunk width (where the window sums restart) and the stencil
// tile shape (bit-identical).
struct TuneSite {
    std::string key;
    std::vector<int> candidates;
};

TuneSite tune_site(const rl_ctx *ctx, int W, int H, const rl_thinning *thin) {
    TuneSite t;
    if (ctx->flags & RL_FLAG_PER_ITERATION) return t;
    const int path = choose_path(ctx, W);
    char buf[192];
    const char *sto = ctx->storage == RL_STORAGE_F32 ? "f32" : ctx->storage == RL_STORAGE_BF16 ? "bf16" : "f16";
    const char *bnd = ctx->boundary == RL_BOUNDARY_CLAMP ? "clamp" : "mirror";
    const char *th = thin ? (thin->schedule ? "replay" : "thin") : "plain";
    if (ctx->kind == RL_PSF_MOTION && (path == RL_PATH_RUNSUM || needs_fold(ctx))) {
        const int L = ctx->axis == 0 ? ctx->kw : ctx->kh;
        const int line = ctx->axis == 0 ? W : H;
        for (int c : {13, 17, 33})
            if (rl::motion_x_tb_fits(line, L, thin != nullptr, c)) t.candidates.push_back(c);
        snprintf(buf, sizeof buf, "motion-chunk:L%d%s:%dx%d:%s:%s:%s:sm%d", L, ctx->axis ? "y" : "x", W, H, sto,
                 bnd, th, ctx->sms);
    } else if (path == RL_PATH_SPAN && ctx->kind == RL_PSF_DISC && ctx->disc_radius >= 1 &&
               ctx->disc_radius <= rl::kDiscMaxRadius && !thin && !needs_fold(ctx) &&
               !(ctx->flags & RL_FLAG_PERSISTENT)) {
        // (RL_FLAG_PERSISTENT is the caller's decision -- a batch sets it: a
        // small persistent solve is slower alone, which is what the timing
        // sees, but shares the GPU with the other streams better)
        // 0 = two launches per iteration; c >= 1 = persistent with c CTAs per
        // SM, around the rule's count (the launch caps c at its occupancy)
        const long long tiles = (long long)((W + rl::disc_tile() - 1) / rl::disc_tile()) *
                                ((H + rl::disc_persist_tile_h() - 1) / rl::disc_persist_tile_h());
        const int cmax = rl::disc_min_blocks(ctx->disc_radius, false);
        const int c = std::min(rl::disc_persist_ctas(tiles, ctx->sms), cmax);
        t.candidates = {0};
        for (int d = c - 1; d <= c + 1; ++d)
            if (d >= 1 && d <= cmax) t.candidates.push_back(d);
        snprintf(buf, sizeof buf, "disc-launch:r%d:%dx%d:%s:%s:%s:sm%d", ctx->disc_radius, W, H, sto, bnd, th,
                 ctx->sms);
    } else if (path == RL_PATH_STENCIL && !ctx->sq_k) {
        t.candidates = {64 << 16 | 32, 64 << 16 | 64, 128 << 16 | 32, 128 << 16 | 64};
        snprintf(buf, sizeof buf, "stencil-tile:%dx%da%d,%d:%dx%d:%s:%s:%s:sm%d", ctx->kw, ctx->kh, ctx->ax, ctx->ay,
                 W, H, sto, bnd, th, ctx->sms);
    } else {
        return t;
    }
    if (t.candidates.size() > 1) t.key = buf;
    return t;
}

// With RL_FLAG_AUTOTUNE: the first call for a key times every candidate on
// the call's own inputs (a warm-up run, then the faster of two timed runs of
// up to 10 iterations, into library scratch; CUDA events on the context
// stream) and caches the fastest; later calls with the key take the cached
// choice.  The device is drained first, so that in a batch the other
// streams' work does not decide the choice.
rl_status tune_if_needed(rl_ctx *ctx, const void *f, const void *u0, int W, int H, long long pitch, int K,
                         const rl_thinning *thin) {
    ctx->tune_choice = -1;
    if (!(ctx->flags & RL_FLAG_AUTOTUNE) || K < 1) return RL_OK;
    const TuneSite site = tune_site(ctx, W, H, thin);
    if (site.key.empty()) return RL_OK;
    int choice = -1;
    if (rl::tune_get(site.key, &choice)) {
        ctx->tune_choice = choice;
        return RL_OK;
    }
    const size_t bytes = (size_t)pitch * H * elem_size(ctx->storage);
    rl_status st = grow(ctx, &ctx->tunebuf, &ctx->tunebuf_bytes, bytes, "rl_iterate: tuning buffer");
    if (st != RL_OK) return st;
    const int kt = K < 10 ? K : 10;
    float best_ms = 0.f;
    std::string times;
    // time the candidates on a quiet GPU: in a batch the other streams'
    // work would otherwise decide the choice (a one-time stall per key)
    CK(cudaDeviceSynchronize(), "rl_iterate: tuning");
    for (int c : site.candidates) {
        ctx->tune_choice = c;
        int path = 0;
        float ms = -1.f;
        st = run_device(ctx, f, u0, ctx->tunebuf, W, H, pitch, kt, thin, &path);  // warm-up
        for (int rep = 0; rep < 2 && st == RL_OK; ++rep) {  // the faster of two timed runs
            CK(cudaEventRecord(ctx->ev0, ctx->stream), "rl_iterate: tuning");
            st = run_device(ctx, f, u0, ctx->tunebuf, W, H, pitch, kt, thin, &path);
            CK(cudaEventRecord(ctx->ev1, ctx->stream), "rl_iterate: tuning");
            CK(cudaEventSynchronize(ctx->ev1), "rl_iterate: tuning");
            float t = 0.f;
            if (st == RL_OK) CK(cudaEventElapsedTime(&t, ctx->ev0, ctx->ev1), "rl_iterate: tuning");
            if (st == RL_OK && (ms < 0.f || t < ms)) ms = t;
        }
        if (st != RL_OK) {  // a candidate that cannot run here (shared memory) is skipped
            CK(cudaStreamSynchronize(ctx->stream), "rl_iterate: tuning");
            (void)cudaGetLastError();
        }
        char b[32];
        snprintf(b, sizeof b, "%s%.1f", times.empty() ? "" : " ", ms >= 0.f ? 1e3f * ms / kt : -1.f);
        times += b;
        if (ms >= 0.f && (choice < 0 || ms < best_ms)) {
            best_ms = ms;
            choice = c;
        }
    }
    if (choice < 0) return fail(ctx, RL_ERR_CUDA, "rl_iterate: no tuning candidate ran");
    rl::tune_put(site.key, choice, times);
    ctx->tune_choice = choice;
    return RL_OK;
}

}  // namespace

namespace rl {
void set_status_sink(rl_ctx *ctx, int *host_word) {
    if (ctx) ctx->status_sink = host_word;
}
}  // namespace rl

static rl_status iterate_impl(rl_ctx *ctx, const void *f, const void *u0, void *u_out, int W, int H,
                              long long pitch, int iterations, const rl_thinning *thin, rl_stats *stats) {
    if (!ctx) return RL_ERR_INVALID_ARG;
    if (!f || !u_out) return fail(ctx, RL_ERR_INVALID_ARG, "rl_iterate: f and u_out must not be NULL");
    if (W < 1 || H < 1 || pitch < W || iterations < 0)
        return fail(ctx, RL_ERR_INVALID_ARG, "rl_iterate: need W, H >= 1, pitch >= W, iterations >= 0");
    if (u_out == f) return fail(ctx, RL_ERR_INVALID_ARG, "rl_iterate: u_out must not alias f");
    if (!ctx->has_psf) return fail(ctx, RL_ERR_STATE, "rl_iterate: no PSF set");
    const int bx = ctx->kw - 1 - ctx->ax, by = ctx->kh - 1 - ctx->ay;
    if (ctx->ax >= W || bx >= W || ctx->ay >= H || by >= H)
        return fail(ctx, RL_ERR_INVALID_ARG, "rl_iterate: PSF extent must be smaller than the image");
    if (thin) {
        if (!(thin->threshold >= 0.f) || thin->reset_period < 1 ||
            (thin->update_period != 1 && thin->update_period != thin->reset_period))
            return fail(ctx, RL_ERR_INVALID_ARG,
                        "rl_iterate: thinning needs threshold >= 0, reset_period >= 1, "
                        "update_period 1 or reset_period");
    }
    const size_t es = elem_size(ctx->storage);
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    struct Restore {
        int d, p;
        ~Restore() { if (d != p) cudaSetDevice(p); }
    } restore{ctx->device, prev};
    // Default-stream contexts: the call's work goes to the internal stream,
    // after everything already queued on the caller's stream, and the
    // caller's stream waits for it on every return path.
    struct Fence {
        rl_ctx *c;
        cudaStream_t user;
        ~Fence() {
            if (!c) return;
            cudaEventRecord(c->ev_out, c->own);
            cudaStreamWaitEvent(user, c->ev_out, 0);
            c->stream = user;
        }
    } fence{nullptr, ctx->stream};
    if (ctx->own) {
        CK(cudaEventRecord(ctx->ev_in, ctx->stream), "rl_iterate: stream fence");
        CK(cudaStreamWaitEvent(ctx->own, ctx->ev_in, 0), "rl_iterate: stream fence");
        ctx->stream = ctx->own;
        fence.c = ctx;
    }

    const bool dev_f = is_device_ptr(f), dev_o = is_device_ptr(u_out);
    const bool dev_u = u0 ? is_device_ptr(u0) : true;
    const bool staged = !(dev_f && dev_o && dev_u);
    const void *df = f, *du = u0;
    void *dout = u_out;
    long long dp = pitch;
    if (staged) {
        // Any host buffer: stage every input into library-owned device
        // buffers with a packed pitch, run there, and copy the result back.
        dp = W;
        const size_t bytes = (size_t)W * H * es;
        const void *src[2] = {f, u0};
        const bool on_dev[2] = {dev_f, dev_u};
        for (int i = 0; i < 3; ++i) {
            if (i == 1 && !u0) continue;
            rl_status st = grow(ctx, &ctx->stage[i], &ctx->stage_bytes[i], bytes, "rl_iterate: staging");
            if (st != RL_OK) return st;
            if (i < 2)
                CK(cudaMemcpy2DAsync(ctx->stage[i], W * es, src[i], pitch * es, W * es, H,
                                     on_dev[i] ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                     ctx->stream),
                   "rl_iterate: upload");
        }
        df = ctx->stage[0];
        du = u0 ? ctx->stage[1] : nullptr;
        dout = ctx->stage[2];
    }
    {
        rl_status st = tune_if_needed(ctx, df, du, W, H, dp, iterations, thin);
        if (st != RL_OK) return st;
    }
    ctx->launches = 0;
    if (stats) CK(cudaEventRecord(ctx->ev0, ctx->stream), "rl_iterate: event");
    int path = 0;
    rl_status st = run_device(ctx, df, du, dout, W, H, dp, iterations, thin, &path);
    if (st != RL_OK) return st;
    if (staged) {
        CK(cudaMemcpy2DAsync(u_out, pitch * es, dout, W * es, W * es, H,
                             dev_o ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream),
           "rl_iterate: download");
    }
    if (stats) {
        CK(cudaEventRecord(ctx->ev1, ctx->stream), "rl_iterate: event");
        CK(cudaEventSynchronize(ctx->ev1), "rl_iterate: sync");
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1), "rl_iterate: timing");
        unsigned long long act = (unsigned long long)W * H * iterations;
        if (thin) CK(cudaMemcpy(&act, ctx->d_counter, sizeof act, cudaMemcpyDeviceToHost), "rl_iterate: counter");
        stats->iterations = iterations;
        stats->pixel_iterations = (long long)W * H * iterations;
        stats->active_pixel_iterations = (long long)act;
        stats->device_ms = ms;
        stats->path = path;
        stats->launches = ctx->launches;
        // FP64 flux of the input and the result (diagnostics, after the timing)
        const int nb = rl::flux_blocks();
        CK(rl::launch_flux(df, dp, W, H, ctx->storage, ctx->d_flux, ctx->d_flux + nb, ctx->stream),
           "rl_iterate: flux");
        CK(rl::launch_flux(staged ? dout : u_out, dp, W, H, ctx->storage, ctx->d_flux,
                           ctx->d_flux + nb + 1, ctx->stream),
           "rl_iterate: flux");
        double fl[2] = {0.0, 0.0};
        CK(cudaMemcpyAsync(fl, ctx->d_flux + nb, sizeof fl, cudaMemcpyDeviceToHost, ctx->stream),
           "rl_iterate: flux");
        CK(cudaStreamSynchronize(ctx->stream), "rl_iterate: flux");
        stats->flux_f = fl[0];
        stats->flux_u = fl[1];
    } else if (staged) {
        CK(cudaStreamSynchronize(ctx->stream), "rl_iterate: sync");
    }
    if ((stats || staged) && ctx->pstatus) {
        // the stream is synchronised: did a persistent launch give up waiting?
        int pst = 0;
        CK(cudaMemcpy(&pst, ctx->pstatus, sizeof pst, cudaMemcpyDeviceToHost), "rl_iterate: status");
        if (pst != 0)
            return fail(ctx, RL_ERR_TIMEOUT, "rl_iterate: the persistent disc kernel gave up waiting for a tile");
    }
    CK(cudaGetLastError(), "rl_iterate");
    ctx->err.clear();
    return RL_OK;
}

static rl_status iterate_tiles_impl(rl_ctx *ctx, const rl_job *jobs, int n) {
    if (!ctx) return RL_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && !jobs)) return fail(ctx, RL_ERR_INVALID_ARG, "rl_iterate_tiles: need n >= 0 and jobs");
    if (!ctx->has_psf) return fail(ctx, RL_ERR_STATE, "rl_iterate_tiles: no PSF set");
    if (ctx->storage != RL_STORAGE_F32)
        return fail(ctx, RL_ERR_UNSUPPORTED, "rl_iterate_tiles: FP32 storage only");
    if (needs_fold(ctx))
        return fail(ctx, RL_ERR_UNSUPPORTED, "rl_iterate_tiles: no exact-transpose band in the batched form");
    if (ctx->path_pref != RL_PATH_AUTO && ctx->path_pref != RL_PATH_SPAN)
        return fail(ctx, RL_ERR_UNSUPPORTED, "rl_iterate_tiles: runs the span path (AUTO or SPAN) only");
    int op = -1, R = 0;
    if (ctx->kind == RL_PSF_DISC && ctx->disc_radius >= 1 && ctx->disc_radius <= rl::kDiscMaxRadius) {
        op = 0;
        R = ctx->disc_radius;
    } else if (ctx->box_radius) {
        op = 1;
        R = ctx->box_radius;
    } else {
        return fail(ctx, RL_ERR_UNSUPPORTED,
                    "rl_iterate_tiles: the PSF must take the disc or box kernel (disc radius 1..16, or a "
                    "uniform centred odd square up to 33 x 33)");
    }
    for (int j = 0; j < n; ++j) {
        const rl_job &jb = jobs[j];
        if (!jb.f || !jb.u_out || jb.u_out == jb.f || jb.W < 1 || jb.H < 1 || jb.pitch < jb.W ||
            jb.iterations < 0)
            return fail(ctx, RL_ERR_INVALID_ARG,
                        "rl_iterate_tiles: each job needs f, u_out (not aliasing f), W, H >= 1, pitch >= W, "
                        "iterations >= 0");
        if (jb.thin || jb.f_host || jb.u_host)
            return fail(ctx, RL_ERR_UNSUPPORTED, "rl_iterate_tiles: no thinning or host buffers in the batched form");
        if (R >= jb.W || R >= jb.H)
            return fail(ctx, RL_ERR_INVALID_ARG, "rl_iterate_tiles: PSF extent must be smaller than the image");
        if (!is_device_ptr(jb.f) || !is_device_ptr(jb.u_out) || (jb.u0 && !is_device_ptr(jb.u0)))
            return fail(ctx, RL_ERR_INVALID_ARG, "rl_iterate_tiles: f, u0 and u_out must be device pointers");
    }
    if (n == 0) return RL_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    struct Restore {
        int d, p;
        ~Restore() { if (d != p) cudaSetDevice(p); }
    } restore{ctx->device, prev};
    // default-stream contexts run on the internal stream, fenced (as rl_iterate)
    struct Fence {
        rl_ctx *c;
        cudaStream_t user;
        ~Fence() {
            if (!c) return;
            cudaEventRecord(c->ev_out, c->own);
            cudaStreamWaitEvent(user, c->ev_out, 0);
            c->stream = user;
        }
    } fence{nullptr, ctx->stream};
    if (ctx->own) {
        CK(cudaEventRecord(ctx->ev_in, ctx->stream), "rl_iterate_tiles: stream fence");
        CK(cudaStreamWaitEvent(ctx->own, ctx->ev_in, 0), "rl_iterate_tiles: stream fence");
        ctx->stream = ctx->own;
        fence.c = ctx;
    }
    // Jobs by iteration count, descending: the jobs still iterating at
    // iteration k are a prefix, and so are their tiles in the work list.
    std::vector<int> ord(n);
    for (int j = 0; j < n; ++j) ord[j] = j;
    std::stable_sort(ord.begin(), ord.end(),
                     [&](int x, int y) { return jobs[x].iterations > jobs[y].iterations; });
    std::vector<long long> sp(n);
    size_t plane_bytes = 0;
    for (int j = 0; j < n; ++j) {
        const rl_job &jb = jobs[ord[j]];
        sp[j] = ((long long)jb.W + 63) / 64 * 64;
        plane_bytes += (size_t)sp[j] * jb.H * sizeof(float) * 2;  // u and q
    }
    std::vector<rl::TileJob> tj(n);
    std::vector<int2> items;
    std::vector<long long> prefix(n + 1, 0);
    for (int j = 0; j < n; ++j) {
        const rl_job &jb = jobs[ord[j]];
        const int tiles = ((jb.W + 63) / 64) * ((jb.H + 63) / 64);
        for (int t = 0; t < (jb.iterations > 0 ? tiles : 0); ++t) items.push_back(make_int2(j, t));
        prefix[j + 1] = (long long)items.size();
    }
    const size_t jobs_bytes = (n * sizeof(rl::TileJob) + 255) / 256 * 256;
    const size_t items_bytes = (std::max<size_t>(items.size(), 1) * sizeof(int2) + 255) / 256 * 256;
    // the persistent form's tables: half-step starts and counts, per-job first
    // item and tile columns, per-item progress, ticket and status
    const int kmax = jobs[ord[0]].iterations;
    // The persistent form only when RL_FLAG_PERSISTENT asks for it: each job's
    // tiles form a small grid whose per-tile chain of items sets the pace
    // (measured: 64 frames of 128^2..512^2 under a disc r8, about 1300
    // tiles, 46.6 Gpx-it/s persistent against 50.6 with a launch pair per
    // iteration).
    const bool persistent = !(ctx->flags & RL_FLAG_PER_ITERATION) && kmax > 0 &&
                            (ctx->flags & RL_FLAG_PERSISTENT);
    std::vector<int> tstart, tcount, tfirst(n), ttx(n);
    if (persistent) {
        int active = n, acc = 0;
        for (int k = 0; k < kmax; ++k) {
            while (active > 0 && jobs[ord[active - 1]].iterations <= k) --active;
            for (int h = 0; h < 2; ++h) {
                tstart.push_back(acc);
                tcount.push_back((int)prefix[active]);
                acc += (int)prefix[active];
            }
        }
        tstart.push_back(acc);
        for (int j = 0; j < n; ++j) {
            tfirst[j] = (int)prefix[j];
            ttx[j] = (jobs[ord[j]].W + 63) / 64;
        }
    }
    const size_t tab_ints = persistent ? tstart.size() + tcount.size() + 2 * (size_t)n + items.size() + 2 : 0;
    char *scratch = nullptr;
    SALLOC((void **)&scratch, plane_bytes + jobs_bytes + items_bytes + tab_ints * sizeof(int),
           "rl_iterate_tiles: scratch");
    struct Free {
        char *p;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } release{scratch, ctx->stream};
    char *cur = scratch + jobs_bytes + items_bytes + tab_ints * sizeof(int);
    for (int j = 0; j < n; ++j) {
        const rl_job &jb = jobs[ord[j]];
        float *work = (float *)cur;
        cur += (size_t)sp[j] * jb.H * sizeof(float);
        float *q = (float *)cur;
        cur += (size_t)sp[j] * jb.H * sizeof(float);
        IterArgs a;
        memset(&a, 0, sizeof a);
        a.f = jb.f;
        a.W = jb.W;
        a.H = jb.H;
        a.f_pitch = jb.pitch;
        a.clamp = ctx->boundary == RL_BOUNDARY_CLAMP;
        a.ax = a.bx = a.ay = a.by = R;
        a.weight = ctx->weight;
        a.m_pitch = a.mi_pitch = sp[j];
        a.u_out = work;
        a.out_pitch = sp[j];
        tj[j].a[0] = a;
        tj[j].a[0].u_in = jb.u0 ? jb.u0 : jb.f;  // first iteration reads the start image
        tj[j].a[0].in_pitch = jb.pitch;
        tj[j].a[1] = a;
        tj[j].a[1].u_in = work;  // later ones update the work plane in place
        tj[j].a[1].in_pitch = sp[j];
        tj[j].qplane = q;
        tj[j].q_pitch = sp[j];
    }
    auto *djobs = (rl::TileJob *)scratch;
    auto *ditems = (int2 *)(scratch + jobs_bytes);
    CK(cudaMemcpyAsync(djobs, tj.data(), n * sizeof(rl::TileJob), cudaMemcpyHostToDevice, ctx->stream),
       "rl_iterate_tiles: job table");
    if (!items.empty())
        CK(cudaMemcpyAsync(ditems, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, ctx->stream),
           "rl_iterate_tiles: work list");
    if (persistent) {
        // one cooperative launch: every iteration of every job
        int *tab = (int *)(scratch + jobs_bytes + items_bytes);
        std::vector<int> host;
        host.insert(host.end(), tstart.begin(), tstart.end());
        host.insert(host.end(), tcount.begin(), tcount.end());
        host.insert(host.end(), tfirst.begin(), tfirst.end());
        host.insert(host.end(), ttx.begin(), ttx.end());
        CK(cudaMemcpyAsync(tab, host.data(), host.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream),
           "rl_iterate_tiles: tables");
        int *progress = tab + host.size();
        CK(cudaMemsetAsync(progress, 0, (items.size() + 2) * sizeof(int), ctx->stream), "rl_iterate_tiles: progress");
        rl::TilesPersistArgs tp;
        memset(&tp, 0, sizeof tp);
        tp.jobs = djobs;
        tp.items = ditems;
        tp.start = tab;
        tp.count = tab + tstart.size();
        tp.first = tp.count + tcount.size();
        tp.tiles_x = tp.first + n;
        tp.n_halves = 2 * kmax;
        tp.n_items0 = (int)items.size();
        tp.progress = progress;
        tp.ticket = (unsigned *)(progress + items.size());
        tp.status = progress + items.size() + 1;
        tp.wait_ns = 2000000000ull;
        CK(rl::launch_tiles_persist(op, R, tp, ctx->stream), "rl_iterate_tiles: persistent launch");
        // the status word lives in this call's scratch: read it before release
        int pst = 0;
        CK(cudaMemcpyAsync(&pst, tp.status, sizeof pst, cudaMemcpyDeviceToHost, ctx->stream), "rl_iterate_tiles: status");
        CK(cudaStreamSynchronize(ctx->stream), "rl_iterate_tiles: status");
        if (pst != 0)
            return fail(ctx, RL_ERR_TIMEOUT, "rl_iterate_tiles: the persistent kernel gave up waiting for a tile");
    } else {
        int active = n;
        for (int k = 0; k < kmax; ++k) {
            while (active > 0 && jobs[ord[active - 1]].iterations <= k) --active;
            CK(rl::launch_tiles(op, R, djobs, ditems, (int)prefix[active], k == 0 ? 0 : 1, ctx->stream),
               "rl_iterate_tiles: kernel launch");
        }
    }
    for (int j = 0; j < n; ++j) {
        const rl_job &jb = jobs[ord[j]];
        const void *src = jb.iterations > 0 ? (const void *)tj[j].a[1].u_in : (jb.u0 ? jb.u0 : jb.f);
        const long long spitch = jb.iterations > 0 ? sp[j] : jb.pitch;
        if (src != jb.u_out)
            CK(cudaMemcpy2DAsync(jb.u_out, jb.pitch * sizeof(float), src, spitch * sizeof(float), jb.W * sizeof(float),
                                 jb.H, cudaMemcpyDeviceToDevice, ctx->stream),
               "rl_iterate_tiles: copy out");
    }
    CK(cudaGetLastError(), "rl_iterate_tiles");
    ctx->err.clear();
    return RL_OK;
}

static rl_status get_mask_impl(rl_ctx *ctx, void *dst, long long dst_pitch) {
    if (!ctx) return RL_ERR_INVALID_ARG;
    if (!dst) return fail(ctx, RL_ERR_INVALID_ARG, "rl_get_mask: dst is NULL");
    if (!ctx->last_mask) return fail(ctx, RL_ERR_STATE, "rl_get_mask: no thinned iteration has run");
    if (dst_pitch < ctx->last_W) return fail(ctx, RL_ERR_INVALID_ARG, "rl_get_mask: dst_pitch < W");
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaMemcpy2DAsync(dst, dst_pitch, ctx->last_mask, ctx->last_mp, ctx->last_W,
                                      ctx->last_H, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "rl_get_mask");
    return RL_OK;
}

// Failure detection of the persistent disc kernel without a GPU fault: a
// small launch whose ticket counter starts past the forward half of its only
// iteration, so every adjoint item waits for neighbours that never finish.
// Each wait gives up after wait_ms, the kernel records status 1 and every CTA
// returns; the context stays usable.
static rl_status selftest_wait_timeout_impl(int device, int wait_ms) {
    if (wait_ms < 1 || wait_ms > 10000) return RL_ERR_INVALID_ARG;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        (void)cudaGetLastError();
        return RL_ERR_CUDA;
    }
    const int W = 128, H = 128, tiles = (W / rl::disc_tile()) * (H / rl::disc_persist_tile_h());
    float *buf = nullptr;  // f, work u, out, q
    int *scratch = nullptr;
    cudaStream_t s = nullptr;
    rl_status st = RL_ERR_CUDA;
    cudaError_t e = cudaMalloc(&buf, 4 * sizeof(float) * W * H);
    if (e == cudaSuccess) e = cudaMalloc(&scratch, (tiles + 2) * sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, 4 * sizeof(float) * W * H, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, (tiles + 2) * sizeof(int), s);
    const unsigned first = (unsigned)tiles;  // the forward half of iteration 0 is never handed out
    if (e == cudaSuccess) e = cudaMemcpyAsync(scratch + tiles, &first, sizeof first, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        rl::PersistArgs p;
        memset(&p, 0, sizeof p);
        IterArgs a;
        memset(&a, 0, sizeof a);
        a.f = buf;
        a.u_in = buf;
        a.u_out = buf + 2 * W * H;
        a.W = W;
        a.H = H;
        a.f_pitch = a.in_pitch = a.out_pitch = W;
        a.ax = a.bx = a.ay = a.by = 2;
        a.weight = 1.f / 13.f;
        for (int i = 0; i < 4; ++i) p.a[i] = a;
        p.qplane = buf + 3 * W * H;
        p.q_pitch = W;
        p.K = 1;
        p.tiles_x = W / rl::disc_tile();
        p.tiles_y = H / rl::disc_persist_tile_h();
        p.progress = scratch;
        p.ticket = (unsigned *)(scratch + tiles);
        p.status = scratch + tiles + 1;
        p.wait_ns = (unsigned long long)wait_ms * 1000000ull;
        e = rl::launch_disc_persist(p, rl::ST_F32, 2, s);
    }
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, scratch + tiles + 1, sizeof status, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) st = status == 1 ? RL_ERR_TIMEOUT : RL_ERR_STATE;
    (void)cudaGetLastError();
    if (s) cudaStreamDestroy(s);
    cudaFree(buf);
    cudaFree(scratch);
    cudaSetDevice(prev);
    return st;
}

// ---- C ABI entry points ------------------------------------------------------
extern "C" {

rl_status rl_create(const rl_config *cfg, rl_ctx **out) {
    return abi_guard(nullptr, [&] { return create_impl(cfg, out); });
}

rl_status rl_destroy(rl_ctx *ctx) { return abi_guard(nullptr, [&] { return destroy_impl(ctx); }); }

rl_status rl_set_psf(rl_ctx *ctx, const rl_psf_desc *d) {
    return abi_guard(ctx, [&] { return set_psf_impl(ctx, d); });
}

rl_status rl_iterate(rl_ctx *ctx, const void *f, const void *u0, void *u_out, int W, int H, long long pitch,
                     int iterations, const rl_thinning *thin, rl_stats *stats) {
    return abi_guard(ctx, [&] { return iterate_impl(ctx, f, u0, u_out, W, H, pitch, iterations, thin, stats); });
}

rl_status rl_iterate_tiles(rl_ctx *ctx, const rl_job *jobs, int n) {
    return abi_guard(ctx, [&] { return iterate_tiles_impl(ctx, jobs, n); });
}

rl_status rl_get_mask(rl_ctx *ctx, void *dst, long long dst_pitch) {
    return abi_guard(ctx, [&] { return get_mask_impl(ctx, dst, dst_pitch); });
}

rl_status rl_selftest_wait_timeout(int device, int wait_ms) {
    return abi_guard(nullptr, [&] { return selftest_wait_timeout_impl(device, wait_ms); });
}

void rl_test_fail_allocation(int nth) { g_fail_alloc.store(nth > 0 ? nth : 0); }

void rl_test_persist_ctas(int n) { g_test_persist_ctas.store(n > 0 ? n : 0); }

void rl_test_persist_wait_ns(unsigned long long ns) { g_test_wait_ns.store(ns); }

}  // extern "C"
