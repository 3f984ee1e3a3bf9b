/*
 * rl.h -- C ABI of the GB300 (sm_103a) Richardson-Lucy deconvolution library.
 *
 * The library runs the hot path of non-blind Richardson-Lucy (RL)
 * deconvolution as described by Welk & Erler, "Algorithmic Optimisations for
 * Iterative Deconvolution Methods":
 *
 *   Sec. 1, Eq. 2   given the observed image f and the PSF h, find u with
 *                   f ~ u (x) h;
 *   Sec. 2, Eq. 3   u^{k+1} = ( h* (x) ( f / (u^k (x) h) ) ) . u^k,  u^0 = f,
 *                   h* = h reflected about the origin; the iteration count
 *                   is the only parameter of the method;
 *   Sec. 2          missing pixels outside the image are continued from the
 *                   image (clamp = closest pixel, or half-sample mirror);
 *   Sec. 3          fast convolutions for special PSFs: a running-sum box
 *                   filter for linear motion blur, the "generic box filter"
 *                   (per-row spans) for uniform convex PSFs such as the
 *                   defocus disc, and direct summation / the list filter for
 *                   general PSFs;
 *   Sec. 4, Eq. 4-5 selective convolution ("thinning"): pixels whose change
 *                   falls below a threshold become inactive, keep their last
 *                   re-blurred value v and stop changing; every P (= 10)
 *                   iterations all pixels are active again.
 *
 * Conventions for every entry point:
 *   - Return an rl_status; no call aborts the process and no C++ exception
 *     crosses this boundary.  On failure rl_last_error(ctx) describes it.
 *   - Images are single-channel, row-major (x fastest), with a row pitch
 *     given in ELEMENTS.  The element type is the context's storage type
 *     (float, bfloat16 or float16); arithmetic is FP32 in every mode.
 *   - A context is used by one host thread at a time.  It owns all scratch
 *     device memory it needs; scratch is allocated on first use, grows when a
 *     larger image arrives, and is freed by rl_destroy.
 *   - Work is issued on the context's CUDA stream (rl_config.stream; NULL =
 *     the legacy default stream).  Calls return when the work is queued,
 *     except where stated.  For a context on the legacy or per-thread default
 *     stream, rl_iterate runs its kernels on an internal non-blocking stream
 *     (so that its iteration loop can be replayed as a CUDA graph), ordered
 *     after the work already queued on the default stream, and the default
 *     stream waits for it: the ordering seen by the caller is unchanged.
 */
#ifndef RL_GB300_H
#define RL_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rl_ctx rl_ctx; /* opaque; created by rl_create */

typedef enum {
    RL_OK = 0,
    RL_ERR_INVALID_ARG = 1, /* null pointer, bad size, bad PSF, ...         */
    RL_ERR_UNSUPPORTED = 2, /* valid request this build cannot run          */
    RL_ERR_OOM = 3,         /* device or host allocation failed             */
    RL_ERR_CUDA = 4,        /* a CUDA call failed (message has the reason)  */
    RL_ERR_TIMEOUT = 5,     /* a bounded device wait gave up                */
    RL_ERR_STATE = 6        /* call out of order (e.g. no PSF set yet)      */
} rl_status;

typedef enum {
    RL_PSF_MOTION = 0, /* uniform linear motion blur, Sec. 3 Fig. 1a          */
    RL_PSF_DISC = 1,   /* uniform disc (defocus), Sec. 3 "Defocus blur"      */
    RL_PSF_DENSE = 2   /* arbitrary non-negative taps, Sec. 3 "Sparse blur"  */
} rl_psf_kind;

typedef enum { RL_STORAGE_F32 = 0, RL_STORAGE_BF16 = 1, RL_STORAGE_F16 = 2 } rl_storage;

typedef enum {
    RL_BOUNDARY_MIRROR = 0, /* half-sample symmetric: ... c b a | a b c ...   */
    RL_BOUNDARY_CLAMP = 1   /* closest image pixel (the paper's choice, Sec. 2) */
} rl_boundary;

typedef enum {
    RL_PATH_AUTO = 0,    /* motion -> RUNSUM, disc -> SPAN; dense -> STENCIL,
                            except -> SPAN: a uniform centred odd square up to
                            33 x 33 (box, Sec. 3 rectangular blur), another
                            uniform rectangle reaching 3..16 pixels from the
                            anchor, and other uniform taps reaching more than
                            4 pixels                                            */
    RL_PATH_RUNSUM = 1,  /* sliding-window box filter along x or y (motion only)  */
    RL_PATH_SPAN = 2,    /* per-row span sums of a uniform PSF (motion, disc,
                            or dense taps that are uniform with one contiguous
                            run per row); separable sliding sums for a uniform
                            rectangle reaching up to 16 pixels from the anchor  */
    RL_PATH_STENCIL = 3, /* direct summation over the non-zero taps (any PSF)     */
    RL_PATH_SAT = 4      /* uniform rectangles reaching up to 16 pixels from the
                            anchor only: the summed-area table (2D cumulated
                            sums, Sec. 3), four lookups per output in 64-bit
                            fixed point; no thinning.  AUTO never picks it:
                            the separable sums of SPAN are faster            */
} rl_path;

/*
 * PSF descriptor (Sec. 3, Fig. 1).
 *   RL_PSF_MOTION: `length` >= 1 pixels along `axis` (0 = x, 1 = y); taps
 *       1/length at offsets [-(length/2), length-1-length/2].
 *   RL_PSF_DISC:   `radius` >= 0; support dx^2 + dy^2 <= radius^2 (pixel-
 *       centre inclusion), weight 1/|support|.
 *   RL_PSF_DENSE:  `kw` x `kh` host array `taps` (row-major, taps[j*kw+i] at
 *       offset (i - anchor_x, j - anchor_y)); anchor_x/anchor_y < 0 select the
 *       centre (kw/2, kh/2).  Taps must be finite and >= 0 with a positive
 *       sum; they are copied and normalised to unit sum.
 * Offsets follow convolution: (u (x) h)(p) = sum_t h(t) u(p - t).
 */
typedef struct {
    int kind;                /* rl_psf_kind                     */
    int axis;                /* MOTION: 0 = x, 1 = y            */
    int length;              /* MOTION                          */
    int radius;              /* DISC                            */
    int kw, kh;              /* DENSE                           */
    int anchor_x, anchor_y;  /* DENSE; < 0 = centre             */
    const float *taps;       /* DENSE; host memory, kw*kh items */
} rl_psf_desc;

/*
 * Selective convolution (Sec. 4, Eq. 4-5).  Pass NULL to rl_iterate for
 * plain RL.  Iteration k (counting from 0 in each rl_iterate call) is "full"
 * when k % reset_period == 0: every pixel is used.  Otherwise only active
 * pixels are re-blurred and updated; inactive pixels keep the ratio f/v of
 * their last active iteration and do not change.  The change of a used pixel
 * is |c - 1| (relative = 1, c = the correction factor, 0 where u = 0) or
 * |u' - u| (relative = 0).  A pixel whose change is < threshold becomes
 * inactive: after every iteration when update_period == 1 (Sec. 4), or only
 * after full iterations when update_period == reset_period (the mask is then
 * fixed for the rest of the epoch).
 */
typedef struct {
    float threshold;   /* >= 0; 0 reproduces plain RL (Table 2, first row) */
    int relative;      /* 1: |c - 1|, 0: |u' - u| (absolute, Sec. 4)         */
    int reset_period;  /* P >= 1, the paper uses 10                        */
    int update_period; /* 1 or reset_period                                */
    /* Optional replay of a recorded schedule: iterations x H x W bytes (row
     * pitch W, host or device memory), byte = 1 when the pixel is used in
     * that iteration.  When non-NULL the threshold rule is not evaluated;
     * used pixels are re-blurred and updated and inactive ones keep the
     * ratio of their last used iteration, exactly as above.  NULL = decide
     * by the threshold. */
    const unsigned char *schedule;
} rl_thinning;

/* rl_config.flags */
#define RL_FLAG_PER_ITERATION 1 /* one launch per iteration (per half on
                                   the disc path) even where the running-
                                   sum path could keep whole rows resident
                                   for all iterations, or the disc path run
                                   them all in one persistent launch      */
#define RL_FLAG_AUTOTUNE 8      /* choose the disc path's launch form (not
                                   with RL_FLAG_PERSISTENT), the
                                   running-sum chunk width and the stencil
                                   tile shape by timing the candidates on the
                                   first call for a (site, PSF, size,
                                   storage, boundary, thinning, SM count)
                                   key -- that call blocks while it tunes --
                                   and caching the fastest for the process
                                   (and, with RL_TUNE_CACHE naming a file,
                                   across processes as JSON lines); the
                                   choice depends on the request alone    */
#define RL_FLAG_PERSISTENT 4    /* disc path: one persistent launch for all
                                   iterations even where the image has too
                                   few tiles for it to pay (under about 6
                                   per SM), plain or thinned; tests and
                                   tuning                                 */
/* The adjoint convolution of Eq. 3.  Default: h* (x) q with the same
 * boundary continuation as the forward one -- h reflected about the origin
 * (Sec. 2), the "pad-flip" operator B.  With this flag: the exact matrix
 * transpose A^T of the forward operator A (u -> h (x) u with the boundary
 * continuation), i.e. the zero-padded correlation of q folded back onto the
 * pixels the boundary map sends each padded position to.  The two are the
 * same operator for a PSF symmetric in each axis under the mirror boundary
 * (those keep their fast paths); otherwise (clamp, off-centre or asymmetric
 * taps) A^T makes RL conserve flux exactly and the solve runs on the
 * generic stencil path. */
#define RL_FLAG_ADJOINT_TRANSPOSE 2

typedef struct {
    int device;     /* CUDA device ordinal                                   */
    void *stream;   /* cudaStream_t to issue work on; NULL = default stream */
    int storage;    /* rl_storage of f, u0, u_out (and internal u buffers)  */
    int boundary;   /* rl_boundary                                          */
    int path;       /* rl_path                                              */
    int flags;      /* RL_FLAG_* bits, 0 = defaults                         */
} rl_config;

typedef struct {
    long long iterations;             /* iterations run                        */
    long long pixel_iterations;       /* W * H * iterations                    */
    long long active_pixel_iterations;/* pixel-iterations actually re-blurred  */
    double device_ms;                 /* stream time of the call (CUDA events) */
    int path;                         /* rl_path that ran                      */
    int launches;                     /* kernel launches the call issued       */
    double flux_f;                    /* sum of f in FP64 (diagnostics)        */
    double flux_u;                    /* sum of u_out in FP64; equals flux_f for
                                         unthinned RL under the mirror boundary
                                         with an axis-symmetric PSF           */
} rl_stats;

/*
 * Create a context on cfg->device.  cfg may be NULL (device 0, default
 * stream, FP32, mirror boundary, AUTO path).  On success *out owns the
 * context; release it with rl_destroy.  Errors: RL_ERR_INVALID_ARG for a null
 * `out` or an unknown enum value, RL_ERR_UNSUPPORTED when the device is not a
 * compute capability 10.3 GPU, RL_ERR_CUDA/RL_ERR_OOM when setup fails.
 */
rl_status rl_create(const rl_config *cfg, rl_ctx **out);

/*
 * Set the PSF h of Eq. 3 (descriptor semantics above).  Copies and
 * normalises the taps, derives the per-row span table (Sec. 3, generic box
 * filter) and uploads both to the device.  Errors: RL_ERR_INVALID_ARG for a
 * bad descriptor (negative or non-finite taps, zero sum, length < 1,
 * radius < 0, null taps, kw/kh < 1, anchor outside the array, more than
 * 65536 taps); RL_ERR_UNSUPPORTED when the context's forced path cannot
 * represent the PSF (RUNSUM needs a motion PSF; SPAN needs a uniform PSF with
 * one contiguous run per row).
 */
rl_status rl_set_psf(rl_ctx *ctx, const rl_psf_desc *psf);

/*
 * Run `iterations` RL iterations (Eq. 3) of the current PSF on a W x H image.
 *   f      observed image (read only).
 *   u0     starting image; NULL means u0 = f (the paper's choice).
 *   u_out  receives u^iterations; may alias u0 but not f.
 *   pitch  row pitch in elements for f, u0 and u_out (>= W).
 *   thin   NULL for plain RL, else selective convolution (see rl_thinning).
 *   stats  NULL, or receives counters; a non-NULL stats makes the call wait
 *          for the stream (active counts and timing are read back).
 * Pointers may be device memory or host memory (pageable or pinned); host
 * buffers are staged through library-owned device buffers with copies on the
 * context stream, and the call then returns only after u_out is written.
 * Device pointers must be on the context's device and aligned to the element
 * size.  The boundary continuation is the context's.  The PSF's extent on
 * each side must be smaller than the image along that axis.
 * Errors: RL_ERR_INVALID_ARG (null f/u_out, W or H < 1, pitch < W,
 * iterations < 0, u_out == f, PSF larger than the image, bad thinning
 * parameters), RL_ERR_STATE (no PSF set), RL_ERR_OOM, RL_ERR_CUDA.
 */
rl_status rl_iterate(rl_ctx *ctx, const void *f, const void *u0, void *u_out,
                     int W, int H, long long pitch, int iterations,
                     const rl_thinning *thin, rl_stats *stats);

/*
 * Diagnostics for selective convolution (Sec. 4): copy the active-pixel mask
 * left by the last thinned rl_iterate on this context into dst, W x H bytes
 * with a row pitch of dst_pitch bytes (host or device memory).  A byte is 1
 * when the pixel would be re-blurred in the next (non-full) iteration.  Waits
 * for the context stream.  Errors: RL_ERR_INVALID_ARG (null dst, pitch < W),
 * RL_ERR_STATE (no thinned iteration has run on this context), RL_ERR_CUDA.
 */
rl_status rl_get_mask(rl_ctx *ctx, void *dst, long long dst_pitch);

/* Release the context and all device memory it owns.  NULL is a no-op. */
rl_status rl_destroy(rl_ctx *ctx);

/* Message of the last failure on ctx ("" if none).  With ctx == NULL, the
 * message of the last failed rl_create on this thread.  The pointer stays
 * valid until the next call on the same context. */
const char *rl_last_error(const rl_ctx *ctx);

/*
 * Batched execution of many independent deconvolutions (the batched and
 * served workloads): a batch owns `slots` CUDA streams, each with its own
 * context and scratch.  rl_batch_submit copies the job into a host queue and
 * returns at once; queued jobs are issued in submission order, each to the
 * slot with the least queued work (pixel-iterations), while that slot has
 * fewer than two jobs on the GPU.  Every batch call issues what fits.  Jobs on
 * different slots overlap on the GPU, jobs on one slot run in order.  Each
 * job's result depends only on its own inputs (no cross-job state), so a job
 * gives the same image alone and in any mix, and a job that fails (bad PSF,
 * out of memory) fails alone: the others run on.
 *
 *   f, u0 (NULL = f), u_out: device pointers, caller-owned, valid until the
 *       job is done; u_out may alias u0 but not f.
 *   f_host (nullable): pinned or pageable host image uploaded into f on the
 *       job's stream before it runs.  u_host (nullable): u_out is copied there
 *       after it runs.  Both use row pitch W elements.
 *   psf: copied at submit.  thin: nullable, copied at submit (a schedule
 *       pointer inside must stay valid until the job is done).
 * Errors: as rl_set_psf / rl_iterate, returned by rl_batch_submit when the
 * job is issued inside that call, else by rl_batch_query / rl_batch_wait of
 * its ticket; RL_ERR_TIMEOUT there when the job's persistent launch gave up
 * a bounded wait (its image is then incomplete; the other jobs are not
 * affected); RL_ERR_INVALID_ARG for a bad ticket.  No C++ exception crosses
 * the ABI: host allocation failures come back as RL_ERR_OOM.
 */
typedef struct {
    const void *f;
    const void *u0;
    void *u_out;
    const void *f_host;
    void *u_host;
    int W, H;
    long long pitch;
    int iterations;
    rl_psf_desc psf;
    const rl_thinning *thin;
} rl_job;

typedef struct rl_batch rl_batch;

/* Create a batch of `slots` >= 1 streams on cfg->device (cfg->stream is
 * ignored: the batch creates its own non-blocking streams).  Unless
 * cfg->flags has RL_FLAG_PER_ITERATION, plain disc solves run as one
 * persistent launch each, which shares the GPU between streams better than
 * two launches per iteration; thinned ones take the form the image size
 * picks (a small thinned solve in one launch would hold its SMs for the
 * whole solve). */
rl_status rl_batch_create(const rl_config *cfg, int slots, rl_batch **out);
/* Queue a job; *ticket identifies it for rl_batch_query / rl_batch_wait. */
rl_status rl_batch_submit(rl_batch *b, const rl_job *job, long long *ticket);
/* *done = 1 when the job's work (and its download) has finished, or when it
 * was cancelled or failed (then its status is returned). */
rl_status rl_batch_query(rl_batch *b, long long ticket, int *done);
/* Block until the job has finished. */
rl_status rl_batch_wait(rl_batch *b, long long ticket);
/* Block until every submitted job has finished. */
rl_status rl_batch_sync(rl_batch *b);
/* Cancel a job.  Not yet issued: it is dropped and never runs (*was_running
 * = 0).  Already on the GPU: it cannot be stopped; it runs to the end, may
 * still write u_out / u_host, and its result is to be discarded (*was_running
 * = 1).  Either way its ticket then reports done with RL_OK.  RL_ERR_STATE if
 * the job has already finished, failed or been cancelled; RL_ERR_INVALID_ARG
 * for an unknown ticket.  was_running may be NULL. */
rl_status rl_batch_cancel(rl_batch *b, long long ticket, int *was_running);
/* Drop the jobs not yet issued, wait for the issued ones, then release
 * streams, contexts and scratch.  NULL-safe. */
rl_status rl_batch_destroy(rl_batch *b);
/* Message of the last failure on b. */
const char *rl_batch_last_error(const rl_batch *b);

/*
 * Batched (request, tile) form of the disc and box kernels (Eq. 3 per job;
 * Sec. 3 defocus disc and rectangular box blur): n jobs that share ctx's PSF
 * run over the 64 x 64 tiles of every job still iterating, so many small
 * images fill the GPU that one image alone would leave mostly idle: one
 * forward and one adjoint launch per iteration, or, with RL_FLAG_PERSISTENT
 * on ctx, every iteration of every job in one persistent cooperative launch
 * in which each tile waits only for the tiles around it in its own job.  A job leaves the work list when its own iteration count ends;
 * each job's result is, bit for bit, the image that rl_iterate on ctx gives
 * for it alone.
 *   ctx: its PSF must take the disc or box kernel (RL_PSF_DISC of radius
 *       1..16, or dense taps forming a uniform centred odd square up to
 *       33 x 33); path AUTO or SPAN; FP32 storage; no exact-transpose band
 *       (clamp with RL_FLAG_ADJOINT_TRANSPOSE).
 *   jobs[j]: f, u0 (NULL = f), u_out device pointers, caller-owned, valid
 *       until the work is done; u_out may alias u0 but not f; W, H, pitch
 *       (elements), iterations.  psf is ignored (ctx's PSF applies); thin,
 *       f_host and u_host must be NULL.
 * Enqueued on ctx's stream (as rl_iterate); the persistent form then waits
 * for the stream, to read the kernel's status word before its scratch is
 * released.  The library's scratch, one u and one q plane per job, is
 * allocated and released in stream order.
 * Errors: RL_ERR_INVALID_ARG, RL_ERR_STATE (no PSF), RL_ERR_UNSUPPORTED (PSF,
 * storage, band, thinning or host buffers), RL_ERR_TIMEOUT (a bounded wait of
 * the persistent form gave up), RL_ERR_CUDA, RL_ERR_OOM.
 */
rl_status rl_iterate_tiles(rl_ctx *ctx, const rl_job *jobs, int n);

/* Library version string, e.g. "rl-gb300 0.1 sm_103a". */
const char *rl_version(void);

/*
 * Self-test of failure detection in the persistent disc kernel (the one
 * launch that runs every iteration of a plain disc solve; its work items wait
 * for neighbouring tiles with bounded waits).  Runs a 128 x 128 launch on
 * `device` whose first half is never handed out, so every later item waits
 * for tiles that never finish; each wait gives up after wait_ms (1..10000)
 * and the kernel records it and returns without faulting.  Returns
 * RL_ERR_TIMEOUT when the give-up was detected and reported (the expected
 * outcome), RL_ERR_STATE if the kernel finished without reporting it,
 * RL_ERR_CUDA or RL_ERR_INVALID_ARG otherwise.  Allocates and frees its own
 * small buffers; no context is needed.  No counterpart in the paper.
 */
rl_status rl_selftest_wait_timeout(int device, int wait_ms);

/*
 * Fault injection for tests (host side, no GPU fault): with nth > 0 the
 * nth scratch allocation that rl_iterate, rl_iterate_tiles or a batch job
 * makes from now on, in any context of the process, fails as if the device
 * were out of memory -- the call returns RL_ERR_OOM with a message and the
 * context stays usable.  0 disables.  No counterpart in the paper.
 */
void rl_test_fail_allocation(int nth);

/*
 * Launch shape for tests: with n > 0, every persistent disc launch of the
 * process (plain or thinned, RL_FLAG_PERSISTENT or chosen by size) runs n
 * CTAs per SM (at most its occupancy, at most one per tile) instead of the
 * rule's about two tiles per CTA; results are bit-identical for every n.
 * 0 restores the rule.  Host side only; no counterpart in the paper.
 */
void rl_test_persist_ctas(int n);

/*
 * Failure detection for tests (no GPU fault): with ns > 0, every persistent
 * disc launch of the process gives up a wait for a neighbouring tile after
 * ns nanoseconds instead of 2 s -- with a few ns and about one tile per
 * CTA (rl_test_persist_ctas), where each half starts while the previous
 * one still finishes, a launch over many tiles almost surely gives up.  The launch then records it and returns; the solve
 * reports RL_ERR_TIMEOUT (rl_iterate on its next synchronising call, a
 * batch job through rl_batch_query / rl_batch_wait) and its image is
 * incomplete.  0 restores the bound.  No counterpart in the paper.
 */
void rl_test_persist_wait_ns(unsigned long long ns);

/*
 * Allocation-free variant of the running-sum path.  The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc -- code
 * running inside an allocator or memory-pool hook, latency-critical threads
 * where an allocation may block on the device, processes whose device memory
 * is partitioned in advance.
 *
 * Runs `iterations` RL iterations of the running-sum path for horizontal
 * linear motion blur of `length` pixels (RL_PSF_MOTION, axis 0), FP32,
 * `boundary` as in
 * rl_boundary, on `stream` (cudaStream_t; NULL = default stream) of the
 * CURRENT device.  f, u0 (NULL = f) and u_out are caller-owned device
 * pointers of the current device (or managed memory) with row pitch `pitch`
 * elements; anything else -- a host buffer, another device's memory -- is
 * rejected with RL_ERR_INVALID_ARG before any launch, since staging it would
 * allocate.  u_out must alias neither f nor u0.
 * No context is needed and the call allocates nothing: its only scratch (the
 * second buffer of the iteration ping-pong) is a fixed array of
 * RL_NOALLOC_MAX_PIXELS floats (16 MiB) in the library image, which every GPU
 * that loads the library holds until the process exits.  W * H above that
 * limit is rejected with RL_ERR_INVALID_ARG.
 *
 * The first call on each device looks up the array's device address (once,
 * with that device current); make that first call before any stream capture.
 * The cached address does not survive a cudaDeviceReset of that device.
 * All calls on a device share the array and it keeps the last call's
 * contents; nothing in it needs clearing (every pixel is written before it is
 * read), but calls whose work overlaps on the GPU race on it.  Returns when
 * the work is queued.  On failure a message is written to err (err_len bytes,
 * may be NULL).  Errors: RL_ERR_INVALID_ARG, RL_ERR_UNSUPPORTED (rows too
 * long for the running-sum kernel), RL_ERR_CUDA.
 */
#define RL_NOALLOC_MAX_PIXELS 4194304
rl_status rl_motion_x_noalloc(const float *f, const float *u0, float *u_out, int W, int H,
                              long long pitch, int length, int boundary, int iterations,
                              void *stream, char *err, int err_len);

#ifdef __cplusplus
}
#endif
#endif /* RL_GB300_H */
