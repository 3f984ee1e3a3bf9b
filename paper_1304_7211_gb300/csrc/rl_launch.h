// rl_launch.h -- host-side launch entry points of the RL kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <string>

#include "rl_common.cuh"

struct rl_ctx;  // include/rl.h

namespace rl {

enum Storage { ST_F32 = 0, ST_BF16 = 1, ST_F16 = 2 };
enum TileMode { TILE_SPAN = 0, TILE_STENCIL = 1 };

// Running-sum box filter along x (Sec. 3 "Linear motion blur"): one fused RL
// iteration, whole rows resident in shared memory.
cudaError_t launch_motion_x(const IterArgs &a, int storage, bool thin, cudaStream_t s);
size_t motion_x_smem_bytes(int W, int L);
bool motion_x_fits(int W, int L);

// Running-sum box filter along x with the rows resident in shared memory for
// all tb.K iterations (one launch per rl_iterate call).
cudaError_t launch_motion_x_tb(const IterArgs &a, const TBArgs &tb, int storage, bool thin,
                               cudaStream_t s);
// chunk: 0 = the built-in width for the row length, else 13, 17 or 33
size_t motion_x_tb_smem_bytes(int W, int L, bool thin, int chunk = 0);
bool motion_x_tb_fits(int W, int L, bool thin, int chunk = 0);
// per storage type and thinning mode (k_motion_tb_*.cu)
cudaError_t launch_motion_tb_f32(const IterArgs &a, const TBArgs &tb, cudaStream_t s);
cudaError_t launch_motion_tb_f32_thin(const IterArgs &a, const TBArgs &tb, cudaStream_t s);
cudaError_t launch_motion_tb_bf16(const IterArgs &a, const TBArgs &tb, cudaStream_t s);
cudaError_t launch_motion_tb_bf16_thin(const IterArgs &a, const TBArgs &tb, cudaStream_t s);
cudaError_t launch_motion_tb_f16(const IterArgs &a, const TBArgs &tb, cudaStream_t s);
cudaError_t launch_motion_tb_f16_thin(const IterArgs &a, const TBArgs &tb, cudaStream_t s);

// FP64 sum of a W x H plane (pitch in elements) of the given storage into
// *out (device); `partial` holds flux_blocks() doubles.
int flux_blocks();
cudaError_t launch_flux(const void *p, long long pitch, int W, int H, int storage, double *partial,
                        double *out, cudaStream_t s);

// Transpose n_planes planes of W x H elements of `elem_bytes` (4, 2 or 1)
// from src (pitch sp elements) to dst (H x W, pitch dp elements).
cudaError_t launch_transpose(const void *src, long long sp, long long s_plane, void *dst,
                             long long dp, long long d_plane, int W, int H, int n_planes,
                             int elem_bytes, cudaStream_t s);

// Running-sum box filter along y: column strips streamed through shared
// memory, one fused RL iteration.
cudaError_t launch_motion_y(const IterArgs &a, int storage, bool thin, cudaStream_t s);

// 2D tile kernel: per-row span sums of a uniform PSF (Sec. 3 "generic box
// filter") or direct summation over dense taps (naive / list filter).
struct TileShape { int tx, ty; };
TileShape tile_shape_for(int ax, int bx, int ay, int by);
cudaError_t launch_tile(const IterArgs &a, int storage, bool thin, int mode, TileShape ts,
                        cudaStream_t s);
cudaError_t launch_tile_f32(const IterArgs &a, bool thin, int mode, TileShape ts, cudaStream_t s);
cudaError_t launch_tile_bf16(const IterArgs &a, bool thin, int mode, TileShape ts, cudaStream_t s);
cudaError_t launch_tile_f16(const IterArgs &a, bool thin, int mode, TileShape ts, cudaStream_t s);

// Register-blocked disc kernels (k_disc.cuh, one translation unit per
// radius): the defocus disc of radius 1..16 with compile-time runs.  One RL
// iteration = two launches sharing the library-owned FP32 q plane.
constexpr int kDiscMaxRadius = 16;
constexpr int disc_tile() { return 64; }  // output tile edge of the two-half kernels
// The persistent disc kernel's tiles are 64 x this (64: the two-half
// kernels' tile).  A 64 x 32 tile (64 threads) doubles the work items but
// measured slower at every size (halo staging and prefix passes per output
// grow by a fifth).
constexpr int disc_persist_tile_h() { return 64; }
// Resident CTAs per SM the two-half kernels are compiled for (register cap of
// their launch bounds; the staged tile fits as many): seven up to R = 8, six
// up to 12, five beyond, five with selective convolution or R = 1.
constexpr int disc_min_blocks(int R, bool thin) { return R > 12 ? 5 : R > 8 ? 6 : thin || R == 1 ? 5 : 7; }
cudaError_t launch_disc(const IterArgs &a, int storage, bool thin, int radius, float *qplane,
                        long long q_pitch, cudaStream_t s);
#define RL_DECLARE_DISC_R(R)                                                                 \
    cudaError_t launch_disc_r##R(const IterArgs &a, int storage, bool thin, float *qplane,   \
                                 long long q_pitch, cudaStream_t s);
RL_DECLARE_DISC_R(1) RL_DECLARE_DISC_R(2) RL_DECLARE_DISC_R(3) RL_DECLARE_DISC_R(4)
RL_DECLARE_DISC_R(5) RL_DECLARE_DISC_R(6) RL_DECLARE_DISC_R(7) RL_DECLARE_DISC_R(8)
RL_DECLARE_DISC_R(9) RL_DECLARE_DISC_R(10) RL_DECLARE_DISC_R(11) RL_DECLARE_DISC_R(12)
RL_DECLARE_DISC_R(13) RL_DECLARE_DISC_R(14) RL_DECLARE_DISC_R(15) RL_DECLARE_DISC_R(16)
#undef RL_DECLARE_DISC_R

// Batched (request, tile) form of the disc and box halves: one job's
// arguments for its first iteration (a[0]) and the later ones (a[1]), with
// its q plane.  A launch pair runs one iteration of every listed item
// (int2: job, tile index in row-major tile order).  FP32 storage, no
// thinning, no transpose band.
struct TileJob {
    IterArgs a[2];
    float *qplane;
    long long q_pitch;
};
// op 0 = disc, 1 = box; radius 1..16
cudaError_t launch_tiles(int op, int radius, const TileJob *jobs, const int2 *items, int n_items, int phase,
                         cudaStream_t s);

// Persistent form of the batched (request, tile) launches: every iteration
// of every job in one cooperative launch.  The items of half-step hk (hk = 2k:
// forward of iteration k, 2k + 1: adjoint) are the first count[hk] entries of
// `items` (jobs sorted by iteration count, descending); half-step hk's
// tickets start at start[hk] (start[2 kmax] = total).  An item waits for the
// tiles around it in its own job (`first[j]`: index of job j's first item,
// `tiles_x[j]` its tile columns) to finish half-step hk - 1.  progress (one
// per item of half-step 0), ticket and status are zeroed before the launch.
struct TilesPersistArgs {
    const TileJob *jobs;
    const int2 *items;
    const int *start;          // 2 kmax + 1 ticket offsets
    const int *count;          // items per half-step
    const int *first;          // per job: index of its first item
    const int *tiles_x;        // per job: tile columns
    int n_halves;              // 2 kmax
    int n_items0;              // items of half-step 0
    int *progress;
    unsigned *ticket;
    int *status;
    unsigned long long wait_ns;
};
cudaError_t launch_tiles_persist(int op, int radius, const TilesPersistArgs &p, cudaStream_t s);
#define RL_DECLARE_TILES_R(R)                                                                 \
    cudaError_t launch_disc_tiles_r##R(const TileJob *, const int2 *, int, int, cudaStream_t); \
    cudaError_t launch_box_tiles_r##R(const TileJob *, const int2 *, int, int, cudaStream_t);  \
    cudaError_t launch_disc_tiles_persist_r##R(const TilesPersistArgs &, cudaStream_t);        \
    cudaError_t launch_box_tiles_persist_r##R(const TilesPersistArgs &, cudaStream_t);
RL_DECLARE_TILES_R(1) RL_DECLARE_TILES_R(2) RL_DECLARE_TILES_R(3) RL_DECLARE_TILES_R(4)
RL_DECLARE_TILES_R(5) RL_DECLARE_TILES_R(6) RL_DECLARE_TILES_R(7) RL_DECLARE_TILES_R(8)
RL_DECLARE_TILES_R(9) RL_DECLARE_TILES_R(10) RL_DECLARE_TILES_R(11) RL_DECLARE_TILES_R(12)
RL_DECLARE_TILES_R(13) RL_DECLARE_TILES_R(14) RL_DECLARE_TILES_R(15) RL_DECLARE_TILES_R(16)
#undef RL_DECLARE_TILES_R

// Persistent form of the disc halves: all K iterations of one image in one
// cooperative launch.  Work items (iteration k, half, tile) are handed out in
// that order by a ticket counter; an item starts once the 3 x 3 tiles around
// its tile have finished the previous half (per-tile progress counters,
// release / acquire at GPU scope), so no grid-wide barrier separates the
// halves and one tile's staging overlaps other tiles' sums.  a[] holds the
// arguments of the four kinds of iteration, index (k > 0) + 2 (k == K - 1):
// the first reads the start image, the last writes the caller's buffer, the
// others work in place on a library u plane.  progress, ticket and status
// are zeroed before the launch; a wait longer than wait_ns sets status to 1
// and every CTA returns.  Selective convolution (thin_p > 0) on the default
// tile with its tile flags and an in-place mask; no replayed schedules, no
// transpose band.
struct PersistArgs {
    IterArgs a[4];
    float *qplane;
    long long q_pitch;
    int K;
    int tiles_x, tiles_y;
    int *progress;             // per tile: halves completed
    unsigned *ticket;          // next work item
    int *status;               // 0, or 1 when a wait gave up
    unsigned long long wait_ns;
    int thin_p, thin_q;        // selective convolution: reset and mask-update periods (0 = none)
    int ctas_per_sm;           // grid cap per SM (0 or above the occupancy: the occupancy)
};
// rl_config.flags bit that a batch sets on its slot contexts, beside
// RL_FLAG_PERSISTENT: the persistent form is forced on plain disc solves
// only; thinned ones keep the size rule.  Not part of the public flags.
constexpr int kFlagBatchSlot = 1 << 24;
// Every later persistent launch of ctx copies its status word (0, or 1 when
// a wait gave up) into *host_word (pinned host memory) on the context's
// stream after the launch; NULL stops it.  Lets a batch report the outcome
// of each job without a synchronising call.
void set_status_sink(rl_ctx *ctx, int *host_word);

// CTAs per SM for a persistent solve over `tiles` tiles: about two work items
// per CTA and half, round(tiles / (2 sms)), at least 1.  Fewer items per CTA
// run the halves in lock step (every CTA waits at once); more leave SMs idle
// (measured on GB300, disc r 4..16, 1024^2..4096^2: 2048^2, 1024 tiles, is
// fastest with 3 CTAs per SM, 4096^2 with every resident one).
inline int disc_persist_ctas(long long tiles, int sms) {
    const long long c = (tiles + sms) / (2LL * sms);
    return c < 1 ? 1 : (c > 64 ? 64 : (int)c);
}
// Launch with a grid of p.ctas_per_sm (else every co-resident) CTAs per SM,
// at most one per tile; returns cudaErrorNotSupported when the radius has no
// persistent kernel.
cudaError_t launch_disc_persist(const PersistArgs &p, int storage, int radius, cudaStream_t s);
#define RL_DECLARE_PERSIST_R(R) \
    cudaError_t launch_disc_persist_r##R(const PersistArgs &p, int storage, cudaStream_t s);
RL_DECLARE_PERSIST_R(1) RL_DECLARE_PERSIST_R(2) RL_DECLARE_PERSIST_R(3) RL_DECLARE_PERSIST_R(4)
RL_DECLARE_PERSIST_R(5) RL_DECLARE_PERSIST_R(6) RL_DECLARE_PERSIST_R(7) RL_DECLARE_PERSIST_R(8)
RL_DECLARE_PERSIST_R(9) RL_DECLARE_PERSIST_R(10) RL_DECLARE_PERSIST_R(11) RL_DECLARE_PERSIST_R(12)
RL_DECLARE_PERSIST_R(13) RL_DECLARE_PERSIST_R(14) RL_DECLARE_PERSIST_R(15) RL_DECLARE_PERSIST_R(16)
#undef RL_DECLARE_PERSIST_R

// Register-blocked uniform square box (2R + 1)^2, R = 1..16 (k_box_*.cu): the
// disc's run sums with every run at half-width R.
cudaError_t launch_box(const IterArgs &a, int storage, bool thin, int radius, float *qplane, long long q_pitch,
                       cudaStream_t s);
#define RL_DECLARE_BOX_R(R)                                                                  \
    cudaError_t launch_box_r##R(const IterArgs &a, int storage, bool thin, float *qplane,    \
                                long long q_pitch, cudaStream_t s);
RL_DECLARE_BOX_R(1) RL_DECLARE_BOX_R(2) RL_DECLARE_BOX_R(3) RL_DECLARE_BOX_R(4)
RL_DECLARE_BOX_R(5) RL_DECLARE_BOX_R(6) RL_DECLARE_BOX_R(7) RL_DECLARE_BOX_R(8)
RL_DECLARE_BOX_R(9) RL_DECLARE_BOX_R(10) RL_DECLARE_BOX_R(11) RL_DECLARE_BOX_R(12)
RL_DECLARE_BOX_R(13) RL_DECLARE_BOX_R(14) RL_DECLARE_BOX_R(15) RL_DECLARE_BOX_R(16)
#undef RL_DECLARE_BOX_R

// Register-blocked uniform rectangle [lox, hix] x [loy, hiy] (tap offsets
// about the anchor, each within the halo R in {4, 8, 16}; k_rect.cu):
// separable sliding sums through a shared-memory plane of vertical sums.
constexpr int kRectMaxReach = 16;
int rect_halo(int reach);  // the halo class for a reach, 0 if none
cudaError_t launch_rect(const IterArgs &a, int lox, int hix, int loy, int hiy, int storage, bool thin,
                        float *qplane, long long q_pitch, cudaStream_t s);
cudaError_t launch_rect_r4(const IterArgs &, int, int, int, int, int, bool, float *, long long, cudaStream_t);
cudaError_t launch_rect_r8(const IterArgs &, int, int, int, int, int, bool, float *, long long, cudaStream_t);
cudaError_t launch_rect_r16(const IterArgs &, int, int, int, int, int, bool, float *, long long, cudaStream_t);

// Uniform rectangle by a summed-area table in 64-bit fixed point (k_sat.cu):
// the same tap offsets and halo classes as launch_rect; no thinning.
cudaError_t launch_sat(const IterArgs &a, int lox, int hix, int loy, int hiy, int storage, float *qplane,
                       long long q_pitch, cudaStream_t s);
cudaError_t launch_sat_r4(const IterArgs &, int, int, int, int, int, float *, long long, cudaStream_t);
cudaError_t launch_sat_r8(const IterArgs &, int, int, int, int, int, float *, long long, cudaStream_t);
cudaError_t launch_sat_r16(const IterArgs &, int, int, int, int, int, float *, long long, cudaStream_t);

// Exact-transpose band between the two halves (a.fold_ct set): A^T q on the
// pixels within (fold_rx, fold_ry) of the border, from the full q plane.
cudaError_t launch_fold_band(const IterArgs &a, const float *qplane, long long q_pitch, cudaStream_t s);

// Register-blocked dense stencil (same two-launch structure as the disc):
// centred K x K taps, K in {3, 5, 7, 9}; `taps` is a host array of K*K.
cudaError_t launch_stencil(const IterArgs &a, const float *taps, int K, int storage, bool thin,
                           float *qplane, long long q_pitch, cudaStream_t s);
cudaError_t launch_stencil_k3(const IterArgs &, const float *, int, bool, float *, long long, cudaStream_t);
cudaError_t launch_stencil_k5(const IterArgs &, const float *, int, bool, float *, long long, cudaStream_t);
cudaError_t launch_stencil_k7(const IterArgs &, const float *, int, bool, float *, long long, cudaStream_t);
cudaError_t launch_stencil_k9(const IterArgs &, const float *, int, bool, float *, long long, cudaStream_t);

// Autotuner choice cache (rl_tune.cu): keyed by the request alone; backed by
// the file named in RL_TUNE_CACHE (JSON lines) when that is set.
bool tune_get(const std::string &key, int *choice);
void tune_put(const std::string &key, int choice, const std::string &timings_us);
void tune_clear();
}  // namespace rl
