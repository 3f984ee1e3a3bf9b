// rl_noalloc.cu -- a Richardson-Lucy entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a custom
// allocator or memory-pool hook (re-entering the allocator would deadlock or
// recurse), real-time or latency-critical threads where an allocation can
// block on a device-wide synchronisation, and processes whose device memory is
// carved up in advance so that a late allocation may fail.  For them
// rl_motion_x_noalloc runs the running-sum RL iteration for horizontal motion
// blur (the same kernel as rl_iterate's RUNSUM path) with its only scratch --
// the second image buffer of the ping-pong -- in a fixed-size array that is
// part of the library image.  Every GPU that loads the library holds that
// array (RL_NOALLOC_MAX_PIXELS floats, 16 MiB) until the process exits.
//
// The array is shared by every call on a device and keeps the contents of the
// last call; nothing in it has to start at zero because every pixel is written
// before it is read.  Calls whose work overlaps on the GPU (different
// streams, or different host threads on one device) race on it.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/rl.h"
#include "rl_launch.h"

static __device__ __align__(256) float g_rl_noalloc_scratch[RL_NOALLOC_MAX_PIXELS];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
float *g_scratch_addr[kMaxDevices];  // device address of the array, per device

void set_err(char *err, int err_len, const char *msg) {
    if (err && err_len > 0) snprintf(err, (size_t)err_len, "%s", msg);
}

// Device (or managed) memory of device `dev`.  The entry point cannot stage a
// host buffer the way rl_iterate does (that would allocate), so anything else
// is rejected before a kernel could dereference it.
bool on_device(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

static rl_status noalloc_impl(const float *f, const float *u0, float *u_out, int W, int H, long long pitch,
                              int length, int boundary, int iterations, void *stream, char *err, int err_len) {
    set_err(err, err_len, "");
    if (!f || !u_out || u_out == f || (u0 && u_out == u0)) {
        set_err(err, err_len, "rl_motion_x_noalloc: f and u_out are required; u_out must not alias f or u0");
        return RL_ERR_INVALID_ARG;
    }
    if (W < 1 || H < 1 || pitch < W || iterations < 0 || length < 1 ||
        (boundary != RL_BOUNDARY_MIRROR && boundary != RL_BOUNDARY_CLAMP)) {
        set_err(err, err_len, "rl_motion_x_noalloc: need W, H, length >= 1, pitch >= W, "
                              "iterations >= 0 and a known boundary");
        return RL_ERR_INVALID_ARG;
    }
    const int ax = length / 2, bx = length - 1 - ax;
    if (ax >= W || bx >= W) {
        set_err(err, err_len, "rl_motion_x_noalloc: half the motion length must be smaller than W");
        return RL_ERR_INVALID_ARG;
    }
    if ((long long)W * H > RL_NOALLOC_MAX_PIXELS) {
        char buf[160];
        snprintf(buf, sizeof buf, "rl_motion_x_noalloc: %d x %d = %lld pixels exceeds the fixed "
                 "scratch of %d pixels", W, H, (long long)W * H, RL_NOALLOC_MAX_PIXELS);
        set_err(err, err_len, buf);
        return RL_ERR_INVALID_ARG;
    }
    if (!rl::motion_x_fits(W, length)) {
        set_err(err, err_len, "rl_motion_x_noalloc: rows too long for the running-sum kernel");
        return RL_ERR_UNSUPPORTED;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_err(err, err_len, "rl_motion_x_noalloc: no current CUDA device");
        return RL_ERR_CUDA;
    }
    if (!on_device(f, dev) || !on_device(u_out, dev) || (u0 && !on_device(u0, dev))) {
        set_err(err, err_len, "rl_motion_x_noalloc: f, u0 and u_out must be device memory of the "
                              "current device (host buffers cannot be staged without allocating)");
        return RL_ERR_INVALID_ARG;
    }
    float *scratch = nullptr;
    {
        // One-time set-up per device, with that device current: the host-side
        // name of the array is not a device address, so ask the runtime.  The
        // cached address belongs to the device's primary context and does not
        // survive a cudaDeviceReset.
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_rl_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                (void)cudaGetLastError();
                set_err(err, err_len, "rl_motion_x_noalloc: cudaGetSymbolAddress failed");
                return RL_ERR_CUDA;
            }
            g_scratch_addr[dev] = (float *)p;
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const float *start = u0 ? u0 : f;
    if (iterations == 0) {
        e = cudaMemcpy2DAsync(u_out, pitch * sizeof(float), start, pitch * sizeof(float),
                              W * sizeof(float), H, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) {
            set_err(err, err_len, cudaGetErrorString(e));
            return RL_ERR_CUDA;
        }
        return RL_OK;
    }
    rl::IterArgs a = {};
    a.f = f;
    a.W = W;
    a.H = H;
    a.f_pitch = pitch;
    a.clamp = boundary == RL_BOUNDARY_CLAMP;
    a.ax = ax;
    a.bx = bx;
    a.weight = (float)(1.0 / (double)length);
    // Iterations alternate between the scratch array (pitch W) and u_out so
    // that the last one lands in u_out.
    const void *in = start;
    long long in_pitch = pitch;
    for (int k = 0; k < iterations; ++k) {
        const bool to_out = ((iterations - 1 - k) & 1) == 0;
        a.u_in = in;
        a.in_pitch = in_pitch;
        a.u_out = to_out ? (void *)u_out : (void *)scratch;
        a.out_pitch = to_out ? pitch : W;
        e = rl::launch_motion_x(a, rl::ST_F32, false, s);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            set_err(err, err_len, cudaGetErrorString(e));
            return RL_ERR_CUDA;
        }
        in = a.u_out;
        in_pitch = a.out_pitch;
    }
    return RL_OK;
}

// No C++ exception crosses the C ABI (the set-up lock is the only thing here
// that could throw).
extern "C" rl_status rl_motion_x_noalloc(const float *f, const float *u0, float *u_out, int W,
                                         int H, long long pitch, int length, int boundary,
                                         int iterations, void *stream, char *err, int err_len) {
    try {
        return noalloc_impl(f, u0, u_out, W, H, pitch, length, boundary, iterations, stream, err, err_len);
    } catch (...) {
        set_err(err, err_len, "rl_motion_x_noalloc: internal error");
        return RL_ERR_STATE;
    }
}
