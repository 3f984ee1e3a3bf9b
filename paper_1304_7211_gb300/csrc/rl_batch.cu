// rl_batch.cu -- batched execution of independent deconvolutions on several
// CUDA streams (declared in include/rl.h).  Each slot is a non-blocking
// stream with its own context (PSF, scratch); the scheduler places a job on
// the slot with the least queued pixel-iterations, so small images from
// different jobs share the GPU while each job's own iterations stay in order.
#include <cuda_runtime.h>

#include <deque>
#include <new>
#include <string>
#include <vector>

#include "../../include/rl.h"

namespace {

struct Pending {
    long long ticket;
    cudaEvent_t done;
    long long work;  // pixel-iterations
};

struct Slot {
    cudaStream_t stream = nullptr;
    rl_ctx *ctx = nullptr;
    std::deque<Pending> queue;  // submitted, possibly unfinished
    long long queued_work = 0;
};

}  // namespace

struct rl_batch {
    int device = 0;
    int storage = RL_STORAGE_F32;
    std::vector<Slot> slots;
    std::vector<cudaEvent_t> free_events;
    long long next_ticket = 1;
    std::string err;
};

namespace {

rl_status bfail(rl_batch *b, rl_status st, const std::string &m) {
    b->err = m;
    return st;
}

// Retire finished jobs at the front of each slot's queue.
void reap(rl_batch *b) {
    for (auto &s : b->slots) {
        while (!s.queue.empty() && cudaEventQuery(s.queue.front().done) == cudaSuccess) {
            s.queued_work -= s.queue.front().work;
            b->free_events.push_back(s.queue.front().done);
            s.queue.pop_front();
        }
        (void)cudaGetLastError();
    }
}

Pending *find(rl_batch *b, long long ticket) {
    for (auto &s : b->slots)
        for (auto &p : s.queue)
            if (p.ticket == ticket) return &p;
    return nullptr;
}

struct DeviceGuard {
    int prev = 0;
    explicit DeviceGuard(int d) {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard() { cudaSetDevice(prev); }
};

}  // namespace

extern "C" {

rl_status rl_batch_create(const rl_config *cfg, int slots, rl_batch **out) {
    if (!out || slots < 1 || slots > 256) return RL_ERR_INVALID_ARG;
    *out = nullptr;
    rl_config c = {0, nullptr, RL_STORAGE_F32, RL_BOUNDARY_MIRROR, RL_PATH_AUTO, 0};
    if (cfg) c = *cfg;
    rl_batch *b = new (std::nothrow) rl_batch;
    if (!b) return RL_ERR_OOM;
    b->device = c.device;
    b->storage = c.storage;
    DeviceGuard g(c.device);
    b->slots.resize(slots);
    for (auto &s : b->slots) {
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess) {
            (void)cudaGetLastError();
            rl_batch_destroy(b);
            return RL_ERR_CUDA;
        }
        rl_config sc = c;
        sc.stream = s.stream;
        rl_status st = rl_create(&sc, &s.ctx);
        if (st != RL_OK) {
            rl_batch_destroy(b);
            return st;
        }
    }
    *out = b;
    return RL_OK;
}

rl_status rl_batch_submit(rl_batch *b, const rl_job *job, long long *ticket) {
    if (!b) return RL_ERR_INVALID_ARG;
    if (!job || !ticket) return bfail(b, RL_ERR_INVALID_ARG, "rl_batch_submit: job and ticket are required");
    if (!job->f || !job->u_out || job->W < 1 || job->H < 1 || job->pitch < job->W || job->iterations < 0)
        return bfail(b, RL_ERR_INVALID_ARG, "rl_batch_submit: bad job geometry or buffers");
    DeviceGuard g(b->device);
    reap(b);
    Slot *best = &b->slots[0];
    for (auto &s : b->slots)
        if (s.queued_work < best->queued_work) best = &s;
    Slot &s = *best;
    rl_status st = rl_set_psf(s.ctx, &job->psf);
    if (st != RL_OK) return bfail(b, st, rl_last_error(s.ctx));
    const size_t esz = b->storage == RL_STORAGE_F32 ? 4 : 2;
    if (job->f_host) {
        cudaError_t e = cudaMemcpy2DAsync((void *)job->f, job->pitch * esz, job->f_host, job->W * esz,
                                          job->W * esz, job->H, cudaMemcpyHostToDevice, s.stream);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return bfail(b, RL_ERR_CUDA, std::string("rl_batch_submit: upload: ") + cudaGetErrorString(e));
        }
    }
    st = rl_iterate(s.ctx, job->f, job->u0, job->u_out, job->W, job->H, job->pitch, job->iterations,
                    job->thin, nullptr);
    if (st != RL_OK) return bfail(b, st, rl_last_error(s.ctx));
    if (job->u_host) {
        cudaError_t e = cudaMemcpy2DAsync(job->u_host, job->W * esz, job->u_out, job->pitch * esz,
                                          job->W * esz, job->H, cudaMemcpyDeviceToHost, s.stream);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return bfail(b, RL_ERR_CUDA, std::string("rl_batch_submit: download: ") + cudaGetErrorString(e));
        }
    }
    cudaEvent_t ev;
    if (!b->free_events.empty()) {
        ev = b->free_events.back();
        b->free_events.pop_back();
    } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        (void)cudaGetLastError();
        return bfail(b, RL_ERR_CUDA, "rl_batch_submit: event");
    }
    cudaEventRecord(ev, s.stream);
    const long long work = (long long)job->W * job->H * (job->iterations > 0 ? job->iterations : 1);
    s.queue.push_back({b->next_ticket, ev, work});
    s.queued_work += work;
    *ticket = b->next_ticket++;
    return RL_OK;
}

rl_status rl_batch_query(rl_batch *b, long long ticket, int *done) {
    if (!b || !done) return RL_ERR_INVALID_ARG;
    DeviceGuard g(b->device);
    Pending *p = find(b, ticket);
    if (!p) {
        // not queued any more: finished and reaped, or never issued
        *done = ticket > 0 && ticket < b->next_ticket;
        return *done ? RL_OK : bfail(b, RL_ERR_INVALID_ARG, "rl_batch_query: unknown ticket");
    }
    const cudaError_t e = cudaEventQuery(p->done);
    if (e != cudaSuccess && e != cudaErrorNotReady) {
        (void)cudaGetLastError();
        return bfail(b, RL_ERR_CUDA, std::string("rl_batch_query: ") + cudaGetErrorString(e));
    }
    (void)cudaGetLastError();
    *done = e == cudaSuccess;
    return RL_OK;
}

rl_status rl_batch_wait(rl_batch *b, long long ticket) {
    if (!b) return RL_ERR_INVALID_ARG;
    DeviceGuard g(b->device);
    Pending *p = find(b, ticket);
    if (!p) return ticket > 0 && ticket < b->next_ticket ? RL_OK
                                                         : bfail(b, RL_ERR_INVALID_ARG, "rl_batch_wait: unknown ticket");
    const cudaError_t e = cudaEventSynchronize(p->done);
    if (e != cudaSuccess) return bfail(b, RL_ERR_CUDA, std::string("rl_batch_wait: ") + cudaGetErrorString(e));
    reap(b);
    return RL_OK;
}

rl_status rl_batch_sync(rl_batch *b) {
    if (!b) return RL_ERR_INVALID_ARG;
    DeviceGuard g(b->device);
    for (auto &s : b->slots) {
        const cudaError_t e = cudaStreamSynchronize(s.stream);
        if (e != cudaSuccess) return bfail(b, RL_ERR_CUDA, std::string("rl_batch_sync: ") + cudaGetErrorString(e));
    }
    reap(b);
    return RL_OK;
}

rl_status rl_batch_destroy(rl_batch *b) {
    if (!b) return RL_OK;
    {
        DeviceGuard g(b->device);
        for (auto &s : b->slots) {
            if (s.stream) cudaStreamSynchronize(s.stream);
            rl_destroy(s.ctx);
            for (auto &p : s.queue) cudaEventDestroy(p.done);
            if (s.stream) cudaStreamDestroy(s.stream);
        }
        for (auto ev : b->free_events) cudaEventDestroy(ev);
    }
    delete b;
    return RL_OK;
}

const char *rl_batch_last_error(const rl_batch *b) { return b ? b->err.c_str() : ""; }

}  // extern "C"
