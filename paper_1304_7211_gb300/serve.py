"""Continuous-batching request loop over the C batch executor.

Requests (observed image on the host or already on the device, PSF,
iteration count, optional thinning) arrive on a timeline.  The loop admits
waiting requests in arrival order while the bytes resident on the device stay
under an HBM budget, allocates each admitted request's device buffers (f and
u stay resident until it finishes), and submits it to an ``rl_batch``: the
upload, all RL iterations and the download into a pooled pinned host buffer
run on one of the batch's streams, interleaved on the GPU with every other
request in flight.  Finished requests are retired by polling (no blocking
wait), their memory is released and later arrivals are admitted.  Latency
is measured from arrival to result-on-host.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import rl


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    f: object                # observed image: host array, or a CUDA tensor of the storage dtype
    spec: object             # PSF spec (kind/axis/length/radius/taps/kw/kh)
    iterations: int
    thin: tuple | None = None  # (threshold, relative, reset_period, update_period)
    result: np.ndarray | None = None
    t_admit: float = 0.0
    t_done: float = 0.0

    @property
    def latency_ms(self) -> float:
        return 1e3 * (self.t_done - self.arrival_s)


@dataclasses.dataclass
class ServeReport:
    n: int
    wall_s: float
    p50_ms: float
    p99_ms: float
    mean_ms: float
    px_it: float
    mpx_it_per_s: float
    peak_resident_bytes: int

    def as_dict(self) -> dict:
        return dataclasses.asdict(self)


class Server:
    """Admission by HBM budget + continuous batching on ``slots`` streams."""

    def __init__(self, device: int = 0, slots: int = 8, hbm_budget_bytes: float = 150e9,
                 storage: str = "f32", boundary: str = "mirror"):
        import torch
        self.torch = torch
        self.device = device
        self.storage = storage
        self.dtype = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[storage]
        self.esize = 4 if storage == "f32" else 2
        self.budget = hbm_budget_bytes
        self.batch = rl.Batch(slots, device=device, storage=storage, boundary=boundary)
        self._pinned = {}  # size class -> free pinned host buffers (result downloads)

    def close(self):
        self.batch.close()

    def _pinned_buffer(self, shape):
        """A pinned host buffer of at least H x W elements from a pool of
        power-of-two size classes (page-locking memory per request would
        cost more than the download it serves)."""
        n = shape[0] * shape[1]
        cls = 1 << max(16, (n - 1).bit_length())
        free = self._pinned.setdefault(cls, [])
        buf = free.pop() if free else self.torch.empty(cls, dtype=self.dtype).pin_memory()
        return buf, buf[:n].view(shape)

    def _release_pinned(self, buf):
        self._pinned[buf.numel()].append(buf)

    def _bytes(self, r: Request) -> int:
        # f and u on the device plus the stale-ratio/mask planes of thinning
        n = r.f.shape[0] * r.f.shape[1]
        return n * (2 * self.esize + (9 if r.thin else 0))

    def run(self, requests: list[Request], realtime: bool = True) -> ServeReport:
        """Serve ``requests`` (sorted by arrival).  With ``realtime`` the loop
        waits for each arrival time; otherwise every request is available at
        once (arrival = start)."""
        torch = self.torch
        dev = torch.device("cuda", self.device)
        waiting = list(requests)
        waiting.sort(key=lambda r: r.arrival_s)
        inflight = {}   # ticket -> (request, buffers, host result, bytes)
        resident = 0
        peak = 0
        t0 = time.perf_counter()
        if not realtime:
            for r in waiting:
                r.arrival_s = 0.0
        i = 0
        done = []
        while i < len(waiting) or inflight:
            now = time.perf_counter() - t0
            # admit arrived requests in order while the budget allows
            while i < len(waiting) and waiting[i].arrival_s <= now:
                r = waiting[i]
                need = self._bytes(r)
                if inflight and resident + need > self.budget:
                    break
                H, W = r.f.shape
                on_dev = hasattr(r.f, "is_cuda") and r.f.is_cuda
                if on_dev:  # in the server's storage type (a converted copy if it differs)
                    f_dev, f_host = (r.f if r.f.dtype == self.dtype else r.f.to(self.dtype)), None
                else:
                    f_dev = torch.empty((H, W), dtype=self.dtype, device=dev)
                    f_host = torch.from_numpy(np.ascontiguousarray(r.f)).to(self.dtype).pin_memory()
                u_dev = torch.empty((H, W), dtype=self.dtype, device=dev)
                u_buf, u_host = self._pinned_buffer((H, W))
                th = rl.thinning(*r.thin) if r.thin else None
                r.t_admit = time.perf_counter() - t0
                ticket = self.batch.submit(r.spec, f_dev, u_dev, r.iterations, W, H,
                                           f_host=f_host, u_host=u_host, thin=th)
                inflight[ticket] = (r, (f_dev, u_dev, f_host), (u_buf, u_host), need)
                resident += need
                peak = max(peak, resident)
                i += 1
            # retire finished requests
            for ticket in [t for t in inflight if self.batch.query(t)]:
                r, bufs, (u_buf, u_host), need = inflight.pop(ticket)
                r.t_done = time.perf_counter() - t0
                r.result = u_host.to(torch.float32, copy=True).numpy()
                self._release_pinned(u_buf)
                resident -= need
                done.append(r)
                del bufs
            if i < len(waiting) and not inflight:
                # idle: sleep until the next arrival
                time.sleep(max(0.0, min(0.001, waiting[i].arrival_s - now)))
            elif inflight:
                time.sleep(0.0002)
        wall = time.perf_counter() - t0
        lat = np.array([r.latency_ms for r in done])
        px_it = float(sum(r.f.shape[0] * r.f.shape[1] * r.iterations for r in done))
        return ServeReport(len(done), wall, float(np.percentile(lat, 50)),
                           float(np.percentile(lat, 99)), float(lat.mean()), px_it,
                           px_it / wall / 1e6, peak)


def sequential(requests: list[Request], device: int = 0, storage: str = "f32",
               boundary: str = "mirror") -> float:
    """Plain one-at-a-time solves of the same requests (the baseline the
    served throughput is compared with); returns the wall time in seconds."""
    return sum(service_times(requests, device, storage, boundary))


def service_times(requests: list[Request], device: int = 0, storage: str = "f32",
                  boundary: str = "mirror") -> list[float]:
    """Each request solved alone, one after another, with nothing else on
    the GPU: seconds from its start to its result on the host (upload if the
    image is on the host, the solve, the download)."""
    import torch
    dtype = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[storage]
    out = []
    for r in requests:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with rl.Deconvolver(r.spec, device=device, storage=storage, boundary=boundary) as d:
            on_dev = hasattr(r.f, "is_cuda") and r.f.is_cuda
            f = (r.f.to(dtype) if on_dev else
                 torch.from_numpy(np.ascontiguousarray(r.f)).to(dtype).cuda(device))
            th = rl.thinning(*r.thin) if r.thin else None
            u = d.run(f, r.iterations, thin=th)
            r.result = u.float().cpu().numpy()
        out.append(time.perf_counter() - t0)
    return out


def fifo_report(requests: list[Request], service_s: list[float]) -> ServeReport:
    """The plain path as a server: one request at a time in arrival order,
    each taking its measured alone-time (service_s), on the same arrival
    trace -- request i starts at max(arrival_i, end of request i - 1)."""
    end = 0.0
    lat = []
    t_first = min(r.arrival_s for r in requests)
    for r, s in sorted(zip(requests, service_s), key=lambda p: p[0].arrival_s):
        end = max(end, r.arrival_s) + s
        lat.append(1e3 * (end - r.arrival_s))
    lat = np.array(lat)
    px_it = float(sum(r.f.shape[0] * r.f.shape[1] * r.iterations for r in requests))
    wall = end - min(0.0, t_first)
    return ServeReport(len(requests), wall, float(np.percentile(lat, 50)), float(np.percentile(lat, 99)),
                       float(lat.mean()), px_it, px_it / wall / 1e6, 0)
