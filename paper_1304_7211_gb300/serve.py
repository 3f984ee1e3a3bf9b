"""Continuous-batching request loop over the C batch executor.

Requests (observed image on the host, PSF, iteration count, optional
thinning) arrive on a timeline.  The loop admits waiting requests in arrival
order while the bytes resident on the device stay under an HBM budget,
allocates each admitted request's device buffers (f and u stay resident
until it finishes), and submits it to an ``rl_batch``: the upload, all RL
iterations and the download run on one of the batch's streams, interleaved on
the GPU with every other request in flight.  Finished requests are retired
by polling (no blocking wait), their memory is released and later arrivals
are admitted.  Latency is measured from arrival to result-on-host.
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
    f: np.ndarray            # observed image, host (float32 or the storage dtype)
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

    def close(self):
        self.batch.close()

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
                f_dev = torch.empty((H, W), dtype=self.dtype, device=dev)
                u_dev = torch.empty((H, W), dtype=self.dtype, device=dev)
                f_host = torch.from_numpy(np.ascontiguousarray(r.f)).to(self.dtype).pin_memory()
                u_host = torch.empty((H, W), dtype=self.dtype).pin_memory()
                th = rl.thinning(*r.thin) if r.thin else None
                r.t_admit = time.perf_counter() - t0
                ticket = self.batch.submit(r.spec, f_dev, u_dev, r.iterations, W, H,
                                           f_host=f_host, u_host=u_host, thin=th)
                inflight[ticket] = (r, (f_dev, u_dev, f_host), u_host, need)
                resident += need
                peak = max(peak, resident)
                i += 1
            # retire finished requests
            for ticket in [t for t in inflight if self.batch.query(t)]:
                r, bufs, u_host, need = inflight.pop(ticket)
                r.t_done = time.perf_counter() - t0
                r.result = u_host.float().numpy()
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
        px_it = float(sum(r.f.size * r.iterations for r in done))
        return ServeReport(len(done), wall, float(np.percentile(lat, 50)),
                           float(np.percentile(lat, 99)), float(lat.mean()), px_it,
                           px_it / wall / 1e6, peak)


def sequential(requests: list[Request], device: int = 0, storage: str = "f32",
               boundary: str = "mirror") -> float:
    """Plain one-at-a-time solves of the same requests (the baseline the
    served throughput is compared with); returns the wall time in seconds."""
    import torch
    dtype = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[storage]
    t0 = time.perf_counter()
    for r in requests:
        with rl.Deconvolver(r.spec, device=device, storage=storage, boundary=boundary) as d:
            f = torch.from_numpy(np.ascontiguousarray(r.f)).to(dtype).cuda(device)
            th = rl.thinning(*r.thin) if r.thin else None
            u = d.run(f, r.iterations, thin=th)
            r.result = u.float().cpu().numpy()
    torch.cuda.synchronize()
    return time.perf_counter() - t0
