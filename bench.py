"""Benchmark: Richardson-Lucy deconvolution throughput on one GB300.

Workload (one "step"): the 2048 x 2048 FP32 synthetic image deconvolved with
each of the three PSFs of the plain-RL workload -- horizontal motion length
31, vertical motion length 31, and a disc of radius 8 -- for 200 iterations
each (Poisson noise at peak 1000, mirror boundaries, u0 = f, no thinning),
every solve on its production path (running sum, running sum, span).
Metric: Mpixel-iterations per second (3 x 2048^2 x 200 pixel-iterations per
step).

``value`` times the device path with inputs already resident in HBM; ``e2e``
times the same call through the C ABI with pinned HOST buffers, so the library
stages f and u in and out inside the timed region.  Under torchrun every rank
runs its own replica (the solves are independent; no collective on the data
path) and ``value`` sums all ranks' work over the slowest rank's time.

``--impl reference`` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload and prints the same JSON line.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mpixel-iter/s per GB300 vs plain path at <=1e-4 rel err; serve p50/p99 ms"
UNIT = "Mpixel-iter/s"
SIZE = 2048
ITERS = 200
WORKLOAD = "plain RL 2048x2048 fp32, PSFs motion-x 31 / motion-y 31 / disc r8, 200 it each"
L2_FLUSH_BYTES = 512 << 20
CPU_ITERS = 3          # oracle iterations per PSF in the CPU baseline sample
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_plain_2048.json")


def source_sha() -> str:
    """Hash of every CUDA source and the ABI header: a DRAM-traffic capture
    counts only for the library built from the sources it was taken on."""
    h = hashlib.sha256()
    files = sorted(glob.glob(os.path.join(ROOT, "paper_1304_7211_gb300", "csrc", "*")))
    for path in files + [os.path.join(ROOT, "include", "rl.h")]:
        h.update(os.path.basename(path).encode())
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


_T0 = time.perf_counter()


def progress(stage: str) -> None:
    """One line per finished stage on stderr (the JSON line goes to stdout)."""
    print(f"bench: {stage} done at {time.perf_counter() - _T0:.1f} s", file=sys.stderr, flush=True)


def kernel_key(name: str) -> str:
    """Short kernel name from ncu's demangled one: template arguments kept,
    namespaces and the parameter list dropped."""
    name = name.replace("(anonymous namespace)::", "").split("(")[0].replace("void ", "").strip()
    # ncu prints the anonymous namespace as "<unnamed>::" or "unnamed>::"
    return re.sub(r"(<?unnamed>|\(anonymous namespace\)|\b\w+)::", "", name)


def ingest_ncu(csv_path: str, out_path: str, workload: str, command: str) -> dict:
    """Per-kernel launches, DRAM bytes and device time per launch from an ncu
    CSV (``--csv --page raw``: one row per launch, a row of units under the
    header) of gpu__time_duration.sum and dram__bytes_{read,write}.sum,
    tagged with the hash of the current sources."""
    import csv
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9,
             "nsecond": 1e-9, "ns": 1e-9, "usecond": 1e-6, "us": 1e-6, "msecond": 1e-3, "ms": 1e-3,
             "second": 1.0, "s": 1.0}
    with open(csv_path) as fh:
        rows = list(csv.reader(ln for ln in fh if ln.startswith('"')))
    hdr, units = rows[0], rows[1]
    col = {n: i for i, n in enumerate(hdr)}
    name_col = col.get("Kernel Name", col.get("Function Name"))
    kernels = {}
    for r in rows[2:]:
        def val(metric):
            i = col.get(metric)
            if i is None or not r[i]:
                return 0.0
            return float(r[i].replace(",", "")) * scale.get(units[i], 1.0)
        k = kernel_key(r[name_col])
        e = kernels.setdefault(k, {"launches": 0, "dram_bytes": 0.0, "seconds": 0.0})
        e["launches"] += 1
        e["dram_bytes"] += val("dram__bytes_read.sum") + val("dram__bytes_write.sum")
        e["seconds"] += val("gpu__time_duration.sum")
    out = {"build_sha": source_sha(), "workload": workload, "command": command,
           "kernels": {k: {"launches": e["launches"],
                           "dram_bytes_per_launch": e["dram_bytes"] / e["launches"],
                           "us_per_launch": 1e6 * e["seconds"] / e["launches"]}
                       for k, e in sorted(kernels.items())}}
    with open(out_path, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    return out


def measured_traffic():
    """The DRAM-traffic capture of the current sources (profiles/), or None when the
    sources changed since it was taken."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    d = json.load(open(TRAFFIC_FILE))
    return d if d.get("build_sha") == source_sha() else None


def traffic_of(cap, pred):
    """Summed DRAM bytes per launch of the captured kernels matching pred."""
    if cap is None:
        return None
    ks = [v for k, v in cap["kernels"].items() if pred(k)]
    return sum(v["dram_bytes_per_launch"] for v in ks) if ks else None


def whole_job_rate(units_per_rank: float, seconds: float, world_size: int, device=None) -> tuple:
    """Weak-scaling aggregate: every rank processes `units_per_rank` units in
    its own `seconds`; the job takes as long as the slowest rank (max over
    ranks), and the rate is all ranks' units over that time.  Returns
    (rate, max_seconds).  Works with any initialised process group (NCCL on
    GPUs, gloo on CPU)."""
    if world_size > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        seconds = float(t.item())
    return world_size * units_per_rank / seconds, seconds


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_inputs():
    import numpy as np
    from paper_1304_7211_gb300 import synth
    out = []
    for spec in synth.CONFIG2_PSFS:
        c = synth.config2(spec, SIZE)
        out.append((spec, c.f.astype(np.float32)))
    return out


def oracle_sample(inputs, its=CPU_ITERS):
    """The FP64 oracle, as it stands, on the full 2048^2 image of each PSF for
    `its` iterations: (pixel-iterations, seconds, per-PSF notes)."""
    import numpy as np
    import oracle
    oracle.build()
    px_it, t_total, per = 0, 0.0, []
    for spec, f32 in inputs:
        t = spec.dense()
        psf = oracle.psf_dense(t, t.shape[1] // 2, t.shape[0] // 2)
        f64 = f32.astype(np.float64)
        t0 = time.perf_counter()
        oracle.rl(f64, psf, its)
        dt = time.perf_counter() - t0
        t_total += dt
        px_it += f64.size * its
        per.append(f"{spec.name}:{its}it/{dt:.2f}s")
    return px_it, t_total, per


def _single_thread_sample(inputs) -> dict:
    """The same sample in a fresh process limited to one OpenMP thread."""
    import numpy as np
    with tempfile.TemporaryDirectory() as td:
        names = []
        for i, (spec, f32) in enumerate(inputs):
            np.save(os.path.join(td, f"f{i}.npy"), f32)
            names.append(spec.name)
        code = (
            "import json, sys, numpy as np; sys.path.insert(0, %r)\n"
            "import bench\n"
            "from paper_1304_7211_gb300 import synth\n"
            "specs = {s.name: s for s in synth.CONFIG2_PSFS}\n"
            "inp = [(specs[n], np.load(%r + '/f%%d.npy' %% i)) for i, n in enumerate(%r)]\n"
            "print(json.dumps(bench.oracle_sample(inp)))\n" % (ROOT, td, names))
        env = dict(os.environ, OMP_NUM_THREADS="1")
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                             timeout=600)
        px_it, secs, per = json.loads(out.stdout.strip().splitlines()[-1])
    return {"value": px_it / secs / 1e6, "unit": UNIT, "cores": 1, "seconds": secs,
            "sample": f"full 2048x2048 image, {CPU_ITERS} iterations per PSF ({', '.join(per)})"}


def cpu_baseline_run(inputs, single_thread: bool = True):
    """Time the FP64 oracle (as it stands) on the host cores on a bounded
    sample: the full 2048^2 image of each PSF for CPU_ITERS iterations, with
    every core (OpenMP over rows) and, in a fresh process, with one."""
    px_it, secs, per = oracle_sample(inputs)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    d = {"value": px_it / secs / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
         "seconds": secs,
         "sample": f"full 2048x2048 image, {CPU_ITERS} iterations per PSF ({', '.join(per)}); "
                   f"FP64 direct summation, OpenMP over rows"}
    if single_thread:
        try:
            d["single_thread"] = _single_thread_sample(inputs)
        except Exception as e:  # reported, not fatal: the all-core figure stands
            d["single_thread"] = {"error": str(e)[:200]}
    return d


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    # Each step is a bounded sample of the workload: the full 2048^2 image of
    # every PSF for CPU_ITERS iterations (not the 200 of the GPU step), timed
    # as it runs; the rate is over the sample's own pixel-iterations.
    inputs = make_inputs()
    oracle_sample(inputs, its=1)  # warm-up: builds and loads the oracle
    secs, px = [], 0
    for _ in range(args.steps):
        px, t, per = oracle_sample(inputs)
        secs.append(t)
    v = px * len(secs) / sum(secs) / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"full 2048x2048 image, {CPU_ITERS} iterations per PSF per step ({', '.join(per)}); "
              f"FP64 direct summation, OpenMP over rows")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + f" (CPU oracle; a step is the {CPU_ITERS}-iteration sample)",
                       "size": SIZE, "iterations": CPU_ITERS},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_case(args):
    """One solve of one PSF at --size for --iters iterations (for ncu)."""
    import numpy as np
    import torch
    from paper_1304_7211_gb300 import _build, rl, synth
    _build.build()
    specs = {s.name: s for s in (synth.motion(31, 0), synth.motion(31, 1), synth.disc(8),
                                 synth.disc(12), synth.gaussian(7, 1.5), synth.motion(15, 0),
                                 synth.motion(8, 0), synth.motion(8, 1),
                                 synth.dense(np.eye(9)[::-1]))}
    # uniform centred squares (register-blocked box kernel)
    specs.update({f"box{k}": synth.dense(np.ones((k, k))) for k in (3, 9, 17, 33)})
    # other uniform rectangles (register-blocked rectangle kernel)
    specs.update({f"rect{h}x{w}": synth.dense(np.ones((h, w))) for h, w in ((3, 5), (9, 7), (9, 31), (31, 9),
                                                                           (33, 31))})
    spec = specs[args.case]
    g = synth.latent_image(args.size, args.size, synth.SEED_BASE + 2)
    f32 = np.maximum(synth.blur(g, spec), 0.0).astype(np.float32)
    dt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[args.storage]
    f = torch.from_numpy(f32).cuda().to(dt)
    u = torch.empty_like(f)
    th = None if args.tau is None else rl.thinning(args.tau, True, 10, args.q)
    with rl.Deconvolver(spec, path=args.path, storage=args.storage, adjoint=args.adjoint,
                        boundary=args.boundary) as d:
        rl.rl_iterate(d.ctx, f, None, u, args.size, args.size, args.size, args.iters, th)
        torch.cuda.synchronize()
        runs = [rl.rl_iterate(d.ctx, f, None, u, args.size, args.size, args.size, args.iters, th,
                              stats=True) for _ in range(max(1, args.repeat))]
    ms = sorted(r.device_ms for r in runs)
    med = ms[len(ms) // 2]
    st = runs[-1]
    act = st.active_pixel_iterations / max(st.pixel_iterations, 1)
    print(f"case {spec.name} {args.size}^2 x {args.iters} it {args.storage} tau={args.tau} "
          f"adjoint={args.adjoint} boundary={args.boundary}: "
          f"{med:.3f} ms ({med / args.iters * 1e3:.1f} us/it; min {ms[0] / args.iters * 1e3:.1f}, "
          f"{len(ms)} runs) path={rl.PATH_NAME[st.path]} active={100 * act:.1f}% launches={st.launches}")
    return 0


def batch_run(local, n_images=64, slots=32, storage="f32"):
    """Batched workload: 64 images, sides log-uniform in [128, 1536], PSF and
    iteration count (50..300) per image, all submitted to one rl_batch
    (32 streams: small images fill few CTA slots each) vs the same solves one
    at a time; the batch runs with the built-in launch choices and with the
    autotuner's (its cache filled by a first, untimed pass).  Returns a
    dict."""
    import numpy as np
    import torch
    from paper_1304_7211_gb300 import rl, synth
    dev = torch.device("cuda", local)
    dt = {"f32": torch.float32, "bf16": torch.bfloat16}[storage]
    jobs = []
    for (w, h, spec, its, seed) in synth.batch_specs(n_images):
        c = synth.batch_case(w, h, spec, its, seed)
        f = torch.from_numpy(c.f.astype(np.float32)).to(dev).to(dt)
        jobs.append((spec, f, torch.empty_like(f), its, w, h))
    px_it = float(sum(w * h * its for (_, _, _, its, w, h) in jobs))

    def batched(flags=0):
        with rl.Batch(slots, device=local, storage=storage, flags=flags) as b:
            for spec, f, u, its, w, h in jobs:
                b.submit(spec, f, u, its, w, h)
            b.sync()

    def tuned():
        batched(rl.RL_FLAG_AUTOTUNE)

    def sequential():
        for spec, f, u, its, w, h in jobs:
            with rl.Deconvolver(spec, device=local, storage=storage) as d:
                rl.rl_iterate(d.ctx, f, None, u, w, h, w, its)
        torch.cuda.synchronize(dev)

    batched()  # warm-up (scratch growth, module load)
    tuned()    # fills the tuning cache for every job's key
    sequential()
    ts = {}
    for name, fn in (("batched", batched), ("tuned", tuned), ("sequential", sequential)):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize(dev)
        ts[name] = time.perf_counter() - t0
    return {"workload": f"{n_images} images, sides log-uniform [128,1536], motion x/y 5-41, "
                        f"disc r 3-15, gaussian 7x7; 50-300 it; {storage}", "slots": slots,
            "px_it": px_it, "batched_ms": 1e3 * ts["batched"], "tuned_ms": 1e3 * ts["tuned"],
            "sequential_ms": 1e3 * ts["sequential"],
            "value": px_it / ts["batched"] / 1e6, "tuned_value": px_it / ts["tuned"] / 1e6,
            "sequential_value": px_it / ts["sequential"] / 1e6,
            "speedup_vs_plain": ts["sequential"] / ts["batched"], "unit": UNIT,
            "timing": "host wall clock around submit..sync, inputs resident"}


def tiles_run(local, n_images=64, slots=32):
    """Batched (request, tile) workload: 64 frames under one disc r = 8 PSF,
    sides log-uniform in [128, 512], 50..150 iterations each, as one
    rl_iterate_tiles call (one launch pair per iteration over every frame's
    tiles) vs rl_batch on 32 streams vs one solve at a time.  Returns a dict."""
    import numpy as np
    import torch
    from paper_1304_7211_gb300 import rl, synth
    dev = torch.device("cuda", local)
    rng = np.random.default_rng(synth.SEED_BASE + 90)
    spec = synth.disc(8)
    jobs = []
    for j in range(n_images):
        w, h = (int(round(np.exp(rng.uniform(np.log(128), np.log(512))))) for _ in range(2))
        its = int(rng.integers(50, 151))
        c = synth.make_case(w, h, spec, 0, "poisson", synth.SEED_BASE + 900 + j)
        f = torch.from_numpy(c.f.astype(np.float32)).to(dev)
        jobs.append((f, torch.empty_like(f), its, w, h))
    px_it = float(sum(w * h * its for (_, _, its, w, h) in jobs))
    ctx = rl.Deconvolver(spec, device=local)

    def tiles():
        rl.rl_iterate_tiles(ctx.ctx, [(f, None, u, w, h, w, its) for (f, u, its, w, h) in jobs])

    def streams():
        with rl.Batch(slots, device=local) as b:
            for f, u, its, w, h in jobs:
                b.submit(spec, f, u, its, w, h)
            b.sync()

    def sequential():
        for f, u, its, w, h in jobs:
            rl.rl_iterate(ctx.ctx, f, None, u, w, h, w, its)

    ts = {}
    for name, fn in (("tiles", tiles), ("streams", streams), ("sequential", sequential)):
        fn()  # warm-up
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize(dev)
        ts[name] = time.perf_counter() - t0
    ctx.close()
    return {"workload": f"{n_images} frames, one disc r8 PSF, sides log-uniform [128,512], 50-150 it; fp32",
            "px_it": px_it, "unit": UNIT, "value": px_it / ts["tiles"] / 1e6,
            "streams_value": px_it / ts["streams"] / 1e6, "sequential_value": px_it / ts["sequential"] / 1e6,
            "tiles_ms": 1e3 * ts["tiles"], "streams_ms": 1e3 * ts["streams"],
            "sequential_ms": 1e3 * ts["sequential"], "slots": slots,
            "timing": "host wall clock around the call(s)..sync, inputs resident"}


def serve_run(local, n=400, rates=(100.0, 200.0), slots=16):
    """Served workload: a Poisson-arrival trace of n requests, sides
    log-uniform in [256, 4096], PSF as in the batched workload, 50..500
    iterations, thinning threshold 1e-4 (mask recomputed every 10
    iterations), admission under a 150 GB budget.  Each request's observed
    image is its own latent crop blurred by its own PSF with Poisson noise,
    made on the GPU before the run (it arrives on the device; the result goes
    back to pinned host memory).  The same requests are served at every rate
    (arrival times scale with 1 / rate).  Baseline: the plain path as a
    server -- one request at a time in arrival order, each taking its
    measured alone-time -- on the same trace.  Returns a dict."""
    import numpy as np
    from paper_1304_7211_gb300 import serve, synth
    trace = synth.serve_trace(n, 1.0)
    fs = synth.serve_inputs_device(trace, local)
    thin = (1e-4, True, 10, 10)

    def requests(rate):
        return [serve.Request(j, t / rate, f, spec, its, thin)
                for j, ((t, w, h, spec, its, _), f) in enumerate(zip(trace, fs))]

    alone = requests(1.0)
    svc = serve.service_times(alone, device=local)
    progress("serve: alone-solve times")
    srv = serve.Server(device=local, slots=slots, hbm_budget_bytes=150e9)
    rows = []
    try:
        srv.run([serve.Request(-1, 0.0, r.f, r.spec, 5, r.thin) for r in alone[:8]], realtime=False)
        for rate in rates:
            reqs = requests(rate)
            rep = srv.run(reqs, realtime=True)
            fifo = serve.fifo_report(reqs, svc)
            same = sum(bool(np.array_equal(r.result, a.result)) for r, a in zip(reqs, alone))
            rows.append({"rate_per_s": rate, "served": rep.as_dict(), "fifo_sequential": fifo.as_dict(),
                         "served_over_sequential": rep.mpx_it_per_s / fifo.mpx_it_per_s,
                         "results_bitwise_same_as_alone": f"{same}/{len(reqs)}"})
            progress(f"serve at {rate:g} requests/s")
    finally:
        srv.close()
    px_it = float(sum(r.f.shape[0] * r.f.shape[1] * r.iterations for r in alone))
    return {"workload": f"{n} requests, Poisson arrivals, sides log-uniform [256,4096], motion x/y 5-41, "
                        f"disc r 3-15, gaussian 7x7, 50-500 it, thinning 1e-4 (P=Q=10), budget 150 GB, "
                        f"{slots} streams; fp32",
            "unit": UNIT, "px_it": px_it, "sequential_offline_value": px_it / sum(svc) / 1e6,
            "inputs": "per request: crop of a seeded 4096^2 latent, blurred by its own PSF, Poisson peak 1000",
            "rates": rows}


def thinned_run(local, size=4096, iters=300, oracle_size=384, pending=None):
    """Thinned workload: disc radius 12, Poisson noise at peak 500, 300
    iterations, relative thresholds {1e-3, 1e-4, 1e-5} with the mask
    recomputed every 10 iterations, FP32 and BF16 storage.  Reports time,
    active pixel-iterations and PSNR against the latent image; each variant
    also runs on a smaller image of the same generator, whose error against
    the FP64 oracle the CPU-baseline leg fills in (``pending``)."""
    import numpy as np
    import torch
    from paper_1304_7211_gb300 import rl, synth
    c = synth.config3(size)
    rows = []
    variants = [(None, "f32"), (None, "bf16")] + [(t, sto) for t in (1e-3, 1e-4, 1e-5)
                                                   for sto in ("f32", "bf16")]
    small = synth.config3(oracle_size)
    outputs = []
    key = f"rel_linf_vs_oracle_{oracle_size}"
    for tau, sto in variants:
        dt = {"f32": torch.float32, "bf16": torch.bfloat16}[sto]
        f = torch.from_numpy(c.f.astype(np.float32)).to(dt).cuda(local)
        u = torch.empty_like(f)
        th = None if tau is None else rl.thinning(tau, True, 10, 10)
        with rl.Deconvolver(c.spec, device=local, storage=sto) as d:
            rl.rl_iterate(d.ctx, f, None, u, size, size, size, 20, th)  # warm-up
            st = rl.rl_iterate(d.ctx, f, None, u, size, size, size, iters, th, stats=True)
            psnr = psnr_db(u.float().cpu().numpy(), c.g)
            fs = torch.from_numpy(small.f.astype(np.float32)).to(dt).cuda(local)
            us = torch.empty_like(fs)
            rl.rl_iterate(d.ctx, fs, None, us, oracle_size, oracle_size, oracle_size, iters, th)
            u_small = us.float().cpu().numpy()
        row = {"tau": tau, "storage": sto, "ms": st.device_ms,
               "mpx_it_per_s": size * size * iters / st.device_ms / 1e3,
               "active_pct": 100.0 * st.active_pixel_iterations / st.pixel_iterations,
               "psnr_vs_latent_db": psnr, key: None}
        rows.append(row)
        outputs.append((row, tau, u_small))
    out = {"workload": f"{size}^2 disc r12 Poisson peak 500, {iters} it, mask every 10 it",
           "oracle_cpu_s": None, "rows": rows}
    if pending is not None:
        # the oracle runs on the input as the GPU saw it (FP32-rounded f)
        pending.append({"kind": "thinned", "f": small.f.astype(np.float32).astype(np.float64),
                        "iters": iters, "outputs": outputs, "key": key, "report": out})
    return out


def solve_roofline(spec, ms_solve, launches, pk, pk_kind, sms, cap) -> dict:
    """Roofline of one 200-iteration 2048^2 solve's kernel, from its live
    CUDA-event time.  Disc (span path): 2 (2r + 1) run-end additions per pixel
    per convolution (Sec. 3, generic box filter), two convolutions, plus the
    ratio, the update and two scalings, against the FP32 issue peak (SMs x 128
    lanes x max SM clock); the unit of work is one iteration (its forward and
    adjoint launches).  Running sum with rows resident (Sec. 3, linear motion
    blur): the fused per-iteration pass would move 12 B/px-it (f and u in, u'
    out), counted as effective bytes against the measured copy bandwidth;
    the unit of work is the one launch of the solve.  traffic: DRAM bytes per
    unit from the ncu capture of these sources (profiles/), else None."""
    px = SIZE * SIZE
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    if spec.kind == "disc":
        r = spec.radius
        per_unit = px * (4 * (2 * r + 1) + 4)
        unit_ms = ms_solve / ITERS
        peak = sms * 128 * sm_mhz * 1e6 / 1e12
        achieved = per_unit / (unit_ms * 1e-3) / 1e12
        persistent = launches == 1
        if persistent:
            kern = f"k_disc_persist<float, DiscOp<{r}>> (all {ITERS} iterations in one launch)"
            traffic = traffic_of(cap, lambda k: re.match(rf"k_disc_persist<float, DiscOp<{r}[,>]", k) is not None)
            traffic = traffic / ITERS if traffic is not None else None
        else:
            kern = f"k_disc_half<float, 0, DiscOp<{r}>, FWD> + <.., ADJ> (both launches of one iteration)"
            traffic = traffic_of(cap, lambda k: re.match(rf"k_disc_half<float, 0, DiscOp<{r}[,>]", k) is not None)
        return {"solve": spec.name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": kern,
                "unit_of_work": "one RL iteration on the 2048^2 image",
                "algorithmic_per_unit": per_unit, "algorithmic_unit": "FP32 additions",
                "peak_source": f"{sms} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz (additions)",
                "hbm_equiv_gbs": 12 * px / (unit_ms * 1e-3) / 1e9,
                "hbm_equiv_frac": 12 * px / (unit_ms * 1e-3) / 1e9 / pk["hbm_gbs"]}
    per_unit = 12 * px * ITERS
    achieved = per_unit / (ms_solve * 1e-3) / 1e9
    traffic = traffic_of(cap, lambda k: k.startswith("k_motion_x_tb<float, 0,"))
    return {"solve": spec.name, "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
            "kernel": f"k_motion_x_tb<float> (rows resident for all {ITERS} iterations; "
                      + ("along x)" if spec.axis == 0 else "on the transposed image)"),
            "unit_of_work": f"one launch = the {ITERS}-iteration solve",
            "algorithmic_per_unit": per_unit, "algorithmic_unit": "bytes of the fused per-iteration pass "
                                                                 "(12 B/px-it), effective",
            "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({pk_kind})"}


def config1_run(local, pending=None) -> dict:
    """The 256^2 workload: motion-x 15, Gaussian noise sigma 2, 50 iterations,
    FP32; its rate, and its output for the CPU-baseline leg to compare with
    the FP64 oracle on the same input (``pending``)."""
    import numpy as np
    import torch
    from paper_1304_7211_gb300 import rl, synth
    c = synth.config1()
    f32 = c.f.astype(np.float32)
    H, W = f32.shape
    f = torch.from_numpy(f32).cuda(local)
    u = torch.empty_like(f)
    with rl.Deconvolver(c.spec, device=local) as d:
        rl.rl_iterate(d.ctx, f, None, u, W, H, W, c.iterations)
        ms = sorted(rl.rl_iterate(d.ctx, f, None, u, W, H, W, c.iterations, stats=True).device_ms
                    for _ in range(7))
    med = ms[len(ms) // 2]
    out = {"workload": f"{W}x{H} fp32, motion-x 15, Gaussian noise sigma 2, {c.iterations} it",
           "value": W * H * c.iterations / med / 1e3, "unit": UNIT, "ms_per_solve": med,
           "rel_linf_vs_oracle": None,
           "timing": "CUDA events around rl_iterate (stats), median of 7; latency-bound at this size"}
    if pending is not None:
        pending.append({"kind": "config1", "f": f32.astype(np.float64), "taps": c.spec.dense(),
                        "iters": c.iterations, "u": u.cpu().numpy(), "report": out})
    return out


def rel_linf(a, b) -> float:
    """Relative L-infinity difference max|a - b| / max|b| (FP64)."""
    import numpy as np
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


def psnr_db(u, g) -> float:
    """PSNR of u against the latent image g, peak = max(g)."""
    import numpy as np
    u, g = np.asarray(u, np.float64), np.asarray(g, np.float64)
    mse = float(np.mean((u - g) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(float(g.max()) ** 2 / mse)


def oracle_checks(pending) -> float:
    """The CPU-baseline leg's comparisons: the FP64 oracle run on the inputs
    of the GPU sub-measurements (``pending``), its relative L-inf difference
    written into their reports.  Returns the oracle's seconds."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    for p in pending:
        if p["kind"] == "config1":
            t = p["taps"]
            ref = oracle.rl(p["f"], oracle.psf_dense(t, t.shape[1] // 2, t.shape[0] // 2), p["iters"]).u
            p["report"]["rel_linf_vs_oracle"] = rel_linf(p["u"], ref)
        elif p["kind"] == "thinned":
            refs = {}
            for row, tau, u in p["outputs"]:
                if tau not in refs:
                    refs[tau] = oracle.rl(p["f"], oracle.psf_disc(12), p["iters"], threshold=tau,
                                          update_period=10).u
                row[p["key"]] = rel_linf(u, refs[tau])
            p["report"]["oracle_cpu_s"] = time.perf_counter() - t0
    return time.perf_counter() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case", default=None,
                    help="profiling mode: run one solve of this PSF (e.g. disc8, motionx31, "
                         "motiony31, dense7x7) and print its time; no JSON line")
    ap.add_argument("--repeat", type=int, default=1, help="case mode: timed solves (median reported)")
    ap.add_argument("--adjoint", default="padflip", choices=["padflip", "transpose"],
                    help="case mode: adjoint of Eq. 3 (pad-flip or exact transpose)")
    ap.add_argument("--boundary", default="mirror", choices=["mirror", "clamp"],
                    help="case mode: boundary continuation")
    ap.add_argument("--size", type=int, default=SIZE)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--path", default="auto")
    ap.add_argument("--tau", type=float, default=None, help="case mode: relative thinning threshold")
    ap.add_argument("--q", type=int, default=10, help="case mode: mask update period (1 or 10)")
    ap.add_argument("--storage", default="f32")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched sub-measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the served sub-measurement")
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--workload", default="plain", choices=["plain", "thinned", "serve"],
                    help="'thinned' prints the thinned-workload table, 'serve' the full served "
                         "workload (2000 requests at 20 / 50 / 100 / 200 per second), instead of "
                         "the bench line")
    ap.add_argument("--no-config3", action="store_true", help="skip the 4096^2 thinned sub-measurement")
    ap.add_argument("--no-config1", action="store_true", help="skip the 256^2 sub-measurement")
    ap.add_argument("--ingest-ncu", nargs=2, metavar=("CSV", "COMMAND"), default=None,
                    help="write profiles/traffic_plain_2048.json from an ncu CSV (launch list with "
                         "dram__bytes_{read,write}.sum) of COMMAND, tagged with the current sources' hash")
    args = ap.parse_args()
    if args.ingest_ncu:
        out = ingest_ncu(args.ingest_ncu[0], TRAFFIC_FILE, WORKLOAD, args.ingest_ncu[1])
        print(json.dumps(out, indent=1))
        return 0
    ws, rank, local = dist_init()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.case:
        return run_case(args)
    if args.workload in ("thinned", "serve"):
        import torch
        torch.cuda.set_device(local)
        from paper_1304_7211_gb300 import _build
        _build.build()
        if args.workload == "thinned":
            pending = []
            out = thinned_run(local, pending=pending)
            if not args.no_cpu_baseline:
                oracle_checks(pending)  # the CPU-baseline leg of this mode
        else:
            out = serve_run(local, n=2000, rates=(20.0, 50.0, 100.0, 200.0))
        print(json.dumps(out), flush=True)
        return 0

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1304_7211_gb300 import _build, rl
    _build.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    inputs = make_inputs()
    solves = []
    for spec, f32 in inputs:
        d = rl.Deconvolver(spec, device=local, stream=stream)
        f_dev = torch.from_numpy(f32).to(dev)
        u_dev = torch.empty_like(f_dev)
        f_host = torch.from_numpy(f32).pin_memory()
        u_host = torch.empty_like(f_host).pin_memory()
        solves.append((spec, d, f_dev, u_dev, f_host, u_host))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step_device():
        for spec, d, f, u, _, _ in solves:
            rl.rl_iterate(d.ctx, f, None, u, SIZE, SIZE, SIZE, ITERS)

    def step_host():
        for spec, d, _, _, fh, uh in solves:
            rl.rl_iterate(d.ctx, fh, None, uh, SIZE, SIZE, SIZE, ITERS)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # per-kernel timing of one solve of each PSF (same stream, CUDA events)
    def solve_ms(idx, reps=3):
        spec, d, f, u, _, _ = solves[idx]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ts = []
        for _ in range(reps):
            flush.zero_()
            ev[0].record(stream)
            rl.rl_iterate(d.ctx, f, None, u, SIZE, SIZE, SIZE, ITERS)
            ev[1].record(stream)
            ev[1].synchronize()
            ts.append(ev[0].elapsed_time(ev[1]))
        return statistics.median(ts)

    for _ in range(max(args.warmup, 3)):
        step_device()
    barrier()

    clocks = Clocks(local)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    for i in range(args.steps):
        flush.zero_()  # L2 flush between steps, outside the events
        starts[i].record(stream)
        step_device()
        ends[i].record(stream)
    barrier()
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    px_step = 3 * SIZE * SIZE * ITERS
    rate, t_s = whole_job_rate(px_step * args.steps, sum(step_ms) * 1e-3, ws, dev)
    t_ms = t_s * 1e3
    value = rate / 1e6

    # end to end through the C ABI with host buffers
    for _ in range(2):
        step_host()
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(2, min(args.steps, 5))
    for _ in range(e2e_steps):
        step_host()
    barrier()
    e2e_rate, _ = whole_job_rate(px_step * e2e_steps, time.perf_counter() - t0, ws, dev)
    e2e = e2e_rate / 1e6
    plane = SIZE * SIZE * 4

    # kernel launches inside the timed region, as counted by the library
    launches_per_step = 0
    launches = {}
    for spec, d, f, u, _, _ in solves:
        st = rl.rl_iterate(d.ctx, f, None, u, SIZE, SIZE, SIZE, ITERS, stats=True)
        launches_per_step += st.launches
        launches[spec.name] = st.launches

    # roofline of every solve's kernel; the top-level one is the slowest solve's
    per = {solves[i][0].name: solve_ms(i) for i in range(3)}
    pk, pk_kind = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    cap = measured_traffic()
    rooflines = [solve_roofline(solves[i][0], per[solves[i][0].name], launches[solves[i][0].name], pk,
                                pk_kind, sms, cap) for i in range(3)]
    dom = max(range(3), key=lambda i: per[solves[i][0].name])
    roof = dict(rooflines[dom])
    roof["per_solve"] = rooflines
    roof["traffic_capture"] = (os.path.relpath(TRAFFIC_FILE, ROOT) if cap is not None else
                               "none for the current sources (profiles/ capture predates a kernel change)")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "size": SIZE, "iterations": ITERS,
                       "psfs": [s[0].name for s in solves], "boundary": "mirror",
                       "l2": "512 MiB write between steps, outside the timed events",
                       "parallelism": f"replicas x{ws}"},
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 3 * plane,
                    "d2h_bytes_per_step": 3 * plane},
            "gpu_launches": launches_per_step * args.steps,
            "roofline": roof, "clocks": clk}
    progress("main step, e2e and rooflines")
    pending = []  # GPU outputs the CPU-baseline leg compares with the oracle
    if not args.no_config1:
        line["config1"] = config1_run(local, pending)
        progress("config1")
    if not args.no_batch:
        line["batch"] = batch_run(local)
        progress("batch f32")
        line["batch_bf16"] = batch_run(local, storage="bf16")
        progress("batch bf16")
        line["batch_tiles"] = tiles_run(local)
        progress("batch tiles")
    if not args.no_config3 and ws == 1:
        line["config3"] = thinned_run(local, pending=pending)
        progress("config3")
    if not args.no_serve:
        line["serve"] = serve_run(local, n=args.serve_requests)
        progress("serve")
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_run(inputs)
        if pending:
            line["cpu_baseline"]["oracle_checks_s"] = oracle_checks(pending)
        progress("cpu baseline")
    if rank == 0:
        print(json.dumps(line), flush=True)
    for s in solves:
        s[1].close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
