"""Batched execution and the continuous-batching server on the GPU.

Every job's image must be the same whether it runs alone or among other jobs
on concurrent streams (bitwise: the kernels are deterministic and no state is
shared between jobs), and a sample of them must match the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1304_7211_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-4

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1304_7211_gb300 import _build, rl
    _build.build()
    return rl.load()


def oracle_psf(spec):
    t = spec.dense()
    return oracle.psf_dense(t, t.shape[1] // 2, t.shape[0] // 2)


def small_jobs(n=12, seed=synth.SEED_BASE + 70):
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(n):
        W = int(rng.integers(40, 300))
        H = int(rng.integers(40, 300))
        spec = synth.random_psf(rng)
        t = spec.dense()
        if t.shape[1] // 2 >= W or t.shape[0] // 2 >= H:
            spec = synth.disc(2)
        its = int(rng.integers(5, 40))
        thin = (1e-4, True, 10, 10) if j % 3 == 0 else None
        c = synth.make_case(W, H, spec, its, "poisson", seed + j)
        jobs.append((spec, c.f.astype(np.float32), its, thin))
    return jobs


def alone(spec, f32, its, thin):
    from paper_1304_7211_gb300 import rl
    with rl.Deconvolver(spec) as d:
        u = d.run(torch.from_numpy(f32).cuda(), its, thin=rl.thinning(*thin) if thin else None)
    torch.cuda.synchronize()
    return u.cpu().numpy()


def test_batch_jobs_match_alone_and_oracle():
    from paper_1304_7211_gb300 import rl
    jobs = small_jobs()
    outs = []
    with rl.Batch(slots=4) as b:
        tickets = []
        keep = []
        for spec, f32, its, thin in jobs:
            f = torch.from_numpy(f32).cuda()
            u = torch.empty_like(f)
            H, W = f32.shape
            th = rl.thinning(*thin) if thin else None
            tickets.append(b.submit(spec, f, u, its, W, H, thin=th))
            keep.append((f, u))
        for t in tickets:
            b.wait(t)
            assert b.query(t)
        b.sync()
        outs = [u.cpu().numpy() for _, u in keep]
    for (spec, f32, its, thin), got in zip(jobs, outs):
        np.testing.assert_array_equal(got, alone(spec, f32, its, thin))
    for (spec, f32, its, thin), got in list(zip(jobs, outs))[1:4]:
        if thin:
            continue
        ref = oracle.rl(f32.astype(np.float64), oracle_psf(spec), its).u
        assert oracle.rel_linf(got, ref) <= TOL


def test_batch_host_buffers():
    from paper_1304_7211_gb300 import rl
    jobs = small_jobs(5, seed=synth.SEED_BASE + 71)
    with rl.Batch(slots=2) as b:
        res = []
        for spec, f32, its, thin in jobs:
            H, W = f32.shape
            fd = torch.empty((H, W), device="cuda")
            ud = torch.empty((H, W), device="cuda")
            fh = torch.from_numpy(f32).pin_memory()
            uh = torch.empty((H, W)).pin_memory()
            t = b.submit(spec, fd, ud, its, W, H, f_host=fh, u_host=uh)
            res.append((t, uh, fd, ud, fh))
        b.sync()
        for (spec, f32, its, thin), (t, uh, *_r) in zip(jobs, res):
            np.testing.assert_array_equal(uh.numpy(), alone(spec, f32, its, None))


def test_batch_rejects_bad_jobs():
    from paper_1304_7211_gb300 import rl
    with rl.Batch(slots=1) as b:
        f = torch.ones((8, 8), device="cuda")
        with pytest.raises(rl.RLError):
            b.submit(synth.disc(8), f, f.clone(), 3, 8, 8)   # PSF wider than the image
        with pytest.raises(rl.RLError):
            b.wait(12345)


def test_server_results_same_alone_and_in_the_mix():
    from paper_1304_7211_gb300 import serve
    jobs = small_jobs(16, seed=synth.SEED_BASE + 72)
    reqs = [serve.Request(i, 0.002 * i, f32, spec, its, thin)
            for i, (spec, f32, its, thin) in enumerate(jobs)]
    srv = serve.Server(slots=4, hbm_budget_bytes=2e9)
    try:
        rep = srv.run(reqs, realtime=True)
    finally:
        srv.close()
    assert rep.n == len(reqs)
    assert rep.p99_ms >= rep.p50_ms > 0
    for r, (spec, f32, its, thin) in zip(reqs, jobs):
        np.testing.assert_array_equal(r.result, alone(spec, f32, its, thin))


def test_server_respects_hbm_budget():
    from paper_1304_7211_gb300 import serve
    jobs = small_jobs(8, seed=synth.SEED_BASE + 73)
    reqs = [serve.Request(i, 0.0, f32, spec, its, None) for i, (spec, f32, its, thin) in enumerate(jobs)]
    biggest = max(r.f.size * 8 for r in reqs)
    srv = serve.Server(slots=4, hbm_budget_bytes=biggest)
    try:
        rep = srv.run(reqs, realtime=False)
    finally:
        srv.close()
    assert rep.n == len(reqs)
    assert rep.peak_resident_bytes <= biggest
