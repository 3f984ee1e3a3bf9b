"""Failure handling at the C ABI, injected on the host (no GPU fault).

An allocation failure forced through the library's test hook must come back
as RL_ERR_OOM with a message, leave the context usable, and -- in a batch --
fail only the job it hit: the jobs before and after it give the same images
as alone.  A job cancelled before it starts never runs; one already on the
GPU runs to the end and is reported cancelled.  A persistent launch that
gives up a bounded wait is reported for its own job.
"""
import numpy as np
import pytest

from paper_1304_7211_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1304_7211_gb300 import _build, rl
    _build.build()
    return rl.load()


@pytest.fixture(autouse=True)
def no_injection(lib):
    lib.rl_test_fail_allocation(0)
    yield
    lib.rl_test_fail_allocation(0)


def image(w, h, spec, seed):
    c = synth.make_case(w, h, spec, 0, "poisson", synth.SEED_BASE + seed)
    return torch.from_numpy(c.f.astype(np.float32)).cuda()


def alone(spec, f, its):
    from paper_1304_7211_gb300 import rl
    with rl.Deconvolver(spec) as d:
        u = d.run(f, its)
    torch.cuda.synchronize()
    return u


def test_injected_allocation_failure_in_rl_iterate(lib):
    from paper_1304_7211_gb300 import rl
    spec = synth.disc(5)
    f = image(300, 200, spec, 160)
    with rl.Deconvolver(spec) as d:
        lib.rl_test_fail_allocation(1)
        with pytest.raises(rl.RLError) as e:
            d.run(f, 10)
        assert e.value.status == rl.RL_ERR_OOM
        assert "injected allocation failure" in e.value.message
        u = d.run(f, 10)  # the same context goes on
    torch.cuda.synchronize()
    assert torch.equal(u, alone(spec, f, 10))


def test_injected_failure_in_a_batch_fails_that_job_only(lib):
    from paper_1304_7211_gb300 import rl
    spec = synth.disc(4)
    small = [image(160, 120, spec, 161 + j) for j in range(3)]
    big = image(900, 700, spec, 165)  # needs more scratch than the small jobs: it allocates
    outs = [torch.full_like(f, -1.0) for f in small]
    big_out = torch.full_like(big, -1.0)
    with rl.Batch(slots=1) as b:
        t0 = b.submit(spec, small[0], outs[0], 12, 160, 120)
        lib.rl_test_fail_allocation(1)  # the next scratch allocation: the big job's
        with pytest.raises(rl.RLError) as e:
            b.submit(spec, big, big_out, 12, 900, 700)  # issued at once: the failure comes back here
        assert e.value.status == rl.RL_ERR_OOM
        t1 = b.submit(spec, small[1], outs[1], 12, 160, 120)
        b.sync()
        # the slot full: the big job waits on the host and fails when it is
        # issued later, which its ticket reports; the job after it runs
        t2 = b.submit(spec, small[2], outs[2], 300, 160, 120)
        t3 = b.submit(spec, small[2], outs[2], 300, 160, 120)
        tbig = b.submit(spec, big, big_out, 12, 900, 700)
        t4 = b.submit(spec, small[1], outs[1], 12, 160, 120)
        lib.rl_test_fail_allocation(1)
        with pytest.raises(rl.RLError) as e:
            b.wait(tbig)
        assert e.value.status == rl.RL_ERR_OOM
        lib.rl_test_fail_allocation(0)
        b.sync()
        for t in (t0, t1, t2, t3, t4):
            assert b.query(t)
    for f, u, its in zip(small, outs, (12, 12, 300)):
        assert torch.equal(u, alone(spec, f, its))
    assert bool((big_out == -1.0).all())  # the failed job wrote nothing


def test_cancel_before_start_and_while_running(lib):
    from paper_1304_7211_gb300 import rl
    spec = synth.disc(8)
    f_big = image(2048, 1024, spec, 170)
    f_small = image(200, 150, spec, 171)
    with rl.Batch(slots=1) as b:
        u_a = torch.empty_like(f_big)
        u_b = torch.empty_like(f_big)
        u_c = torch.full_like(f_small, -1.0)
        ta = b.submit(spec, f_big, u_a, 300, 2048, 1024)   # on the GPU at once
        tb = b.submit(spec, f_big, u_b, 300, 2048, 1024)   # second job of the slot, also issued
        tc = b.submit(spec, f_small, u_c, 20, 200, 150)    # the slot is full: waits on the host
        assert b.cancel(tc) is False                       # dropped before it started
        try:
            running = b.cancel(ta)
            assert running is True
        except rl.RLError as e:  # it may already have finished on a fast GPU
            assert e.value.status == rl.RL_ERR_STATE
        b.sync()
        assert b.query(tc) and b.query(ta)
        with pytest.raises(rl.RLError):
            b.cancel(tc)  # already cancelled
    torch.cuda.synchronize()
    assert bool((u_c == -1.0).all())  # never ran
    assert torch.equal(u_b, alone(spec, f_big, 300))


def test_persistent_give_up_is_reported_per_batch_job(lib):
    """A neighbour wait that runs out in a batch job's persistent launch (the
    wait bound shortened to 1 ns through the test hook; with one tile per CTA
    every CTA that finishes a half takes an item of the next one while its
    neighbours still compute, so items do wait; nothing faults, the launch
    records it and returns) fails that job alone with RL_ERR_TIMEOUT; the
    other job is exact, and with the bound restored the same job matches its
    alone-solve bit for bit."""
    from paper_1304_7211_gb300 import rl
    spec, other = synth.disc(7), synth.motion(9, 0)
    f, g = image(2000, 1500, spec, 163), image(300, 200, other, 164)
    u, v = torch.empty_like(f), torch.empty_like(g)
    lib.rl_test_persist_ctas(7)  # 768 CTAs for the 32 x 24 tiles
    lib.rl_test_persist_wait_ns(1)
    try:
        with rl.Batch(2) as b:
            t1 = b.submit(spec, f, u, 40, 2000, 1500)
            t2 = b.submit(other, g, v, 10, 300, 200)
            with pytest.raises(rl.RLError) as e:
                b.wait(t1)
            assert e.value.status == rl.RL_ERR_TIMEOUT
            assert "gave up" in e.value.message
            b.wait(t2)
            torch.cuda.synchronize()
            assert torch.equal(v, alone(other, g, 10))
            lib.rl_test_persist_wait_ns(0)
            t3 = b.submit(spec, f, u, 20, 2000, 1500)
            b.wait(t3)
            assert b.query(t3)
    finally:
        lib.rl_test_persist_wait_ns(0)
        lib.rl_test_persist_ctas(0)
    torch.cuda.synchronize()
    assert torch.equal(u, alone(spec, f, 20))
