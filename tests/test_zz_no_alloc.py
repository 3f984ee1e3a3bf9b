"""The allocation-free entry point ``rl_motion_x_noalloc``.

It exists for callers that cannot call cudaMalloc (allocator or pool hooks,
latency-critical threads, pre-partitioned device memory): its scratch is a
fixed array inside the library.  Here it must give the same images as the
regular entry point ``rl_iterate`` (running-sum path) on two calls in a row --
the second call reuses the array the first one left behind -- and reject an
image larger than the fixed scratch with a clear message.  This file sorts
last so a run that stops at the first failure has run everything else first.
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


def regular(spec, f, iters, boundary):
    from paper_1304_7211_gb300 import rl
    with rl.Deconvolver(spec, boundary=boundary, path="runsum") as d:
        u = d.run(f, iters)
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.float64)


def test_noalloc_matches_rl_iterate_on_two_calls_in_a_row():
    from paper_1304_7211_gb300 import rl
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    calls = [(synth.motion(15, 0), 300, 211, 40, "mirror"),
             (synth.motion(31, 0), 517, 389, 25, "clamp")]
    fs, outs = [], []
    for spec, W, H, iters, boundary in calls:  # two calls in a row
        c = synth.make_case(W, H, spec, 0, "poisson", synth.SEED_BASE + 61 + W)
        f = torch.from_numpy(c.f.astype(np.float32)).cuda()
        out = torch.full_like(f, -1.0)
        rl.rl_motion_x_noalloc(f, None, out, W, H, W, spec.length, boundary, iters, stream)
        fs.append(f)
        outs.append(out)
    torch.cuda.synchronize()
    for (spec, W, H, iters, boundary), f, out in zip(calls, fs, outs):
        ref = regular(spec, f, iters, boundary)
        err = oracle.rel_linf(out.cpu().numpy(), ref)
        assert err <= TOL, err


def test_noalloc_rejects_images_beyond_the_fixed_scratch():
    from paper_1304_7211_gb300 import rl
    W, H = 4096, rl.RL_NOALLOC_MAX_PIXELS // 4096 + 1
    f = torch.ones((2, 2), device="cuda")  # never read: the size check comes first
    with pytest.raises(rl.RLError) as e:
        rl.rl_motion_x_noalloc(f, None, f.clone(), W, H, W, 5, "mirror", 3)
    assert e.value.status == rl.RL_ERR_INVALID_ARG
    assert "exceeds the fixed scratch" in e.value.message
