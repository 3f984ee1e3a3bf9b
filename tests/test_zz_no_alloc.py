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


@pytest.mark.parametrize("iters", [7, 8])
def test_noalloc_padded_pitch_and_start_image(iters):
    """Padded rows (pitch W + 37) and an explicit start image: the ping-pong
    then alternates between the fixed array (pitch W) and u_out (the caller's
    pitch), and the last iteration must land in u_out whether the count is
    odd or even.  Compared with rl_iterate on the same padded buffers."""
    from paper_1304_7211_gb300 import rl
    torch.cuda.set_device(0)
    spec = synth.motion(13, 0)
    W, H, pad = 251, 173, 37
    c = synth.make_case(W, H, spec, 0, "poisson", synth.SEED_BASE + 64)
    fb = torch.zeros((H, W + pad), device="cuda")
    fb[:, :W] = torch.from_numpy(c.f.astype(np.float32)).cuda()
    u0b = torch.zeros_like(fb)
    u0b[:, :W] = fb[:, :W] * 0.9 + 1.0
    out = torch.full_like(fb, -1.0)
    rl.rl_motion_x_noalloc(fb, u0b, out, W, H, W + pad, spec.length, "mirror", iters,
                           torch.cuda.current_stream())
    ref = torch.full_like(fb, -1.0)
    with rl.Deconvolver(spec, path="runsum") as d:
        rl.rl_iterate(d.ctx, fb, u0b, ref, W, H, W + pad, iters)
    torch.cuda.synchronize()
    err = oracle.rel_linf(out[:, :W].cpu().numpy(), ref[:, :W].cpu().numpy().astype(np.float64))
    assert err <= TOL, err
    # the padding columns of u_out are not touched
    assert bool((out[:, W:] == -1.0).all())


def test_noalloc_refuses_host_memory_before_any_launch():
    """The entry point cannot stage host buffers (that would allocate), so a
    numpy array or CPU tensor is refused by the binding, and a raw host
    address by the library itself, before any kernel is launched."""
    from paper_1304_7211_gb300 import rl
    torch.cuda.set_device(0)
    W, H = 64, 32
    f_host = np.ones((H, W), np.float32)
    out = torch.empty((H, W), device="cuda")
    with pytest.raises(TypeError):
        rl.rl_motion_x_noalloc(f_host, None, out, W, H, W, 5, "mirror", 2)
    with pytest.raises(TypeError):
        rl.rl_motion_x_noalloc(torch.ones((H, W)), None, out, W, H, W, 5, "mirror", 2)
    with pytest.raises(TypeError):
        rl.rl_motion_x_noalloc(torch.ones((H, W), device="cuda", dtype=torch.float16), None, out,
                               W, H, W, 5, "mirror", 2)
    with pytest.raises(rl.RLError) as e:
        rl.rl_motion_x_noalloc(f_host.ctypes.data, None, out, W, H, W, 5, "mirror", 2)
    assert e.value.status == rl.RL_ERR_INVALID_ARG
    assert "device memory" in e.value.message
    torch.cuda.synchronize()  # the context is still healthy
