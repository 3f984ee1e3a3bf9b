"""The persistent form of the disc path against its two-launch form.

Without thinning or the exact-transpose band, a disc solve on an image with
enough tiles (RL_FLAG_PERSISTENT forces it on any) runs all of its
iterations in one cooperative launch in which every (iteration, half, tile)
item waits for its 3 x 3 tile neighbourhood to finish the previous half.  It
runs the same tile arithmetic as the two launches per iteration of
RL_FLAG_PER_ITERATION, so the images must agree bit for bit -- for one
tile or many, ragged edges, one to many iterations, every storage type and
both boundaries -- and match the FP64 oracle.
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


def run(spec, f, iters, storage, boundary, per_iteration):
    from paper_1304_7211_gb300 import rl
    flags = rl.RL_FLAG_PER_ITERATION if per_iteration else rl.RL_FLAG_PERSISTENT
    ctx = rl.rl_create(0, None, storage, boundary, "auto", flags)
    try:
        rl.rl_set_psf(ctx, spec)
        H, W = f.shape
        u = torch.empty_like(f)
        st = rl.rl_iterate(ctx, f, None, u, W, H, W, iters, None, stats=True)
    finally:
        rl.rl_destroy(ctx)
    torch.cuda.synchronize()
    return u, st


@pytest.mark.parametrize("radius,W,H,iters", [(1, 40, 33, 1), (3, 64, 64, 2), (8, 203, 157, 3),
                                              (8, 600, 70, 17), (12, 257, 321, 12), (16, 97, 150, 5),
                                              (5, 1030, 515, 20)])
@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_persistent_equals_two_launch_form(radius, W, H, iters, storage):
    spec = synth.disc(radius)
    c = synth.make_case(W, H, spec, 0, "poisson", synth.SEED_BASE + 140 + radius)
    dt = {"f32": torch.float32, "bf16": torch.bfloat16}[storage]
    f = torch.from_numpy(c.f.astype(np.float32)).cuda().to(dt)
    for boundary in ("mirror", "clamp"):
        a, sa = run(spec, f, iters, storage, boundary, per_iteration=False)
        b, sb = run(spec, f, iters, storage, boundary, per_iteration=True)
        assert sa.launches == 1 and sb.launches == 2 * iters
        assert torch.equal(a, b), (boundary, (a.float() - b.float()).abs().max().item())


def test_persistent_matches_oracle_many_tiles():
    spec = synth.disc(8)
    c = synth.make_case(517, 389, spec, 0, "poisson", synth.SEED_BASE + 150)
    f32 = c.f.astype(np.float32)
    u, st = run(spec, torch.from_numpy(f32).cuda(), 40, "f32", "mirror", per_iteration=False)
    assert st.launches == 1
    t = spec.dense()
    ref = oracle.rl(f32.astype(np.float64), oracle.psf_dense(t, t.shape[1] // 2, t.shape[0] // 2), 40).u
    assert oracle.rel_linf(u.cpu().numpy(), ref) <= TOL


def test_bounded_wait_gives_up_and_reports():
    """A launch whose forward half is never handed out: every adjoint item
    waits for neighbours that never finish.  Each wait gives up after 50 ms,
    the status word reports it, every CTA returns, and the GPU stays usable
    for the next solve."""
    from paper_1304_7211_gb300 import rl
    lib = rl.load()
    assert lib.rl_selftest_wait_timeout(0, 50) == rl.RL_ERR_TIMEOUT
    spec = synth.disc(4)
    c = synth.make_case(200, 150, spec, 0, "poisson", synth.SEED_BASE + 151)
    f = torch.from_numpy(c.f.astype(np.float32)).cuda()
    a, _ = run(spec, f, 5, "f32", "mirror", per_iteration=False)
    b, _ = run(spec, f, 5, "f32", "mirror", per_iteration=True)
    assert torch.equal(a, b)


@pytest.mark.parametrize("thin", [(1e-3, True, 10, 10), (1e-3, True, 10, 1), (0.05, False, 10, 1)],
                         ids=["rel-q10", "rel-q1", "abs-q1"])
@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_thinned_persistent_equals_two_launch_form(thin, storage):
    """Selective convolution (Eq. 4-5) in the persistent kernel: the mask,
    the tile flags and the stale ratios are updated in place as in the two
    launches per iteration, so images, final masks and active counts agree
    exactly."""
    from paper_1304_7211_gb300 import rl
    spec = synth.disc(6)
    W, H, K = 333, 250, 27
    c = synth.make_case(W, H, spec, 0, "poisson", synth.SEED_BASE + 152)
    dt = {"f32": torch.float32, "bf16": torch.bfloat16}[storage]
    f = torch.from_numpy(c.f.astype(np.float32)).cuda().to(dt)
    outs = []
    for flags in (rl.RL_FLAG_PERSISTENT, rl.RL_FLAG_PER_ITERATION):
        ctx = rl.rl_create(0, None, storage, "mirror", "auto", flags)
        try:
            rl.rl_set_psf(ctx, spec)
            u = torch.empty_like(f)
            st = rl.rl_iterate(ctx, f, None, u, W, H, W, K, rl.thinning(*thin), stats=True)
            m = np.zeros((H, W), np.uint8)
            rl.rl_get_mask(ctx, m, W)
        finally:
            rl.rl_destroy(ctx)
        torch.cuda.synchronize()
        outs.append((u, m, st))
    (ua, ma, sa), (ub, mb, sb) = outs
    assert sa.launches == 1
    assert torch.equal(ua, ub)
    np.testing.assert_array_equal(ma, mb)
    assert sa.active_pixel_iterations == sb.active_pixel_iterations < W * H * K
