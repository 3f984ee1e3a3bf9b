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


@pytest.mark.parametrize("ctas", [1, 2, 3, 5, 7])
@pytest.mark.parametrize("thin", [None, (1e-3, True, 10, 10)], ids=["plain", "thinned"])
def test_every_grid_size_equals_two_launch_form(ctas, thin):
    """The persistent grid holds `ctas` CTAs per SM (at most one per tile);
    with fewer CTAs than tiles each CTA takes several items per half, in
    ticket order, so every wait is for an item taken earlier.  The result
    must not depend on the grid: bit-identical to the two launches for every
    count, plain and thinned (Eq. 4-5), with many tiles per CTA at 1 CTA per
    SM (2000 x 1500: 32 x 24 tiles)."""
    from paper_1304_7211_gb300 import rl
    lib = rl.load()
    spec = synth.disc(7)
    W, H, K = 2000, 1500, 13
    c = synth.make_case(W, H, spec, 0, "poisson", synth.SEED_BASE + 153)
    f = torch.from_numpy(c.f.astype(np.float32)).cuda()
    outs = []
    for flags in (rl.RL_FLAG_PERSISTENT, rl.RL_FLAG_PER_ITERATION):
        ctx = rl.rl_create(0, None, "f32", "mirror", "auto", flags)
        lib.rl_test_persist_ctas(ctas)
        try:
            rl.rl_set_psf(ctx, spec)
            u = torch.empty_like(f)
            st = rl.rl_iterate(ctx, f, None, u, W, H, W, K, rl.thinning(*thin) if thin else None, stats=True)
        finally:
            lib.rl_test_persist_ctas(0)
            rl.rl_destroy(ctx)
        torch.cuda.synchronize()
        outs.append((u, st))
    (ua, sa), (ub, sb) = outs
    assert sa.launches == 1 and sb.launches > 1
    assert torch.equal(ua, ub)
    assert sa.active_pixel_iterations == sb.active_pixel_iterations


@pytest.mark.parametrize("side,storage,thin,persistent", [
    (1024, "f32", False, False),   # 256 tiles, under 6 per SM: two launches
    (2048, "f32", False, True),    # 1024 tiles: persistent, 3 CTAs per SM
    (2048, "bf16", False, False),  # 16-bit plain keeps 1.25 tiles per resident CTA
    (2048, "bf16", True, True),    # thinned 16-bit: persistent
    (4096, "bf16", False, True)])
def test_launch_form_rule(side, storage, thin, persistent):
    """Without flags the size rule picks the form: persistent from about 6
    tiles per SM (FP32, or thinned), from 1.25 tiles per resident CTA slot
    for plain 16-bit storage; the two forms agree bit for bit, so only the
    launch count tells them apart."""
    from paper_1304_7211_gb300 import rl
    props = torch.cuda.get_device_properties(0)
    if props.multi_processor_count != 152:
        pytest.skip("the sizes assume a 152-SM GB300")
    dt = {"f32": torch.float32, "bf16": torch.bfloat16}[storage]
    torch.manual_seed(7)
    f = (torch.rand(side, side, device="cuda") * 100 + 5).to(dt)
    ctx = rl.rl_create(0, None, storage, "mirror", "auto", 0)
    try:
        rl.rl_set_psf(ctx, synth.disc(8))
        u = torch.empty_like(f)
        st = rl.rl_iterate(ctx, f, None, u, side, side, side, 4,
                           rl.thinning(1e-3, True, 10, 10) if thin else None, stats=True)
    finally:
        rl.rl_destroy(ctx)
    torch.cuda.synchronize()
    assert (st.launches == 1) == persistent
