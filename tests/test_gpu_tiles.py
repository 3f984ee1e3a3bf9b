"""GPU: the batched (request, tile) form, rl_iterate_tiles.

Jobs under one disc or box PSF run as one launch pair per iteration over the
tiles of every job still iterating.  The kernels' per-tile code is the one
rl_iterate runs, so each job's image must equal its single-image solve
bitwise, whatever the mix of sizes and iteration counts; one job is also
checked against the FP64 oracle.
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


# (W, H, iterations): ragged and exact tile multiples, a job smaller than a
# tile, a job with no iterations, and ties in the iteration count
SHAPES = [(150, 117, 30), (64, 64, 12), (300, 70, 30), (33, 21, 7), (129, 200, 0), (257, 65, 19), (40, 40, 30)]


def images(seed):
    out = []
    for i, (W, H, _) in enumerate(SHAPES):
        c = synth.make_case(W, H, synth.disc(2), 0, "poisson", seed + i)
        out.append(torch.from_numpy(c.f.astype(np.float32)).cuda())
    return out


@pytest.mark.parametrize("boundary", ["mirror", "clamp"])
@pytest.mark.parametrize("spec", [synth.disc(4), synth.disc(1), synth.disc(13), synth.dense(np.ones((7, 7))),
                                  synth.dense(np.ones((15, 15)))], ids=lambda s: s.name)
def test_tiles_equal_single_solves(spec, boundary):
    from paper_1304_7211_gb300 import rl
    fs = images(synth.SEED_BASE + 80)
    r = max(spec.dense().shape) // 2
    keep = [j for j, (W, H, _) in enumerate(SHAPES) if r < W and r < H]
    outs = [torch.full_like(f, -1.0) for f in fs]
    with rl.Deconvolver(spec, boundary=boundary) as d:
        rl.rl_iterate_tiles(d.ctx, [(fs[j], None, outs[j], SHAPES[j][0], SHAPES[j][1], SHAPES[j][0], SHAPES[j][2])
                                    for j in keep])
        torch.cuda.synchronize()
        for j in keep:
            W, H, K = SHAPES[j]
            ref = torch.empty_like(fs[j])
            rl.rl_iterate(d.ctx, fs[j], None, ref, W, H, W, K)
            torch.cuda.synchronize()
            assert torch.equal(outs[j], ref), (j, SHAPES[j])
    j = 0
    W, H, K = SHAPES[j]
    f64 = fs[j].cpu().numpy().astype(np.float64)
    t = spec.dense()
    want = oracle.rl(f64, oracle.psf_dense(t, t.shape[1] // 2, t.shape[0] // 2), K, boundary=boundary).u
    assert oracle.rel_linf(outs[j].cpu().numpy().astype(np.float64), want) <= TOL


def test_tiles_u0_and_aliasing():
    from paper_1304_7211_gb300 import rl
    spec = synth.disc(5)
    fs = images(synth.SEED_BASE + 81)[:3]
    u0s = [f * 0.5 + 3.0 for f in fs]
    ref = []
    with rl.Deconvolver(spec) as d:
        for j, f in enumerate(fs):
            W, H, K = SHAPES[j]
            r = torch.empty_like(f)
            rl.rl_iterate(d.ctx, f, u0s[j], r, W, H, W, K)
            ref.append(r)
        # u_out aliasing u0: the result replaces the start image
        rl.rl_iterate_tiles(d.ctx, [(fs[j], u0s[j], u0s[j], SHAPES[j][0], SHAPES[j][1], SHAPES[j][0],
                                     SHAPES[j][2]) for j in range(3)])
        torch.cuda.synchronize()
    for j in range(3):
        assert torch.equal(u0s[j], ref[j])


def test_tiles_pitched_rows():
    # a row pitch larger than W on input and output
    from paper_1304_7211_gb300 import rl
    spec = synth.dense(np.ones((5, 5)))
    W, H, K, P = 150, 90, 20, 192
    f = images(synth.SEED_BASE + 82)[0][:H, :W].contiguous()
    fp = torch.zeros((H, P), device="cuda")
    fp[:, :W] = f
    out = torch.full((H, P), -7.0, device="cuda")
    with rl.Deconvolver(spec) as d:
        rl.rl_iterate_tiles(d.ctx, [(fp, None, out, W, H, P, K)])
        ref = torch.empty_like(f)
        rl.rl_iterate(d.ctx, f, None, ref, W, H, W, K)
        torch.cuda.synchronize()
    assert torch.equal(out[:, :W], ref)
    assert torch.all(out[:, W:] == -7.0)


def test_tiles_errors():
    from paper_1304_7211_gb300 import rl
    f = torch.ones((80, 80), device="cuda")
    u = torch.empty_like(f)
    job = [(f, None, u, 80, 80, 80, 3)]
    for spec, kw in ((synth.motion(9, 0), {}), (synth.gaussian(7, 1.5), {}), (synth.disc(4), {"storage": "bf16"}),
                     (synth.disc(4), {"boundary": "clamp", "adjoint": "transpose"}),
                     (synth.dense(np.ones((3, 5))), {})):
        with rl.Deconvolver(spec, **kw) as d:
            with pytest.raises(rl.RLError) as e:
                rl.rl_iterate_tiles(d.ctx, job)
            assert e.value.status == rl.RL_ERR_UNSUPPORTED
    with rl.Deconvolver(synth.disc(4)) as d:
        host = np.ones((80, 80), np.float32)
        with pytest.raises(rl.RLError) as e:
            rl.rl_iterate_tiles(d.ctx, [(host, None, u, 80, 80, 80, 3)])
        assert e.value.status == rl.RL_ERR_INVALID_ARG
        with pytest.raises(rl.RLError) as e:  # PSF wider than the image
            rl.rl_iterate_tiles(d.ctx, [(f, None, u, 4, 80, 80, 3)])
        assert e.value.status == rl.RL_ERR_INVALID_ARG
        rl.rl_iterate_tiles(d.ctx, [])  # no jobs: nothing to do


@pytest.mark.parametrize("spec", [synth.disc(8), synth.dense(np.ones((9, 9)))], ids=lambda s: s.name)
def test_persistent_tiles_equal_launch_per_iteration(spec):
    """The batched form's one persistent launch (every iteration of every job)
    against its launch pair per iteration (RL_FLAG_PER_ITERATION): same tile
    arithmetic, so the same bits, for a mix of 24 sizes and iteration counts."""
    from paper_1304_7211_gb300 import rl
    rng = np.random.default_rng(synth.SEED_BASE + 83)
    jobs = []
    for j in range(24):
        W, H = int(rng.integers(40, 400)), int(rng.integers(40, 400))
        K = int(rng.integers(0, 45))
        c = synth.make_case(W, H, spec, 0, "poisson", synth.SEED_BASE + 300 + j)
        jobs.append((torch.from_numpy(c.f.astype(np.float32)).cuda(), W, H, K))
    outs = []
    for flags in (rl.RL_FLAG_PERSISTENT, rl.RL_FLAG_PER_ITERATION):
        us = [torch.full_like(f, -1.0) for f, *_ in jobs]
        with rl.Deconvolver(spec, flags=flags) as d:
            rl.rl_iterate_tiles(d.ctx, [(f, None, u, W, H, W, K) for (f, W, H, K), u in zip(jobs, us)])
        torch.cuda.synchronize()
        outs.append(us)
    for a, b in zip(*outs):
        assert torch.equal(a, b)
