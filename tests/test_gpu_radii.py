"""GPU parity for every compiled radius and for the 4096 x 4096 workload's PSF.

The disc (Sec. 3 "Defocus blur") and the uniform square box (Sec. 3
"Rectangular blur") kernels are compiled once per radius 1..16; each radius
is checked here against the FP64 oracle on a small image that is ragged
against the 64 x 64 tiles.  The thinned workload's PSF, the disc of radius
12, is checked at several tiles with both boundaries, with the oracle's
thinning schedule replayed (mask recomputed every 10 iterations, Eq. 4-5,
relative thresholds 1e-3 / 1e-4 / 1e-5) and with BF16 storage.
"""
import numpy as np
import pytest

import oracle
from paper_1304_7211_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-4
BF16_U = 2.0 ** -9  # unit roundoff of BF16 (8 significant bits)

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


def gpu_rl(spec, f32, iters, boundary="mirror", storage="f32", thin=None, path="auto"):
    from paper_1304_7211_gb300 import rl
    dt = {"f32": torch.float32, "bf16": torch.bfloat16}[storage]
    f = torch.from_numpy(f32).cuda().to(dt)
    with rl.Deconvolver(spec, device=0, storage=storage, boundary=boundary, path=path) as d:
        u, st = d.run(f, iters, thin=thin, stats=True)
    torch.cuda.synchronize()
    return u.float().cpu().numpy().astype(np.float64), st


def case(w, h, spec, seed):
    return synth.make_case(w, h, spec, 0, "poisson", seed).f.astype(np.float32)


@pytest.mark.parametrize("radius", range(1, 17))
def test_every_disc_radius(radius):
    # 150 x 97: ragged in both axes; the largest disc (33 pixels) still fits
    spec = synth.disc(radius)
    f32 = case(150, 97, spec, synth.SEED_BASE + 80 + radius)
    boundary = "clamp" if radius % 4 == 0 else "mirror"
    u, st = gpu_rl(spec, f32, 30, boundary=boundary)
    assert st.path == 2
    ref = oracle.rl(f32.astype(np.float64), oracle_psf(spec), 30, boundary=boundary).u
    err = oracle.rel_linf(u, ref)
    assert err <= TOL, err


@pytest.mark.parametrize("radius", range(1, 17))
def test_every_box_radius(radius):
    k = 2 * radius + 1
    spec = synth.dense(np.ones((k, k)))
    f32 = case(150, 97, spec, synth.SEED_BASE + 100 + radius)
    boundary = "mirror" if radius % 3 else "clamp"
    u, st = gpu_rl(spec, f32, 20, boundary=boundary)
    assert st.path == 2
    ref = oracle.rl(f32.astype(np.float64), oracle_psf(spec), 20, boundary=boundary).u
    err = oracle.rel_linf(u, ref)
    assert err <= TOL, err


@pytest.mark.parametrize("boundary", ["mirror", "clamp"])
def test_disc12_several_tiles_50_iterations(boundary):
    # 203 x 157 spans 4 x 3 tiles with ragged right and bottom edges
    spec = synth.disc(12)
    f32 = case(203, 157, spec, synth.SEED_BASE + 120)
    u, _ = gpu_rl(spec, f32, 50, boundary=boundary)
    ref = oracle.rl(f32.astype(np.float64), oracle_psf(spec), 50, boundary=boundary).u
    err = oracle.rel_linf(u, ref)
    print(f"disc12 {boundary}: rel_linf={err:.2e}")
    assert err <= TOL, err


@pytest.mark.parametrize("tau", [1e-3, 1e-4, 1e-5])
def test_disc12_thinned_replay(tau):
    """The thinned workload's selective convolution (relative threshold, mask
    recomputed on full iterations, reset every 10) with the oracle's masks
    replayed: images within 1e-4 and identical active pixel-iteration counts."""
    from paper_1304_7211_gb300 import rl
    spec = synth.disc(12)
    K = 30
    f32 = case(203, 157, spec, synth.SEED_BASE + 121)
    res = oracle.rl(f32.astype(np.float64), oracle_psf(spec), K, threshold=tau, relative=True,
                    update_period=10, want_mask=True)
    sched = np.ascontiguousarray(res.mask_trace)
    u, st = gpu_rl(spec, f32, K, thin=rl.thinning(tau, True, 10, 10, schedule=sched))
    err = oracle.rel_linf(u, res.u)
    print(f"disc12 tau={tau}: rel_linf={err:.2e} active={res.active_pixel_iterations / (K * f32.size):.3f}")
    assert err <= TOL, err
    assert st.active_pixel_iterations == res.active_pixel_iterations


def test_disc12_bf16_storage():
    """BF16 storage, FP32 arithmetic: u is rounded once per iteration, so after
    K iterations the error against the oracle on the same rounded f is at
    most K unit roundoffs."""
    spec = synth.disc(12)
    K = 30
    f32 = case(203, 157, spec, synth.SEED_BASE + 122)
    f_r = torch.from_numpy(f32).to(torch.bfloat16).float().numpy()
    u, _ = gpu_rl(spec, f_r, K, storage="bf16")
    ref = oracle.rl(f_r.astype(np.float64), oracle_psf(spec), K).u
    err = oracle.rel_linf(u, ref)
    print(f"disc12 bf16: rel_linf={err:.2e} (bound {K * BF16_U:.2e})")
    assert err <= K * BF16_U


def test_bf16_jobs_through_the_batch_executor():
    """BF16 jobs submitted to rl_batch give the same bits as alone, and match
    the oracle on the rounded f within K unit roundoffs."""
    from paper_1304_7211_gb300 import rl
    specs = [synth.disc(5), synth.motion(11, 0), synth.motion(9, 1), synth.gaussian(7, 1.5)]
    jobs = []
    for j, spec in enumerate(specs):
        W, H = 97 + 31 * j, 131 - 17 * j
        f32 = case(W, H, spec, synth.SEED_BASE + 130 + j)
        f = torch.from_numpy(f32).cuda().to(torch.bfloat16)
        jobs.append((spec, f, torch.empty_like(f), 20, W, H))
    with rl.Batch(slots=3, storage="bf16") as b:
        for spec, f, u, its, W, H in jobs:
            b.submit(spec, f, u, its, W, H)
        b.sync()
    for spec, f, u, its, W, H in jobs:
        with rl.Deconvolver(spec, storage="bf16") as d:
            alone = d.run(f, its)
        torch.cuda.synchronize()
        assert torch.equal(u, alone)
        f_r = f.float().cpu().numpy().astype(np.float64)
        ref = oracle.rl(f_r, oracle_psf(spec), its).u
        err = oracle.rel_linf(u.float().cpu().numpy(), ref)
        assert err <= its * BF16_U, (spec.name, err)
