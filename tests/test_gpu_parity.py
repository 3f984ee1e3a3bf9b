"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bar (FP32 storage): relative L-inf error <= 1e-4 against the oracle after 50
iterations, on seeded synthetic inputs at sizes that span several tiles with
ragged tails.  Cross-path agreement (running sum / span / stencil) uses the
same bound.  Thinned runs compare images within a bound derived from the
threshold and masks by the count of disagreeing pixels.
"""
import math

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


def gpu_rl(spec, f32, iters, path="auto", boundary="mirror", storage="f32", thin=None,
           u0=None, want_mask=False):
    from paper_1304_7211_gb300 import rl
    dt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[storage]
    f = torch.from_numpy(f32).cuda().to(dt)
    u0t = None if u0 is None else torch.from_numpy(u0).cuda().to(dt)
    with rl.Deconvolver(spec, device=0, storage=storage, boundary=boundary, path=path) as d:
        u, st = d.run(f, iters, u0=u0t, thin=thin, stats=True)
        mask = d.mask() if (want_mask and thin is not None) else None
    torch.cuda.synchronize()
    out = u.float().cpu().numpy().astype(np.float64)
    return (out, st, mask) if want_mask else (out, st)


def case(w, h, spec, noise="poisson", seed=synth.SEED_BASE + 50):
    c = synth.make_case(w, h, spec, 0, noise, seed)
    return c.f.astype(np.float32)


PATH_CASES = [
    (synth.motion(15, 0), "runsum"), (synth.motion(31, 0), "runsum"),
    (synth.motion(6, 0), "runsum"), (synth.motion(31, 1), "runsum"),
    (synth.motion(8, 1), "runsum"), (synth.disc(3), "span"), (synth.disc(8), "span"),
    (synth.motion(9, 0), "span"), (synth.motion(9, 1), "span"),
    (synth.gaussian(7, 1.5), "stencil"), (synth.disc(4), "stencil"),
    (synth.motion(11, 1), "stencil"),
]


@pytest.mark.parametrize("boundary", ["mirror", "clamp"])
@pytest.mark.parametrize("spec,path", PATH_CASES, ids=lambda v: getattr(v, "name", v))
def test_path_matches_oracle(spec, path, boundary):
    # 203 x 301: ragged against every tile width; > 256 rows for the y strips.
    f32 = case(203, 301, spec)
    u, st = gpu_rl(spec, f32, 50, path=path, boundary=boundary)
    ref = oracle.rl(f32.astype(np.float64), oracle_psf(spec), 50, boundary=boundary).u
    err = oracle.rel_linf(u, ref)
    assert err <= TOL, err
    assert st.path == {"runsum": 1, "span": 2, "stencil": 3}[path]


def test_asymmetric_dense_psf_off_centre_anchor():
    rng = np.random.default_rng(3)
    taps = rng.uniform(0.1, 1.0, size=(3, 5))
    spec = synth.PsfSpec("dense", taps=tuple(taps.reshape(-1)), kw=5, kh=3)
    spec_anchor = type("S", (), dict(kind="dense", taps=spec.taps, kw=5, kh=3,
                                     anchor_x=4, anchor_y=0, axis=0, length=0, radius=0))()
    f32 = case(130, 97, synth.gaussian(5, 1.0))
    for boundary in ("mirror", "clamp"):
        u, _ = gpu_rl(spec_anchor, f32, 30, path="stencil", boundary=boundary)
        psf = oracle.psf_dense(taps, 4, 0)
        ref = oracle.rl(f32.astype(np.float64), psf, 30, boundary=boundary).u
        assert oracle.rel_linf(u, ref) <= TOL


@pytest.mark.parametrize("boundary", ["mirror", "clamp"])
@pytest.mark.parametrize("k", [3, 5, 7, 9])
def test_asymmetric_centred_square_taps(k, boundary):
    # Centred odd square taps take the register-blocked stencil kernel; random
    # asymmetric taps catch a flipped or transposed tap index in either half.
    rng = np.random.default_rng(100 + k)
    taps = rng.uniform(0.05, 1.0, size=(k, k))
    spec = synth.dense(taps)
    f32 = case(203, 161, spec, seed=synth.SEED_BASE + 52)
    u, st = gpu_rl(spec, f32, 30, path="stencil", boundary=boundary)
    ref = oracle.rl(f32.astype(np.float64), oracle_psf(spec), 30, boundary=boundary).u
    assert oracle.rel_linf(u, ref) <= TOL
    assert st.path == 3
    # BF16 storage: K x unit roundoff against the oracle on the rounded f
    f_r = torch.from_numpy(f32).to(torch.bfloat16).float().numpy()
    u, _ = gpu_rl(spec, f_r, 30, path="stencil", boundary=boundary, storage="bf16")
    ref = oracle.rl(f_r.astype(np.float64), oracle_psf(spec), 30, boundary=boundary).u
    assert oracle.rel_linf(u, ref) <= 30 * 2.0 ** -9


@pytest.mark.parametrize("boundary", ["mirror", "clamp"])
@pytest.mark.parametrize("k", [3, 5, 9, 15, 23, 33])
def test_uniform_square_box(k, boundary):
    # A uniform centred odd square (Sec. 3, rectangular blur) takes the
    # register-blocked box kernel (path 2): separable sums, every radius
    # 1..16; 203 x 161 is ragged against the 64 x 64 tiles.
    spec = synth.dense(np.ones((k, k)))
    f32 = case(203, 161, spec, seed=synth.SEED_BASE + 53)
    u, st = gpu_rl(spec, f32, 30, boundary=boundary)
    assert st.path == 2
    ref = oracle.rl(f32.astype(np.float64), oracle_psf(spec), 30, boundary=boundary).u
    assert oracle.rel_linf(u, ref) <= TOL
    # the generic stencil tiles compute the same convolution tap by tap
    if k <= 15:
        v, sv = gpu_rl(spec, f32, 30, path="stencil", boundary=boundary)
        assert sv.path == 3
        assert oracle.rel_linf(u, v) <= TOL


def anchored(taps, ax, ay):
    """Dense taps with an explicit anchor, as the PSF descriptor takes them."""
    t = np.asarray(taps, np.float64)
    return type("S", (), dict(kind="dense", taps=tuple(t.reshape(-1)), kw=t.shape[1], kh=t.shape[0],
                              anchor_x=ax, anchor_y=ay, axis=0, length=0, radius=0,
                              name=f"rect{t.shape[0]}x{t.shape[1]}_a{ax}_{ay}", t=t))()


# (rows, cols, anchor x, anchor y): centred and off-centre, even and odd,
# thin in either axis, reaching 1..16 pixels from the anchor
RECTS = [(3, 5, 2, 1), (9, 31, 15, 4), (31, 9, 4, 15), (1, 17, 8, 0), (17, 1, 0, 8), (8, 8, 4, 4),
         (6, 11, 0, 0), (2, 33, 16, 1), (12, 4, 3, 11), (21, 15, 7, 10)]


@pytest.mark.parametrize("boundary", ["mirror", "clamp"])
@pytest.mark.parametrize("rect", RECTS, ids=lambda r: "x".join(map(str, r)))
def test_uniform_rectangle(rect, boundary):
    # A uniform rectangle of any anchor within 16 pixels (Sec. 3,
    # rectangular blur) takes the register-blocked rectangle kernel on the
    # span path: vertical sums in shared memory, horizontal sums slid along
    # them.
    kh, kw, ax, ay = rect
    spec = anchored(np.ones((kh, kw)), ax, ay)
    f32 = case(203, 161, synth.disc(2), seed=synth.SEED_BASE + 55)
    u, st = gpu_rl(spec, f32, 30, path="span", boundary=boundary)
    assert st.path == 2
    ref = oracle.rl(f32.astype(np.float64), oracle.psf_dense(spec.t, ax, ay), 30, boundary=boundary).u
    assert oracle.rel_linf(u, ref) <= TOL


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("shape", [(11, 11), (7, 15)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_uniform_box_and_rectangle_reduced_storage(storage, shape):
    # RL under a box PSF amplifies a perturbation of u by more than the
    # factor one the general storage test assumes, so the bound here is
    # measured on the oracle itself: its FP64 iterates with u rounded to the
    # storage format after every iteration (what 16-bit storage does) drift
    # from the unrounded ones by e; the GPU may differ from the unrounded
    # oracle by 2 e (its FP32 arithmetic flips some of the rounding
    # decisions).
    K = 30
    spec = synth.dense(np.ones(shape))
    f32 = case(150, 133, spec, seed=synth.SEED_BASE + 54)
    dt = {"bf16": torch.bfloat16, "f16": torch.float16}[storage]
    f_r = torch.from_numpy(f32).to(dt).float().numpy()
    u, st = gpu_rl(spec, f_r, K, storage=storage)
    assert st.path == 2
    f64, psf = f_r.astype(np.float64), oracle_psf(spec)
    ref = oracle.rl(f64, psf, K).u
    rounded = f64
    for _ in range(K):
        rounded = oracle.rl(f64, psf, 1, u0=rounded).u
        rounded = torch.from_numpy(rounded).to(dt).double().numpy()
    e = oracle.rel_linf(rounded, ref)
    assert e >= UNIT_ROUNDOFF[storage] / 2  # the rounding did happen
    assert oracle.rel_linf(u, ref) <= 2 * e


def test_uniform_rectangle_from_dense_taps_auto_path():
    # uniform centred squares: the box kernel; other uniform rectangles
    # within 2 pixels of the anchor: the register stencil; up to 16: the
    # rectangle kernel; beyond: the span tiles
    for shape, path in (((3, 5), 3), ((3, 11), 2), ((13, 1), 2), ((5, 5), 2), ((35, 35), 2), ((3, 41), 2),
                        ((9, 7), 2), ((7, 3), 2)):
        spec = synth.dense(np.ones(shape))
        f32 = case(150, 90, spec)
        u, st = gpu_rl(spec, f32, 40)
        assert st.path == path
        ref = oracle.rl(f32.astype(np.float64), oracle_psf(spec), 40).u
        assert oracle.rel_linf(u, ref) <= TOL


@pytest.mark.parametrize("spec,paths", [(synth.motion(31, 0), ("runsum", "span", "stencil")),
                                        (synth.motion(31, 1), ("runsum", "span", "stencil")),
                                        (synth.disc(8), ("span", "stencil"))],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_cross_path_agreement(spec, paths):
    f32 = case(257, 263, spec, seed=synth.SEED_BASE + 51)
    outs = [gpu_rl(spec, f32, 50, path=p)[0] for p in paths]
    for o in outs[1:]:
        assert oracle.rel_linf(o, outs[0]) <= TOL


@pytest.mark.parametrize("spec", [synth.motion(5, 0), synth.motion(5, 1), synth.disc(1),
                                  synth.gaussian(3, 0.8)], ids=lambda s: s.name)
@pytest.mark.parametrize("shape", [(1, 7), (7, 1), (6, 6), (3, 40), (65, 2), (17, 33)])
def test_small_and_degenerate_shapes(spec, shape):
    H, W = shape
    t = spec.dense()
    if t.shape[1] // 2 >= W or t.shape[0] // 2 >= H:
        pytest.skip("PSF larger than the image")
    rng = np.random.default_rng(H * 100 + W)
    f32 = rng.uniform(5, 250, size=(H, W)).astype(np.float32)
    u, _ = gpu_rl(spec, f32, 12)
    ref = oracle.rl(f32.astype(np.float64), oracle_psf(spec), 12).u
    assert oracle.rel_linf(u, ref) <= TOL


def test_delta_psf_and_zero_iterations():
    f32 = case(70, 50, synth.motion(1, 0))
    u, _ = gpu_rl(synth.motion(1, 0), f32, 5)
    np.testing.assert_allclose(u, f32, rtol=1e-6)
    u0 = np.full_like(f32, 3.0)
    u, _ = gpu_rl(synth.disc(2), f32, 0, u0=u0)
    np.testing.assert_array_equal(u, u0)


def test_explicit_u0_and_aliasing_and_pitch():
    from paper_1304_7211_gb300 import rl
    spec = synth.disc(3)
    f32 = case(120, 77, spec)
    u0 = (f32 * 0.5 + 10).astype(np.float32)
    ref = oracle.rl(f32.astype(np.float64), oracle_psf(spec), 7,
                    u0=u0.astype(np.float64)).u
    # pitched buffers: rows of 128 elements
    fpad = torch.zeros((77, 128), device="cuda")
    fpad[:, :120] = torch.from_numpy(f32).cuda()
    upad = torch.zeros((77, 128), device="cuda")
    upad[:, :120] = torch.from_numpy(u0).cuda()
    with rl.Deconvolver(spec) as d:
        for iters in (1, 7):
            buf = upad.clone()
            rl.rl_iterate(d.ctx, fpad, buf, buf, 120, 77, 128, iters)  # u_out aliases u0
            torch.cuda.synchronize()
            if iters == 7:
                err = oracle.rel_linf(buf[:, :120].cpu().numpy(), ref)
                assert err <= TOL
            assert torch.all(buf[:, 120:] == 0)  # padding untouched


def test_host_buffers_are_staged():
    from paper_1304_7211_gb300 import rl
    spec = synth.motion(15, 0)
    f32 = case(200, 64, spec)
    with rl.Deconvolver(spec) as d:
        u = d.run(f32, 20)  # numpy in, numpy out
    ref = oracle.rl(f32.astype(np.float64), oracle_psf(spec), 20).u
    assert oracle.rel_linf(u, ref) <= TOL


def test_errors_are_reported():
    from paper_1304_7211_gb300 import rl
    ctx = rl.rl_create(0)
    try:
        f = torch.ones((8, 8), device="cuda")
        with pytest.raises(rl.RLError) as e:
            rl.rl_iterate(ctx, f, None, f.clone(), 8, 8, 8, 3)
        assert e.value.status == rl.RL_ERR_STATE
        rl.rl_set_psf(ctx, synth.disc(8))  # extent 8 >= 8
        with pytest.raises(rl.RLError) as e:
            rl.rl_iterate(ctx, f, None, f.clone(), 8, 8, 8, 3)
        assert e.value.status == rl.RL_ERR_INVALID_ARG
        with pytest.raises(rl.RLError) as e:
            rl.rl_iterate(ctx, f, None, f, 8, 8, 8, 3)  # u_out aliases f
        assert e.value.status == rl.RL_ERR_INVALID_ARG
        with pytest.raises(rl.RLError) as e:
            rl.rl_set_psf(ctx, synth.dense([[1.0, -1.0, 1.0]]))
        assert e.value.status == rl.RL_ERR_INVALID_ARG
        with pytest.raises(rl.RLError) as e:
            rl.rl_set_psf(ctx, synth.dense([[0.0, 0.0]]))
        assert e.value.status == rl.RL_ERR_INVALID_ARG
    finally:
        rl.rl_destroy(ctx)
    ctx = rl.rl_create(0, path="runsum")
    try:
        with pytest.raises(rl.RLError) as e:
            rl.rl_set_psf(ctx, synth.disc(3))
        assert e.value.status == rl.RL_ERR_UNSUPPORTED
    finally:
        rl.rl_destroy(ctx)
    ctx = rl.rl_create(0, path="span")
    try:
        with pytest.raises(rl.RLError) as e:
            rl.rl_set_psf(ctx, synth.gaussian(5, 1.0))
        assert e.value.status == rl.RL_ERR_UNSUPPORTED
    finally:
        rl.rl_destroy(ctx)


# ---- invariants at the benchmark size ----------------------------------------

@pytest.mark.parametrize("spec", synth.CONFIG2_PSFS, ids=lambda s: s.name)
def test_full_size_launch_configuration(spec):
    """2048 x 2048 in the benchmark's launch configuration: element-wise
    parity with the oracle after 3 iterations, and flux / nonnegativity after
    the full 200 iterations."""
    c = synth.config2(spec)
    f32 = c.f.astype(np.float32)
    f64 = f32.astype(np.float64)
    u3, _ = gpu_rl(spec, f32, 3)
    ref3 = oracle.rl(f64, oracle_psf(spec), 3).u
    assert oracle.rel_linf(u3, ref3) <= TOL
    u, st = gpu_rl(spec, f32, c.iterations)
    assert u.min() >= 0.0
    assert abs(u.sum() - f64.sum()) <= 1e-4 * f64.sum()


@pytest.mark.parametrize("spec", synth.CONFIG2_PSFS, ids=lambda s: s.name)
def test_200_iterations_against_oracle(spec):
    """The full iteration count of the 2048 x 2048 workload on a 512 x 512
    image from the same generator: element-wise parity after 200 iterations."""
    c = synth.config2(spec, size=512)
    f32 = c.f.astype(np.float32)
    u, _ = gpu_rl(spec, f32, c.iterations)
    ref = oracle.rl(f32.astype(np.float64), oracle_psf(spec), c.iterations).u
    err = oracle.rel_linf(u, ref)
    print(f"{spec.name}: 200 it rel_linf={err:.3e}")
    assert err <= TOL


def test_constant_image_is_reproduced():
    f32 = np.full((300, 310), 77.0, np.float32)
    for spec in (synth.motion(31, 0), synth.motion(31, 1), synth.disc(8), synth.gaussian(7, 1.5)):
        for boundary in ("mirror", "clamp"):
            u, _ = gpu_rl(spec, f32, 20, boundary=boundary)
            np.testing.assert_allclose(u, 77.0, rtol=2e-6)


# ---- storage modes --------------------------------------------------------------

# Unit roundoff of the storage format: bf16 keeps 8 significant bits, f16 11.
UNIT_ROUNDOFF = {"bf16": 2.0 ** -9, "f16": 2.0 ** -11}


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("spec", [synth.motion(15, 0), synth.motion(15, 1), synth.disc(4),
                                  synth.gaussian(7, 1.5)], ids=lambda s: s.name)
def test_reduced_precision_storage(spec, storage):
    """BF16/FP16 storage of f and u with FP32 arithmetic.  Every iteration
    rounds u once to the storage format (relative error <= unit roundoff),
    and the multiplicative update carries a relative error of u into u' with
    factor about one, so after K iterations the error against the FP64 oracle
    (run on the same rounded f) is bounded by K times the unit roundoff."""
    K = 30
    tol = K * UNIT_ROUNDOFF[storage]
    f32 = case(180, 140, spec)
    dt = {"bf16": torch.bfloat16, "f16": torch.float16}[storage]
    f_r = torch.from_numpy(f32).to(dt).float().numpy()
    u, _ = gpu_rl(spec, f_r, K, storage=storage)
    ref = oracle.rl(f_r.astype(np.float64), oracle_psf(spec), K).u
    err = oracle.rel_linf(u, ref)
    print(f"{storage} {spec.name}: rel_linf={err:.2e}")
    assert err <= tol


# ---- selective convolution (Eq. 4-5) -------------------------------------------

def test_zero_threshold_equals_plain():
    from paper_1304_7211_gb300 import rl
    for spec in (synth.motion(15, 0), synth.motion(15, 1), synth.disc(4), synth.gaussian(7, 1.5)):
        f32 = case(150, 120, spec)
        plain, _ = gpu_rl(spec, f32, 25)
        for q in (1, 10):
            thin, st = gpu_rl(spec, f32, 25, thin=rl.thinning(0.0, update_period=q))
            np.testing.assert_array_equal(thin, plain)
            assert st.active_pixel_iterations == 150 * 120 * 25


def test_infinite_threshold_keeps_only_full_iterations():
    from paper_1304_7211_gb300 import rl
    for spec in (synth.motion(15, 0), synth.motion(15, 1), synth.disc(4)):
        f32 = case(140, 110, spec)
        for K in (9, 10, 11, 23):
            thin, st = gpu_rl(spec, f32, K, thin=rl.thinning(math.inf))
            plain, _ = gpu_rl(spec, f32, -(-K // 10))
            np.testing.assert_array_equal(thin, plain)
            assert st.active_pixel_iterations == 140 * 110 * (-(-K // 10))


THIN_CASES = [(True, 1e-4, 1), (True, 1e-3, 1), (True, 1e-4, 10), (False, 0.01, 1),
              (False, 0.05, 10)]
THIN_PATHS = [(synth.disc(4), "span"), (synth.disc(4), "stencil"), (synth.motion(15, 0), "runsum"),
              (synth.motion(15, 1), "runsum"), (synth.dense(np.ones((7, 7))), "span"),
              (synth.dense(np.ones((5, 13))), "span")]


@pytest.mark.parametrize("relative,tau,q", THIN_CASES)
@pytest.mark.parametrize("spec,path", THIN_PATHS, ids=lambda v: getattr(v, "name", v))
def test_thinned_replay_matches_oracle(spec, path, relative, tau, q):
    """The oracle's per-iteration used-pixel masks (Eq. 4-5) replayed on the
    GPU: same selective convolutions, so the images agree to 1e-4 and the
    active pixel-iteration counts exactly."""
    from paper_1304_7211_gb300 import rl
    K = 34
    f32 = case(170, 150, spec, seed=synth.SEED_BASE + 52)
    res = oracle.rl(f32.astype(np.float64), oracle_psf(spec), K, threshold=tau,
                    relative=relative, update_period=q, want_mask=True)
    sched = np.ascontiguousarray(res.mask_trace)
    u, st = gpu_rl(spec, f32, K, path=path, thin=rl.thinning(tau, relative, 10, q, schedule=sched))
    err = oracle.rel_linf(u, res.u)
    assert err <= TOL, err
    assert st.active_pixel_iterations == res.active_pixel_iterations
    assert res.active_pixel_iterations < K * f32.size  # thinning did something


@pytest.mark.parametrize("relative,tau,q", THIN_CASES)
@pytest.mark.parametrize("spec,path", THIN_PATHS, ids=lambda v: getattr(v, "name", v))
def test_thinned_free_running_masks(spec, path, relative, tau, q):
    """GPU decisions (FP32) against the oracle's (FP64): the final masks are
    compared by the count of disagreeing pixels, the active counts by their
    relative difference.  A disagreement needs a change within rounding of
    the threshold, so both stay tiny.  The image difference those flips cause
    depends on the PSF, so its bound is measured on the oracle: its own
    iterates with tau moved by 1e-3 relative (the FP32 rounding of the Eq. 4
    statistic near tau = 1e-4) differ by `spread`; the GPU may differ by
    twice that, and never needs to be closer than 1e-2."""
    from paper_1304_7211_gb300 import rl
    K = 34
    f32 = case(170, 150, spec, seed=synth.SEED_BASE + 52)
    f64 = f32.astype(np.float64)
    th = rl.thinning(tau, relative=relative, update_period=q)
    u, st, mask = gpu_rl(spec, f32, K, path=path, thin=th, want_mask=True)
    res = oracle.rl(f64, oracle_psf(spec), K, threshold=tau, relative=relative, update_period=q)
    nxt = oracle.rl(f64, oracle_psf(spec), K + 1, threshold=tau, relative=relative,
                    update_period=q, want_mask=True).mask_trace[K]
    dis = int(np.sum(mask != nxt))
    act_rel = abs(st.active_pixel_iterations - res.active_pixel_iterations) / res.active_pixel_iterations
    err = oracle.rel_linf(u, res.u)
    print(f"{spec.name} {path} tau={tau} q={q}: mask_disagree={dis}/{mask.size} "
          f"act_rel={act_rel:.2e} image_rel_linf={err:.2e}")
    assert dis <= 0.005 * mask.size
    assert act_rel <= 0.005
    spread = max(oracle.rel_linf(oracle.rl(f64, oracle_psf(spec), K, threshold=tau * (1 + d), relative=relative,
                                           update_period=q).u, res.u) for d in (1e-3, -1e-3))
    assert err <= max(1e-2, 2 * spread)


# ---- running sum: whole rows resident vs one launch per iteration -------------

def run_flags(spec, f32, iters, flags, boundary="mirror", storage="f32", thin=None):
    from paper_1304_7211_gb300 import rl
    dt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[storage]
    f = torch.from_numpy(f32).cuda().to(dt)
    with rl.Deconvolver(spec, storage=storage, boundary=boundary, path="runsum", flags=flags) as d:
        u, st = d.run(f, iters, thin=thin, stats=True)
        m = d.mask() if thin is not None and thin.schedule is None else None
    torch.cuda.synchronize()
    return u.float().cpu().numpy(), st, m


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("boundary", ["mirror", "clamp"])
@pytest.mark.parametrize("spec", [synth.motion(15, 0), synth.motion(8, 0), synth.motion(15, 1),
                                  synth.motion(8, 1)], ids=lambda s: s.name)
def test_resident_rows_match_per_iteration(spec, boundary, storage):
    from paper_1304_7211_gb300 import rl
    f32 = case(203, 157, spec, seed=synth.SEED_BASE + 53)
    res, _, _ = run_flags(spec, f32, 23, 0, boundary, storage)
    per, _, _ = run_flags(spec, f32, 23, rl.RL_FLAG_PER_ITERATION, boundary, storage)
    # same iteration, running sums restarted at different chunk boundaries
    tol = 1e-5 if storage == "f32" else 23 * UNIT_ROUNDOFF["bf16"]
    assert oracle.rel_linf(res, per) <= tol


@pytest.mark.parametrize("q", [1, 10])
@pytest.mark.parametrize("spec", [synth.motion(15, 0), synth.motion(15, 1)], ids=lambda s: s.name)
def test_resident_rows_thinning(spec, q):
    from paper_1304_7211_gb300 import rl
    f32 = case(170, 150, spec, seed=synth.SEED_BASE + 52)
    th = rl.thinning(1e-3, update_period=q)
    res, st_r, m_r = run_flags(spec, f32, 34, 0, thin=th)
    per, st_p, m_p = run_flags(spec, f32, 34, rl.RL_FLAG_PER_ITERATION, thin=th)
    assert int(np.sum(m_r != m_p)) <= 0.005 * m_r.size
    assert abs(st_r.active_pixel_iterations - st_p.active_pixel_iterations) <= \
        0.005 * st_p.active_pixel_iterations
    # replay of the oracle's schedule through the resident kernel
    resq = oracle.rl(f32.astype(np.float64), oracle_psf(spec), 34, threshold=1e-3,
                     update_period=q, want_mask=True)
    th2 = rl.thinning(1e-3, update_period=q, schedule=np.ascontiguousarray(resq.mask_trace))
    rep, st, _ = run_flags(spec, f32, 34, 0, thin=th2)
    assert oracle.rel_linf(rep, resq.u) <= TOL
    assert st.active_pixel_iterations == resq.active_pixel_iterations


# ---- CUDA-graph replay of iteration segments ------------------------------------

@pytest.mark.parametrize("thin", [None, (2e-3, True, 10, 1), (2e-3, True, 10, 10)])
@pytest.mark.parametrize("spec", [synth.disc(4), synth.gaussian(7, 1.5), synth.motion(9, 0)],
                         ids=lambda s: s.name)
def test_graph_replay_matches_direct_launches(spec, thin):
    """On an explicit stream the middle iterations are replayed from a captured
    CUDA graph; on the legacy default stream they are launched one by one.
    Same kernels, same arguments: identical images, masks and counts."""
    from paper_1304_7211_gb300 import rl
    f32 = case(190, 170, spec, seed=synth.SEED_BASE + 54)
    outs = []
    for use_stream in (False, True):
        s = torch.cuda.Stream() if use_stream else None
        ctx_stream = s.cuda_stream if s is not None else None
        with torch.cuda.stream(s) if s is not None else torch.cuda.stream(torch.cuda.default_stream()):
            f = torch.from_numpy(f32).cuda()
            u = torch.empty_like(f)
            ctx = rl.rl_create(0, ctx_stream)
            try:
                rl.rl_set_psf(ctx, spec)
                th = rl.thinning(*thin) if thin else None
                for _ in range(2):  # the second call reuses the cached graph
                    st = rl.rl_iterate(ctx, f, None, u, 190, 170, 190, 47, th, stats=True)
                m = np.zeros((170, 190), np.uint8)
                if thin:
                    rl.rl_get_mask(ctx, m, 190)
            finally:
                rl.rl_destroy(ctx)
            torch.cuda.synchronize()
            outs.append((u.cpu().numpy(), m, st.active_pixel_iterations, st.launches))
    (u0, m0, a0, l0), (u1, m1, a1, l1) = outs
    np.testing.assert_array_equal(u0, u1)
    np.testing.assert_array_equal(m0, m1)
    assert a0 == a1 and l0 == l1


def test_flux_diagnostics():
    from paper_1304_7211_gb300 import rl
    for spec in (synth.disc(5), synth.motion(13, 1), synth.gaussian(7, 1.5)):
        f32 = case(230, 170, spec, seed=synth.SEED_BASE + 55)
        _, st = gpu_rl(spec, f32, 30)
        ref = float(f32.astype(np.float64).sum())
        assert abs(st.flux_f - ref) <= 1e-12 * ref
        assert abs(st.flux_u - st.flux_f) <= 2e-5 * st.flux_f  # flux conservation
