"""GPU parity of the exact-transpose adjoint (rl_config flag
RL_FLAG_ADJOINT_TRANSPOSE) against the oracle's A^T.

Where the pad-flip operator of Eq. 3 (h reflected about the origin with the
same boundary continuation, Sec. 2) is not the transpose of the forward
operator -- any PSF under clamp, an axis-asymmetric PSF under the mirror --
the library folds the zero-padded correlation of q back onto the pixels the
boundary map sends each padded position to.  Checked: images against the FP64
oracle with adjoint="transpose" (<= 1e-4 relative L-inf after 30
iterations), exact flux conservation (which A^T gives RL and B in general does
not), and that symmetric PSFs under the mirror keep their fast paths.
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


class Anchored:
    """Dense taps with an explicit anchor (the PSF descriptor's anchor_x/y)."""

    def __init__(self, taps, ax, ay, name):
        t = np.asarray(taps, np.float64)
        self.kind, self.axis, self.length, self.radius = "dense", 0, 0, 0
        self.taps = tuple(t.reshape(-1))
        self.kh, self.kw = t.shape
        self.anchor_x, self.anchor_y = ax, ay
        self.name = name
        self.t = t

    def oracle_psf(self):
        return oracle.psf_dense(self.t, self.anchor_x, self.anchor_y)


class Motion:
    """A motion PSF as the library takes it (running-sum path), with its
    oracle taps anchored at floor(L/2)."""

    def __init__(self, length, axis):
        self.spec = synth.motion(length, axis)
        self.kind, self.axis, self.length, self.radius = "motion", axis, length, 0
        self.taps, self.kw, self.kh = None, 0, 0
        self.t = self.spec.dense()
        self.anchor_x, self.anchor_y = self.t.shape[1] // 2, self.t.shape[0] // 2
        self.name = self.spec.name + "_motion"

    def oracle_psf(self):
        return oracle.psf_dense(self.t, self.anchor_x, self.anchor_y)


class Disc:
    """A disc PSF as the library takes it (register-blocked disc kernel)."""

    def __init__(self, radius):
        self.spec = synth.disc(radius)
        self.kind, self.axis, self.length, self.radius = "disc", 0, 0, radius
        self.taps, self.kw, self.kh = None, 0, 0
        self.t = self.spec.dense()
        self.anchor_x = self.anchor_y = radius
        self.name = self.spec.name + "_disc"

    def oracle_psf(self):
        return oracle.psf_dense(self.t, self.anchor_x, self.anchor_y)


def axis_symmetric(spec):
    t = spec.t
    return (spec.anchor_x == t.shape[1] - 1 - spec.anchor_x and spec.anchor_y == t.shape[0] - 1 - spec.anchor_y
            and np.array_equal(t, t[:, ::-1]) and np.array_equal(t, t[::-1, :]))


def centred(spec):
    t = spec.dense()
    return Anchored(t, t.shape[1] // 2, t.shape[0] // 2, spec.name)


def asym_taps(shape, seed):
    return np.random.default_rng(seed).uniform(0.05, 1.0, size=shape)


CASES = [
    Anchored(asym_taps((3, 5), 3), 4, 0, "dense3x5_anchor40"),
    Anchored(asym_taps((5, 5), 4), 2, 2, "dense5x5_asym"),
    Anchored(np.eye(7)[::-1], 3, 3, "line45_7"),
    centred(synth.motion(6, 0)),
    centred(synth.motion(8, 1)),
    centred(synth.disc(3)),
    Motion(6, 0), Motion(8, 1), Motion(9, 0),
    Disc(5),
    # reaches 10 pixels from its anchor: the generic stencil tiles fold it
    Anchored(asym_taps((3, 11), 5), 10, 1, "dense3x11_anchor101"),
    # uniform centred squares: the box kernel with the band fold
    Anchored(np.ones((9, 9)), 4, 4, "box9"),
    Anchored(np.ones((25, 25)), 12, 12, "box25"),
    # uniform rectangles off their centre: the rectangle kernel with the fold
    Anchored(np.ones((6, 11)), 0, 0, "rect6x11_corner"),
    Anchored(np.ones((3, 21)), 15, 1, "rect3x21_a15"),
]


def uniform_rectangle(spec):
    """Equal taps filling a rectangle reaching <= 16 pixels from the anchor:
    the library runs those on the box / rectangle kernels (path 2)."""
    t = spec.t
    if spec.kind != "dense":
        return False
    ys, xs = np.nonzero(t)
    if len(ys) != (np.ptp(ys) + 1) * (np.ptp(xs) + 1) or not np.all(t[ys, xs] == t[ys[0], xs[0]]):
        return False
    reach = max(abs(xs.min() - spec.anchor_x), abs(xs.max() - spec.anchor_x),
                abs(ys.min() - spec.anchor_y), abs(ys.max() - spec.anchor_y))
    return reach <= 16


def gpu_run(spec, f32, iters, boundary, adjoint, thin=None, stats=False):
    from paper_1304_7211_gb300 import rl
    f = torch.from_numpy(f32).cuda()
    with rl.Deconvolver(spec, boundary=boundary, adjoint=adjoint) as d:
        u, st = d.run(f, iters, thin=thin, stats=True)
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.float64), st


def case_image(w, h, seed):
    c = synth.make_case(w, h, synth.disc(2), 0, "poisson", seed)
    return c.f.astype(np.float32)


@pytest.mark.parametrize("boundary", ["mirror", "clamp"])
@pytest.mark.parametrize("spec", CASES, ids=lambda s: s.name)
def test_transpose_matches_oracle(spec, boundary):
    # 150 x 117: ragged against the tile shapes, several tiles per axis
    f32 = case_image(150, 117, synth.SEED_BASE + 60)
    u, st = gpu_run(spec, f32, 30, boundary, "transpose")
    ref = oracle.rl(f32.astype(np.float64), spec.oracle_psf(), 30, boundary=boundary,
                    adjoint="transpose").u
    assert oracle.rel_linf(u, ref) <= TOL
    pf = oracle.rl(f32.astype(np.float64), spec.oracle_psf(), 30, boundary=boundary,
                   adjoint="padflip").u
    if boundary == "mirror" and axis_symmetric(spec):
        # B = A^T: the fast path runs unchanged
        assert oracle.rel_linf(pf, ref) <= 1e-12
        assert st.path != 3 or spec.kind == "dense"
    else:
        # not the pad-flip iterate (the test would be vacuous otherwise); the
        # fold runs in the resident rows for motion PSFs, on the two-half
        # kernels for the disc and uniform rectangles, else in the stencil
        # kernels
        assert oracle.rel_linf(pf, ref) > 10 * TOL
        assert st.path == (2 if uniform_rectangle(spec) else {"motion": 1, "disc": 2}.get(spec.kind, 3))


@pytest.mark.parametrize("shape", [(9, 11), (6, 40), (40, 6), (13, 13)])
@pytest.mark.parametrize("boundary", ["mirror", "clamp"])
def test_transpose_small_images(shape, boundary):
    # PSF extents up to the image size: folds from both ends of an axis
    H, W = shape
    spec = Anchored(asym_taps((3, 5), 7), 1, 2, "dense3x5")
    f32 = np.random.default_rng(H * 100 + W).uniform(5, 250, size=(H, W)).astype(np.float32)
    u, _ = gpu_run(spec, f32, 12, boundary, "transpose")
    ref = oracle.rl(f32.astype(np.float64), spec.oracle_psf(), 12, boundary=boundary,
                    adjoint="transpose").u
    assert oracle.rel_linf(u, ref) <= TOL


@pytest.mark.parametrize("boundary", ["mirror", "clamp"])
def test_transpose_conserves_flux(boundary):
    # with A^T: sum_p u'(p) = sum_p u(p) (A^T q)(p) = sum_p (A u)(p) q(p)
    # = sum_p f(p) wherever A u > 0 -- exactly, for any PSF
    spec = Anchored(asym_taps((5, 3), 11), 0, 4, "dense5x3_corner")
    f32 = case_image(200, 130, synth.SEED_BASE + 61)
    _, st = gpu_run(spec, f32, 20, boundary, "transpose")
    assert abs(st.flux_u - st.flux_f) <= 1e-5 * abs(st.flux_f)
    _, st_pf = gpu_run(spec, f32, 20, boundary, "padflip")
    assert abs(st_pf.flux_u - st_pf.flux_f) > 1e-4 * abs(st_pf.flux_f)


def test_symmetric_psf_under_mirror_is_unchanged():
    # B = A^T there: same fast paths, bitwise the same result
    for spec in (synth.disc(5), synth.gaussian(7, 1.5), synth.motion(15, 0), synth.motion(9, 1)):
        f32 = case_image(140, 100, synth.SEED_BASE + 62)
        a, sa = gpu_run(spec, f32, 15, "mirror", "padflip")
        b, sb = gpu_run(spec, f32, 15, "mirror", "transpose")
        np.testing.assert_array_equal(a, b)
        assert sa.path == sb.path


@pytest.mark.parametrize("spec", [CASES[0], CASES[10], Motion(6, 0), Motion(8, 1), Disc(4), CASES[11], CASES[13]],
                         ids=lambda s: s.name)
@pytest.mark.parametrize("boundary", ["mirror", "clamp"])
def test_transpose_thinned_replay(boundary, spec):
    # the oracle's used-pixel schedule replayed: same selective convolutions
    from paper_1304_7211_gb300 import rl
    f32 = case_image(130, 90, synth.SEED_BASE + 63)
    K = 25
    ref = oracle.rl(f32.astype(np.float64), spec.oracle_psf(), K, boundary=boundary,
                    adjoint="transpose", threshold=1e-3, relative=True, reset_period=10,
                    update_period=1, want_mask=True)
    sched = np.ascontiguousarray(ref.mask_trace)
    u, st = gpu_run(spec, f32, K, boundary, "transpose",
                    thin=rl.thinning(1e-3, True, 10, 1, schedule=sched))
    assert oracle.rel_linf(u, ref.u) <= TOL
    assert st.active_pixel_iterations == ref.active_pixel_iterations
