"""Pins for the FP64 oracle against things other than itself.

* boundary maps against numpy.pad ('symmetric' = half-sample mirror,
  'edge' = closest pixel, Sec. 2);
* the forward operator and the pad-flip adjoint against scipy.ndimage;
* the exact transpose against the dense matrix of the forward operator and
  the adjoint identity;
* Richardson-Lucy (Eq. 3) against an independent numpy/scipy loop;
* closed forms and invariants (delta PSF, constant images, flux, fixed point,
  nonnegativity);
* selective convolution (Eq. 4-5) against an independent loop, the zero
  threshold row of Table 2, and the infinite-threshold limit.
"""
import math
import os

import numpy as np
import pytest
from scipy import ndimage

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_facts.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            out[k] = float(v)
    return out


def centred_kernel(psf):
    """Odd-sized array K with K[R + t] = h(t) (t = offset from the anchor)."""
    kh, kw = psf.taps.shape
    rx = max(psf.ax, kw - 1 - psf.ax)
    ry = max(psf.ay, kh - 1 - psf.ay)
    k = np.zeros((2 * ry + 1, 2 * rx + 1))
    k[ry - psf.ay:ry - psf.ay + kh, rx - psf.ax:rx - psf.ax + kw] = psf.taps
    return k


MODES = {"mirror": "reflect", "clamp": "nearest"}


def scipy_forward(u, psf, boundary):
    return ndimage.correlate(u, centred_kernel(psf)[::-1, ::-1], mode=MODES[boundary])


def scipy_padflip(q, psf, boundary):
    return ndimage.correlate(q, centred_kernel(psf), mode=MODES[boundary])


def rand_psf(rng, kh, kw, anchor=None):
    t = rng.uniform(0.05, 1.0, size=(kh, kw))
    if anchor is None:
        anchor = (int(rng.integers(0, kw)), int(rng.integers(0, kh)))
    return oracle.psf_dense(t, anchor[0], anchor[1])


SYMMETRIC_PSFS = [
    lambda: oracle.psf_motion(5, 0),
    lambda: oracle.psf_motion(7, 1),
    lambda: oracle.psf_disc(2),
    lambda: oracle.psf_disc(3),
    lambda: oracle.psf_dense(np.outer([1, 4, 6, 4, 1], [1, 2, 1])),
]


# ---- boundary maps -------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_mirror_map_matches_numpy_symmetric_pad(n):
    pad = 3 * n + 4
    ref = np.pad(np.arange(n), pad, mode="symmetric")
    got = [oracle.bmap(e, n, "mirror") for e in range(-pad, n + pad)]
    assert got == list(ref)


def test_mirror_map_literal_half_sample():
    # ... c b a | a b c | c b a ...  for n = 3
    assert [oracle.bmap(e, 3) for e in range(-4, 8)] == [2, 2, 1, 0, 0, 1, 2, 2, 1, 0, 0, 1]


@pytest.mark.parametrize("n", [1, 4, 7])
def test_clamp_map_matches_numpy_edge_pad(n):
    pad = 2 * n + 3
    ref = np.pad(np.arange(n), pad, mode="edge")
    got = [oracle.bmap(e, n, "clamp") for e in range(-pad, n + pad)]
    assert got == list(ref)


# ---- PSFs ------------------------------------------------------------------

def test_disc_support_sizes_are_gauss_circle_numbers():
    g = golden()
    for r in (1, 2, 3, 4, 8, 12, 15):
        p = oracle.psf_disc(r)
        assert int((p.taps > 0).sum()) == int(g[f"disc_support_r{r}"])
        assert math.isclose(p.taps.sum(), 1.0, rel_tol=1e-14)
        # uniform weight on the support
        nz = p.taps[p.taps > 0]
        assert np.ptp(nz) == 0.0


def test_motion_psf_layout():
    p = oracle.psf_motion(6, 0)
    assert p.taps.shape == (1, 6) and (p.ax, p.ay) == (3, 0)
    q = oracle.psf_motion(9, 1)
    assert q.taps.shape == (9, 1) and (q.ax, q.ay) == (0, 4)
    assert np.allclose(q.taps, 1.0 / 9.0)


def test_dense_psf_validation():
    with pytest.raises(ValueError):
        oracle.psf_dense([[1.0, -0.5]])
    with pytest.raises(ValueError):
        oracle.psf_dense([[0.0, 0.0]])
    with pytest.raises(ValueError):
        oracle.psf_dense([[1.0, float("nan")]])
    p = oracle.psf_dense([[1.0, 3.0]])
    assert np.allclose(p.taps, [[0.25, 0.75]])


# ---- operators -------------------------------------------------------------

@pytest.mark.parametrize("boundary", ["mirror", "clamp"])
@pytest.mark.parametrize("shape,kshape", [((5, 7), (3, 3)), ((9, 6), (2, 5)),
                                          ((11, 13), (5, 4)), ((4, 9), (1, 7)),
                                          ((8, 3), (6, 1))])
def test_forward_matches_scipy(boundary, shape, kshape):
    rng = np.random.default_rng(hash((shape, kshape)) % 2**32)
    u = rng.uniform(0, 255, size=shape)
    psf = rand_psf(rng, *kshape)
    got = oracle.conv(u, psf, boundary)
    ref = scipy_forward(u, psf, boundary)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-11)


@pytest.mark.parametrize("boundary", ["mirror", "clamp"])
def test_forward_large_psf_multiple_reflections(boundary):
    # PSF wider than the image: the continuation is applied repeatedly.
    rng = np.random.default_rng(3)
    u = rng.uniform(0, 1, size=(3, 4))
    psf = rand_psf(rng, 9, 11, anchor=(5, 4))
    np.testing.assert_allclose(oracle.conv(u, psf, boundary),
                               scipy_forward(u, psf, boundary), rtol=1e-13)


@pytest.mark.parametrize("boundary", ["mirror", "clamp"])
def test_padflip_matches_scipy(boundary):
    rng = np.random.default_rng(11)
    q = rng.uniform(0.5, 2.0, size=(10, 12))
    psf = rand_psf(rng, 4, 5, anchor=(1, 3))
    np.testing.assert_allclose(oracle.conv_adjoint(q, psf, boundary, "padflip"),
                               scipy_padflip(q, psf, boundary), rtol=1e-13)


def dense_matrix(psf, W, H, boundary):
    A = np.zeros((W * H, W * H))
    for j in range(W * H):
        e = np.zeros(W * H)
        e[j] = 1.0
        A[:, j] = oracle.conv(e.reshape(H, W), psf, boundary).reshape(-1)
    return A


@pytest.mark.parametrize("boundary", ["mirror", "clamp"])
def test_transpose_is_dense_matrix_transpose(boundary):
    rng = np.random.default_rng(5)
    H, W = 6, 7
    psf = rand_psf(rng, 3, 4, anchor=(2, 0))
    A = dense_matrix(psf, W, H, boundary)
    q = rng.uniform(0, 1, size=(H, W))
    got = oracle.conv_adjoint(q, psf, boundary, "transpose").reshape(-1)
    np.testing.assert_allclose(got, A.T @ q.reshape(-1), rtol=1e-13, atol=1e-14)
    # adjoint identity <A a, b> = <a, A^T b>
    a = rng.uniform(size=(H, W))
    b = rng.uniform(size=(H, W))
    lhs = np.sum(oracle.conv(a, psf, boundary) * b)
    rhs = np.sum(a * oracle.conv_adjoint(b, psf, boundary, "transpose"))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("make", SYMMETRIC_PSFS)
def test_padflip_equals_transpose_for_axis_symmetric_psf_under_mirror(make):
    psf = make()
    H, W = 9, 8
    A = dense_matrix(psf, W, H, "mirror")
    # A is symmetric and doubly stochastic under the half-sample mirror
    np.testing.assert_allclose(A, A.T, atol=1e-15)
    np.testing.assert_allclose(A.sum(axis=0), 1.0, rtol=1e-13)
    rng = np.random.default_rng(2)
    q = rng.uniform(size=(H, W))
    np.testing.assert_allclose(oracle.conv_adjoint(q, psf, "mirror", "padflip"),
                               oracle.conv_adjoint(q, psf, "mirror", "transpose"),
                               rtol=1e-13)
    # ... and the adjoint identity holds for the pad-flip operator itself
    a = rng.uniform(size=(H, W))
    lhs = np.sum(oracle.conv(a, psf, "mirror") * q)
    rhs = np.sum(a * oracle.conv_adjoint(q, psf, "mirror", "padflip"))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_padflip_differs_from_transpose_when_it_should():
    # Even-length motion blur is not axis-symmetric; clamp is not a
    # symmetric continuation.  Both make B != A^T, so the test above has teeth.
    rng = np.random.default_rng(4)
    q = rng.uniform(size=(6, 9))
    p = oracle.psf_motion(4, 0)
    assert not np.allclose(oracle.conv_adjoint(q, p, "mirror", "padflip"),
                           oracle.conv_adjoint(q, p, "mirror", "transpose"))
    d = oracle.psf_disc(2)
    assert not np.allclose(oracle.conv_adjoint(q, d, "clamp", "padflip"),
                           oracle.conv_adjoint(q, d, "clamp", "transpose"))


# ---- Richardson-Lucy (Eq. 3) ------------------------------------------------

def independent_rl(f, psf, K, boundary, u0=None):
    u = f.copy() if u0 is None else u0.copy()
    for _ in range(K):
        v = scipy_forward(u, psf, boundary)
        q = np.where(v > 0, f / np.where(v > 0, v, 1.0), 0.0)
        u = u * scipy_padflip(q, psf, boundary)
    return u


@pytest.mark.parametrize("boundary", ["mirror", "clamp"])
def test_rl_matches_independent_loop_asymmetric_psf(boundary):
    rng = np.random.default_rng(7)
    f = rng.uniform(5, 250, size=(12, 17))
    psf = rand_psf(rng, 3, 5, anchor=(1, 2))
    got = oracle.rl(f, psf, 6, boundary=boundary).u
    ref = independent_rl(f, psf, 6, boundary)
    np.testing.assert_allclose(got, ref, rtol=1e-12)


def test_rl_explicit_u0_and_zero_iterations():
    rng = np.random.default_rng(8)
    f = rng.uniform(5, 250, size=(7, 9))
    u0 = rng.uniform(5, 250, size=(7, 9))
    psf = oracle.psf_disc(2)
    np.testing.assert_array_equal(oracle.rl(f, psf, 0).u, f)
    np.testing.assert_array_equal(oracle.rl(f, psf, 0, u0=u0).u, u0)
    np.testing.assert_allclose(oracle.rl(f, psf, 3, u0=u0).u,
                               independent_rl(f, psf, 3, "mirror", u0), rtol=1e-12)


def test_delta_psf_closed_form():
    # h = delta: v = u, q = f/u, c = q, so u^1 = f and it stays there.
    rng = np.random.default_rng(9)
    f = rng.uniform(1, 255, size=(6, 11))
    u0 = rng.uniform(1, 255, size=(6, 11))
    for psf in (oracle.psf_motion(1, 0), oracle.psf_disc(0)):
        np.testing.assert_allclose(oracle.rl(f, psf, 1, u0=u0).u, f, rtol=1e-15)
        np.testing.assert_allclose(oracle.rl(f, psf, 5).u, f, rtol=1e-15)


@pytest.mark.parametrize("boundary", ["mirror", "clamp"])
def test_constant_image_is_reproduced(boundary):
    # Any normalised PSF maps a constant to itself, so q = 1 and c = 1.
    rng = np.random.default_rng(10)
    f = np.full((9, 13), 37.5)
    psf = rand_psf(rng, 4, 3, anchor=(0, 2))
    np.testing.assert_allclose(oracle.rl(f, psf, 20, boundary=boundary).u, f,
                               rtol=1e-13)


@pytest.mark.parametrize("make", SYMMETRIC_PSFS)
def test_flux_and_nonnegativity(make):
    psf = make()
    rng = np.random.default_rng(12)
    f = rng.uniform(0, 255, size=(14, 11))
    f[3, 4] = 0.0
    for K in (1, 2, 7):
        u = oracle.rl(f, psf, K).u
        assert u.min() >= 0.0
        assert abs(u.sum() - f.sum()) <= 1e-12 * f.sum()


def test_flux_with_exact_transpose_any_psf():
    rng = np.random.default_rng(13)
    f = rng.uniform(1, 255, size=(10, 8))
    psf = rand_psf(rng, 3, 4, anchor=(3, 1))
    for boundary in ("mirror", "clamp"):
        u = oracle.rl(f, psf, 4, boundary=boundary, adjoint="transpose").u
        assert abs(u.sum() - f.sum()) <= 1e-12 * f.sum()


@pytest.mark.parametrize("make", SYMMETRIC_PSFS)
def test_fixed_point(make):
    # f = A g exactly and u^0 = g  =>  v = f, q = 1, u^1 = g.
    psf = make()
    rng = np.random.default_rng(14)
    g = rng.uniform(10, 250, size=(12, 10))
    f = oracle.conv(g, psf, "mirror")
    np.testing.assert_allclose(oracle.rl(f, psf, 1, u0=g).u, g, rtol=1e-13)


@pytest.mark.parametrize("make", SYMMETRIC_PSFS)
def test_poisson_likelihood_never_decreases(make):
    """RL is the EM algorithm for Poisson data (Shepp-Vardi): when the
    forward operator A is non-negative with unit column sums -- under the
    half-sample mirror, any PSF symmetric in each axis -- every iteration
    leaves the log-likelihood sum_p f_p log (A u)_p - (A u)_p at least where
    it was, for any non-negative f.  A ratio turned upside down, a missing
    factor u or an adjoint taken from the wrong side breaks this."""
    psf = make()
    rng = np.random.default_rng(19)
    g = rng.uniform(10, 250, size=(13, 12))
    f = rng.poisson(oracle.conv(g, psf, "mirror")).astype(np.float64)

    def loglik(u):
        v = oracle.conv(u, psf, "mirror")
        return float(np.sum(np.where(f > 0, f * np.log(np.maximum(v, 1e-300)), 0.0) - v))

    u = f.copy()
    prev = loglik(u)
    gains = []
    for _ in range(12):
        u = oracle.rl(f, psf, 1, u0=u).u
        cur = loglik(u)
        assert cur >= prev - 1e-12 * abs(prev), (cur, prev)
        gains.append(cur - prev)
        prev = cur
    assert gains[0] > 0.0  # the first iteration moves off the blurred start


def test_poisson_likelihood_catches_an_inverted_ratio():
    """The likelihood pin rejects a planted mistake: the update with the
    ratio v / f instead of f / v lowers the likelihood."""
    psf = oracle.psf_disc(2)
    rng = np.random.default_rng(20)
    g = rng.uniform(10, 250, size=(13, 12))
    f = rng.poisson(oracle.conv(g, psf, "mirror")).astype(np.float64)

    def loglik(u):
        v = oracle.conv(u, psf, "mirror")
        return float(np.sum(f * np.log(v) - v))

    def wrong_step(u):
        v = oracle.conv(u, psf, "mirror")
        return u * oracle.conv_adjoint(v / f, psf, "mirror")

    u1 = oracle.rl(f, psf, 1).u
    assert loglik(u1) > loglik(f)
    assert loglik(wrong_step(f)) < loglik(f)


def test_scaling_the_data_scales_the_iterates():
    """Eq. 3 is homogeneous of degree one in (f, u0): scaling f by 4 (exact
    in binary floating point) scales every iterate by 4 bit for bit.  The
    relative rule of Eq. 4-5 (|c - 1|) is scale-free, so the same masks
    result; the absolute rule (|u' - u|) needs the threshold scaled too, and
    with the threshold left alone it decides differently.  A rule that mixed
    the two changes, or a constant added anywhere in the arithmetic, fails."""
    rng = np.random.default_rng(21)
    psf = oracle.psf_disc(2)
    g = rng.uniform(10, 250, size=(16, 15))
    f = rng.poisson(oracle.conv(g, psf, "mirror")).astype(np.float64) + 1.0
    K = 13
    np.testing.assert_array_equal(oracle.rl(4 * f, psf, K).u, 4 * oracle.rl(f, psf, K).u)
    a = oracle.rl(f, psf, K, threshold=2e-3, relative=True)
    b = oracle.rl(4 * f, psf, K, threshold=2e-3, relative=True)
    np.testing.assert_array_equal(b.u, 4 * a.u)
    assert a.active_pixel_iterations == b.active_pixel_iterations
    a = oracle.rl(f, psf, K, threshold=0.05, relative=False)
    b = oracle.rl(4 * f, psf, K, threshold=0.2, relative=False)
    np.testing.assert_array_equal(b.u, 4 * a.u)
    assert a.active_pixel_iterations == b.active_pixel_iterations
    c = oracle.rl(4 * f, psf, K, threshold=0.05, relative=False)
    assert c.active_pixel_iterations > a.active_pixel_iterations  # same threshold, larger changes


def test_zero_ratio_where_reblur_vanishes():
    # f = 0 on a block wider than the PSF: v = 0 there after one step,
    # q must be 0 (not NaN) and u stays finite.
    f = np.full((12, 12), 50.0)
    f[2:10, 2:10] = 0.0
    psf = oracle.psf_disc(1)
    u = oracle.rl(f, psf, 6).u
    assert np.all(np.isfinite(u))
    assert np.all(u[4:8, 4:8] == 0.0)


# ---- selective convolution (Eq. 4-5) ---------------------------------------

def independent_thinned_rl(f, psf, K, tau, relative, P, Q, boundary="mirror"):
    u = f.copy()
    stale = np.zeros_like(f)
    M = np.ones(f.shape, bool)
    masks = []
    for k in range(K):
        full = k % P == 0
        use = np.ones(f.shape, bool) if full else M.copy()
        v = scipy_forward(u, psf, boundary)
        fresh = np.where(v > 0, f / np.where(v > 0, v, 1.0), 0.0)
        q = np.where(use, fresh, stale)
        stale = np.where(use, fresh, stale)
        c = scipy_padflip(q, psf, boundary)
        un = np.where(use, u * c, u)
        if relative:
            d = np.where(use & (u > 0), np.abs(c - 1.0), 0.0)
        else:
            d = np.where(use, np.abs(un - u), 0.0)
        if Q == 1:
            M = use & (d >= tau)
        elif full:
            M = d >= tau
        masks.append(use)
        u = un
    return u, np.array(masks)


@pytest.mark.parametrize("relative,tau,Q", [(True, 2e-3, 1), (False, 0.05, 1),
                                            (True, 2e-3, 10), (False, 0.02, 10)])
def test_thinning_matches_independent_loop(relative, tau, Q):
    rng = np.random.default_rng(15)
    g = np.kron(rng.uniform(20, 240, size=(4, 5)), np.ones((5, 5)))
    f = oracle.conv(g, oracle.psf_disc(2), "mirror") + rng.uniform(0, 1, g.shape)
    psf = oracle.psf_disc(2)
    res = oracle.rl(f, psf, 23, threshold=tau, relative=relative,
                    update_period=Q, want_mask=True)
    ref_u, ref_masks = independent_thinned_rl(f, psf, 23, tau, relative, 10, Q)
    np.testing.assert_array_equal(res.mask_trace.astype(bool), ref_masks)
    np.testing.assert_allclose(res.u, ref_u, rtol=1e-12)
    assert res.active_pixel_iterations == int(ref_masks.sum())
    # thinning really happened in this case
    assert res.active_pixel_iterations < 23 * f.size


def test_zero_threshold_is_plain_rl():
    # Table 2, threshold 0: 0.00 % omitted and the same result as the reference.
    g = golden()
    rng = np.random.default_rng(16)
    f = rng.uniform(10, 240, size=(15, 18))
    psf = oracle.psf_disc(2)
    plain = oracle.rl(f, psf, 25).u
    for Q in (1, 10):
        res = oracle.rl(f, psf, 25, threshold=0.0, update_period=Q)
        omitted = 100.0 * (1 - res.active_pixel_iterations / (25 * f.size))
        assert omitted == g["table2_tau0_omitted_percent"]
        np.testing.assert_array_equal(res.u, plain)


def test_infinite_threshold_keeps_only_full_iterations():
    P = int(golden()["thinning_reset_period"])
    rng = np.random.default_rng(17)
    f = rng.uniform(10, 240, size=(11, 14))
    psf = oracle.psf_motion(5, 0)
    for K in (1, 9, 10, 11, 25):
        res = oracle.rl(f, psf, K, threshold=math.inf)
        np.testing.assert_allclose(res.u, oracle.rl(f, psf, -(-K // P)).u, rtol=1e-14)


def test_mask_only_shrinks_within_an_epoch_and_trend():
    rng = np.random.default_rng(18)
    g = np.kron(rng.uniform(20, 240, size=(5, 5)), np.ones((6, 6)))
    psf = oracle.psf_disc(2)
    f = oracle.conv(g, psf, "mirror")
    omitted = []
    for tau in (0.0, 1e-3, 1e-2, 1e-1):
        res = oracle.rl(f, psf, 30, threshold=tau, want_mask=True)
        m = res.mask_trace.astype(bool)
        for k in range(1, 30):
            if k % 10:
                assert np.all(m[k] <= m[k - 1])
            else:
                assert m[k].all()
        omitted.append(1 - res.active_pixel_iterations / m.size)
    # Table 2 trend: more pixels omitted for larger thresholds.
    assert omitted[0] == 0.0 and all(a <= b for a, b in zip(omitted, omitted[1:]))
    assert omitted[-1] > 0.3
