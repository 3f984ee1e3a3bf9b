"""The seeded input generator: determinism, value ranges, and that its blur
(scipy, half-sample mirror) is the oracle's forward operator A."""
import numpy as np
import pytest

import oracle
from paper_1304_7211_gb300 import synth


def test_latent_image_deterministic_and_in_range():
    a = synth.latent_image(96, 80, 123)
    b = synth.latent_image(96, 80, 123)
    c = synth.latent_image(96, 80, 124)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)
    assert a.shape == (80, 96)
    assert a.min() >= 10.0 and a.max() <= 250.0


@pytest.mark.parametrize("method", ["direct", "fft"])
@pytest.mark.parametrize("spec", [synth.motion(15, 0), synth.motion(9, 1),
                                  synth.motion(6, 0), synth.disc(4),
                                  synth.gaussian(7, 1.5), synth.disc(12)])
def test_generator_blur_is_oracle_forward_operator(spec, method):
    g = synth.latent_image(40, 33, 5)
    t = spec.dense()
    psf = oracle.psf_dense(t, t.shape[1] // 2, t.shape[0] // 2)
    np.testing.assert_allclose(synth.blur(g, spec, method), oracle.conv(g, psf, "mirror"),
                               rtol=1e-11)


def test_generator_psfs_match_oracle_psfs():
    np.testing.assert_allclose(synth.disc(8).dense(), oracle.psf_disc(8).taps, rtol=1e-15)
    np.testing.assert_allclose(synth.motion(31, 1).dense(),
                               oracle.psf_motion(31, 1).taps, rtol=1e-15)


def test_noise_models():
    b = np.full((64, 64), 100.0)
    gz = synth.add_noise(b, "gaussian", 1, sigma=2.0)
    assert abs(gz.std() - 2.0) < 0.2 and gz.min() >= 0.0
    p = synth.add_noise(b, "poisson", 1, peak=1000.0)
    counts = p * 4.0
    np.testing.assert_allclose(counts, np.round(counts))
    assert abs(counts.mean() - 400.0) < 5.0


def test_batch_and_serve_specs():
    specs = synth.batch_specs(64)
    assert len(specs) == 64
    for w, h, spec, its, seed in specs:
        assert 128 <= w <= 1536 and 128 <= h <= 1536 and 50 <= its <= 300
        if spec.kind == "motion":
            assert spec.length % 2 == 1 and 5 <= spec.length <= 41
        if spec.kind == "disc":
            assert 3 <= spec.radius <= 15
    tr = synth.serve_trace(50, rate=100.0)
    ts = [r[0] for r in tr]
    assert ts == sorted(ts) and len(tr) == 50
