"""The autotuner (RL_FLAG_AUTOTUNE): the first call for a request key times
the candidates of its tunable site -- the disc path's launch form, the
running-sum chunk width, the stencil tile shape -- and caches the fastest.
A tuned run must agree with the untuned one within the parity tolerance (the
disc form and the tile shape leave every pixel's arithmetic unchanged, the
chunk width only moves where FP32 window sums restart), and the choice must
be recorded in the cache file named by RL_TUNE_CACHE.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1304_7211_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-4

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    path = tmp_path_factory.mktemp("tune") / "cache.jsonl"
    os.environ["RL_TUNE_CACHE"] = str(path)
    from paper_1304_7211_gb300 import _build, rl
    _build.build()
    yield rl.load()
    os.environ.pop("RL_TUNE_CACHE", None)


def solve(spec, f, its, flags):
    from paper_1304_7211_gb300 import rl
    H, W = f.shape
    with rl.Deconvolver(spec, flags=flags) as d:
        u = torch.empty_like(f)
        st = rl.rl_iterate(d.ctx, f, None, u, W, H, W, its, None, stats=True)
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.float64), st


CASES = [(synth.disc(8), 700, 530, 30, True),                      # launch form
         (synth.motion(15, 0), 1500, 97, 40, False),                # chunk width, rows
         (synth.motion(21, 1), 83, 1400, 40, False),                # chunk width, columns
         (synth.dense(np.outer(np.ones(3), np.hanning(13)[1:-1])), 301, 203, 25, True)]  # stencil tiles


@pytest.mark.parametrize("spec,W,H,its,bitwise", CASES, ids=lambda v: getattr(v, "name", None))
def test_tuned_agrees_with_untuned(spec, W, H, its, bitwise):
    from paper_1304_7211_gb300 import rl
    c = synth.make_case(W, H, spec, 0, "poisson", synth.SEED_BASE + 180 + W)
    f = torch.from_numpy(c.f.astype(np.float32)).cuda()
    plain, _ = solve(spec, f, its, 0)
    tuned, st = solve(spec, f, its, rl.RL_FLAG_AUTOTUNE)   # tunes, then solves
    again, _ = solve(spec, f, its, rl.RL_FLAG_AUTOTUNE)    # takes the cached choice
    assert oracle.rel_linf(tuned, plain) <= TOL
    np.testing.assert_array_equal(tuned, again)
    if bitwise:
        np.testing.assert_array_equal(tuned, plain)
    t = spec.dense()
    ref = oracle.rl(c.f.astype(np.float32).astype(np.float64),
                    oracle.psf_dense(t, t.shape[1] // 2, t.shape[0] // 2), its).u
    assert oracle.rel_linf(tuned, ref) <= TOL


def test_choices_are_written_to_the_cache_file():
    lines = [json.loads(l) for l in open(os.environ["RL_TUNE_CACHE"]) if l.strip()]
    keys = {l["key"].split(":")[0] for l in lines}
    assert {"disc-launch", "motion-chunk", "stencil-tile"} <= keys
    for l in lines:
        assert isinstance(l["choice"], int)
        assert len(l["us"].split()) >= 2  # every candidate's time per iteration
    # one entry per key: the second call of each case took the cached choice
    assert len({l["key"] for l in lines}) == len(lines)
