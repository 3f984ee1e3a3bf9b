"""The summed-area-table path (Sec. 3, rectangular blur by 2D cumulated
sums) for uniform rectangles: element-wise parity with the FP64 oracle,
agreement with the separable rectangle kernel, an image whose values are
thousands of times larger (the fixed-point scale follows each tile's
largest value), and the cases it refuses."""
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


def anchored(rows, cols, ax, ay):
    t = np.ones((rows, cols))
    return type("S", (), dict(kind="dense", taps=tuple(t.reshape(-1)), kw=cols, kh=rows, anchor_x=ax,
                              anchor_y=ay, axis=0, length=0, radius=0, name=f"rect{rows}x{cols}", t=t))()


def gpu(spec, f32, its, path, boundary="mirror"):
    from paper_1304_7211_gb300 import rl
    with rl.Deconvolver(spec, path=path, boundary=boundary) as d:
        u, st = d.run(torch.from_numpy(f32).cuda(), its, stats=True)
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.float64), st


# (rows, cols, anchor x, anchor y): centred and off-centre, thin either way,
# the three halo classes (reach 1..4, 5..8, 9..16), a motion row
RECTS = [(3, 5, 2, 1), (1, 1, 0, 0), (9, 31, 15, 4), (31, 9, 4, 15), (1, 17, 8, 0), (8, 8, 4, 4),
         (17, 17, 8, 8), (33, 33, 16, 16), (5, 12, 0, 4)]


@pytest.mark.parametrize("boundary", ["mirror", "clamp"])
@pytest.mark.parametrize("rect", RECTS, ids=lambda r: "x".join(map(str, r)))
def test_sat_matches_oracle(rect, boundary):
    rows, cols, ax, ay = rect
    spec = anchored(*rect)
    c = synth.make_case(203, 161, synth.dense(np.ones((3, 3))), 0, "poisson", synth.SEED_BASE + 190)
    f32 = synth.blur(c.g, synth.dense(np.ones((rows, cols)))).astype(np.float32) + 1.0
    u, st = gpu(spec, f32, 30, "sat", boundary)
    assert st.path == 4
    ref = oracle.rl(f32.astype(np.float64), oracle.psf_dense(spec.t, ax, ay), 30, boundary=boundary).u
    err = oracle.rel_linf(u, ref)
    assert err <= TOL, err
    # the separable sliding sums of the span path compute the same operator
    v, _ = gpu(spec, f32, 30, "auto", boundary)
    assert oracle.rel_linf(u, v) <= TOL


def test_sat_large_values_and_motion_row():
    # values around 1e6: the per-tile fixed-point scale shrinks, the sums stay exact
    spec = synth.motion(15, 0)
    c = synth.make_case(300, 200, spec, 0, "poisson", synth.SEED_BASE + 191)
    f32 = (c.f * 4000.0 + 1.0).astype(np.float32)
    u, st = gpu(spec, f32, 25, "sat")
    assert st.path == 4
    t = spec.dense()
    ref = oracle.rl(f32.astype(np.float64), oracle.psf_dense(t, t.shape[1] // 2, 0), 25).u
    assert oracle.rel_linf(u, ref) <= TOL


def test_sat_refuses_other_psfs_and_thinning():
    from paper_1304_7211_gb300 import rl
    f = torch.ones((64, 64), device="cuda")
    with rl.Deconvolver(synth.disc(3), path="sat") as d:
        with pytest.raises(rl.RLError) as e:
            d.run(f, 3)
        assert e.value.status == rl.RL_ERR_UNSUPPORTED
    with rl.Deconvolver(synth.dense(np.ones((5, 5))), path="sat") as d:
        with pytest.raises(rl.RLError) as e:
            d.run(f, 3, thin=rl.thinning(1e-3))
        assert e.value.status == rl.RL_ERR_UNSUPPORTED
        d.run(f, 3)  # the context goes on


def test_sat_bf16_storage():
    """BF16 storage on the table path: f and u rounded to BF16, the table
    built from the staged FP32 values; within K unit roundoffs of the oracle
    on the rounded f (the rectangle's amplification is small at 7 x 5)."""
    spec = synth.dense(np.ones((7, 5)))
    c = synth.make_case(190, 150, spec, 0, "poisson", synth.SEED_BASE + 192)
    f_r = torch.from_numpy(c.f.astype(np.float32)).to(torch.bfloat16)
    from paper_1304_7211_gb300 import rl
    with rl.Deconvolver(spec, path="sat", storage="bf16") as d:
        u = d.run(f_r.cuda(), 10)
    torch.cuda.synchronize()
    with rl.Deconvolver(spec, path="span", storage="bf16") as d:
        v = d.run(f_r.cuda(), 10)
    torch.cuda.synchronize()
    ref = oracle.rl(f_r.float().numpy().astype(np.float64), oracle.psf_dense(np.ones((7, 5)), 2, 3), 10).u
    assert oracle.rel_linf(u.float().cpu().numpy(), ref) <= 10 * 2.0 ** -9
    assert oracle.rel_linf(u.float().cpu().numpy(), v.float().cpu().numpy().astype(np.float64)) <= 10 * 2.0 ** -9
