"""Where selective convolution (Sec. 4, Eq. 4-5) could save GPU time on the
thinned workload (disc radius 12, Poisson noise at peak 500, relative
threshold 1e-3, mask recomputed every 10 iterations).

The GPU kernels share work across an 8x4 block of outputs (staging, the row
prefix, register-blocked run sums), so a skipped pixel only saves time when
its whole block, or its whole 64x64 tile, is inactive.  These tests read the
oracle's used-pixel masks on a 256x256 image of the workload's generator:
with noise, about a third of the pixels are inactive yet every block keeps an
active pixel in every selective iteration; without noise, blocks do go idle.
"""
import numpy as np

import oracle
from paper_1304_7211_gb300 import synth

K = 40


def idle_fractions(mask):
    """(active pixels, idle 8x4 blocks, idle 64x64 tiles) of one used-pixel mask."""
    a = mask.astype(bool)
    H, W = a.shape
    blocks = a.reshape(H // 4, 4, W // 8, 8).any(axis=(1, 3))
    tiles = a.reshape(H // 64, 64, W // 64, 64).any(axis=(1, 3))
    return a.mean(), 1.0 - blocks.mean(), 1.0 - tiles.mean()


def selective_masks(f):
    r = oracle.rl(f.astype(np.float32).astype(np.float64), oracle.psf_disc(12), K, threshold=1e-3,
                  relative=True, reset_period=10, update_period=10, want_mask=True)
    return [r.mask_trace[k] for k in range(K) if k % 10 != 0]


def test_noisy_workload_leaves_no_block_idle():
    c = synth.config3(256)
    fr = [idle_fractions(m) for m in selective_masks(c.f)]
    active = np.array([x[0] for x in fr])
    assert 0.5 < active.min() and active.max() < 0.9   # a third or so omitted
    assert max(x[1] for x in fr) == 0.0                # yet no 8x4 block is idle
    assert max(x[2] for x in fr) == 0.0                # and no tile


def test_noise_free_input_does_idle_blocks():
    g = synth.latent_image(256, 256, synth.SEED_BASE + 3)
    f = synth.blur(g, synth.disc(12))
    fr = [idle_fractions(m) for m in selective_masks(f)]
    assert fr[-1][1] > 0.1  # after 30 iterations more than a tenth of the blocks are idle


def test_idle_fraction_counts():
    m = np.zeros((128, 128), np.uint8)
    m[0, 0] = 1     # block (0, 0), tile (0, 0)
    m[127, 64] = 1  # block (31, 8), tile (1, 1)
    act, blk, til = idle_fractions(m)
    assert act == 2 / 128 ** 2
    assert blk == 1 - 2 / (32 * 16)
    assert til == 0.5
