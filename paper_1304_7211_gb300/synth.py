"""Seeded synthetic inputs for Richardson-Lucy deconvolution.

This module is shared by the tests, the oracle checks and the benchmark.  It
holds none of the deconvolution arithmetic: it draws a latent image, builds
the dense PSF used to blur it, applies the blur model of Eq. 1 (Sec. 1),
``f = g (x) h + n``, through scipy library routines (``scipy.ndimage`` or an
FFT convolution of the symmetrically padded image; half-sample mirror
continuation), and adds noise.

The paper's test image (the 256x256 "cameraman", Sec. 5) is not available;
these images stand in for it: a linear grey-value gradient 16 -> 128 with
axis-aligned rectangles of intensity U[10, 250] painted over it, i.e. an
8-bit-range image with flat regions and sharp edges.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy import ndimage, signal

SEED_BASE = 13047211


@dataclasses.dataclass(frozen=True)
class PsfSpec:
    """A PSF descriptor as the library takes it (motion / disc / dense)."""
    kind: str                      # "motion" | "disc" | "dense"
    axis: int = 0                  # motion: 0 = x, 1 = y
    length: int = 0                # motion length in pixels
    radius: int = 0                # disc radius
    taps: tuple | None = None      # dense: row-major kh x kw
    kw: int = 0
    kh: int = 0

    @property
    def name(self) -> str:
        if self.kind == "motion":
            return f"motion{'xy'[self.axis]}{self.length}"
        if self.kind == "disc":
            return f"disc{self.radius}"
        return f"dense{self.kh}x{self.kw}"

    def dense(self) -> np.ndarray:
        """Dense (kh, kw) taps with unit sum, anchor at the centre index."""
        if self.kind == "motion":
            t = np.full(self.length, 1.0 / self.length)
            return t.reshape(1, -1) if self.axis == 0 else t.reshape(-1, 1)
        if self.kind == "disc":
            r = self.radius
            d = np.arange(-r, r + 1)
            t = ((d[None, :] ** 2 + d[:, None] ** 2) <= r * r).astype(np.float64)
            return t / t.sum()
        t = np.asarray(self.taps, np.float64).reshape(self.kh, self.kw)
        return t / t.sum()


def motion(length: int, axis: int = 0) -> PsfSpec:
    return PsfSpec("motion", axis=axis, length=length)


def disc(radius: int) -> PsfSpec:
    return PsfSpec("disc", radius=radius)


def gaussian(size: int = 7, sigma: float = 1.5) -> PsfSpec:
    """Sampled isotropic Gaussian exp(-(dx^2+dy^2)/(2 sigma^2)), size x size."""
    d = np.arange(size) - size // 2
    t = np.exp(-(d[None, :] ** 2 + d[:, None] ** 2) / (2.0 * sigma * sigma))
    t = t / t.sum()
    return PsfSpec("dense", taps=tuple(float(v) for v in t.reshape(-1)),
                   kw=size, kh=size)


def dense(taps) -> PsfSpec:
    t = np.atleast_2d(np.asarray(taps, np.float64))
    return PsfSpec("dense", taps=tuple(float(v) for v in t.reshape(-1)),
                   kw=t.shape[1], kh=t.shape[0])


def latent_image(width: int, height: int, seed: int) -> np.ndarray:
    """Gradient background 16 -> 128 along a random direction in [0, pi/2]
    plus n = clip(round(16 W H / 65536), 8, 4096) rectangles with
    log-uniform sides in [4, max(8, min(W,H)/4)], uniform positions,
    intensity U[10, 250], painted in order.  float64, shape (H, W)."""
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0.0, math.pi / 2)
    y, x = np.mgrid[0:height, 0:width].astype(np.float64)
    ramp = x * math.cos(theta) + y * math.sin(theta)
    span = max(float(ramp.max()), 1e-12)
    g = 16.0 + 112.0 * ramp / span
    n = int(np.clip(round(16 * width * height / 65536), 8, 4096))
    hi = max(8.0, min(width, height) / 4.0)
    sides = np.exp(rng.uniform(math.log(4.0), math.log(hi), size=(n, 2)))
    sides = np.maximum(1, np.round(sides)).astype(np.int64)
    vals = rng.uniform(10.0, 250.0, size=n)
    ux = rng.uniform(0.0, 1.0, size=n)
    uy = rng.uniform(0.0, 1.0, size=n)
    for k in range(n):
        w = int(min(sides[k, 0], width))
        h = int(min(sides[k, 1], height))
        x0 = int(ux[k] * (width - w + 1))
        y0 = int(uy[k] * (height - h + 1))
        g[y0:y0 + h, x0:x0 + w] = vals[k]
    return g


def blur(g: np.ndarray, spec: PsfSpec, method: str = "auto") -> np.ndarray:
    """Eq. 1 without noise: h (x) g with the half-sample mirror continuation
    (scipy ``mode='reflect'``), anchor at the centre tap.  ``method`` 'direct'
    correlates with scipy.ndimage; 'fft' pads by the symmetric continuation
    and convolves through the FFT (same operator, rounding ~1e-13); 'auto'
    takes the FFT for large kernels on large images."""
    t = spec.dense()
    kh, kw = t.shape
    if method == "auto":
        method = "fft" if (kh * kw > 64 and g.size > 65536) else "direct"
    if method == "fft":
        ay, ax = kh // 2, kw // 2
        # 'valid' convolution reads a[p + k - 1 - j]; shifting the image by the
        # far-side extent (k - 1 - anchor) makes that g(p - (j - anchor)).
        a = np.pad(np.asarray(g, np.float64), ((kh - 1 - ay, ay), (kw - 1 - ax, ax)),
                   mode="symmetric")
        return signal.fftconvolve(a, t, mode="valid")
    # Pad the kernel to odd size around the anchor (kw//2, kh//2) and flip it,
    # so that scipy's centred correlation computes sum_t h(t) g(p - t).
    ax, ay = kw // 2, kh // 2
    rx = max(ax, kw - 1 - ax)
    ry = max(ay, kh - 1 - ay)
    k = np.zeros((2 * ry + 1, 2 * rx + 1))
    k[ry - ay:ry - ay + kh, rx - ax:rx - ax + kw] = t
    return ndimage.correlate(np.asarray(g, np.float64), k[::-1, ::-1],
                             mode="reflect")


def add_noise(b: np.ndarray, kind: str, seed: int, sigma: float = 2.0,
              peak: float = 1000.0) -> np.ndarray:
    """Gaussian (std sigma, clipped at 0) or Poisson noise (image scaled so
    that grey value 250 maps to ``peak`` counts, then scaled back)."""
    rng = np.random.default_rng(seed + 7)
    if kind == "none":
        return b.copy()
    if kind == "gaussian":
        return np.maximum(b + rng.normal(0.0, sigma, size=b.shape), 0.0)
    if kind == "poisson":
        s = peak / 250.0
        return rng.poisson(np.maximum(b, 0.0) * s).astype(np.float64) / s
    raise ValueError(kind)


@dataclasses.dataclass
class Case:
    g: np.ndarray          # latent image (float64)
    f: np.ndarray          # observed image (float64)
    spec: PsfSpec
    iterations: int
    seed: int


def make_case(width: int, height: int, spec: PsfSpec, iterations: int,
              noise: str = "poisson", seed: int = SEED_BASE, **noise_kw) -> Case:
    g = latent_image(width, height, seed)
    f = add_noise(blur(g, spec), noise, seed, **noise_kw)
    return Case(g, f, spec, iterations, seed)


# --- the five workloads ------------------------------------------------------

def config1() -> Case:
    """256x256, horizontal motion length 15, Gaussian noise sigma 2, 50 it."""
    return make_case(256, 256, motion(15, 0), 50, "gaussian", SEED_BASE + 1,
                     sigma=2.0)


CONFIG2_PSFS = (motion(31, 0), motion(31, 1), disc(8))


def config2(spec: PsfSpec, size: int = 2048) -> Case:
    """2048x2048, Poisson noise at peak 1000, 200 iterations; one of the three
    PSFs in CONFIG2_PSFS.  The latent image is the same for all three."""
    return make_case(size, size, spec, 200, "poisson", SEED_BASE + 2,
                     peak=1000.0)


def config3(size: int = 4096) -> Case:
    """4096x4096, disc radius 12, Poisson noise at peak 500, 300 iterations."""
    return make_case(size, size, disc(12), 300, "poisson", SEED_BASE + 3,
                     peak=500.0)


def random_psf(rng: np.random.Generator) -> PsfSpec:
    """Per-image PSF of the batched and served workloads: horizontal or
    vertical motion of odd length 5..41, a disc of radius 3..15, or the
    7x7 Gaussian with sigma 1.5."""
    kind = int(rng.integers(0, 4))
    if kind in (0, 1):
        return motion(int(rng.integers(2, 21)) * 2 + 1, kind)
    if kind == 2:
        return disc(int(rng.integers(3, 16)))
    return gaussian(7, 1.5)


def log_uniform_side(rng, lo: int, hi: int) -> int:
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def batch_specs(n: int = 64, lo: int = 128, hi: int = 1536,
                seed: int = SEED_BASE + 4, it_lo: int = 50, it_hi: int = 300):
    """(width, height, PsfSpec, iterations, seed) per image of the batched
    workload; sides log-uniform and drawn independently."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(n):
        w = log_uniform_side(rng, lo, hi)
        h = log_uniform_side(rng, lo, hi)
        spec = random_psf(rng)
        its = int(rng.integers(it_lo, it_hi + 1))
        out.append((w, h, spec, its, seed + 1000 * (j + 1)))
    return out


def batch_case(w, h, spec, its, seed) -> Case:
    return make_case(w, h, spec, its, "poisson", seed, peak=1000.0)


def serve_trace(n: int = 2000, rate: float = 100.0, lo: int = 256,
                hi: int = 4096, it_lo: int = 50, it_hi: int = 500,
                seed: int = SEED_BASE + 5):
    """Poisson-arrival request trace: list of (arrival_s, width, height,
    PsfSpec, iterations, seed)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for j in range(n):
        t += float(rng.exponential(1.0 / rate))
        w = log_uniform_side(rng, lo, hi)
        h = log_uniform_side(rng, lo, hi)
        spec = random_psf(rng)
        its = int(rng.integers(it_lo, it_hi + 1))
        out.append((t, w, h, spec, its, seed + 100000 + j))
    return out


def serve_inputs_device(trace, device: int = 0, bases: int = 4, base_size: int = 4096,
                        peak: float = 1000.0, seed: int = SEED_BASE + 6):
    """Observed images of a served trace, made on the GPU: request j's latent
    image is a crop of one of `bases` seeded 4096^2 latent images, blurred
    by the request's own PSF (Eq. 1, with the half-sample mirror continuation)
    and given Poisson noise at `peak` counts.  Returns float32 CUDA tensors.
    The blur is torch's library convolution: these are benchmark inputs, not
    reference values."""
    import torch
    import torch.nn.functional as F
    dev = torch.device("cuda", device)
    lat = [torch.from_numpy(latent_image(base_size, base_size, seed + k).astype(np.float32)).to(dev)
           for k in range(bases)]
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    rng = np.random.default_rng(seed)
    out = []
    for j, (_, w, h, spec, _, _) in enumerate(trace):
        g = lat[j % bases]
        y0 = int(rng.integers(0, base_size - h + 1))
        x0 = int(rng.integers(0, base_size - w + 1))
        crop = g[y0:y0 + h, x0:x0 + w][None, None]
        taps = torch.from_numpy(np.ascontiguousarray(spec.dense()[::-1, ::-1]).astype(np.float32)).to(dev)
        kh, kw = taps.shape
        py, px = kh // 2, kw // 2
        # half-sample mirror: ... c b a | a b c ...
        x = torch.cat([crop[..., :, :px].flip(-1), crop, crop[..., :, w - (kw - 1 - px):].flip(-1)], dim=-1) \
            if kw > 1 else crop
        x = torch.cat([x[..., :py, :].flip(-2), x, x[..., h - (kh - 1 - py):, :].flip(-2)], dim=-2) \
            if kh > 1 else x
        b = F.conv2d(x, taps[None, None])[0, 0]
        scale = peak / 250.0
        f = torch.poisson(torch.clamp(b, min=0.0) * scale, generator=gen) / scale
        out.append(f.contiguous())
    return out
