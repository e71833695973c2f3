"""Seeded synthetic inputs for radio-interferometric imaging problems.

This module draws random numbers only: sky images, (u, v) coverages, block
sizes and unit-variance complex noise. It holds none of the imaging method's
arithmetic (no measurement operator, no wavelet, no noise-level or epsilon
computation), so the CPU oracle and the CUDA path can both take their inputs
from here without sharing any of the method.

The paper (Sec. 1, measurement model y = Phi x + n) fixes no dataset; these
generators stand in for the telescope data it motivates. Recipes:

* sky: point sources at uniform positions inside the central 80% of the field,
  Exp(1) fluxes, plus Gaussian blobs with amplitude U(0.2, 1) and width
  U(1, 3) * (n / 64) pixels; optionally a smooth diffuse component (a low-pass
  filtered Gaussian random field, exponentiated, scaled to 10% of the peak).
  The image is positive and its peak is 1.
* (u, v): 2-D Gaussian density with standard deviation pi/4 per axis, truncated
  to [-pi, pi)^2 by rejection; an optional fraction is drawn uniformly on
  [-pi, pi)^2 instead. Units are radians per pixel.
* block sizes: lognormal(sigma) draws normalised to M by largest-remainder
  rounding, each at least 1 (the contiguous partition of Eq. 2).
* noise: complex samples (a + i b) / sqrt(2), a, b ~ N(0, 1).
* block-group sequences: uniform draws from {0, ..., G-1}, one per iteration.

Seeds follow one PCG64 stream per role: sky 1000 + c, uv 2000 + c,
noise 3000 + c, blocks 4000 + c for workload index c.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * np.pi


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _gaussian_blob(ny: int, nx: int, cy: float, cx: float, sigma: float) -> np.ndarray:
    iy = np.arange(ny)[:, None]
    ix = np.arange(nx)[None, :]
    return np.exp(-((iy - cy) ** 2 + (ix - cx) ** 2) / (2.0 * sigma * sigma))


def sky(nx: int, ny: int, seed: int, n_points: int = 20, n_blobs: int = 3,
        diffuse: bool = False) -> np.ndarray:
    """Positive synthetic sky, float64 [ny][nx], peak normalised to 1."""
    g = rng(seed)
    img = np.zeros((ny, nx), dtype=np.float64)
    lo_y, hi_y = 0.1 * ny, 0.9 * ny
    lo_x, hi_x = 0.1 * nx, 0.9 * nx
    py = g.integers(int(np.ceil(lo_y)), int(np.floor(hi_y)), size=n_points)
    px = g.integers(int(np.ceil(lo_x)), int(np.floor(hi_x)), size=n_points)
    flux = g.exponential(1.0, size=n_points)
    np.add.at(img, (py, px), flux)
    scale = max(nx, ny) / 64.0
    for _ in range(n_blobs):
        amp = g.uniform(0.2, 1.0)
        sig = g.uniform(1.0, 3.0) * scale
        cy = g.uniform(0, ny)
        cx = g.uniform(0, nx)
        img += amp * _gaussian_blob(ny, nx, cy, cx, sig)
    if diffuse:
        field_ = g.standard_normal((ny, nx))
        fy = np.fft.fftfreq(ny)[:, None]
        fx = np.fft.fftfreq(nx)[None, :]
        lowpass = np.exp(-(fx * fx + fy * fy) / (2.0 * 0.02 ** 2))
        smooth = np.real(np.fft.ifft2(np.fft.fft2(field_) * lowpass))
        smooth /= max(np.std(smooth), 1e-300)
        diff = np.exp(smooth)
        diff *= 0.1 * img.max() / diff.max()
        img += diff
    img /= img.max()
    return img


def uv_coverage(M: int, seed: int, sigma: float = np.pi / 4.0,
                uniform_fraction: float = 0.0,
                dtype=np.float64) -> tuple[np.ndarray, np.ndarray]:
    """(u, v) in radians/pixel on [-pi, pi): truncated Gaussian plus optional
    uniform fraction. Returned in the requested dtype; values are clamped so
    that rounding to float32 never produces +pi."""
    g = rng(seed)
    n_uni = int(round(uniform_fraction * M))
    n_gau = M - n_uni
    us = np.empty(0)
    vs = np.empty(0)
    while us.size < n_gau:
        need = n_gau - us.size
        cu = g.normal(0.0, sigma, size=int(need * 1.1) + 16)
        cv = g.normal(0.0, sigma, size=cu.size)
        keep = (cu >= -np.pi) & (cu < np.pi) & (cv >= -np.pi) & (cv < np.pi)
        us = np.concatenate([us, cu[keep]])[:n_gau]
        vs = np.concatenate([vs, cv[keep]])[:n_gau]
    if n_uni:
        us = np.concatenate([us, g.uniform(-np.pi, np.pi, size=n_uni)])
        vs = np.concatenate([vs, g.uniform(-np.pi, np.pi, size=n_uni)])
        order = g.permutation(M)
        us, vs = us[order], vs[order]
    u = us.astype(dtype)
    v = vs.astype(dtype)
    top = np.nextafter(dtype(np.pi), dtype(0)) if np.dtype(dtype) == np.float32 else np.nextafter(np.pi, 0)
    u = np.where(u >= np.pi, top, u).astype(dtype)
    v = np.where(v >= np.pi, top, v).astype(dtype)
    return u, v


def block_sizes(M: int, R: int, seed: int, sigma: float = 0.5) -> np.ndarray:
    """R uneven positive block sizes summing to M (lognormal weights,
    largest-remainder rounding, each >= 1)."""
    if R < 1 or M < R:
        raise ValueError("need 1 <= R <= M")
    if R == 1:
        return np.array([M], dtype=np.int64)
    g = rng(seed)
    w = g.lognormal(0.0, sigma, size=R)
    spare = M - R
    share = w / w.sum() * spare
    base = np.floor(share).astype(np.int64)
    left = spare - int(base.sum())
    order = np.argsort(-(share - base), kind="stable")
    base[order[:left]] += 1
    return base + 1


def block_offsets(sizes: np.ndarray) -> np.ndarray:
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def unit_noise(M: int, seed: int) -> np.ndarray:
    """Complex128 noise with E|n_m|^2 = 1: (a + i b)/sqrt(2)."""
    g = rng(seed)
    a = g.standard_normal(M)
    b = g.standard_normal(M)
    return (a + 1j * b) / np.sqrt(2.0)


def group_sequence(n: int, G: int, seed: int) -> np.ndarray:
    """n block-group indices drawn uniformly from {0, ..., G-1} (the group of
    each iteration of a stochastic block-subset solve), int32."""
    return rng(seed).integers(0, G, size=n).astype(np.int32)


@dataclass
class Workload:
    """Sizes and seeds of one synthetic imaging problem."""
    name: str
    nx: int
    ny: int
    M: int
    J: int
    levels: int
    R: int
    snr_db: float
    dtype: str = "f32"
    oversample: float = 2.0
    n_points: int = 20
    n_blobs: int = 3
    diffuse: bool = False
    uniform_fraction: float = 0.0
    index: int = 1
    extra: dict = field(default_factory=dict)

    def draw(self):
        """Return (sky, u, v, block_offsets, unit_noise) for this workload."""
        c = self.index
        fdt = np.float32 if self.dtype == "f32" else np.float64
        x = sky(self.nx, self.ny, 1000 + c, self.n_points, self.n_blobs, self.diffuse)
        u, v = uv_coverage(self.M, 2000 + c, uniform_fraction=self.uniform_fraction, dtype=fdt)
        nz = unit_noise(self.M, 3000 + c)
        offs = block_offsets(block_sizes(self.M, self.R, 4000 + c))
        return x, u, v, offs, nz


# The five imaging workloads: plain FP64 64x64; 256x256 with 8 blocks;
# 1024x1024 with 64 blocks; one 512x512 channel of the 32-channel batch;
# the 256x256 warm-start problem.
WORKLOADS = {
    "sara64_fp64": Workload("sara64_fp64", 64, 64, 8192, 4, 3, 1, 30.0, "f64", index=0),
    "sara256_r8": Workload("sara256_r8", 256, 256, 655360, 6, 4, 8, 30.0, "f32", index=1),
    "sara1024_r64": Workload("sara1024_r64", 1024, 1024, 10485760, 6, 5, 64, 20.0, "f32",
                             n_points=500, n_blobs=40, diffuse=True,
                             uniform_fraction=0.1, index=2),
    "sara256_warm": Workload("sara256_warm", 256, 256, 131072, 4, 3, 1, 30.0, "f32", index=4),
}


def channel_workload(ch: int, n: int = 512) -> Workload:
    """Channel ch of the 32-channel batch: M ~ U(0.5N, 5N), R ~ U{4..16}."""
    g = rng(5000 + ch)
    N = n * n
    M = int(g.integers(N // 2, 5 * N + 1))
    R = int(g.integers(4, 17))
    return Workload(f"chan{ch}", n, n, M, 6, 4, R, 30.0, "f32", index=100 + ch)
