"""Video-shaped robust-PCA instances standing in for the background-subtraction videos of
Section 3 (the recorded videos themselves are not used).

Each column of D is one vectorised frame (pixel p = y * width + x), as in the paper's
video experiment.  The background is exactly rank 2: a static smooth image b (values in
[0.1, 0.7]) plus a slow global illumination ramp l_t (values in [0, 0.2]), so
L*_{p,t} = b_p + l_t.  Three axis-aligned rectangles of U{12..30} x U{16..40} pixels move on
reflecting random walks; each has an intensity drawn uniformly from [0, 1] and occludes
the background, so S*_{p,t} = intensity - L*_{p,t} on its pixels.  Gaussian noise with
standard deviation ``noise`` is added to every entry.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class VideoInstance:
    width: int
    height: int
    frames: int
    seed: int
    background: np.ndarray   # (m,) static image b
    ramp: np.ndarray         # (n,) illumination l
    D: np.ndarray            # m x n float64
    fg_mask: np.ndarray      # m x n bool, pixels covered by a rectangle
    noise: float

    @property
    def m(self) -> int:
        return self.width * self.height

    @property
    def n(self) -> int:
        return self.frames

    @property
    def L(self) -> np.ndarray:
        return self.background[:, None] + self.ramp[None, :]


def _smooth_image(rng: np.random.Generator, width: int, height: int) -> np.ndarray:
    y, x = np.mgrid[0:height, 0:width]
    img = np.zeros((height, width))
    for _ in range(6):
        fx, fy = rng.uniform(0.2, 2.0, size=2)
        ph = rng.uniform(0, 2 * np.pi, size=2)
        a = rng.standard_normal()
        img += a * np.cos(2 * np.pi * fx * x / width + ph[0]) * np.cos(2 * np.pi * fy * y / height + ph[1])
    img -= img.min()
    img /= max(img.max(), 1e-12)
    return 0.1 + 0.6 * img


def video_instance(width: int = 176, height: int = 144, frames: int = 2000, seed: int = 0,
                   noise: float = 1e-3, n_rects: int = 3) -> VideoInstance:
    rng = np.random.Generator(np.random.PCG64(seed))
    m = width * height
    b = _smooth_image(rng, width, height).reshape(-1)
    t = np.arange(frames)
    ramp = 0.2 * t / max(frames - 1, 1)
    D = b[:, None] + ramp[None, :]
    mask = np.zeros((m, frames), dtype=bool)
    hs = rng.integers(12, 31, size=n_rects)
    ws = rng.integers(16, 41, size=n_rects)
    inten = rng.uniform(0.0, 1.0, size=n_rects)
    ys = np.array([rng.integers(0, height - h + 1) for h in hs])
    xs = np.array([rng.integers(0, width - w + 1) for w in ws])
    for f in range(frames):
        col = D[:, f].reshape(height, width).copy()
        cov = np.zeros((height, width), dtype=bool)
        for q in range(n_rects):
            col[ys[q]:ys[q] + hs[q], xs[q]:xs[q] + ws[q]] = inten[q]
            cov[ys[q]:ys[q] + hs[q], xs[q]:xs[q] + ws[q]] = True
        D[:, f] = col.reshape(-1)
        mask[:, f] = cov.reshape(-1)
        for q in range(n_rects):
            dy, dx = rng.integers(-2, 3, size=2)
            ny, nx = ys[q] + dy, xs[q] + dx
            if ny < 0 or ny > height - hs[q]:
                ny = ys[q] - dy
            if nx < 0 or nx > width - ws[q]:
                nx = xs[q] - dx
            ys[q] = min(max(ny, 0), height - hs[q])
            xs[q] = min(max(nx, 0), width - ws[q])
    D += noise * rng.standard_normal(D.shape)
    return VideoInstance(width=width, height=height, frames=frames, seed=seed, background=b,
                         ramp=ramp, D=D, fg_mask=mask, noise=noise)
