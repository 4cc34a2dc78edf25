"""Seeded synthetic rectified stereo pairs.

This module only makes inputs.  It holds none of the stereo method's
arithmetic: it draws a texture, a disparity field and a right view warped
from the left, and it can return the left-grid ground-truth disparity.  The
CUDA path, the CPU oracle, the tests and the benchmark all take their images
from here, so both sides of every parity check see identical bytes.

Two generators stand in for the paper's datasets (synthetic colon 640x480,
SCARED 1280x720, SERV-CT 720x576, Hamlyn), none of which is available:

* ``g1`` -- smoothed Gaussian noise (sigma 1.5 px) scaled to about 40 DN std
  around 128 plus a linear shading ramp of about +-40 DN; disparity is a plane
  plus one Gaussian bump; the right view is the left warped by the disparity
  with linear interpolation plus N(0, 2 DN) noise.
* ``g2`` -- surgical-like statistics: g1 texture, a 5-60 px disparity built
  from six Gaussian bumps, 20% of the area textureless (constant plus
  N(0, 0.5) noise), saturated specular discs (255, radius 5-20 px) placed
  independently in each view, a radial vignette down to 15% and a
  left-to-right gain in [0.9, 1.1].

Convention: disparity d >= 0 with I_r(x - d, y) ~= I_l(x, y).  The warp is
R(x) = C(x + D(x)) where C is the texture canvas (L = C on the image), so the
disparity field D lives on the right-view grid; the left-grid disparity is the
fixed point d(x) = D(x - d(x)).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "StereoPair",
    "g1_pair",
    "g2_pair",
    "shift_pair",
    "quadratic_image",
    "ramp_image",
    "gaussian_blur",
    "config_pair",
    "CONFIGS",
]


@dataclass
class StereoPair:
    left: np.ndarray        # (h, w) uint8 or float64
    right: np.ndarray       # (h, w) uint8 or float64
    disp_right: np.ndarray  # (h, w) float64, D on the right-view grid
    seed: int

    @property
    def shape(self):
        return self.left.shape

    def gt_left(self, iters: int = 30) -> np.ndarray:
        """Left-grid ground-truth disparity by fixed-point iteration of
        d(x) = D(x - d(x)) (linear interpolation of D along x)."""
        h, w = self.disp_right.shape
        xs = np.arange(w, dtype=np.float64)[None, :].repeat(h, 0)
        d = self.disp_right.copy()
        for _ in range(iters):
            xq = np.clip(xs - d, 0.0, w - 1.0)
            x0 = np.floor(xq).astype(np.int64)
            x1 = np.minimum(x0 + 1, w - 1)
            t = xq - x0
            rows = np.arange(h)[:, None]
            d = (1 - t) * self.disp_right[rows, x0] + t * self.disp_right[rows, x1]
        return d


def _gauss_kernel(sigma: float) -> np.ndarray:
    r = int(np.ceil(4.0 * sigma))
    x = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (x / sigma) ** 2)
    return k / k.sum()


def gaussian_blur(img: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian blur with mirror padding (input generator only)."""
    k = _gauss_kernel(sigma)
    r = (len(k) - 1) // 2
    out = np.asarray(img, dtype=np.float64)
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (r, r)
        p = np.pad(out, pad, mode="reflect")
        acc = np.zeros_like(out)
        n = out.shape[axis]
        for i, kv in enumerate(k):
            sl = [slice(None), slice(None)]
            sl[axis] = slice(i, i + n)
            acc += kv * p[tuple(sl)]
        out = acc
    return out


def _canvas_texture(rng: np.random.Generator, h: int, wc: int, w: int) -> np.ndarray:
    """Smoothed-noise texture on a canvas wider than the image (the right
    view samples up to max(D) px to the right of the left image)."""
    noise = rng.standard_normal((h, wc))
    tex = gaussian_blur(noise, 1.5)
    tex = tex / tex.std() * 40.0 + 128.0
    # linear shading ramp of about +-40 DN across the image width
    ramp = 40.0 * (2.0 * np.arange(wc, dtype=np.float64) / max(w - 1, 1) - 1.0)
    return tex + ramp[None, :]


def _warp(canvas: np.ndarray, disp_right: np.ndarray) -> np.ndarray:
    """R(x, y) = C(x + D(x, y), y), linear interpolation along x."""
    h, w = disp_right.shape
    wc = canvas.shape[1]
    xs = np.arange(w, dtype=np.float64)[None, :] + disp_right
    xs = np.clip(xs, 0.0, wc - 1.0)
    x0 = np.floor(xs).astype(np.int64)
    x1 = np.minimum(x0 + 1, wc - 1)
    t = xs - x0
    rows = np.arange(h)[:, None]
    return (1 - t) * canvas[rows, x0] + t * canvas[rows, x1]


def _to_u8(x: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(x), 0, 255).astype(np.uint8)


def _plane_bump(rng, h, w, d0, d1, amp, sigma):
    xs = np.arange(w, dtype=np.float64)[None, :]
    ys = np.arange(h, dtype=np.float64)[:, None]
    cx = rng.uniform(0, w - 1)
    cy = rng.uniform(0, h - 1)
    plane = d0 + (d1 - d0) * xs / max(w - 1, 1)
    bump = amp * np.exp(-((xs - cx) ** 2 + (ys - cy) ** 2) / (2.0 * sigma ** 2))
    return np.broadcast_to(plane, (h, w)) + bump


def g1_pair(w: int, h: int, seed: int, d0: float = 4.0, d1: float = 16.0,
            amp: float = 8.0, sigma: float = 40.0, noise: float = 2.0,
            as_float: bool = False) -> StereoPair:
    """Generator G1: smoothed-noise texture with shading, plane + bump disparity."""
    rng = np.random.default_rng(seed)
    disp = _plane_bump(rng, h, w, d0, d1, amp, sigma)
    wc = w + int(np.ceil(disp.max())) + 4
    canvas = _canvas_texture(rng, h, wc, w)
    left = canvas[:, :w]
    right = _warp(canvas, disp) + rng.normal(0.0, noise, size=(h, w))
    if as_float:
        return StereoPair(left.copy(), right, disp, seed)
    return StereoPair(_to_u8(left), _to_u8(right), disp, seed)


def g2_pair(w: int, h: int, seed: int) -> StereoPair:
    """Generator G2 (surgical-like statistics)."""
    rng = np.random.default_rng(seed)
    xs = np.arange(w, dtype=np.float64)[None, :]
    ys = np.arange(h, dtype=np.float64)[:, None]
    # disparity: 5-60 px from a sum of six Gaussian bumps
    field = np.zeros((h, w))
    for _ in range(6):
        cx, cy = rng.uniform(0, w - 1), rng.uniform(0, h - 1)
        s = rng.uniform(0.06, 0.2) * max(w, h)
        a = rng.uniform(0.3, 1.0)
        field += a * np.exp(-((xs - cx) ** 2 + (ys - cy) ** 2) / (2 * s * s))
    field = (field - field.min()) / max(field.max() - field.min(), 1e-12)
    disp = 5.0 + 55.0 * field
    wc = w + int(np.ceil(disp.max())) + 4
    canvas = _canvas_texture(rng, h, wc, w)
    # 20% of the image area textureless: constant (local shading level) + N(0, 0.5)
    mask = np.zeros((h, wc), dtype=bool)
    target = 0.2 * h * w
    xc = np.arange(wc, dtype=np.float64)[None, :]
    tries = 0
    while mask[:, :w].sum() < target and tries < 200:
        cx, cy = rng.uniform(0, w - 1), rng.uniform(0, h - 1)
        r = rng.uniform(0.05, 0.15) * min(w, h)
        mask |= (xc - cx) ** 2 + (ys - cy) ** 2 <= r * r
        tries += 1
    level = 128.0 + 40.0 * (2.0 * xc / max(w - 1, 1) - 1.0)
    flat = np.broadcast_to(level, (h, wc)) + rng.normal(0.0, 0.5, size=(h, wc))
    canvas = np.where(mask, flat, canvas)
    left = canvas[:, :w].copy()
    right = _warp(canvas, disp)
    right *= rng.uniform(0.9, 1.1)
    # radial vignette down to 15% at the corners (camera effect, per view)
    rr = np.sqrt((xs - (w - 1) / 2) ** 2 + (ys - (h - 1) / 2) ** 2)
    vig = 1.0 - 0.85 * (rr / rr.max()) ** 2
    left *= vig
    right *= vig
    # saturated specular discs, independent per view
    for img in (left, right):
        for _ in range(8):
            cx, cy = rng.uniform(0, w - 1), rng.uniform(0, h - 1)
            r = rng.uniform(5, 20)
            img[(xs - cx) ** 2 + (ys - cy) ** 2 <= r * r] = 255.0
    right += rng.normal(0.0, 2.0, size=(h, w))
    return StereoPair(_to_u8(left), _to_u8(right), disp, seed)


def shift_pair(w: int, h: int, seed: int, shift: int, blur: float = 2.0) -> StereoPair:
    """Right view = left view shifted by a constant integer disparity:
    R(x) = L(x + shift) on the image, from a wider canvas; no noise."""
    rng = np.random.default_rng(seed)
    wc = w + shift + 4
    tex = gaussian_blur(rng.standard_normal((h, wc)), blur)
    tex = tex / tex.std() * 40.0 + 128.0
    left = _to_u8(tex[:, :w])
    right = _to_u8(tex[:, shift:shift + w])
    disp = np.full((h, w), float(shift))
    return StereoPair(left, right, disp, seed)


def quadratic_image(w: int, h: int, beta: float, shift: float = 0.0) -> np.ndarray:
    """I(x, y) = beta * (x + shift)^2, no y dependence (float64)."""
    xs = np.arange(w, dtype=np.float64) + shift
    return np.broadcast_to(beta * xs * xs, (h, w)).copy()


def ramp_image(w: int, h: int, alpha: float, offset: float = 0.0) -> np.ndarray:
    """I(x, y) = alpha * x + offset (float64)."""
    xs = np.arange(w, dtype=np.float64)
    return np.broadcast_to(alpha * xs + offset, (h, w)).copy()


# Workloads.  Each entry: generator, size, method settings.
CONFIGS = {
    # 320x240 G1 pair, 8x8 patches stride 4, 3 levels, 8 GN iterations, fp32 pyramids
    "plain_320x240": dict(gen="g1", w=320, h=240, seed=0, patch=8, stride=4,
                          levels=3, iters=8, variance=0, storage="f32"),
    # 640x480 G2 pair, 12x12 patches stride 6, 4 levels, variance on
    "plain_640x480_var": dict(gen="g2", w=640, h=480, seed=0, patch=12, stride=6,
                              levels=4, iters=8, variance=1, storage="f32"),
    # 1920x1080 G1 pair (10-160 px), 12x12 stride 4, 6 levels, variance on, fp16 pyramids
    "plain_1920x1080_f16": dict(gen="g1_hd", w=1920, h=1080, seed=0, patch=12,
                                stride=4, levels=6, iters=8, variance=1,
                                storage="f16"),
}


def config_pair(name: str, seed: int | None = None) -> StereoPair:
    c = CONFIGS[name]
    s = c["seed"] if seed is None else seed
    if c["gen"] == "g1":
        return g1_pair(c["w"], c["h"], s)
    if c["gen"] == "g2":
        return g2_pair(c["w"], c["h"], s)
    if c["gen"] == "g1_hd":
        return g1_pair(c["w"], c["h"], s, d0=10.0, d1=140.0, amp=20.0, sigma=240.0)
    raise KeyError(name)


def batch_sizes_uneven():
    """The uneven-size video batch: 24x640x480, 16x960x540, 16x1280x720,
    8x1920x1080 (64 pairs, G1 generator, seeds 0..63)."""
    sizes = [(640, 480)] * 24 + [(960, 540)] * 16 + [(1280, 720)] * 16 + [(1920, 1080)] * 8
    return sizes
