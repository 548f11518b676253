"""Seeded synthetic inputs shaped like the paper's tracking workloads.

The paper evaluates on a VOT2016 frame (Sec. 3, Fig. 5) and on wide-area
aerial imagery (Sec. 4, Fig. 7); neither is available here, so these
generators produce stand-ins with the same sizes, bit depths and structure:
a smooth textured background with compact textured objects planted on it.

This module holds no arithmetic of the histogram method itself (no
quantisation, no weighting, no integral histograms). Both the CUDA path and
the CPU oracle consume its outputs, and nothing else is shared between them.
Every generator is a pure function of its arguments and a seed
(``numpy.random.default_rng``), so the same call gives the same array on any
machine with the same numpy.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "uniform_image",
    "fbm_value_noise",
    "blob_scene",
    "Scene",
    "config1",
    "config2",
    "config3",
    "config4",
    "config5_frames",
    "config5_queries",
    "config5_repeat_queries",
    "odd_window",
]


def uniform_image(h: int, w: int, bitdepth: int = 8, seed: int = 1) -> np.ndarray:
    """i.i.d. uniform pixels in [0, 2^bitdepth) as uint8 (bitdepth 8) or uint16."""
    rng = np.random.default_rng(seed)
    dtype = np.uint8 if bitdepth <= 8 else np.uint16
    return rng.integers(0, 1 << bitdepth, size=(h, w), dtype=np.int64).astype(dtype)


def _quintic_fade(t: np.ndarray) -> np.ndarray:
    # Perlin's improved-noise fade curve 6t^5 - 15t^4 + 10t^3 (Perlin, 2002).
    return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)


def fbm_value_noise(h: int, w: int, octaves: int, cell: float, rng: np.random.Generator,
                    gain: float = 0.5) -> np.ndarray:
    """Fractal sum of lattice value noise, normalised to [-1, 1] (float64, h x w).

    Octave o uses a lattice of spacing ``cell / 2^o`` with i.i.d. U[-1, 1]
    values interpolated by the quintic fade; amplitudes fall by ``gain``.
    """
    out = np.zeros((h, w), dtype=np.float64)
    norm = 0.0
    amp = 1.0
    for o in range(octaves):
        c = max(cell / (2.0 ** o), 2.0)
        gy = int(np.ceil(h / c)) + 2
        gx = int(np.ceil(w / c)) + 2
        lat = rng.uniform(-1.0, 1.0, size=(gy, gx))
        ys = np.arange(h) / c
        xs = np.arange(w) / c
        y0 = np.floor(ys).astype(np.int64)
        x0 = np.floor(xs).astype(np.int64)
        fy = _quintic_fade(ys - y0)[:, None]
        fx = _quintic_fade(xs - x0)[None, :]
        v00 = lat[y0][:, x0]
        v01 = lat[y0][:, x0 + 1]
        v10 = lat[y0 + 1][:, x0]
        v11 = lat[y0 + 1][:, x0 + 1]
        top = v00 + (v01 - v00) * fx
        bot = v10 + (v11 - v10) * fx
        out += amp * (top + (bot - top) * fy)
        norm += amp
        amp *= gain
    return out / norm


@dataclass
class Scene:
    """A generated frame plus the ground-truth objects planted in it."""

    image: np.ndarray
    bitdepth: int
    # (cx, cy) integer centres of the planted objects; index 0 is the target.
    centres: list = field(default_factory=list)
    # (semi-axis a, semi-axis b, angle, mean) per planted object
    params: list = field(default_factory=list)


def _plant_ellipse(img: np.ndarray, rng: np.random.Generator, cx: int, cy: int, a: float, b: float,
                   ang: float, mean: float, noise_std: float) -> None:
    """Overwrite the pixels of an ellipse (semi-axes a, b, rotated by ang,
    centred on (cx, cy)) with mean + N(0, noise_std) texture, drawn in
    row-major order. Only the ellipse's bounding square is visited, which
    gives the same pixels and draws as visiting the whole frame."""
    h, w = img.shape
    R = int(np.ceil(max(a, b))) + 1
    ys, ye = max(cy - R, 0), min(cy + R + 1, h)
    xs, xe = max(cx - R, 0), min(cx + R + 1, w)
    yy, xx = np.mgrid[ys:ye, xs:xe]
    ca, sa = np.cos(ang), np.sin(ang)
    u = (xx - cx) * ca + (yy - cy) * sa
    v = -(xx - cx) * sa + (yy - cy) * ca
    inside = (u / a) ** 2 + (v / b) ** 2 <= 1.0
    n_in = int(inside.sum())
    sub = img[ys:ye, xs:xe]
    sub[inside] = mean + rng.normal(0.0, noise_std, size=n_in)


def blob_scene(h: int, w: int, bitdepth: int, seed: int, n_blobs: int,
               axes: tuple = (10, 60), octaves: int = 4, cell: float = 128.0,
               bg_mean_frac: float = 0.5, bg_amp_frac: float = 48.0 / 256.0,
               noise_frac: float = 12.0 / 256.0, margin: int = 64) -> Scene:
    """Smooth fBm background plus textured elliptical objects.

    Background: ``mean + amp * fbm`` with mean and amplitude given as
    fractions of the full range (128 +- 48 for 8-bit images). Each object is
    an ellipse with semi-axes drawn from U[axes], a random orientation, a
    mean level drawn uniformly from the middle 70% of the range and i.i.d.
    Gaussian texture of std ``noise_frac * range`` (12 for 8-bit images).
    Values are rounded and clamped to the pixel range.
    """
    rng = np.random.default_rng(seed)
    full = float(1 << bitdepth)
    img = bg_mean_frac * full + bg_amp_frac * full * fbm_value_noise(h, w, octaves, cell, rng)
    centres = []
    params = []
    lo_mean = int(0.15625 * full)   # 40 for 8-bit
    hi_mean = int(0.83984375 * full)  # 215 for 8-bit
    for _ in range(n_blobs):
        a = rng.uniform(axes[0], axes[1])
        b = rng.uniform(axes[0], axes[1])
        ang = rng.uniform(0.0, np.pi)
        mean = float(rng.integers(lo_mean, hi_mean + 1))
        m = min(margin, h // 2 - 1, w // 2 - 1)
        cx = int(rng.integers(m, w - m))
        cy = int(rng.integers(m, h - m))
        _plant_ellipse(img, rng, cx, cy, a, b, ang, mean, noise_frac * full)
        centres.append((cx, cy))
        params.append((a, b, ang, mean))
    img = np.clip(np.rint(img), 0, full - 1)
    dtype = np.uint8 if bitdepth <= 8 else np.uint16
    return Scene(image=img.astype(dtype), bitdepth=bitdepth, centres=centres, params=params)


def odd_window(size: float) -> int:
    """Nearest odd integer >= 3 to a (possibly fractional) window size."""
    n = 2 * int(round((size - 1.0) / 2.0)) + 1
    return max(n, 3)


def config1(seed: int = 1) -> dict:
    """128x128 uint8 i.i.d. uniform image, B=16, one 31x31 Manhattan window,
    target = the window at the image centre (64, 64)."""
    img = uniform_image(128, 128, 8, seed)
    return dict(image=img, bitdepth=8, B=16, kernels=("manhattan",), windows=(31,),
                target_centre=(64, 64))


def config2(seed: int = 2, size: int = 1024) -> dict:
    """1024x1024 uint8 smooth background + 8 textured elliptical objects,
    B=32, Manhattan / Euclidean / Gaussian kernels at windows 21, 41, 81;
    the target is the window centred on object 0."""
    sc = blob_scene(size, size, 8, seed, n_blobs=8)
    return dict(image=sc.image, bitdepth=8, B=32,
                kernels=("manhattan", "euclidean", "gaussian"), windows=(21, 41, 81),
                target_centre=sc.centres[0], scene=sc)


def feature_channels(image: np.ndarray, seed: int) -> list:
    """Three feature images of one u8 scene, in the roles of the tracker's
    intensity, texture and coarse colour features (Sec. 4): the scene itself
    (u8, 8 bits); a 12-bit texture-like channel mixing the scene with seeded
    uniform noise (u16); and a 6-bit channel derived from the scene (u8).
    Returns [(array, bitdepth)]; the array's dtype gives the pixel type."""
    H, W = image.shape
    sc = image.astype(np.int64)
    tex = uniform_image(H, W, 16, seed=seed).astype(np.int64) >> 4  # 12 significant bits
    tex = ((tex + 16 * sc) % 4096).astype(np.uint16)
    six = (sc * 3 // 4 % 64).astype(np.uint8)
    return [(image, 8), (tex, 12), (six, 6)]


def config3(seed: int = 3, n_rois: int = 64, size: int = 4096, roi_range: tuple = (96, 768),
            box_range: tuple = (24, 64)) -> dict:
    """Batched search regions: a 4096 x 4096 uint16 frame (fBm background
    spanning the 16-bit range with i.i.d. Gaussian texture of std 2% of the
    range, plus one textured elliptical object per region), 64 regions with width and height drawn independently from
    U[96, 768], each with a target box side s ~ U[24, 64] and windows at
    0.8 s, s and 1.25 s rounded to odd sides; B = 64, Gaussian kernel.

    The object of region i sits near the region's centre with semi-axes
    about s / 2, so the region's search map has one true peak. Returns the
    frame, the regions as (x0, y0, width, height), the window sides per
    region, and the object centre per region (frame coordinates)."""
    rng = np.random.default_rng(seed)
    full = float(1 << 16)
    img = 0.5 * full + 0.3 * full * fbm_value_noise(size, size, 5, 512.0, rng)
    img += rng.normal(0.0, 0.02 * full, size=img.shape)  # sensor-like texture
    rois, windows, centres = [], [], []
    for _ in range(n_rois):
        rw = int(rng.integers(roi_range[0], roi_range[1] + 1))
        rh = int(rng.integers(roi_range[0], roi_range[1] + 1))
        x0 = int(rng.integers(0, size - rw + 1))
        y0 = int(rng.integers(0, size - rh + 1))
        s = float(rng.uniform(box_range[0], box_range[1]))
        wins = [odd_window(0.8 * s), odd_window(s), odd_window(1.25 * s)]
        cx = x0 + rw // 2 + int(rng.integers(-rw // 8, rw // 8 + 1))
        cy = y0 + rh // 2 + int(rng.integers(-rh // 8, rh // 8 + 1))
        a = 0.5 * s * float(rng.uniform(0.7, 1.0))
        b = 0.5 * s * float(rng.uniform(0.7, 1.0))
        ang = float(rng.uniform(0.0, np.pi))
        mean = float(rng.integers(int(0.15 * full), int(0.85 * full)))
        _plant_ellipse(img, rng, cx, cy, a, b, ang, mean, 0.05 * full)
        rois.append((x0, y0, rw, rh))
        windows.append(wins)
        centres.append((cx, cy))
    img = np.clip(np.rint(img), 0, full - 1).astype(np.uint16)
    return dict(image=img, bitdepth=16, B=64, kernel="gaussian", rois=rois, windows=windows,
                object_centres=centres)


SERVE_WINDOWS = (15, 25, 43, 75, 127)


def config5_frames(seed: int = 5, n_frames: int = 16, size: int = 2048, n_blobs: int = 50) -> list:
    """Resident frames for the serving workload: one fBm background (16-bit
    range, 2% Gaussian texture) shifted a few pixels per frame, with n_blobs
    textured ellipses of 8-40 px moving at constant velocities; frame i holds
    them at their positions at time i. Even frames are uint8 (the 16-bit
    values >> 8), odd frames uint16. Returns [(image, bitdepth)]."""
    rng = np.random.default_rng(seed)
    full = float(1 << 16)
    bg = 0.5 * full + 0.3 * full * fbm_value_noise(size + 64, size + 64, 4, 256.0, rng)
    blobs = []
    for _ in range(n_blobs):
        a = float(rng.uniform(4, 20))
        b = float(rng.uniform(4, 20))
        blobs.append((float(rng.uniform(64, size - 64)), float(rng.uniform(64, size - 64)),
                      float(rng.uniform(-6, 6)), float(rng.uniform(-6, 6)), a, b,
                      float(rng.uniform(0, np.pi)), float(rng.integers(int(0.15 * full), int(0.85 * full)))))
    frames = []
    for i in range(n_frames):
        dx, dy = (3 * i) % 64, (2 * i) % 64
        img = bg[dy: dy + size, dx: dx + size].copy()
        img += rng.normal(0.0, 0.02 * full, size=img.shape)
        for (x, y, vx, vy, a, b, ang, mean) in blobs:
            cx = int(np.clip(x + vx * i, 0, size - 1))
            cy = int(np.clip(y + vy * i, 0, size - 1))
            _plant_ellipse(img, rng, cx, cy, a, b, ang, mean, 0.05 * full)
        img = np.clip(np.rint(img), 0, full - 1)
        if i % 2 == 0:
            frames.append(((img.astype(np.uint32) >> 8).astype(np.uint8), 8))
        else:
            frames.append((img.astype(np.uint16), 16))
    return frames


def config5_queries(seed: int = 5, n: int = 1000, rate: float = 2000.0, n_frames: int = 16,
                    size: int = 2048, crop_range: tuple = (64, 1024)) -> list:
    """A Poisson stream of tracking queries: arrival times with mean rate
    ``rate`` per second, a frame drawn uniformly, crop width and height drawn
    independently from U{64..1024} at a uniform position, B from {16, 32, 64},
    kernel from {Manhattan, Euclidean, Gaussian}, 1-8 targets (seeded
    normalised histograms) and 1-5 windows drawn from the sizes
    15/25/43/75/127 that fit the crop. Returns a list of dicts."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    kernels = ("manhattan", "euclidean", "gaussian")
    for _ in range(n):
        t += float(rng.exponential(1.0 / rate))
        w = int(rng.integers(crop_range[0], crop_range[1] + 1))
        h = int(rng.integers(crop_range[0], crop_range[1] + 1))
        x0 = int(rng.integers(0, size - w + 1))
        y0 = int(rng.integers(0, size - h + 1))
        B = int(rng.choice([16, 32, 64]))
        kernel = kernels[int(rng.integers(0, 3))]
        nt = int(rng.integers(1, 9))
        fit = [s for s in SERVE_WINDOWS if s <= min(w, h)]
        ns = min(int(rng.integers(1, 6)), len(fit))
        wins = sorted(int(v) for v in rng.choice(fit, ns, replace=False))
        targets = rng.gamma(0.5, 1.0, size=(nt, B))
        targets /= targets.sum(1, keepdims=True)
        out.append(dict(t=t, frame=int(rng.integers(0, n_frames)), x0=x0, y0=y0, w=w, h=h, B=B,
                        kernel=kernel, windows=[(v, v) for v in wins], targets=targets.astype(np.float32)))
    return out


def config5_repeat_queries(seed: int = 6, n_frames: int = 16, size: int = 2048, regions_per_frame: int = 5,
                           repeats: int = 5, rate: float = 2000.0, crop_range: tuple = (256, 512)) -> list:
    """Tracking queries that come back to the same search regions: on each
    frame, regions_per_frame search regions (side U{256..512} at a uniform
    position, B from {16, 32}, kernel Manhattan or Euclidean), each queried
    `repeats` times (a tracker asking again for other targets or scales of a
    candidate region) at Poisson arrival times of mean rate `rate`, in a
    seeded random order. Each query has 1-4 targets and 1-3 windows of
    15/25/43/75/127 that fit the crop. Same dict layout as config5_queries."""
    rng = np.random.default_rng(seed)
    regions = []
    for f in range(n_frames):
        for _ in range(regions_per_frame):
            w = int(rng.integers(crop_range[0], crop_range[1] + 1))
            h = int(rng.integers(crop_range[0], crop_range[1] + 1))
            regions.append((f, int(rng.integers(0, size - w + 1)), int(rng.integers(0, size - h + 1)), w, h,
                            int(rng.choice([16, 32])), ("manhattan", "euclidean")[int(rng.integers(0, 2))]))
    order = [r for r in range(len(regions)) for _ in range(repeats)]
    rng.shuffle(order)
    out = []
    t = 0.0
    for r in order:
        f, x0, y0, w, h, B, kernel = regions[r]
        t += float(rng.exponential(1.0 / rate))
        nt = int(rng.integers(1, 5))
        fit = [v for v in SERVE_WINDOWS if v <= min(w, h)]
        ns = min(int(rng.integers(1, 4)), len(fit))
        wins = sorted(int(v) for v in rng.choice(fit, ns, replace=False))
        targets = rng.gamma(0.5, 1.0, size=(nt, B))
        targets /= targets.sum(1, keepdims=True)
        out.append(dict(t=t, frame=f, x0=x0, y0=y0, w=w, h=h, B=B, kernel=kernel,
                        windows=[(v, v) for v in wins], targets=targets.astype(np.float32)))
    return out


def fbm_value_noise_rows(h: int, w: int, octaves: int, cell: float, rng: np.random.Generator,
                         gain: float = 0.5, chunk: int = 512) -> np.ndarray:
    """fbm_value_noise computed in float32, a block of rows at a time (for
    frames of tens of megapixels). The lattices are drawn in the same order;
    values agree with fbm_value_noise to float32 rounding."""
    lats = []
    for o in range(octaves):
        c = max(cell / (2.0 ** o), 2.0)
        gy = int(np.ceil(h / c)) + 2
        gx = int(np.ceil(w / c)) + 2
        lats.append((c, rng.uniform(-1.0, 1.0, size=(gy, gx)).astype(np.float32)))
    out = np.zeros((h, w), dtype=np.float32)
    norm = sum(gain ** o for o in range(octaves))
    for o, (c, lat) in enumerate(lats):
        amp = np.float32(gain ** o / norm)
        xs = np.arange(w) / c
        x0 = np.floor(xs).astype(np.int64)
        fx = _quintic_fade(xs - x0).astype(np.float32)[None, :]
        for r0 in range(0, h, chunk):
            ys = np.arange(r0, min(h, r0 + chunk)) / c
            y0 = np.floor(ys).astype(np.int64)
            fy = _quintic_fade(ys - y0).astype(np.float32)[:, None]
            l0 = lat[y0]
            l1 = lat[y0 + 1]
            top = l0[:, x0] + (l0[:, x0 + 1] - l0[:, x0]) * fx
            bot = l1[:, x0] + (l1[:, x0 + 1] - l1[:, x0]) * fx
            out[r0: r0 + len(ys)] += amp * (top + (bot - top) * fy)
    return out


def config4(seed: int = 4, size: int = 8192, n_blobs: int = 200, frame_index: int = 0) -> dict:
    """Large single frame: 8192 x 8192 uint16 wide-area-like synthetic, a
    fractal terrain (6 octaves of value noise, lattice 1024 px, 0.5 +- 0.35 of
    the range, 2% Gaussian texture) plus 200 textured ellipses of 8-40 px
    moving at constant velocities (shown at time frame_index); B = 64,
    Gaussian and Euclidean kernels, windows 15/25/43/75/127 (geometric)."""
    rng = np.random.default_rng(seed)
    full = float(1 << 16)
    img = 0.5 * full + 0.35 * full * fbm_value_noise_rows(size, size, 6, 1024.0, rng)
    img += rng.normal(0.0, 0.02 * full, size=img.shape).astype(np.float32)
    centres = []
    for _ in range(n_blobs):
        x, y = float(rng.uniform(64, size - 64)), float(rng.uniform(64, size - 64))
        vx, vy = float(rng.uniform(-8, 8)), float(rng.uniform(-8, 8))
        d = float(rng.uniform(8, 40))
        a = 0.5 * d
        b = 0.5 * d * float(rng.uniform(0.5, 1.0))
        ang = float(rng.uniform(0, np.pi))
        mean = float(rng.integers(int(0.1 * full), int(0.9 * full)))
        cx = int(np.clip(x + vx * frame_index, 0, size - 1))
        cy = int(np.clip(y + vy * frame_index, 0, size - 1))
        _plant_ellipse(img, rng, cx, cy, a, b, ang, mean, 0.05 * full)
        centres.append((cx, cy))
    np.rint(img, out=img)
    np.clip(img, 0, full - 1, out=img)
    return dict(image=img.astype(np.uint16), bitdepth=16, B=64, kernels=("gaussian", "euclidean"),
                windows=SERVE_WINDOWS, object_centres=centres)
