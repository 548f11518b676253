"""CPU FP64 oracle for spatially weighted local histograms (SWIH).

TEST INFRASTRUCTURE ONLY. The only code allowed to import, call or execute
anything under ``oracle/`` is the test suite, the package smoke check in
``__graft_entry__.py`` and the CPU-baseline leg of ``bench.py``. The CUDA
library never links it and this module never imports the CUDA library; the
two share nothing but the seeded input generators.

Every function states the passage of the paper it writes out. Where the
paper is silent the reading taken is stated in the docstring:

* ``quantize`` -- the quantiser Q of Sec. 2.1 (named after Eq. 2, not
  defined): equal-width bins, b = floor(v * B / 2^bitdepth).
* ``weighted_ih`` -- Eq. 2 with the pixel weight w(i, j) = i^p j^q, as a
  plain double cumulative sum. Kept in the ring Z / 2^bits, which is exact
  modular arithmetic: the CUDA path stores the same ring elements, so the
  comparison is bit for bit.
* ``kernel_weights`` -- the spatial kernels of Fig. 1 / Sec. 2:
  Manhattan from the city-block distance of Eq. 1, Euclidean and Gaussian
  (the paper names these without a formula; readings below).
* ``hist_*`` / ``likelihood_*`` -- the brute-force approach of Sec. 2
  (visit every pixel of every window), normalised by the window's own
  total weight, scored by the Bhattacharyya coefficient (the paper leaves
  the similarity unnamed).

The exponential kernel's four directional integral histograms
(``exp_directional_ih``) are Eq. 2 with the weights exp(+-lam x) exp(+-lam y),
each summed from the side where its weight is smallest and divided by the
weight at the point (the paper names the kernel without a decomposition).

Parity unpinned: the Gaussian kernel is a polynomial approximant (the paper
gives no decomposition of it); its distance from the true Gaussian is
reported by the tests, not pinned to a value printed in the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from functools import lru_cache

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "brute.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD_DIR, "libswih_oracle.so")

KINDS = ("plain", "manhattan", "euclidean", "gaussian", "exponential")
EXP_LAMBDA = 0.1  # default decay rate of the exponential kernel, per pixel


# --------------------------------------------------------------------------
# build / load the brute-force C routines
# --------------------------------------------------------------------------
def build(force: bool = False) -> str:
    """Compile brute.c into a shared object with gcc (-O2, OpenMP, no fast-math)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


@lru_cache(maxsize=1)
def _lib() -> ctypes.CDLL:
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    I = ctypes.c_int
    L = ctypes.c_long
    lib.swih_oracle_threads.restype = I
    lib.swih_oracle_hist_at.argtypes = [P, I, I, I, P, I, I, P, P, L, P]
    lib.swih_oracle_hist_rect.argtypes = [P, I, I, I, P, I, I, I, I, I, I, P]
    lib.swih_oracle_likelihood_at.argtypes = [P, I, I, I, P, I, I, P, P, L, P, P]
    lib.swih_oracle_likelihood_rect.argtypes = [P, I, I, I, P, I, I, I, I, I, I, P, P]
    return lib


def threads() -> int:
    """OpenMP threads the brute-force loops use."""
    return int(_lib().swih_oracle_threads())


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# --------------------------------------------------------------------------
# quantiser Q (Sec. 2.1, after Eq. 2)
# --------------------------------------------------------------------------
def quantize(image: np.ndarray, bitdepth: int, B: int) -> np.ndarray:
    """Equal-width quantiser: b = floor(v * B / 2^bitdepth), as uint8 (B <= 256).

    The paper names Q as "the quantization function that determines which
    bin to increase" without fixing it; equal-width bins over the full
    pixel range are the reading taken. Values above 2^bitdepth - 1 (stray
    high bits of a wider pixel type) count in the last bin.
    """
    if not (1 <= B <= 256):
        raise ValueError("B must be in [1, 256]")
    v = np.minimum(image.astype(np.int64), (1 << bitdepth) - 1)
    return ((v * B) >> bitdepth).astype(np.uint8)


# --------------------------------------------------------------------------
# Eq. 2: weighted integral histogram with weight x^p y^q
# --------------------------------------------------------------------------
def weighted_ih(bins: np.ndarray, b: int, p: int, q: int, bits: int = 64) -> np.ndarray:
    """IH_w(x, y, b) = sum_{i<=x, j<=y} [Q(f(i, j)) = b] * w(i, j), w = i^p j^q (Eq. 2).

    i is the column and j the row, so the result is indexed [y, x]. The
    sums are taken modulo 2^bits (bits = 32 or 64): unsigned numpy
    arithmetic wraps, which is exact arithmetic in that ring. bits = 128
    uses Python integers (an object array, for small images) reduced mod 2^128.
    """
    if bits == 128:
        h, w = bins.shape
        term = np.zeros((h, w), dtype=object)
        for y in range(h):
            for x in range(w):
                term[y, x] = (x ** p) * (y ** q) if bins[y, x] == b else 0
        return np.cumsum(np.cumsum(term, axis=0), axis=1) % (1 << 128)
    if bits not in (32, 64):
        raise ValueError("bits must be 32, 64 or 128")
    h, w = bins.shape
    xs = np.arange(w, dtype=np.uint64)
    ys = np.arange(h, dtype=np.uint64)
    wx = np.ones(w, dtype=np.uint64)
    for _ in range(p):
        wx = wx * xs
    wy = np.ones(h, dtype=np.uint64)
    for _ in range(q):
        wy = wy * ys
    weight = wy[:, None] * wx[None, :]
    term = np.where(bins == b, weight, np.uint64(0))
    ih = np.cumsum(np.cumsum(term, axis=0, dtype=np.uint64), axis=1, dtype=np.uint64)
    if bits == 32:
        return (ih & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    return ih


def plain_ih(bins: np.ndarray, B: int) -> np.ndarray:
    """Porikli's plain integral histogram, int64 [B, H, W] (Eq. 2 with w = 1)."""
    onehot = (bins[None, :, :] == np.arange(B, dtype=bins.dtype)[:, None, None])
    return np.cumsum(np.cumsum(onehot.astype(np.int64), axis=1), axis=2)


# --------------------------------------------------------------------------
# spatial kernels (Fig. 1, Eq. 1)
# --------------------------------------------------------------------------
def gauss_degree(r: int, degree: int) -> int:
    """Polynomial degree actually fitted on a half-width r: at most r, because
    the samples t = d^2 / r^2, d = 0..r, take only r + 1 distinct values."""
    return max(0, min(degree, r))


def gauss_fit(r: int, sigma: float, degree: int) -> np.ndarray:
    """Least-squares fit of P(t) = sum_i c_i t^i to exp(-d^2 / (2 sigma^2)).

    Samples are the integer offsets d = -r..r of one window axis with
    t = d^2 / r^2. Returns c (length gauss_degree(r, degree) + 1), float64.
    Solved with numpy's SVD-based least squares.
    """
    D = gauss_degree(r, degree)
    d = np.arange(-r, r + 1, dtype=np.float64)
    t = (d * d) / float(r * r)
    A = np.stack([t ** i for i in range(D + 1)], axis=1)
    y = np.exp(-(d * d) / (2.0 * sigma * sigma))
    c, *_ = np.linalg.lstsq(A, y, rcond=None)
    return c


def gauss_axis(r: int, sigma: float, degree: int) -> np.ndarray:
    """g(d) = P(d^2 / r^2) sampled at d = -r..r."""
    c = gauss_fit(r, sigma, degree)
    d = np.arange(-r, r + 1, dtype=np.float64)
    t = (d * d) / float(r * r)
    return sum(ci * t ** i for i, ci in enumerate(c))


def wedding_half_sides(r: int, n: int) -> list:
    """Half-sides of the n nested windows of one axis (Sec. 2, Fig. 4(a): the
    paper gives no sizes): i * r / n rounded half up, i = 1..n."""
    return [int(np.floor(i * r / n + 0.5)) for i in range(1, n + 1)]


def wedding_weights(w: int, h: int, rings: int = 4) -> np.ndarray:
    """Wedding-cake approximation (Sec. 2, Fig. 4(a)) of the Manhattan kernel:
    n nested windows around the centre split the window into rings (the
    innermost window is the first ring); every pixel of a ring gets the mean
    Manhattan weight of that ring's pixels. Reading: the paper only says the
    ring histograms are 'weighted appropriately with respect to their distance
    from P'; the ring mean is the least-squares ring-constant fit, and it keeps
    the kernel's total weight."""
    rx, ry = (w - 1) // 2, (h - 1) // 2
    K = kernel_weights("manhattan", w, h)
    dx = np.abs(np.arange(-rx, rx + 1))[None, :]
    dy = np.abs(np.arange(-ry, ry + 1))[:, None]
    out = np.zeros_like(K)
    taken = np.zeros(K.shape, dtype=bool)
    for a, b in zip(wedding_half_sides(rx, rings), wedding_half_sides(ry, rings)):
        ring = (dx <= a) & (dy <= b) & ~taken
        if ring.any():
            out[ring] = K[ring].mean()
            taken |= ring
    return out


def kernel_weights(kind: str, w: int, h: int, degree: int = 2,
                   sigma_frac: float = 0.25, rings: int = 4, lam: float = EXP_LAMBDA) -> np.ndarray:
    """Weight table K[dy + ry, dx + rx] (float64, h x w) of one window.

    * plain: K = 1 (Porikli's unweighted local histogram).
    * manhattan: K = (rx - |dx|) + (ry - |dy|). Eq. 1's city-block distance
      |dx| + |dy| subtracted from its value at the window corner, so the
      weight is largest at the centre, falls linearly and is zero at the
      four corners (Sec. 2: low weights near the contour; Sec. 2.1: weights
      rise linearly from each quadrant's outer corner to the centre).
    * euclidean: K = (rx^2 - dx^2) + (ry^2 - dy^2), the same construction
      on the squared Euclidean distance dx^2 + dy^2 (the square root of
      the true distance has no finite decomposition into integral
      histograms).
    * gaussian: K = Px(dx^2 / rx^2) * Py(dy^2 / ry^2), each factor the
      least-squares polynomial (gauss_fit) of the axis Gaussian with
      sigma = sigma_frac * (window length along that axis).
    * wedding: the wedding-cake approximation of the Manhattan kernel with
      ``rings`` nested windows (wedding_weights).
    * exponential: K = exp(-lam (|dx| + |dy|)), the exponential weighting of
      the city-block distance (Sec. 2 and Fig. 1 name an exponential kernel
      without a formula). lam is a decay rate per pixel, the same for every
      window size, so one set of integral histograms serves every scale.
    """
    if w < 3 or h < 3 or w % 2 == 0 or h % 2 == 0:
        raise ValueError("window sides must be odd and >= 3")
    rx, ry = (w - 1) // 2, (h - 1) // 2
    dx = np.arange(-rx, rx + 1, dtype=np.float64)[None, :]
    dy = np.arange(-ry, ry + 1, dtype=np.float64)[:, None]
    if kind == "plain":
        return np.ones((h, w), dtype=np.float64)
    if kind == "manhattan":
        return (rx - np.abs(dx)) + (ry - np.abs(dy))
    if kind == "euclidean":
        return (rx * rx - dx * dx) + (ry * ry - dy * dy)
    if kind == "wedding":
        return wedding_weights(w, h, rings)
    if kind == "exponential":
        if not lam > 0.0:
            raise ValueError("the exponential kernel needs a positive decay rate")
        return np.exp(-lam * (np.abs(dx) + np.abs(dy)))
    if kind == "gaussian":
        gx = gauss_axis(rx, sigma_frac * w, degree)[None, :]
        gy = gauss_axis(ry, sigma_frac * h, degree)[:, None]
        K = gy * gx
        if (K < 0).any():
            raise ValueError("Gaussian approximant is negative inside the window")
        return K
    raise ValueError(f"unknown kernel {kind!r}")


def exp_directional_ih(bins: np.ndarray, b: int, lam: float) -> np.ndarray:
    """The four directional integral histograms of the exponential kernel,
    float64 [4, H, W], direction d = (x side) + 2 (y side):

        J_d(x, y) = sum over x' on the x side, y' on the y side of
                    [Q(f(x', y')) = b] * exp(-lam (|x - x'| + |y - y'|)),

    x side 0: x' <= x, 1: x' >= x; y side 0: y' <= y, 1: y' >= y. J_0 is
    Eq. 2 with the weight w(i, j) = exp(lam (i + j)), divided by w(x, y);
    the other three are the same for the weights exp(-+lam i) exp(-+lam j)
    with the sums taken from the opposite side (Sec. 2.1: one weighted IH
    per quadrant, each rising towards the centre). Dividing by the weight at
    (x, y) keeps the values below 1 / (1 - exp(-lam))^2 on any image size.
    Written as two triangular matrix products (a library matmul per axis).
    """
    H, W = bins.shape
    c = (bins == b).astype(np.float64)

    def tri(n, side):
        i = np.arange(n)
        d = i[:, None] - i[None, :]  # row index minus column index
        if side == 0:
            return np.where(d >= 0, np.exp(-lam * np.maximum(d, 0)), 0.0)
        return np.where(d <= 0, np.exp(-lam * np.maximum(-d, 0)), 0.0)

    out = np.empty((4, H, W), dtype=np.float64)
    for d in range(4):
        tx, ty = tri(W, d & 1), tri(H, d >> 1)
        out[d] = ty @ c @ tx.T
    return out


def true_gaussian(w: int, h: int, sigma_frac: float = 0.25) -> np.ndarray:
    """exp(-dx^2 / 2 sx^2 - dy^2 / 2 sy^2) on the window (for reporting only)."""
    rx, ry = (w - 1) // 2, (h - 1) // 2
    dx = np.arange(-rx, rx + 1, dtype=np.float64)[None, :]
    dy = np.arange(-ry, ry + 1, dtype=np.float64)[:, None]
    sx, sy = sigma_frac * w, sigma_frac * h
    return np.exp(-dx * dx / (2 * sx * sx) - dy * dy / (2 * sy * sy))


# --------------------------------------------------------------------------
# brute-force local histograms and likelihood (Sec. 2, "Brute-force Approach")
# --------------------------------------------------------------------------
def _check(bins: np.ndarray, B: int, K: np.ndarray):
    if bins.dtype != np.uint8 or bins.ndim != 2:
        raise TypeError("bins must be a 2-D uint8 array")
    if int(bins.max(initial=0)) >= B:
        raise ValueError("bin index out of range")
    h, w = K.shape
    if h % 2 == 0 or w % 2 == 0:
        raise ValueError("odd window required")
    return (np.ascontiguousarray(bins), np.ascontiguousarray(K, dtype=np.float64))


def valid_centres(H: int, W: int, w: int, h: int):
    """(x0, y0, nx, ny): centres whose whole window lies inside the image."""
    rx, ry = (w - 1) // 2, (h - 1) // 2
    return rx, ry, W - w + 1, H - h + 1


def hist_rect(bins, B, K, cx0, cy0, ncx, ncy) -> np.ndarray:
    """Unnormalised U_c(b) for a rectangle of centres, float64 [ncy, ncx, B]."""
    bins, K = _check(bins, B, K)
    H, W = bins.shape
    h, w = K.shape
    rx, ry = (w - 1) // 2, (h - 1) // 2
    if cx0 - rx < 0 or cy0 - ry < 0 or cx0 + ncx - 1 + rx >= W or cy0 + ncy - 1 + ry >= H:
        raise ValueError("a window leaves the image")
    U = np.empty((ncy, ncx, B), dtype=np.float64)
    _lib().swih_oracle_hist_rect(_ptr(bins), H, W, B, _ptr(K), w, h, cx0, cy0, ncx, ncy, _ptr(U))
    return U


def hist_at(bins, B, K, cx, cy) -> np.ndarray:
    """Unnormalised U_c(b) at listed centres, float64 [n, B]."""
    bins, K = _check(bins, B, K)
    H, W = bins.shape
    h, w = K.shape
    cx = np.ascontiguousarray(cx, dtype=np.int32)
    cy = np.ascontiguousarray(cy, dtype=np.int32)
    rx, ry = (w - 1) // 2, (h - 1) // 2
    if cx.size and (cx.min() < rx or cy.min() < ry or cx.max() >= W - rx or cy.max() >= H - ry):
        raise ValueError("a window leaves the image")
    U = np.empty((cx.size, B), dtype=np.float64)
    _lib().swih_oracle_hist_at(_ptr(bins), H, W, B, _ptr(K), w, h, _ptr(cx), _ptr(cy),
                               cx.size, _ptr(U))
    return U


def normalise(U: np.ndarray) -> np.ndarray:
    """H_c(b) = U_c(b) / sum_b U_c(b) (Sec. 2.1: normalise the histogram)."""
    return U / U.sum(axis=-1, keepdims=True)


def likelihood_rect(bins, B, K, q, cx0, cy0, ncx, ncy) -> np.ndarray:
    """Bhattacharyya coefficient of each normalised window histogram vs q, [ncy, ncx]."""
    bins, K = _check(bins, B, K)
    H, W = bins.shape
    h, w = K.shape
    rx, ry = (w - 1) // 2, (h - 1) // 2
    if cx0 - rx < 0 or cy0 - ry < 0 or cx0 + ncx - 1 + rx >= W or cy0 + ncy - 1 + ry >= H:
        raise ValueError("a window leaves the image")
    q = np.ascontiguousarray(q, dtype=np.float64)
    L = np.empty((ncy, ncx), dtype=np.float64)
    _lib().swih_oracle_likelihood_rect(_ptr(bins), H, W, B, _ptr(K), w, h, cx0, cy0, ncx, ncy,
                                       _ptr(q), _ptr(L))
    return L


def likelihood_at(bins, B, K, q, cx, cy) -> np.ndarray:
    """Bhattacharyya coefficient at listed centres, float64 [n]."""
    bins, K = _check(bins, B, K)
    H, W = bins.shape
    h, w = K.shape
    cx = np.ascontiguousarray(cx, dtype=np.int32)
    cy = np.ascontiguousarray(cy, dtype=np.int32)
    rx, ry = (w - 1) // 2, (h - 1) // 2
    if cx.size != cy.size:
        raise ValueError("cx and cy differ in length")
    if cx.size and (cx.min() < rx or cy.min() < ry or cx.max() >= W - rx or cy.max() >= H - ry):
        raise ValueError("a window leaves the image")
    q = np.ascontiguousarray(q, dtype=np.float64)
    if q.size != B:
        raise ValueError("the target needs B entries")
    L = np.empty(cx.size, dtype=np.float64)
    _lib().swih_oracle_likelihood_at(_ptr(bins), H, W, B, _ptr(K), w, h, _ptr(cx), _ptr(cy),
                                     cx.size, _ptr(q), _ptr(L))
    return L


def likelihood_map(bins, B, K, q) -> np.ndarray:
    """Likelihood at every valid centre, [H - h + 1, W - w + 1]."""
    H, W = bins.shape
    h, w = K.shape
    x0, y0, nx, ny = valid_centres(H, W, w, h)
    return likelihood_rect(bins, B, K, q, x0, y0, nx, ny)


def likelihood_channels_map(bins_list, B_list, K, q_list) -> np.ndarray:
    """Per-feature likelihood maps, float64 [C, H - h + 1, W - w + 1].

    Sec. 4: the tracker computes one likelihood map per feature (chromatic,
    shape, texture) by sliding-window histogram matching. Each feature c is its
    own image of bins in [0, B_c); its map is the brute-force likelihood of its
    own kernel-weighted histograms against its own target q_c.
    """
    if not (len(bins_list) == len(B_list) == len(q_list)) or not bins_list:
        raise ValueError("one bin image, bin count and target per channel")
    return np.stack([likelihood_map(b, B, K, q) for b, B, q in zip(bins_list, B_list, q_list)])


def target_hist(bins, B, K, xc, yc) -> np.ndarray:
    """Normalised weighted histogram of the window centred at (xc, yc), float64 [B]."""
    return normalise(hist_at(bins, B, K, [xc], [yc]))[0]
