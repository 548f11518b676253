"""Why the integral histograms are integers in a ring, not floating point.

The stated alternative stores the integral histograms in FP32 (with
compensated or FP64 carries during the scan). Its best case is that every
stored element is the correctly rounded FP32 value of the exact prefix sum;
the window sums are then differences of four such values. These CPU tests
compute that best case on the 1024 x 1024 benchmark scene (B = 32) at
windows of the benchmark's sizes and measure the error on the normalised bin
values against exact integer arithmetic: FP32 storage misses the 1e-5
tolerance (Manhattan), or loses every digit (the Gaussian's x^4 y^4 moments,
whose translation to the centre cancels them by many orders of magnitude),
while the integer ring is exact by construction (checked in
test_oracle_pins.py and bit for bit on the GPU)."""
import numpy as np

from oracle import swih_oracle as O
from paper_1705_03524_gb300 import synth


def scene():
    cfg = synth.config2()
    return O.quantize(cfg["image"], 8, cfg["B"]), cfg["B"]


def prefix_table(mask, weight):
    """Exact 2-D prefix sums of mask * weight (int64 suffices here)."""
    return np.cumsum(np.cumsum(np.where(mask, weight, 0), axis=0), axis=1)


def corner(t, x, y):
    return 0 if (x < 0 or y < 0) else t[y, x]


def rect(t, x0, x1, y0, y1):
    """Sum over columns (x0, x1] and rows (y0, y1]."""
    return corner(t, x1, y1) - corner(t, x0, y1) - corner(t, x1, y0) + corner(t, x0, y0)


def test_fp32_storage_misses_the_tolerance_for_the_manhattan_kernel():
    bins, B = scene()
    H, W = bins.shape
    w = 81
    r = (w - 1) // 2
    M = w * r * r * 2  # h rx^2 + w ry^2 for a square window
    ys, xs = np.mgrid[0:H, 0:W]
    worst = 0.0
    rng = np.random.default_rng(0)
    for b in range(B):
        mask = bins == b
        if mask.sum() < 1000:
            continue
        t = {k: prefix_table(mask, wgt).astype(np.int64) for k, wgt in (("1", 1), ("x", xs), ("y", ys))}
        t32 = {k: v.astype(np.float32).astype(np.float64) for k, v in t.items()}
        # windows towards the bottom-right, where the prefix sums are largest
        for _ in range(40):
            xc = int(rng.integers(W - 300, W - r))
            yc = int(rng.integers(H - 300, H - r))

            def U(tab):
                # K = (rx - |dx|) + (ry - |dy|): column and row splits at the centre
                n = rect(tab["1"], xc - r - 1, xc + r, yc - r - 1, yc + r)
                left_n = rect(tab["1"], xc - r - 1, xc, yc - r - 1, yc + r)
                left_x = rect(tab["x"], xc - r - 1, xc, yc - r - 1, yc + r)
                right_n, right_x = n - left_n, rect(tab["x"], xc - r - 1, xc + r, yc - r - 1, yc + r) - left_x
                top_n = rect(tab["1"], xc - r - 1, xc + r, yc - r - 1, yc)
                top_y = rect(tab["y"], xc - r - 1, xc + r, yc - r - 1, yc)
                bot_n, bot_y = n - top_n, rect(tab["y"], xc - r - 1, xc + r, yc - r - 1, yc + r) - top_y
                sum_abs_dx = (right_x - xc * right_n) - (left_x - xc * left_n)
                sum_abs_dy = (bot_y - yc * bot_n) - (top_y - yc * top_n)
                return 2 * r * n - sum_abs_dx - sum_abs_dy

            exact = U(t)
            approx = U(t32)
            worst = max(worst, abs(float(approx) - float(exact)) / M)
    assert worst > 1e-5, worst  # the best-case FP32 storage misses the bins' tolerance


def test_fp32_storage_loses_the_gaussian_moments():
    bins, B = scene()
    H, W = bins.shape
    w = 41
    r = (w - 1) // 2
    b = int(np.bincount(bins[H - 200:, W - 200:].ravel(), minlength=B).argmax())
    mask = bins == b
    rng = np.random.default_rng(1)
    xc, yc = W - 60, H - 60
    # exact raw moments sum x^k y^l over the window from four corners of exact
    # prefix sums (Python integers), and the same from FP32-rounded corners
    rows = [np.nonzero(mask[j])[0] for j in range(H)]

    def prefix(x, y, k, l):
        if x < 0 or y < 0:
            return 0
        s = 0
        for j in range(y + 1):
            ii = rows[j][rows[j] <= x]
            if ii.size:
                s += int(sum(int(i) ** k for i in ii)) * j ** l
        return s

    worst = 0.0
    for (k, l) in ((4, 4), (4, 2), (2, 4)):
        cs = [(xc + r, yc + r), (xc - r - 1, yc + r), (xc + r, yc - r - 1), (xc - r - 1, yc - r - 1)]
        vals = [prefix(x, y, k, l) for x, y in cs]
        exact = vals[0] - vals[1] - vals[2] + vals[3]
        approx = float(np.float32(vals[0])) - float(np.float32(vals[1])) - float(np.float32(vals[2])) + \
            float(np.float32(vals[3]))
        # the centred moment sum dx^4 dy^4 is far smaller than these raw
        # moments: compare the error with the largest centred moment possible
        bound = (2 * r + 1) ** 2 * r ** (k + l)
        worst = max(worst, abs(approx - exact) / bound)
    assert worst > 1.0, worst  # errors larger than any window's centred moment
    _ = rng
