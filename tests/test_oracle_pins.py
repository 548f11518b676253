"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each test checks the oracle against something the paper or the mathematics
fixes: hand-summed fixtures, closed-form kernel masses (Sec. 2.1: the total
weight of a window does not depend on where the window is), the plain
histogram as the K = 1 special case, exhaustive tiny inputs, mirror
symmetry, and the paper's own decomposition (Sec. 2.1, Eq. 2) evaluated in
exact integer arithmetic, which must agree with brute force (Sec. 3: the
method is exact).
"""
import itertools
import os

import numpy as np
import pytest

from oracle import swih_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# helpers written independently of the oracle
# ----------------------------------------------------------------------------
def read_hand_fixture(name):
    rows, cases = [], []
    with open(os.path.join(GOLDEN, name)) as f:
        lines = [ln.split("#")[0].strip() for ln in f]
    lines = [ln for ln in lines if ln]
    _, h, w = lines[0].split()
    h, w = int(h), int(w)
    for ln in lines[1:1 + h]:
        rows.append([int(v) for v in ln.split()])
    for ln in lines[1 + h:]:
        parts = ln.split()
        cases.append((parts[0], *map(int, parts[1:5]), [int(v) for v in parts[5:]]))
    return np.array(rows, dtype=np.uint8), cases


def rect_sum(ih, x_lo, x_hi, y_lo, y_hi):
    """Sum over x in (x_lo, x_hi], y in (y_lo, y_hi] from an inclusive prefix table."""
    def at(x, y):
        return 0 if (x < 0 or y < 0) else ih[y][x]
    return at(x_hi, y_hi) - at(x_lo, y_hi) - at(x_hi, y_lo) + at(x_lo, y_lo)


def exact_ih(bins, b, weight):
    """Eq. 2 in Python integers: prefix sums of [bin == b] * weight(x, y)."""
    h, w = bins.shape
    ih = [[0] * w for _ in range(h)]
    for y in range(h):
        run = 0
        for x in range(w):
            if bins[y, x] == b:
                run += weight(x, y)
            ih[y][x] = run + (ih[y - 1][x] if y > 0 else 0)
    return ih


def faulhaber_even(r, k):
    """sum_{d=-r..r} d^(2k) for k = 0, 1, 2 (closed forms)."""
    if k == 0:
        return 2 * r + 1
    if k == 1:
        return r * (r + 1) * (2 * r + 1) // 3
    if k == 2:
        return r * (r + 1) * (2 * r + 1) * (3 * r * r + 3 * r - 1) // 15
    raise ValueError(k)


# ----------------------------------------------------------------------------
# quantiser and integral histograms
# ----------------------------------------------------------------------------
def test_quantize_bin_edges():
    v8 = np.arange(256, dtype=np.uint8)[None, :]
    b = O.quantize(v8, 8, 16)[0]
    assert b[0] == 0 and b[15] == 0 and b[16] == 1 and b[255] == 15
    assert np.all(np.bincount(b, minlength=16) == 16)
    v16 = np.array([[0, 1023, 1024, 65535]], dtype=np.uint16)
    assert list(O.quantize(v16, 16, 64)[0]) == [0, 0, 1, 63]
    # 12 significant bits in a 16-bit pixel: values past 4095 land in the last bin
    v12 = np.array([[0, 63, 64, 4095, 4096, 65535]], dtype=np.uint16)
    assert list(O.quantize(v12, 12, 64)[0]) == [0, 0, 1, 63, 63, 63]
    # non-power-of-two bin count still gives equal-width bins
    b24 = O.quantize(v8, 8, 24)[0]
    assert b24.max() == 23 and np.all(np.diff(b24.astype(int)) >= 0)
    counts = np.bincount(b24, minlength=24)
    assert counts.min() >= 10 and counts.max() <= 11


def test_plain_ih_matches_counts():
    rng = np.random.default_rng(5)
    bins = rng.integers(0, 4, size=(7, 9)).astype(np.uint8)
    ih = O.plain_ih(bins, 4)
    assert np.array_equal(ih[:, -1, -1], np.bincount(bins.ravel(), minlength=4))
    for b in range(4):
        for y in range(7):
            for x in range(9):
                assert ih[b, y, x] == int((bins[: y + 1, : x + 1] == b).sum())
        assert np.array_equal(O.weighted_ih(bins, b, 0, 0, 64).astype(np.int64), ih[b])


@pytest.mark.parametrize("bits", [32, 64, 128])
@pytest.mark.parametrize("p,q", [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2), (4, 4), (3, 2), (8, 8), (7, 6)])
def test_weighted_ih_exact_in_ring(bits, p, q):
    rng = np.random.default_rng(11 + p + 7 * q)
    bins = rng.integers(0, 3, size=(6, 8)).astype(np.uint8)
    for b in range(3):
        ref = exact_ih(bins, b, lambda x, y: x ** p * y ** q)
        got = O.weighted_ih(bins, b, p, q, bits)
        mod = 1 << bits
        for y in range(6):
            for x in range(8):
                assert int(got[y, x]) == ref[y][x] % mod


def test_weighted_ih_128_wraps_exactly_on_large_coordinates():
    # x^8 y^8 prefix sums pass 2^128 at these coordinates; the oracle keeps
    # them mod 2^128, and its 64-bit ring is the same values mod 2^64
    rng = np.random.default_rng(13)
    H, W = 40, 3000
    bins = rng.integers(0, 2, size=(H, W)).astype(np.uint8)
    got = O.weighted_ih(bins, 1, 8, 8, 128)
    ys, xs = np.nonzero(bins == 1)
    exact = sum(int(a) ** 8 * int(c) ** 8 for a, c in zip(xs, ys))
    assert exact >= 1 << 128
    assert int(got[H - 1, W - 1]) == exact % (1 << 128)
    got64 = O.weighted_ih(bins, 1, 3, 2, 64)
    got128 = O.weighted_ih(bins, 1, 3, 2, 128)
    assert all(int(got128[y, x]) % (1 << 64) == int(got64[y, x]) for y in (0, 11, 39) for x in (0, 100, 2999))


def test_weighted_ih_wraps_exactly_on_large_coordinates():
    # x^4 y^4 prefix sums overflow 64 bits by far at these coordinates; the
    # oracle must return the exact value reduced mod 2^64.
    rng = np.random.default_rng(3)
    H, W = 40, 300
    bins = rng.integers(0, 2, size=(H, W)).astype(np.uint8)
    got = O.weighted_ih(bins, 1, 4, 4, 64)
    ys, xs = np.nonzero(bins == 1)
    for (x, y) in [(299, 39), (150, 20), (0, 0), (299, 0)]:
        sel = (xs <= x) & (ys <= y)
        exact = sum(int(a) ** 4 * int(c) ** 4 for a, c in zip(xs[sel], ys[sel]))
        assert int(got[y, x]) == exact % (1 << 64)


# ----------------------------------------------------------------------------
# brute-force local histograms
# ----------------------------------------------------------------------------
def test_hand_fixture():
    bins, cases = read_hand_fixture("hand_5x5.txt")
    for kind, w, h, xc, yc, expect in cases:
        K = O.kernel_weights(kind, w, h)
        U = O.hist_at(bins, 3, K, [xc], [yc])[0]
        assert np.array_equal(U, np.array(expect, dtype=np.float64)), (kind, w, h)


def test_uniform_kernel_is_plain_histogram():
    rng = np.random.default_rng(8)
    bins = rng.integers(0, 6, size=(23, 31)).astype(np.uint8)
    K = O.kernel_weights("plain", 7, 5)
    U = O.hist_rect(bins, 6, K, 3, 2, 31 - 6, 23 - 4)
    for yc in range(2, 23 - 2):
        for xc in range(3, 31 - 3):
            win = bins[yc - 2: yc + 3, xc - 3: xc + 4]
            assert np.array_equal(U[yc - 2, xc - 3], np.bincount(win.ravel(), minlength=6))


@pytest.mark.parametrize("w,h", [(3, 3), (5, 9), (21, 7), (31, 31)])
def test_bin_mass_is_closed_form_everywhere(w, h):
    rng = np.random.default_rng(w * 100 + h)
    H, W = h + 12, w + 15
    bins = rng.integers(0, 5, size=(H, W)).astype(np.uint8)
    rx, ry = (w - 1) // 2, (h - 1) // 2
    x0, y0, nx, ny = O.valid_centres(H, W, w, h)
    closed = {
        "plain": w * h,
        "manhattan": h * rx * rx + w * ry * ry,
        "euclidean": (h * rx * (2 * rx + 1) * (2 * rx - 1) // 3
                      + w * ry * (2 * ry + 1) * (2 * ry - 1) // 3),
    }
    for kind, M in closed.items():
        U = O.hist_rect(bins, 5, O.kernel_weights(kind, w, h), x0, y0, nx, ny)
        assert np.all(U.sum(-1) == M), kind
    # Gaussian approximant: M = (sum_i c_i S_2i(rx) / rx^2i) * (same for y)
    def axis_mass(r, sigma):
        c = O.gauss_fit(r, sigma, 2)
        return sum(ci * faulhaber_even(r, i) / float(r) ** (2 * i) for i, ci in enumerate(c))
    Mg = axis_mass(rx, 0.25 * w) * axis_mass(ry, 0.25 * h)
    U = O.hist_rect(bins, 5, O.kernel_weights("gaussian", w, h), x0, y0, nx, ny)
    np.testing.assert_allclose(U.sum(-1), Mg, rtol=1e-12)


def test_manhattan_config1_mass_value():
    # the 31 x 31 Manhattan window has total weight 31*15^2 * 2 = 13950
    assert O.kernel_weights("manhattan", 31, 31).sum() == 13950


@pytest.mark.parametrize("kind", O.KINDS)
def test_constant_image(kind):
    bins = np.full((20, 25), 3, dtype=np.uint8)
    K = O.kernel_weights(kind, 9, 7)
    H = O.normalise(O.hist_rect(bins, 5, K, 4, 3, 25 - 8, 20 - 6))
    e = np.zeros(5)
    e[3] = 1.0
    assert np.all(H == e)
    q = O.target_hist(bins, 5, K, 10, 10)
    L = O.likelihood_map(bins, 5, K, q)
    assert np.all(L == 1.0)


@pytest.mark.parametrize("kind", O.KINDS)
def test_likelihood_is_one_at_target_centre(kind):
    img = np.random.default_rng(1).integers(0, 256, size=(128, 128)).astype(np.uint8)
    bins = O.quantize(img, 8, 16)
    K = O.kernel_weights(kind, 31, 31)
    q = O.target_hist(bins, 16, K, 64, 64)
    L = O.likelihood_map(bins, 16, K, q)
    assert abs(L[64 - 15, 64 - 15] - 1.0) < 1e-12
    assert L.max() <= 1.0 + 1e-12


def test_bhattacharyya_hand_values():
    # A 3 x 3 plain window with six pixels of bin 0 and three of bin 1 has
    # H = (2/3, 1/3). Against q = (1/3, 2/3), L = 2 sqrt(2/9) = 2 sqrt(2) / 3;
    # against q = (1/4, 3/4), L = sqrt(1/6) + sqrt(1/4).
    bins = np.array([[0, 1, 0],
                     [0, 1, 0],
                     [0, 1, 0]], dtype=np.uint8)
    K = O.kernel_weights("plain", 3, 3)
    L = O.likelihood_at(bins, 2, K, [1.0 / 3.0, 2.0 / 3.0], [1], [1])
    assert abs(L[0] - 2.0 * np.sqrt(2.0) / 3.0) < 1e-15
    L = O.likelihood_at(bins, 2, K, [0.25, 0.75], [1], [1])
    assert abs(L[0] - (np.sqrt(1.0 / 6.0) + 0.5)) < 1e-15
    # Manhattan 3 x 3 weights: corners 0, edge midpoints 1, centre 2 (M = 6).
    # Bin 1 holds the centre and the top edge: U = (3, 3), H = (1/2, 1/2);
    # against q = (1, 0), L = sqrt(1/2).
    bins = np.array([[1, 1, 1],
                     [0, 1, 0],
                     [0, 0, 0]], dtype=np.uint8)
    K = O.kernel_weights("manhattan", 3, 3)
    L = O.likelihood_at(bins, 2, K, [1.0, 0.0], [1], [1])
    assert abs(L[0] - np.sqrt(0.5)) < 1e-15


def test_likelihood_at_listed_centres_by_slicing():
    # Listed centres on a non-square image with a non-square window, near
    # opposite borders (cx != cy everywhere, and a swapped pair would leave the
    # image or land on other pixels), checked against a histogram of the
    # window taken by numpy slicing and against the rectangle routine.
    rng = np.random.default_rng(31)
    H, W, B = 23, 41, 5
    bins = rng.integers(0, B, size=(H, W)).astype(np.uint8)
    w, h = 7, 5
    rx, ry = 3, 2
    K = O.kernel_weights("manhattan", w, h)
    q = rng.gamma(0.5, size=B)
    q = q / q.sum()
    cx = np.array([rx, W - 1 - rx, rx + 1, W - 2 - rx, 20, 37], dtype=np.int32)
    cy = np.array([H - 1 - ry, ry, ry + 1, H - 2 - ry, 11, 3], dtype=np.int32)
    got = O.likelihood_at(bins, B, K, q, cx, cy)
    for i in range(cx.size):
        win = bins[cy[i] - ry: cy[i] + ry + 1, cx[i] - rx: cx[i] + rx + 1]
        U = np.array([K[win == b].sum() for b in range(B)])
        Hc = U / U.sum()
        assert abs(got[i] - np.sqrt(Hc * q).sum()) < 1e-14, i
    L = O.likelihood_rect(bins, B, K, q, rx, ry, W - w + 1, H - h + 1)
    np.testing.assert_array_equal(got, L[cy - ry, cx - rx])
    # the listed-centre histograms agree with the same slicing
    U = O.hist_at(bins, B, K, cx, cy)
    for i in range(cx.size):
        win = bins[cy[i] - ry: cy[i] + ry + 1, cx[i] - rx: cx[i] + rx + 1]
        assert np.array_equal(U[i], [K[win == b].sum() for b in range(B)])
    with pytest.raises(ValueError):
        O.likelihood_at(bins, B, K, q, cy, cx)  # swapped: windows leave the image


@pytest.mark.parametrize("kind", O.KINDS)
def test_mirror_invariance(kind):
    rng = np.random.default_rng(21)
    bins = rng.integers(0, 7, size=(30, 40)).astype(np.uint8)
    w, h = 11, 9
    K = O.kernel_weights(kind, w, h)
    x0, y0, nx, ny = O.valid_centres(30, 40, w, h)
    U = O.hist_rect(bins, 7, K, x0, y0, nx, ny)
    Ux = O.hist_rect(np.ascontiguousarray(bins[:, ::-1]), 7, K, x0, y0, nx, ny)
    Uy = O.hist_rect(np.ascontiguousarray(bins[::-1, :]), 7, K, x0, y0, nx, ny)
    np.testing.assert_allclose(Ux, U[:, ::-1], rtol=1e-14, atol=1e-12)
    np.testing.assert_allclose(Uy, U[::-1, :], rtol=1e-14, atol=1e-12)


def test_exhaustive_binary_3x3():
    # all 512 binary 3x3 windows: U(1) is the sum of the hand-written
    # weight table over the set pixels.
    table = {"plain": [[1, 1, 1], [1, 1, 1], [1, 1, 1]],
             "manhattan": [[0, 1, 0], [1, 2, 1], [0, 1, 0]],
             "euclidean": [[0, 1, 0], [1, 2, 1], [0, 1, 0]]}
    masks = np.array(list(itertools.product([0, 1], repeat=9)), dtype=np.uint8)
    # tile the 512 windows side by side with a 1-pixel gap so each is one centre
    bins = np.zeros((3, 512 * 4), dtype=np.uint8)
    for i, m in enumerate(masks):
        bins[:, 4 * i: 4 * i + 3] = m.reshape(3, 3)
    cx = np.arange(512) * 4 + 1
    cy = np.ones(512, dtype=np.int64)
    for kind, t in table.items():
        U = O.hist_at(bins, 2, O.kernel_weights(kind, 3, 3), cx, cy)
        expect = masks.reshape(512, 3, 3) * np.array(t)[None]
        assert np.array_equal(U[:, 1], expect.reshape(512, 9).sum(1)), kind
        assert np.all(U.sum(1) == np.array(t).sum())


# ----------------------------------------------------------------------------
# the paper's decomposition, evaluated exactly, reproduces brute force
# ----------------------------------------------------------------------------
def swih_manhattan_quadrants(bins, B, w, h, xc, yc):
    """Sec. 2.1 with four directional weighted IHs (weights +-x +-y, Eq. 2)
    and the plain IH: each quadrant's local histogram from its own IH,
    translated from the centre, then summed. Python integers."""
    rx, ry = (w - 1) // 2, (h - 1) // 2
    X0, X1, X2 = xc - rx - 1, xc, xc + rx
    Y0, Y1, Y2 = yc - ry - 1, yc, yc + ry
    # quadrant: (x range, y range, weight function, constant after translation)
    quads = [
        ((X0, X1), (Y0, Y1), lambda x, y: x + y, rx + ry - xc - yc),     # TL, rises to SE
        ((X1, X2), (Y0, Y1), lambda x, y: -x + y, rx + ry + xc - yc),    # TR, rises to SW
        ((X0, X1), (Y1, Y2), lambda x, y: x - y, rx + ry - xc + yc),     # BL, rises to NE
        ((X1, X2), (Y1, Y2), lambda x, y: -x - y, rx + ry + xc + yc),    # BR, rises to NW
    ]
    U = []
    for b in range(B):
        plain = exact_ih(bins, b, lambda x, y: 1)
        total = 0
        for (xa, xb), (ya, yb), wdir, const in quads:
            ihw = exact_ih(bins, b, wdir)
            total += const * rect_sum(plain, xa, xb, ya, yb) + rect_sum(ihw, xa, xb, ya, yb)
        U.append(total)
    return U


def swih_polynomial(bins, B, w, h, xc, yc, coef):
    """U(b) = sum_{i,j} coef[i][j] * S_ij(b), where S_ij = sum over the window of
    dx^i dy^j [bin = b] comes from the monomial IHs x^k y^l (Eq. 2) by the
    binomial translation to the centre. Python integers."""
    from math import comb
    rx, ry = (w - 1) // 2, (h - 1) // 2
    X0, X2, Y0, Y2 = xc - rx - 1, xc + rx, yc - ry - 1, yc + ry
    P = len(coef) - 1
    Q = len(coef[0]) - 1
    out = []
    for b in range(B):
        R = {}
        for k in range(P + 1):
            for l in range(Q + 1):
                ih = exact_ih(bins, b, lambda x, y, k=k, l=l: x ** k * y ** l)
                R[k, l] = rect_sum(ih, X0, X2, Y0, Y2)
        total = 0
        for i in range(P + 1):
            for j in range(Q + 1):
                if coef[i][j] == 0:
                    continue
                S = sum(comb(i, k) * comb(j, l) * (-xc) ** (i - k) * (-yc) ** (j - l) * R[k, l]
                        for k in range(i + 1) for l in range(j + 1))
                total += coef[i][j] * S
        out.append(total)
    return out


def test_paper_quadrant_decomposition_is_exact():
    rng = np.random.default_rng(4)
    bins = rng.integers(0, 3, size=(12, 14)).astype(np.uint8)
    for (w, h, xc, yc) in [(5, 5, 6, 6), (7, 3, 3, 1), (9, 11, 9, 5), (3, 3, 1, 1)]:
        K = O.kernel_weights("manhattan", w, h)
        ref = O.hist_at(bins, 3, K, [xc], [yc])[0]
        assert swih_manhattan_quadrants(bins, 3, w, h, xc, yc) == [int(v) for v in ref]


def test_polynomial_decomposition_is_exact():
    rng = np.random.default_rng(9)
    bins = rng.integers(0, 3, size=(13, 15)).astype(np.uint8)
    for (w, h, xc, yc) in [(5, 7, 6, 6), (9, 3, 4, 1), (3, 13, 7, 6)]:
        rx, ry = (w - 1) // 2, (h - 1) // 2
        # Euclidean: (rx^2 + ry^2) - dx^2 - dy^2
        coef = [[rx * rx + ry * ry, 0, -1], [0, 0, 0], [-1, 0, 0]]
        ref = O.hist_at(bins, 3, O.kernel_weights("euclidean", w, h), [xc], [yc])[0]
        assert swih_polynomial(bins, 3, w, h, xc, yc, coef) == [int(v) for v in ref]
        # Gaussian approximant: product of the axis polynomials in dx^2/rx^2, dy^2/ry^2
        cx = O.gauss_fit(rx, 0.25 * w, 2)
        cy = O.gauss_fit(ry, 0.25 * h, 2)
        coef = [[0.0] * 5 for _ in range(5)]
        for i, ci in enumerate(cx):
            for j, cj in enumerate(cy):
                coef[2 * i][2 * j] = ci / rx ** (2 * i) * cj / ry ** (2 * j)
        ref = O.hist_at(bins, 3, O.kernel_weights("gaussian", w, h), [xc], [yc])[0]
        got = swih_polynomial(bins, 3, w, h, xc, yc, coef)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------------------------
# the Gaussian approximant
# ----------------------------------------------------------------------------
def test_gauss_fit_interpolates_when_exactly_determined():
    # r = 1: t in {0, 1}, degree capped at 1 -> the line through both samples;
    # r = 2: t in {0, 1/4, 1}, degree 2 -> the parabola through all three.
    for r, sigma in [(1, 0.75), (2, 1.25)]:
        c = O.gauss_fit(r, sigma, 2)
        assert len(c) == min(2, r) + 1
        for d in range(0, r + 1):
            t = d * d / (r * r)
            val = sum(ci * t ** i for i, ci in enumerate(c))
            assert abs(val - np.exp(-d * d / (2 * sigma * sigma))) < 1e-13


@pytest.mark.parametrize("r", [3, 10, 20, 40, 63])
def test_gauss_fit_normal_equations(r):
    # least squares <=> the residual is orthogonal to every basis column
    sigma = 0.25 * (2 * r + 1)
    c = O.gauss_fit(r, sigma, 2)
    d = np.arange(-r, r + 1, dtype=np.float64)
    t = d * d / (r * r)
    A = np.stack([np.ones_like(t), t, t * t], 1)
    resid = A @ c - np.exp(-d * d / (2 * sigma * sigma))
    assert np.abs(A.T @ resid).max() < 1e-11 * len(d)
    # any perturbation of c increases the squared residual
    base = float(resid @ resid)
    for k in range(3):
        for eps in (1e-4, -1e-4):
            c2 = c.copy()
            c2[k] += eps
            r2 = A @ c2 - np.exp(-d * d / (2 * sigma * sigma))
            assert float(r2 @ r2) > base


def test_gauss_approximant_distance_from_true_gaussian():
    # reported, not a paper value: the degree-2 approximant stays within a few
    # percent of the Gaussian it replaces at the benchmark's window sizes
    for w in (21, 41, 81):
        err = np.abs(O.kernel_weights("gaussian", w, w) - O.true_gaussian(w, w)).max()
        assert err < 0.05, (w, err)


@pytest.mark.parametrize("r", [7, 10, 20, 40, 63])
def test_gauss_fit_residual_falls_with_the_degree(r):
    # the fits of degree 2, 3, 4 minimise the squared error over nested spaces
    # of polynomials, so their residuals on the samples cannot grow with the degree
    d = np.arange(-r, r + 1, dtype=np.float64)
    sigma = 0.25 * (2 * r + 1)
    y = np.exp(-d * d / (2 * sigma * sigma))
    t = d * d / float(r * r)
    res = []
    for D in (2, 3, 4):
        c = O.gauss_fit(r, sigma, D)
        res.append(float(np.sum((sum(ci * t ** i for i, ci in enumerate(c)) - y) ** 2)))
    assert res[0] >= res[1] - 1e-15 and res[1] >= res[2] - 1e-15, res


# --------------------------------------------------------------------------- wedding cake
def test_wedding_cake_hand_case():
    """5 x 5 window, 2 nested windows (half-sides 1 and 2). Manhattan weights
    (2 - |dx|) + (2 - |dy|): the inner 3 x 3 holds 4 (centre), 3 (x4), 2 (x4)
    = 24 over 9 pixels; the outer ring holds the rest of the total 40
    (h rx^2 + w ry^2 = 5*4 + 5*4) = 16 over 16 pixels."""
    K = O.kernel_weights("wedding", 5, 5, rings=2)
    want = np.ones((5, 5))
    want[1:4, 1:4] = 24.0 / 9.0
    assert np.allclose(K, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("w,h,rings", [(5, 5, 1), (31, 31, 4), (41, 21, 3), (9, 45, 8), (7, 7, 16), (3, 3, 4)])
def test_wedding_cake_keeps_the_manhattan_mass(w, h, rings):
    rx, ry = (w - 1) // 2, (h - 1) // 2
    K = O.kernel_weights("wedding", w, h, rings=rings)
    assert abs(K.sum() - (h * rx * rx + w * ry * ry)) <= 1e-9 * K.sum()
    # ring weights do not increase away from the centre (Manhattan falls off)
    prof = [K[ry, rx + d] for d in range(rx + 1)]
    assert all(a >= b - 1e-12 for a, b in zip(prof, prof[1:]))


def test_wedding_cake_with_one_ring_is_the_plain_histogram():
    rng = np.random.default_rng(4)
    bins = rng.integers(0, 6, size=(30, 40)).astype(np.uint8)
    Kw = O.kernel_weights("wedding", 11, 9, rings=1)
    Kp = O.kernel_weights("plain", 11, 9)
    cx, cy = rng.integers(5, 35, 20), rng.integers(4, 26, 20)
    hw = O.normalise(O.hist_at(bins, 6, Kw, cx, cy))
    hp = O.normalise(O.hist_at(bins, 6, Kp, cx, cy))
    assert np.abs(hw - hp).max() <= 1e-14


# ----------------------------------------------------------------------------
# the exponential kernel
# ----------------------------------------------------------------------------
def geometric_axis_mass(r, lam):
    """sum_{d=-r..r} exp(-lam |d|) = (1 + q - 2 q^(r+1)) / (1 - q), q = exp(-lam)
    (two geometric series and the centre)."""
    import math
    q = math.exp(-lam)
    return (1.0 + q - 2.0 * q ** (r + 1)) / (1.0 - q)


@pytest.mark.parametrize("w,h,lam", [(3, 3, 0.1), (21, 9, 0.5), (41, 81, 0.02), (7, 5, 3.0)])
def test_exponential_mass_is_closed_form_everywhere(w, h, lam):
    rx, ry = (w - 1) // 2, (h - 1) // 2
    M = geometric_axis_mass(rx, lam) * geometric_axis_mass(ry, lam)
    K = O.kernel_weights("exponential", w, h, lam=lam)
    assert abs(K.sum() - M) <= 1e-12 * M
    rng = np.random.default_rng(w * 100 + h)
    bins = rng.integers(0, 4, size=(h + 6, w + 5)).astype(np.uint8)
    x0, y0, nx, ny = O.valid_centres(h + 6, w + 5, w, h)
    U = O.hist_rect(bins, 4, K, x0, y0, nx, ny)
    np.testing.assert_allclose(U.sum(-1), M, rtol=1e-12)


def test_exponential_small_rate_is_the_plain_histogram():
    rng = np.random.default_rng(31)
    bins = rng.integers(0, 5, size=(24, 30)).astype(np.uint8)
    x0, y0, nx, ny = O.valid_centres(24, 30, 9, 7)
    U = O.hist_rect(bins, 5, O.kernel_weights("exponential", 9, 7, lam=1e-10), x0, y0, nx, ny)
    C = O.hist_rect(bins, 5, O.kernel_weights("plain", 9, 7), x0, y0, nx, ny)
    np.testing.assert_allclose(U, C, rtol=1e-8, atol=1e-8)


def test_exp_directional_ih_by_brute_force():
    import math
    rng = np.random.default_rng(5)
    bins = rng.integers(0, 2, size=(4, 6)).astype(np.uint8)
    lam = 0.7
    J = O.exp_directional_ih(bins, 1, lam)
    for d in range(4):
        sx, sy = d & 1, d >> 1
        for y in range(4):
            for x in range(6):
                tot = 0.0
                for yy in range(4):
                    for xx in range(6):
                        on_x = xx <= x if sx == 0 else xx >= x
                        on_y = yy <= y if sy == 0 else yy >= y
                        if on_x and on_y and bins[yy, xx] == 1:
                            tot += math.exp(-lam * (abs(x - xx) + abs(y - yy)))
                assert abs(J[d, y, x] - tot) <= 1e-12 * max(1.0, tot), (d, x, y)


def exp_quadrant_sums(J, lam, w, h, xc, yc):
    """U(b) of the exponential kernel at (xc, yc) from the four directional IHs
    J[d] of bin b: each quadrant's sum is a corner difference of its own
    direction's table, with the decay across the window supplied by powers of
    q = exp(-lam); the centre row and column belong to the top-left quadrant,
    the others start one pixel further out (factors q). Reads outside the image
    are zero."""
    import math
    q = math.exp(-lam)
    rx, ry = (w - 1) // 2, (h - 1) // 2
    Hh, Ww = J.shape[1:]

    def at(d, x, y):
        return J[d, y, x] if (0 <= x < Ww and 0 <= y < Hh) else 0.0

    xl, xr, yu, yd = xc - rx - 1, xc + rx + 1, yc - ry - 1, yc + ry + 1

    def quad(d, xa, xf, ya, yf, fx, fy):
        # xa/ya: the corner next to the centre; xf/yf: one past the far edge
        return at(d, xa, ya) - fx * at(d, xf, ya) - fy * at(d, xa, yf) + fx * fy * at(d, xf, yf)

    tl = quad(0, xc, xl, yc, yu, q ** (rx + 1), q ** (ry + 1))
    tr = q * quad(1, xc + 1, xr, yc, yu, q ** rx, q ** (ry + 1))
    bl = q * quad(2, xc, xl, yc + 1, yd, q ** (rx + 1), q ** ry)
    br = q * q * quad(3, xc + 1, xr, yc + 1, yd, q ** rx, q ** ry)
    return tl + tr + bl + br


@pytest.mark.parametrize("lam", [0.05, 0.3, 1.5])
def test_exponential_quadrant_decomposition_matches_brute_force(lam):
    rng = np.random.default_rng(int(lam * 100))
    H, W, B = 20, 23, 3
    bins = rng.integers(0, B, size=(H, W)).astype(np.uint8)
    J = [O.exp_directional_ih(bins, b, lam) for b in range(B)]
    for (w, h) in [(3, 3), (5, 9), (11, 7), (23, 19), (21, 3)]:
        K = O.kernel_weights("exponential", w, h, lam=lam)
        x0, y0, nx, ny = O.valid_centres(H, W, w, h)
        # every valid centre: includes windows touching each image border
        cx, cy = np.meshgrid(np.arange(x0, x0 + nx), np.arange(y0, y0 + ny))
        cx, cy = cx.ravel(), cy.ravel()
        ref = O.hist_at(bins, B, K, cx, cy)
        got = np.array([[exp_quadrant_sums(J[b], lam, w, h, x, y) for b in range(B)]
                        for x, y in zip(cx, cy)])
        np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-11)


# ----------------------------------------------------------------------------
# feature channels (Sec. 4: one likelihood map per feature)
# ----------------------------------------------------------------------------
def read_channel_fixture():
    with open(os.path.join(GOLDEN, "channels_3x3.txt")) as f:
        lines = [ln.split("#")[0].strip() for ln in f]
    lines = [ln for ln in lines if ln]
    chans = []
    i = 0
    while i < len(lines):
        _, c, _, B = lines[i].split()
        rows = [[int(v) for v in lines[i + k].split()] for k in (1, 2, 3)]
        U = [int(v) for v in lines[i + 4].split()[1:]]
        chans.append((int(B), np.array(rows, dtype=np.uint8), U))
        i += 5
    return chans


def test_channel_hand_fixture():
    chans = read_channel_fixture()
    K = O.kernel_weights("manhattan", 3, 3)
    for B, bins, U in chans:
        assert np.array_equal(O.hist_at(bins, B, K, [1], [1])[0], np.array(U, dtype=np.float64))
    q = [np.array([0.5, 0.5]), np.array([1.0, 1.0, 1.0]) / 3.0]
    L = O.likelihood_channels_map([c[1] for c in chans], [c[0] for c in chans], K, q)
    assert L.shape == (2, 1, 1)
    assert abs(L[0, 0, 0] - (np.sqrt(1 / 6) + np.sqrt(1 / 3))) < 1e-15
    assert abs(L[1, 0, 0] - (np.sqrt(1 / 6) + np.sqrt(1 / 9) + np.sqrt(1 / 18))) < 1e-15


def test_channels_reduce_to_one_image_and_share_the_mass():
    rng = np.random.default_rng(41)
    H, W = 21, 30
    imgs = [rng.integers(0, 256, size=(H, W)).astype(np.uint8), rng.integers(0, 4096, size=(H, W)).astype(np.uint16)]
    Bs = [8, 5]
    bins = [O.quantize(imgs[0], 8, 8), O.quantize(imgs[1], 12, 5)]
    K = O.kernel_weights("euclidean", 7, 5)
    qs = []
    for b, B in zip(bins, Bs):
        q = rng.gamma(0.5, size=B)
        qs.append(q / q.sum())
    L = O.likelihood_channels_map(bins, Bs, K, qs)
    for c in range(2):
        np.testing.assert_array_equal(L[c], O.likelihood_map(bins[c], Bs[c], K, qs[c]))
    # one channel is the single-image path
    np.testing.assert_array_equal(O.likelihood_channels_map(bins[:1], Bs[:1], K, qs[:1])[0],
                                  O.likelihood_map(bins[0], Bs[0], K, qs[0]))
    # every pixel is in one bin of each channel: both channels' windows weigh M
    M = 5 * 3 * 7 * 5 // 3 + 7 * 2 * 5 * 3 // 3  # h rx(2rx+1)(2rx-1)/3 + w ry(2ry+1)(2ry-1)/3
    x0, y0, nx, ny = O.valid_centres(H, W, 7, 5)
    for b, B in zip(bins, Bs):
        assert np.all(O.hist_rect(b, B, K, x0, y0, nx, ny).sum(-1) == M)
