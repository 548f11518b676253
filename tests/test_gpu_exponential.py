"""Exponential kernel K = exp(-lambda (|dx| + |dy|)) on the GPU against the
oracle: likelihood maps and histograms within 1e-5 for decay rates across the
accepted range, windows from 3 x 3 to the whole image, ragged widths (4, 8 and
16 columns per scan thread), band heights that leave short last bands, both
pixel types and B = 1..64; the scan's directional integral histograms against
their definition; bins absent from a window exactly 0 (bins whose weight in the window is below
the fixed-point resolution may round to 0 too)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import swih_oracle as O  # noqa: E402
from paper_1705_03524_gb300 import swih as S  # noqa: E402
from paper_1705_03524_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5
DEV = "cuda:0"


class _DevView:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def make(H, W, u16, seed, smooth):
    if smooth:
        img = synth.blob_scene(H, W, 16 if u16 else 8, seed, n_blobs=3, margin=2).image
    else:
        img = synth.uniform_image(H, W, 16 if u16 else 8, seed)
    raw = img.view(np.int16) if u16 else img
    return img, torch.from_numpy(np.ascontiguousarray(raw)).to(DEV)


CASES = [
    # H, W, u16, B, lambda, windows, band_rows, smooth
    (40, 77, False, 8, 0.1, [(3, 3), (21, 21), (5, 39)], 0, False),
    (45, 300, True, 16, 0.02, [(41, 41), (3, 45), (77, 9)], 0, True),
    (33, 129, False, 1, 0.7, [(9, 11), (129, 33)], 3, False),
    (64, 200, False, 64, 4.0, [(3, 3), (25, 25)], 1, True),
    (50, 96, True, 32, 1.0 / 1024, [(7, 7), (95, 49)], 0, False),
    (37, 160, False, 12, 16.0, [(3, 5), (31, 31)], 0, True),
    (11, 3000, True, 8, 0.2, [(3, 3), (13, 11)], 0, False),
    (9, 4100, False, 16, 0.3, [(3, 3), (9, 9)], 0, False),
    (7, 8192, True, 8, 0.05, [(5, 7), (61, 5)], 0, False),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_exponential_matches_the_oracle(case):
    H, W, u16, B, lam, windows, band_rows, smooth = CASES[case]
    img, d = make(H, W, u16, 50 + case, smooth and H >= 8 and W >= 8)
    bd = 16 if u16 else 8
    mw = max(w for w, _ in windows)
    mh = max(h for _, h in windows)
    desc = S.make_desc(H, W, pixel_type=S.SWIH_PIXEL_U16 if u16 else S.SWIH_PIXEL_U8, bitdepth=bd, bins=B,
                       kernels=("exponential",), max_win=(mw, mh), band_rows=band_rows, exp_lambda=lam)
    bins = O.quantize(img, bd, B)
    rng = np.random.default_rng(case)
    with S.Plan(desc) as plan:
        plan.build_ih(d)
        for (w, h) in windows:
            K = O.kernel_weights("exponential", w, h, lam=lam)
            x0, y0, nx, ny = O.valid_centres(H, W, w, h)
            q = O.target_hist(bins, B, K, x0 + int(rng.integers(0, nx)), y0 + int(rng.integers(0, ny)))
            m = torch.full((ny, nx), -1.0, device=DEV)
            plan.likelihood("exponential", w, h, torch.tensor(q, dtype=torch.float32, device=DEV), m)
            if nx * ny * w * h <= 40_000_000:
                ref = O.likelihood_map(bins, B, K, q)
                got = m.cpu().numpy()
            else:  # sampled centres, borders included
                cx = np.concatenate([[x0, x0 + nx - 1], rng.integers(x0, x0 + nx, 400)])
                cy = np.concatenate([[y0, y0 + ny - 1], rng.integers(y0, y0 + ny, 400)])
                ref = O.likelihood_at(bins, B, K, q, cx, cy)
                got = m.cpu().numpy()[cy - y0, cx - x0]
            err = np.abs(got - ref).max()
            assert err <= TOL, (case, w, h, err)
            # histograms on a block of centres at the top-left corner and one at the bottom-right
            for (bx, by) in ((x0, y0), (x0 + max(0, nx - 6), y0 + max(0, ny - 5))):
                cw, ch = min(6, nx), min(5, ny)
                hist = torch.empty((ch, cw, B), device=DEV)
                plan.local_hist("exponential", w, h, bx, by, cw, ch, hist)
                U = O.hist_rect(bins, B, K, bx, by, cw, ch)
                refh = O.normalise(U)
                gh = hist.cpu().numpy()
                assert np.abs(gh - refh).max() <= TOL, (case, w, h)
                # a bin absent from the window is exactly zero (count gate); a bin whose
                # weight is above the fixed-point resolution is positive (a far corner
                # pixel at lambda = 4 weighs e^-96 and may round to 0 like in float32)
                assert (gh[U == 0.0] == 0.0).all()
                assert (gh[refh > 1e-9] > 0.0).all()
                np.testing.assert_allclose(gh.sum(-1), 1.0, atol=1e-5)
        plan.sync_status()


@pytest.mark.parametrize("lam,band_rows", [(0.02, 0), (0.5, 5), (3.0, 1)])
def test_directional_tables_match_their_definition(lam, band_rows):
    H, W, B = 70, 150, 5
    img, d = make(H, W, False, 7, True)
    bins = O.quantize(img, 8, B)
    desc = S.make_desc(H, W, bins=B, kernels=("exponential",), max_win=(9, 9), band_rows=band_rows,
                       exp_lambda=lam)
    with S.Plan(desc) as plan:
        plan.build_ih(d)
        plan.sync_status()
        info = S.swih_plan_get_info(plan.handle)
        assert info.d_exp and 30 <= info.exp_frac_bits <= 59
        rows = 4 * B * H  # planes (d, b) of H rows each, back to back
        raw = torch.as_tensor(_DevView(info.d_exp, (rows, info.ih_pitch), "<i8"), device=DEV).cpu().numpy()
    J = raw.view(np.uint64).reshape(4, B, H, info.ih_pitch)[..., :W]
    scale = 2.0 ** -info.exp_frac_bits
    jmax = 1.0 / (1.0 - np.exp(-lam)) ** 2
    for b in range(B):
        ref = O.exp_directional_ih(bins, b, lam)
        got = J[:, b].astype(np.float64) * scale
        assert np.abs(got - ref).max() <= 1e-12 * jmax, (b, np.abs(got - ref).max())


def test_exponential_beside_the_polynomial_kernels():
    """One plan serving Manhattan, Gaussian and the exponential kernel: each map
    matches the oracle, so the exponential tables and the integer ones coexist."""
    H, W, B = 96, 140, 16
    img, d = make(H, W, True, 3, True)
    bins = O.quantize(img, 16, B)
    desc = S.make_desc(H, W, pixel_type=S.SWIH_PIXEL_U16, bitdepth=16, bins=B,
                       kernels=("manhattan", "gaussian", "exponential"), max_win=(41, 41), exp_lambda=0.15)
    with S.Plan(desc) as plan:
        plan.build_ih(d)
        for kind, kw in (("manhattan", {}), ("gaussian", {}), ("exponential", {"lam": 0.15})):
            K = O.kernel_weights(kind, 41, 31, **kw)
            x0, y0, nx, ny = O.valid_centres(H, W, 41, 31)
            q = O.target_hist(bins, B, K, x0 + 5, y0 + 7)
            m = torch.empty((ny, nx), device=DEV)
            plan.likelihood(kind, 41, 31, torch.tensor(q, dtype=torch.float32, device=DEV), m)
            err = np.abs(m.cpu().numpy() - O.likelihood_map(bins, B, K, q)).max()
            assert err <= TOL, (kind, err)
        plan.sync_status()
