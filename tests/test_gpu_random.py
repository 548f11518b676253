"""Seeded random plans against the oracle: image size, pixel type and bit
depth, bin count, kernel set, band height and windows drawn at random, on
uniform noise (every bin everywhere) and on smooth scenes (bins absent from
rows and from whole CTA regions, so the sparse paths of the scan and the
gather run). Likelihoods and histograms within 1e-5."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import swih_oracle as O  # noqa: E402
from paper_1705_03524_gb300 import swih as S  # noqa: E402
from paper_1705_03524_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5
DEV = "cuda:0"
KERNELS = ("plain", "manhattan", "euclidean", "gaussian", "wedding")


def odd(rng, lo, hi):
    v = int(rng.integers(lo, hi + 1))
    return v if v % 2 else max(3, v - 1)


@pytest.mark.parametrize("seed", range(18))
def test_random_plan_matches_oracle(seed):
    rng = np.random.default_rng(1000 + seed)
    H = int(rng.integers(3, 141))
    W = int(rng.integers(3, 321))
    u16 = bool(rng.integers(0, 2))
    bd = 12 if u16 else 8
    B = int(rng.integers(1, 41))
    smooth = bool(rng.integers(0, 2)) and H >= 8 and W >= 8
    if smooth:
        img = synth.blob_scene(H, W, 16 if u16 else 8, seed, n_blobs=2, margin=2).image
    else:
        img = synth.uniform_image(H, W, 16 if u16 else 8, seed)
    k = [kk for kk in KERNELS if rng.integers(0, 2)] or ["manhattan"]
    windows = []
    for _ in range(3):
        windows.append((odd(rng, 3, min(W, 61)), odd(rng, 3, min(H, 61))))
    mw = max(w for w, _ in windows)
    mh = max(h for _, h in windows)
    band_rows = int(rng.choice([0, 1, 3, 8, 33]))
    pt = S.SWIH_PIXEL_U16 if u16 else S.SWIH_PIXEL_U8
    raw = img.view(np.int16) if u16 else img
    d = torch.from_numpy(np.ascontiguousarray(raw)).to(DEV)
    desc = S.make_desc(H, W, pixel_type=pt, bitdepth=bd, bins=B, kernels=tuple(k), max_win=(mw, mh),
                       band_rows=band_rows, wedding_rings=int(rng.integers(1, 6)))
    try:
        plan = S.Plan(desc)
    except S.SwihError as e:  # a Gaussian window beyond the exact 64-bit moments is refused
        assert e.status == S.SWIH_ERR_UNSUPPORTED and "gaussian" in k
        return
    bins = O.quantize(np.minimum(img.astype(np.int64), (1 << bd) - 1), bd, B)
    with plan:
        plan.build_ih(d)
        for kind in k:
            for (w, h) in windows:
                K = O.kernel_weights(kind, w, h, rings=desc.wedding_rings)
                x0, y0, nx, ny = O.valid_centres(H, W, w, h)
                q = O.target_hist(bins, B, K, x0 + int(rng.integers(0, nx)), y0 + int(rng.integers(0, ny)))
                m = torch.full((ny, nx), -1.0, device=DEV)
                plan.likelihood(kind, w, h, torch.tensor(q, dtype=torch.float32, device=DEV), m)
                ref = O.likelihood_map(bins, B, K, q)
                err = np.abs(m.cpu().numpy() - ref).max()
                assert err <= TOL, (kind, w, h, H, W, B, err)
                hist = torch.empty((ny, nx, B), device=DEV)
                plan.local_hist(kind, w, h, x0, y0, nx, ny, hist)
                refh = O.normalise(O.hist_rect(bins, B, K, x0, y0, nx, ny))
                errh = np.abs(hist.cpu().numpy() - refh).max()
                assert errh <= TOL, (kind, w, h, errh)
        plan.sync_status()
