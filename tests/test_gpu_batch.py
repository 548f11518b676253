"""Batches of regions of interest (swih_batch_*) against the FP64 oracle and
against the one-region plan path.

Every map of every region is the likelihood map of that region's own crop
(the paper's problem for one search region, Sec. 1 and Sec. 4), so the oracle
for a batch is the single-region oracle applied region by region. Tolerance:
max abs error <= 1e-5 on likelihoods, as for the single-region path.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import swih_oracle as O  # noqa: E402
from paper_1705_03524_gb300 import swih as S  # noqa: E402
from paper_1705_03524_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5
DEV = "cuda:0"


def upload(img: np.ndarray, pitch_bytes=None, offset=0):
    h, w = img.shape
    pb = img.dtype.itemsize
    pitch = pitch_bytes or w * pb
    raw = np.zeros((h, pitch), dtype=np.uint8)
    raw[:, : w * pb] = img.view(np.uint8).reshape(h, w * pb)
    buf = torch.zeros(h * pitch + offset + 64, dtype=torch.uint8, device=DEV)
    buf[offset: offset + h * pitch] = torch.from_numpy(raw.reshape(-1)).to(DEV)
    return buf, buf.data_ptr() + offset, pitch


def oracle_bins(img, bitdepth, B):
    vmax = (1 << bitdepth) - 1
    return O.quantize(np.minimum(img.astype(np.int64), vmax), bitdepth, B)


class Spec:
    """One region: frame rectangle, kernel, windows; targets and maps on the device."""

    def __init__(self, x0, y0, w, h, kernel, windows):
        self.x0, self.y0, self.w, self.h = x0, y0, w, h
        self.kernel, self.windows = kernel, list(windows)
        self.target = None
        self.q = None
        self.maps = [torch.full((h - wh + 1, w - ww + 1), -1.0, device=DEV) for ww, wh in self.windows]

    def crop(self, img):
        return img[self.y0: self.y0 + self.h, self.x0: self.x0 + self.w]

    def set_target(self, bins, B, seed):
        ww, wh = self.windows[0]
        K = O.kernel_weights(self.kernel, ww, wh)
        x0, y0, nx, ny = O.valid_centres(self.h, self.w, ww, wh)
        rng = np.random.default_rng(seed)
        tx = int(rng.integers(x0, x0 + nx))
        ty = int(rng.integers(y0, y0 + ny))
        self.q = O.target_hist(bins, B, K, tx, ty)
        self.target = torch.tensor(self.q, dtype=torch.float32, device=DEV)

    def roi(self):
        return S.make_roi(self.x0, self.y0, self.w, self.h, self.kernel, self.windows, self.target, self.maps)


def make_batch(img, bitdepth, B, kernels, specs, pitch_bytes=None, offset=0, **kw):
    buf, ptr, pitch = upload(img, pitch_bytes, offset)
    pt = S.SWIH_PIXEL_U8 if img.dtype == np.uint8 else S.SWIH_PIXEL_U16
    for i, sp in enumerate(specs):
        if sp.target is None:
            sp.set_target(oracle_bins(sp.crop(img), bitdepth, B), B, seed=100 + i)
    desc = S.make_batch_desc(img.shape[0], img.shape[1], pitch_bytes=pitch, pixel_type=pt,
                             bitdepth=bitdepth, bins=B, kernels=kernels, **kw)
    keep = [buf] + [sp.target for sp in specs] + [m for sp in specs for m in sp.maps]
    return S.Batch(desc, [sp.roi() for sp in specs], ptr, keep=keep), buf, ptr


def check_against_oracle(img, bitdepth, B, specs):
    worst = 0.0
    for sp in specs:
        bins = oracle_bins(sp.crop(img), bitdepth, B)
        for (ww, wh), m in zip(sp.windows, sp.maps):
            K = O.kernel_weights(sp.kernel, ww, wh)
            ref = O.likelihood_map(bins, B, K, sp.q)
            got = m.cpu().numpy().astype(np.float64)
            assert got.shape == ref.shape
            err = np.abs(got - ref).max()
            assert err <= TOL, (sp.kernel, sp.w, sp.h, ww, wh, err)
            worst = max(worst, err)
    return worst


MIXED = [
    (0, 0, 53, 37, "manhattan", [(9, 7), (53, 3)]),
    (17, 5, 96, 64, "gaussian", [(21, 21), (15, 9), (31, 25)]),
    (101, 77, 40, 120, "euclidean", [(3, 3), (39, 45)]),
    (367, 150, 33, 50, "plain", [(5, 5)]),
    (3, 60, 130, 140, "gaussian", [(41, 41)]),
    (200, 10, 150, 31, "manhattan", [(3, 31), (149, 3)]),
    (0, 197, 5, 3, "gaussian", [(3, 3), (5, 3)]),
    (397, 197, 3, 3, "plain", [(3, 3)]),
]


@pytest.mark.parametrize("layout", ["aligned", "pitched_offset"])
def test_mixed_regions_match_oracle(layout):
    img = synth.uniform_image(200, 400, 16, seed=21)  # values above 2^12 - 1 exercise the clamp
    specs = [Spec(*r) for r in MIXED]
    kw = dict(pitch_bytes=812, offset=2) if layout == "pitched_offset" else {}
    batch, _buf, _ptr = make_batch(img, 12, 24, ("plain", "manhattan", "euclidean", "gaussian"), specs,
                                   band_rows=16, **kw)
    with batch:
        batch.run()
        batch.sync_status()
        check_against_oracle(img, 12, 24, specs)


def test_bands_taller_than_64_rows_store_every_row():
    """Work sets store only the rows that hold each bin when bands are at most
    64 rows; with 65-row bands they store every row (no row maps). Both paths
    match the oracle on the same regions."""
    img = synth.blob_scene(200, 400, 8, seed=9, n_blobs=6, margin=10).image
    for band_rows in (65, 16):
        specs = [Spec(*r) for r in MIXED]
        batch, buf, _ptr = make_batch(img, 8, 16, ("plain", "manhattan", "euclidean", "gaussian"), specs,
                                      band_rows=band_rows)
        with batch:
            batch.run()
            batch.sync_status()
        torch.cuda.synchronize()
        check_against_oracle(img, 8, 16, specs)


def test_batch_equals_single_region_plans():
    img = synth.blob_scene(300, 500, 8, seed=5, n_blobs=5, margin=40).image
    specs = [Spec(0, 0, 200, 150, "manhattan", [(21, 21), (41, 41)]),
             Spec(150, 100, 333, 181, "euclidean", [(15, 15), (81, 61)]),
             Spec(60, 200, 96, 100, "manhattan", [(9, 33)])]
    B = 32
    batch, _buf, _ptr = make_batch(img, 8, B, ("manhattan", "euclidean"), specs)
    with batch:
        batch.run()
        batch.sync_status()
        for sp in specs:
            crop = np.ascontiguousarray(sp.crop(img))
            cbuf, cptr, pitch = upload(crop)
            maxw = max(w for w, _ in sp.windows)
            maxh = max(h for _, h in sp.windows)
            d = S.make_desc(sp.h, sp.w, pitch_bytes=pitch, bins=B, kernels=("manhattan", "euclidean"),
                            max_win=(maxw, maxh))
            with S.Plan(d) as p:
                p.build_ih(cptr)
                for (ww, wh), m in zip(sp.windows, sp.maps):
                    alone = torch.empty_like(m)
                    p.likelihood(sp.kernel, ww, wh, sp.target, alone)
                    p.sync_status()
                    assert (alone - m).abs().max().item() <= 1e-6
        check_against_oracle(img, 8, B, specs)


def test_rerun_is_deterministic_follows_the_frame_and_survives_autotune():
    img = synth.uniform_image(160, 260, 8, seed=8)
    specs = [Spec(10, 10, 120, 100, "gaussian", [(15, 15), (31, 21)]),
             Spec(100, 40, 150, 120, "manhattan", [(25, 25)]),
             Spec(0, 100, 90, 60, "euclidean", [(11, 11), (41, 21)])]
    B = 16
    batch, buf, ptr = make_batch(img, 8, B, ("manhattan", "euclidean", "gaussian"), specs)
    with batch:
        batch.run()
        batch.sync_status()
        first = [m.clone() for sp in specs for m in sp.maps]
        batch.run()
        batch.sync_status()
        second = [m.clone() for sp in specs for m in sp.maps]
        assert all(torch.equal(a, b) for a, b in zip(first, second))
        check_against_oracle(img, 8, B, specs)
        # the frame is read at every run: new contents, new maps
        img2 = synth.uniform_image(160, 260, 8, seed=9)
        buf[: img2.size].copy_(torch.from_numpy(img2.reshape(-1)).to(DEV))
        batch.run()
        batch.sync_status()
        check_against_oracle(img2, 8, B, specs)
        # autotuning picks launch shapes, not results
        before = [m.clone() for sp in specs for m in sp.maps]
        batch.autotune()
        for sp in specs:
            for m in sp.maps:
                m.fill_(-1.0)
        batch.run()
        batch.sync_status()
        after = [m for sp in specs for m in sp.maps]
        assert max((a - b).abs().max().item() for a, b in zip(before, after)) <= 1e-6
        check_against_oracle(img2, 8, B, specs)


def test_autotune_of_32bit_groups_keeps_results():
    """A Manhattan + Euclidean batch keeps 32-bit integral histograms, where the
    autotuner also tries steps of 2 bins (256-column tiles only); whatever it
    picks, the maps are unchanged and match the oracle."""
    img = synth.blob_scene(300, 500, 8, seed=5, n_blobs=5, margin=40).image
    specs = [Spec(0, 0, 300, 150, "euclidean", [(21, 21), (41, 41)]),
             Spec(150, 100, 333, 181, "manhattan", [(15, 15), (41, 21)])]
    B = 16
    batch, _buf, _ptr = make_batch(img, 8, B, ("manhattan", "euclidean"), specs)
    with batch:
        batch.run()
        batch.sync_status()
        before = [m.clone() for sp in specs for m in sp.maps]
        batch.autotune()
        for sp in specs:
            for m in sp.maps:
                m.fill_(-1.0)
        batch.run()
        batch.sync_status()
        after = [m for sp in specs for m in sp.maps]
        assert max((a - b).abs().max().item() for a, b in zip(before, after)) <= 1e-6
        check_against_oracle(img, 8, B, specs)


def test_runs_on_a_user_stream():
    img = synth.uniform_image(100, 120, 8, seed=3)
    specs = [Spec(0, 0, 120, 100, "manhattan", [(11, 11)]), Spec(20, 30, 64, 64, "euclidean", [(9, 9)])]
    batch, _buf, _ptr = make_batch(img, 8, 8, ("manhattan", "euclidean"), specs)
    s = torch.cuda.Stream()
    with batch:
        for _ in range(3):
            batch.run(s)
        batch.sync_status(s)
        check_against_oracle(img, 8, 8, specs)


def test_search_regions_workload_sampled():
    """64 regions of 96-768 px cut from a 4096 x 4096 uint16 frame, B = 64,
    Gaussian kernel at three scales per region, in the layout the benchmark
    times; sampled centres vs the oracle, and properties at every centre."""
    cfg = synth.config3()
    img = cfg["image"]
    B = cfg["B"]
    specs = []
    for (x0, y0, w, h), wins, (ox, oy) in zip(cfg["rois"], cfg["windows"], cfg["object_centres"]):
        sp = Spec(x0, y0, w, h, "gaussian", [(k, k) for k in wins])
        bins = oracle_bins(sp.crop(img), 16, B)
        K = O.kernel_weights("gaussian", wins[1], wins[1])
        r = wins[1] // 2
        tx = min(max(ox - x0, r), w - 1 - r)
        ty = min(max(oy - y0, r), h - 1 - r)
        sp.q = O.target_hist(bins, B, K, tx, ty)
        sp.target = torch.tensor(sp.q, dtype=torch.float32, device=DEV)
        sp.bins = bins
        sp.t = (tx, ty)
        specs.append(sp)
    batch, _buf, _ptr = make_batch(img, 16, B, ("gaussian",), specs)
    rng = np.random.default_rng(31)
    with batch:
        batch.run()
        batch.sync_status()
        for sp in specs:
            for k, ((ww, wh), m) in enumerate(zip(sp.windows, sp.maps)):
                got = m.cpu().numpy()
                assert got.min() >= 0.0 and got.max() <= 1.0 + 1e-5
                K = O.kernel_weights("gaussian", ww, wh)
                x0, y0, nx, ny = O.valid_centres(sp.h, sp.w, ww, wh)
                cx = np.concatenate([rng.integers(x0, x0 + nx, 150), [x0, x0 + nx - 1]])
                cy = np.concatenate([rng.integers(y0, y0 + ny, 150), [y0 + ny - 1, y0]])
                ref = O.likelihood_at(sp.bins, B, K, sp.q, cx, cy)
                err = np.abs(got[cy - y0, cx - x0] - ref).max()
                assert err <= TOL, (sp.x0, sp.y0, ww, err)
                if k == 1:  # the target window itself scores 1
                    tx, ty = sp.t
                    assert abs(got[ty - y0, tx - x0] - 1.0) <= TOL


@pytest.mark.parametrize("kernel", ["plain", "manhattan", "euclidean", "gaussian"])
def test_every_binary_4x4_image_in_one_batch(kernel):
    """All 2^16 binary 4 x 4 images, B = 2, 3 x 3 windows: 65536 regions in one
    batched launch. Image t sits at tile (t % 256, t // 256) of a 1024 x 1024
    frame, pixel (i, j) = 255 * bit (4 i + j) of t. The 3 x 3 windows around a
    tile's four centres stay inside the tile, so the oracle on the tiled frame
    gives every image's own answer."""
    t = np.arange(1 << 16, dtype=np.int64)
    bits = (t[:, None] >> np.arange(16)[None, :]) & 1          # [image][4 i + j]
    tiles = (bits.reshape(256, 256, 4, 4) * 255).astype(np.uint8)  # [ty][tx][i][j]
    img = np.ascontiguousarray(tiles.transpose(0, 2, 1, 3).reshape(1024, 1024))
    B = 2
    q = np.array([0.3, 0.7])
    target = torch.tensor(q, dtype=torch.float32, device=DEV)
    maps = torch.full((1 << 16, 2, 2), -1.0, device=DEV)
    buf, ptr, pitch = upload(img)
    rois = [S.make_roi(4 * (k % 256), 4 * (k // 256), 4, 4, kernel, [(3, 3)], target, [maps[k]])
            for k in range(1 << 16)]
    desc = S.make_batch_desc(1024, 1024, pitch_bytes=pitch, bins=B, kernels=(kernel,))
    with S.Batch(desc, rois, ptr, keep=[buf, target, maps]) as b:
        b.run()
        b.sync_status()
    got = maps.cpu().numpy()
    bins = oracle_bins(img, 8, B)
    K = O.kernel_weights(kernel, 3, 3)
    ty, tx = np.divmod(np.arange(1 << 16), 256)
    for dy in (0, 1):
        for dx in (0, 1):
            ref = O.likelihood_at(bins, B, K, q, 4 * tx + 1 + dx, 4 * ty + 1 + dy)
            err = np.abs(got[:, dy, dx] - ref).max()
            assert err <= TOL, (kernel, dx, dy, err)


def test_regions_with_their_own_bin_counts():
    """ROIs of one batch with different bin counts (one work set per count,
    all in the one graph) match the oracle at their own B, survive autotuning,
    and the sync status covers every set."""
    img = synth.blob_scene(260, 420, 8, seed=15, n_blobs=6, margin=30).image
    rows = [(0, 0, 120, 90, "manhattan", [(21, 21)], 8), (100, 40, 200, 150, "gaussian", [(25, 25), (41, 31)], 32),
            (250, 120, 160, 130, "euclidean", [(15, 15)], 64), (30, 150, 90, 100, "gaussian", [(9, 9)], 8),
            (300, 10, 100, 80, "plain", [(7, 7)], 0)]  # 0: the batch's own bin count
    B_default = 16
    specs, bs = [], []
    for (x0, y0, w, h, k, wins, B) in rows:
        sp = Spec(x0, y0, w, h, k, wins)
        Bi = B or B_default
        sp.set_target(oracle_bins(sp.crop(img), 8, Bi), Bi, seed=x0 + y0)
        specs.append(sp)
        bs.append(B)
    buf, ptr, pitch = upload(img)
    desc = S.make_batch_desc(img.shape[0], img.shape[1], pitch_bytes=pitch, bins=B_default,
                             kernels=("plain", "manhattan", "euclidean", "gaussian"))
    rois = [S.make_roi(sp.x0, sp.y0, sp.w, sp.h, sp.kernel, sp.windows, sp.target, sp.maps, bins=B)
            for sp, B in zip(specs, bs)]
    keep = [buf] + [sp.target for sp in specs] + [m for sp in specs for m in sp.maps]
    with S.Batch(desc, rois, ptr, keep=keep) as batch:
        batch.run()
        batch.sync_status()
        first = [m.clone() for sp in specs for m in sp.maps]
        batch.autotune()
        for sp in specs:
            for m in sp.maps:
                m.fill_(-1.0)
        batch.run()
        batch.sync_status()
    for a, m in zip(first, [m for sp in specs for m in sp.maps]):
        assert torch.equal(a, m)
    for sp, B in zip(specs, bs):
        check_against_oracle(img, 8, B or B_default, [sp])
