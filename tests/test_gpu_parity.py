"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

* K1 bins and every K2 integral-histogram plane: bit-exact against the
  oracle's quantiser and Eq. 2 sums in the same ring (mod 2^32 or 2^64).
* K3 normalised histograms and likelihoods: max abs error <= 1e-5 against
  the brute-force oracle (normalised bins and Bhattacharyya coefficients).

Sizes are small enough for the oracle to finish in seconds while spanning
several scan bands, several warps of centres and ragged tails; the
benchmark's full-size workload is checked on sampled centres.
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


class _DevView:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def device_rows(ptr, rows, pitch_elems, typestr):
    """Copy a pitched device array to the host as numpy (rows x pitch)."""
    t = torch.as_tensor(_DevView(ptr, (rows, pitch_elems), typestr), device=DEV)
    return t.cpu().numpy()


def upload(img: np.ndarray, pitch_bytes=None, offset=0):
    """Image to the device as raw bytes with an optional row pitch and base offset."""
    h, w = img.shape
    pb = img.dtype.itemsize
    pitch = pitch_bytes or w * pb
    raw = np.zeros((h, pitch), dtype=np.uint8)
    raw[:, : w * pb] = img.view(np.uint8).reshape(h, w * pb)
    buf = torch.zeros(h * pitch + offset + 64, dtype=torch.uint8, device=DEV)
    buf[offset: offset + h * pitch] = torch.from_numpy(raw.reshape(-1)).to(DEV)
    return buf, buf.data_ptr() + offset, pitch


def make_plan(img, bitdepth, B, kernels, max_win, **kw):
    h, w = img.shape
    pt = S.SWIH_PIXEL_U8 if img.dtype == np.uint8 else S.SWIH_PIXEL_U16
    pitch = kw.pop("pitch_bytes", None)
    offset = kw.pop("offset", 0)
    buf, ptr, pitch = upload(img, pitch, offset)
    desc = S.make_desc(h, w, pitch_bytes=pitch, pixel_type=pt, bitdepth=bitdepth, bins=B,
                       kernels=kernels, max_win=max_win, **kw)
    plan = S.Plan(desc)
    plan.build_ih(ptr)
    plan.sync_status()
    return plan, buf


def oracle_bins(img, bitdepth, B):
    vmax = (1 << bitdepth) - 1
    return O.quantize(np.minimum(img.astype(np.int64), vmax), bitdepth, B)


def check_ih(plan, img, bitdepth, B):
    info = plan.info()
    H, W = img.shape
    bins = oracle_bins(img, bitdepth, B)
    got_bins = device_rows(info.d_bins, H, info.bins_pitch, "|u1")[:, :W]
    assert np.array_equal(got_bins, bins)
    bits = 8 * info.elem_bytes
    ts = "<i4" if info.elem_bytes == 4 else "<i8"
    udt = np.uint32 if info.elem_bytes == 4 else np.uint64
    # rows of a bin the scan did not store (no pixel of the bin) are read at the
    # stored row the plan's row map gives (-1: zero)
    rmap = device_rows(info.d_row_map, B, H, "<i4") if info.d_row_map else None
    if rmap is not None:
        for b in range(B):
            holds = (bins == b).any(axis=1)
            last = np.maximum.accumulate(np.where(holds, np.arange(H), -1))
            assert np.array_equal(rmap[b], last), f"row map of bin {b}"
    for t in range(info.n_terms):
        p, q = info.term_p[t], info.term_q[t]
        for b in range(B):
            ptr = info.d_ih + (t * B + b) * info.plane_elems * info.elem_bytes
            got = device_rows(ptr, H, info.ih_pitch, ts)[:, :W].view(udt)
            if rmap is not None:
                got = np.where((rmap[b] >= 0)[:, None], got[np.maximum(rmap[b], 0)], 0).astype(udt)
            ref = O.weighted_ih(bins, b, p, q, bits)
            if not np.array_equal(got, ref):
                bad = np.argwhere(got != ref)[0]
                raise AssertionError(f"IH term x^{p} y^{q} bin {b} differs at {tuple(bad)}")
    return bins


def check_windows(plan, bins, B, kind, w, h, rect=None):
    H, W = bins.shape
    K = O.kernel_weights(kind, w, h)
    x0, y0, nx, ny = O.valid_centres(H, W, w, h)
    # local histograms over a (sub)rectangle of centres
    cx0, cy0, ncx, ncy = rect or (x0, y0, nx, ny)
    hist = torch.empty((ncy, ncx, B), dtype=torch.float32, device=DEV)
    plan.local_hist(kind, w, h, cx0, cy0, ncx, ncy, hist)
    ref_h = O.normalise(O.hist_rect(bins, B, K, cx0, cy0, ncx, ncy))
    err_h = np.abs(hist.cpu().numpy().astype(np.float64) - ref_h).max()
    assert err_h <= TOL, (kind, w, h, err_h)
    # likelihood over every valid centre, target = a window histogram
    tx, ty = x0 + nx // 3, y0 + ny // 2
    q = O.target_hist(bins, B, K, tx, ty)
    qd = torch.tensor(q, dtype=torch.float32, device=DEV)
    m = torch.empty((ny, nx), dtype=torch.float32, device=DEV)
    plan.likelihood(kind, w, h, qd, m)
    ref_l = O.likelihood_map(bins, B, K, q)
    got_l = m.cpu().numpy().astype(np.float64)
    err_l = np.abs(got_l - ref_l).max()
    assert err_l <= TOL, (kind, w, h, err_l)
    plan.sync_status()
    return err_h, err_l


# --------------------------------------------------------------------------- K1 + K2
IH_CASES = [
    # name, (H, W), pixel bits, B, kernels, max window, extra plan args
    ("config1", (128, 128), 8, 16, ("manhattan",), (31, 31), {}),
    ("ragged_all", (37, 53), 8, 5, ("plain", "manhattan", "euclidean"), (9, 7), dict(band_rows=4)),
    ("wide_E8", (61, 1100), 8, 3, ("manhattan",), (21, 15), dict(band_rows=8)),
    ("wide_E16", (16, 4200), 8, 2, ("manhattan",), (15, 5), dict(band_rows=4)),
    ("plain_2500", (40, 2500), 8, 4, ("plain",), (5, 5), {}),
    ("gauss_u16", (20, 33), 12, 7, ("gaussian",), (15, 9), dict(band_rows=3)),
    ("ring64_forced", (45, 70), 8, 6, ("manhattan", "euclidean"), (11, 11),
     dict(precision=S.SWIH_PREC_RING64, band_rows=5)),
    ("one_bin", (9, 40), 8, 1, ("manhattan",), (5, 5), dict(band_rows=2)),
    ("bins256", (33, 64), 8, 256, ("plain",), (3, 3), {}),
    ("single_band", (24, 96), 8, 4, ("euclidean",), (7, 7), dict(band_rows=100)),
]


def _image(shape, bits, seed):
    h, w = shape
    if bits <= 8:
        return synth.uniform_image(h, w, 8, seed)
    img = synth.uniform_image(h, w, 16, seed)  # values beyond 'bits' exercise clamping
    return img


@pytest.mark.parametrize("case", IH_CASES, ids=[c[0] for c in IH_CASES])
def test_bins_and_integral_histograms_bit_exact(case):
    name, shape, bits, B, kernels, max_win, kw = case
    img = _image(shape, bits, seed=len(name))
    plan, _buf = make_plan(img, bits, B, kernels, max_win, **dict(kw))
    with plan:
        check_ih(plan, img, bits, B)


@pytest.mark.parametrize("pitch_extra,offset", [(0, 0), (7, 0), (64, 0), (3, 1), (0, 5)])
def test_pitched_and_unaligned_u8_input(pitch_extra, offset):
    img = synth.uniform_image(29, 77, 8, seed=3)
    plan, _buf = make_plan(img, 8, 8, ("manhattan",), (9, 9), pitch_bytes=77 + pitch_extra,
                           offset=offset)
    with plan:
        check_ih(plan, img, 8, 8)


def test_u16_offset_input():
    img = synth.uniform_image(21, 45, 16, seed=4)
    plan, _buf = make_plan(img, 10, 16, ("plain",), (5, 5), pitch_bytes=45 * 2 + 6, offset=2)
    with plan:
        check_ih(plan, img, 10, 16)


# --------------------------------------------------------------------------- K3
WIN_CASES = [
    ("config1", (128, 128), 16, ("manhattan",), [(31, 31)]),
    ("tall_chains", (300, 40), 3, ("plain", "manhattan", "euclidean", "gaussian"),
     [(3, 3), (5, 3), (3, 29), (39, 45), (17, 299)]),
    ("ragged", (37, 53), 5, ("plain", "manhattan", "euclidean", "gaussian"),
     [(3, 3), (9, 7), (7, 9), (53, 37), (5, 37), (53, 3)]),
    ("wide", (30, 1100), 4, ("manhattan", "euclidean", "gaussian"), [(21, 15), (1099, 3)]),
    ("bins64", (70, 90), 64, ("manhattan", "gaussian"), [(21, 21), (41, 11)]),
]


@pytest.mark.parametrize("path", ["tiled", "direct"])
@pytest.mark.parametrize("case", WIN_CASES, ids=[c[0] for c in WIN_CASES])
def test_local_hist_and_likelihood_parity(case, path):
    name, shape, B, kernels, windows = case
    H, W = shape
    img = synth.uniform_image(H, W, 8, seed=10 + len(name))
    maxw = max(w for w, _ in windows)
    maxh = max(h for _, h in windows)
    plan, _buf = make_plan(img, 8, B, kernels, (maxw, maxh), band_rows=8)
    if path == "direct":
        S.swih_debug_inject(plan.handle, S.SWIH_INJECT_DIRECT_GATHER)
    with plan:
        bins = oracle_bins(img, 8, B)
        for kind in kernels:
            for (w, h) in windows:
                if kind == "gaussian" and (w * h > 60000):
                    continue
                check_windows(plan, bins, B, kind, w, h)


def test_window_too_wide_for_shared_memory_uses_direct_gather():
    # a 4001-wide window with 64-bit Euclidean terms needs more shared memory
    # than a CTA has; the library falls back to the direct gather on its own
    img = synth.uniform_image(7, 4200, 8, seed=9)
    plan, _buf = make_plan(img, 8, 6, ("euclidean", "manhattan"), (4001, 5),
                           precision=S.SWIH_PREC_RING64)
    with plan:
        bins = oracle_bins(img, 8, 6)
        check_windows(plan, bins, 6, "euclidean", 4001, 5)
        check_windows(plan, bins, 6, "manhattan", 4001, 3)


def test_sub_rectangle_of_centres():
    img = synth.uniform_image(50, 60, 8, seed=2)
    plan, _buf = make_plan(img, 8, 8, ("manhattan", "euclidean"), (11, 11))
    with plan:
        bins = oracle_bins(img, 8, 8)
        check_windows(plan, bins, 8, "manhattan", 11, 9, rect=(7, 6, 13, 1))
        check_windows(plan, bins, 8, "euclidean", 5, 11, rect=(30, 20, 1, 9))


def test_constant_image_gives_delta_histogram():
    img = np.full((40, 44), 200, dtype=np.uint8)
    plan, _buf = make_plan(img, 8, 16, ("manhattan", "euclidean", "gaussian"), (15, 15))
    with plan:
        for kind in ("manhattan", "euclidean", "gaussian"):
            hist = torch.empty((40 - 14, 44 - 14, 16), device=DEV)
            plan.local_hist(kind, 15, 15, 7, 7, 44 - 14, 40 - 14, hist)
            e = torch.zeros(16, device=DEV)
            e[200 * 16 // 256] = 1
            assert (hist - e).abs().max().item() <= TOL


def test_window_argument_errors():
    img = synth.uniform_image(20, 20, 8, seed=1)
    plan, _buf = make_plan(img, 8, 4, ("manhattan",), (9, 9))
    with plan:
        m = torch.empty(400, device=DEV)
        q = torch.full((4,), 0.25, device=DEV)
        for args in [("manhattan", 8, 9), ("manhattan", 11, 9), ("euclidean", 5, 5), ("manhattan", 1, 3)]:
            with pytest.raises(S.SwihError) as ei:
                plan.likelihood(args[0], args[1], args[2], q, m)
            assert ei.value.status == S.SWIH_ERR_INVALID_ARG
        with pytest.raises(S.SwihError):
            plan.local_hist("manhattan", 9, 9, 3, 4, 5, 5, m)  # window leaves the image


def test_injected_stall_reports_timeout_and_recovers():
    img = synth.uniform_image(64, 96, 8, seed=6)
    plan, buf = make_plan(img, 8, 4, ("manhattan",), (9, 9), band_rows=8)
    with plan:
        S.swih_debug_inject(plan.handle, S.SWIH_INJECT_STALL_SCAN_TILE)
        plan.build_ih(buf.data_ptr())
        with pytest.raises(S.SwihError) as ei:
            plan.sync_status()
        assert ei.value.status == S.SWIH_ERR_TIMEOUT
        # the context stays usable: the next build is complete and exact
        plan.build_ih(buf.data_ptr())
        plan.sync_status()
        check_ih(plan, img, 8, 4)


@pytest.mark.parametrize("band_rows", [16, 24, 47, 48, 64])
def test_band_heights_at_the_shared_memory_limit(band_rows):
    """Band heights whose band of bins (band_rows x 1024 bytes kept in shared
    memory) sits on either side of the default 48 KB limit, beside the scan's
    static shared memory: both plans of the benchmark frame build and equal the
    default band height's integral histograms through their maps."""
    cfg = synth.config2()
    img = cfg["image"]
    H, W = img.shape
    B = cfg["B"]
    d = torch.from_numpy(img).to(DEV)
    for kernels, kind, w in ((("gaussian",), "gaussian", 81), (("manhattan", "euclidean"), "euclidean", 41)):
        q = torch.full((B,), 1.0 / B, device=DEV)
        maps = []
        for br in (0, band_rows):
            with S.Plan(S.make_desc(H, W, bins=B, kernels=kernels, max_win=(w, w), band_rows=br)) as p:
                p.build_ih(d)
                m = torch.empty((H - w + 1, W - w + 1), device=DEV)
                p.likelihood(kind, w, w, q, m)
                p.sync_status()
                maps.append(m)
        assert torch.equal(maps[0], maps[1]), (kind, band_rows)


# --------------------------------------------------------------------------- full size
def test_benchmark_workload_sampled_centres():
    """1024 x 1024 synthetic scene, B = 32, the three weighted kernels at windows
    21/41/81, in the plan layout the benchmark uses; sampled centres vs oracle,
    properties (unit mass, L <= 1) at every centre."""
    cfg = synth.config2()
    img = cfg["image"]
    H, W = img.shape
    B = cfg["B"]
    bins = oracle_bins(img, 8, B)
    rng = np.random.default_rng(12)
    plans = []
    buf, ptr, pitch = upload(img)
    for kernels in (("manhattan", "euclidean"), ("gaussian",)):
        d = S.make_desc(H, W, pitch_bytes=pitch, bins=B, kernels=kernels, max_win=(81, 81))
        p = S.Plan(d)
        p.build_ih(ptr)
        plans.append((kernels, p))
    tx, ty = cfg["target_centre"]
    try:
        for kernels, p in plans:
            p.sync_status()
            for kind in kernels:
                for w in cfg["windows"]:
                    K = O.kernel_weights(kind, w, w)
                    q = O.target_hist(bins, B, K, tx, ty)
                    x0, y0, nx, ny = O.valid_centres(H, W, w, w)
                    m = torch.empty((ny, nx), device=DEV)
                    p.likelihood(kind, w, w, torch.tensor(q, dtype=torch.float32, device=DEV), m)
                    got = m.cpu().numpy()
                    assert got.max() <= 1 + 1e-5 and got.min() >= 0
                    cx = rng.integers(x0, x0 + nx, 3000)
                    cy = rng.integers(y0, y0 + ny, 3000)
                    cx = np.concatenate([cx, [x0, x0 + nx - 1, x0, x0 + nx - 1, tx]])
                    cy = np.concatenate([cy, [y0, y0, y0 + ny - 1, y0 + ny - 1, ty]])
                    ref = O.likelihood_at(bins, B, K, q, cx, cy)
                    err = np.abs(got[cy - y0, cx - x0] - ref).max()
                    assert err <= TOL, (kind, w, err)
                    assert abs(got[ty - y0, tx - x0] - 1.0) <= TOL
                    # histograms of one full centre row and one column
                    hist = torch.empty((1, nx, B), device=DEV)
                    p.local_hist(kind, w, w, x0, ty, nx, 1, hist)
                    hh = hist.cpu().numpy()[0]
                    assert np.abs(hh.sum(-1) - 1).max() <= 1e-5
                    sel = np.arange(0, nx, 97)
                    refh = O.normalise(O.hist_at(bins, B, K, x0 + sel, np.full(sel.size, ty)))
                    assert np.abs(hh[sel] - refh).max() <= TOL
            p.sync_status()
    finally:
        for _, p in plans:
            p.close()


def test_benchmark_step_two_streams():
    """The benchmark's step as it is timed: the Gaussian plan on one stream, the
    Manhattan+Euclidean plan forked onto a second stream and joined back each
    step, several steps in a row. The nine maps equal those of the same step on
    one stream bit for bit, and match the oracle at sampled centres."""
    import bench

    cfg = synth.config2()
    img = cfg["image"]
    H, W = img.shape
    B = cfg["B"]
    tx, ty = cfg["target_centre"]
    stream = torch.cuda.Stream(device=DEV)
    fr = bench.FrameStep(S, DEV, img, B, bench.KERNELS, tx, ty, stream, streams=2)
    try:
        assert fr.side is not fr.stream
        for _ in range(4):
            fr.step()
        torch.cuda.synchronize()
        two = [m.cpu().numpy().copy() for m in fr.maps]
        for m in fr.maps:
            m.fill_(-1.0)
        side, fr.side = fr.side, fr.stream
        fr.step()
        fr.side = side
        torch.cuda.synchronize()
        for pl in fr.plans:
            pl.sync_status(stream)
        one = [m.cpu().numpy() for m in fr.maps]
        bins = oracle_bins(img, 8, B)
        rng = np.random.default_rng(13)
        for j, (kind, w) in enumerate(fr.jobs):
            assert np.array_equal(two[j], one[j]), (kind, w)
            K = O.kernel_weights(kind, w, w)
            q = O.target_hist(bins, B, K, tx, ty)
            x0, y0, nx, ny = O.valid_centres(H, W, w, w)
            cx = rng.integers(x0, x0 + nx, 300)
            cy = rng.integers(y0, y0 + ny, 300)
            ref = O.likelihood_at(bins, B, K, q, cx, cy)
            err = np.abs(two[j][cy - y0, cx - x0] - ref).max()
            assert err <= TOL, (kind, w, err)
    finally:
        fr.close()


# --------------------------------------------------------------------------- wedding cake
@pytest.mark.parametrize("rings", [1, 2, 4, 8, 16])
def test_wedding_cake_parity(rings):
    img = synth.uniform_image(90, 120, 8, seed=20 + rings)
    B = 12
    plan, _buf = make_plan(img, 8, B, ("manhattan", "wedding"), (41, 31), wedding_rings=rings)
    with plan:
        bins = oracle_bins(img, 8, B)
        for (w, h) in [(3, 3), (9, 9), (41, 21), (7, 31), (41, 31)]:
            K = O.kernel_weights("wedding", w, h, rings=rings)
            x0, y0, nx, ny = O.valid_centres(90, 120, w, h)
            hist = torch.empty((ny, nx, B), dtype=torch.float32, device=DEV)
            plan.local_hist("wedding", w, h, x0, y0, nx, ny, hist)
            ref_h = O.normalise(O.hist_rect(bins, B, K, x0, y0, nx, ny))
            assert np.abs(hist.cpu().numpy() - ref_h).max() <= TOL, (w, h)
            q = O.target_hist(bins, B, K, x0 + nx // 2, y0 + ny // 3)
            m = torch.empty((ny, nx), device=DEV)
            plan.likelihood("wedding", w, h, torch.tensor(q, dtype=torch.float32, device=DEV), m)
            ref = O.likelihood_map(bins, B, K, q)
            assert np.abs(m.cpu().numpy() - ref).max() <= TOL, (w, h)
        plan.sync_status()


def test_wedding_cake_and_plain_are_approximations_swih_is_exact():
    """Fig. 5: likelihood maps of the weighted (Manhattan) target against the
    brute-force weighted map: SWIH within 1e-5, the wedding cake and the
    plain histogram off by more (printed: max and mean abs error)."""
    cfg = synth.config2()
    img = np.ascontiguousarray(cfg["image"][300:556, 400:656])
    B = cfg["B"]
    bins = oracle_bins(img, 8, B)
    w = 41
    Km = O.kernel_weights("manhattan", w, w)
    q = O.target_hist(bins, B, Km, 128, 128)
    ref = O.likelihood_map(bins, B, Km, q)
    qd = torch.tensor(q, dtype=torch.float32, device=DEV)
    errs = {}
    for kind, rings in [("manhattan", 0), ("plain", 0), ("wedding", 2), ("wedding", 4), ("wedding", 8)]:
        plan, _buf = make_plan(img, 8, B, (kind,), (w, w), wedding_rings=rings)
        with plan:
            m = torch.empty(ref.shape, device=DEV)
            plan.likelihood(kind, w, w, qd, m)
            plan.sync_status()
            d = np.abs(m.cpu().numpy() - ref)
            errs[f"{kind}{rings or ''}"] = (float(d.max()), float(d.mean()))
    print("likelihood error vs brute force (max, mean):", errs)
    assert errs["manhattan"][0] <= TOL
    for k in ("plain", "wedding2", "wedding4", "wedding8"):
        assert errs[k][0] > 100 * TOL, k
    assert errs["wedding8"][1] < errs["plain"][1]


def test_launch_counter_counts_enqueued_kernels():
    img = synth.uniform_image(64, 80, 8, seed=5)
    c0 = S.swih_launch_count()
    plan, _buf = make_plan(img, 8, 8, ("manhattan",), (9, 9))  # one build: quantise + scan + row map
    with plan:
        c1 = S.swih_launch_count()
        m = torch.empty((56, 72), device=DEV)
        plan.likelihood("manhattan", 9, 9, torch.full((8,), 0.125, device=DEV), m)
        plan.sync_status()
        c2 = S.swih_launch_count()
    assert c1 - c0 == 3
    assert c2 - c1 in (1, 2)  # the gather, plus the reduction when the bins were split


@pytest.mark.parametrize("pattern", ["stripes", "blobs", "wide_stripes", "uncached_stripes"])
def test_integral_histograms_with_rows_missing_bins(pattern):
    """Rows that hold no pixel of a bin are not stored by the scan (they are read
    through the plan's row map); check every plane bit for bit where that happens
    often (horizontal stripes of one value, a smooth scene), across several
    bands (the first row of a band is always computed). With 3000 columns and
    64-row bands the band's bins do not fit the scan's shared-memory copy, so its
    sweep prefetches the next row holding the bin from global memory."""
    band_rows = 6
    if pattern in ("stripes", "wide_stripes", "uncached_stripes"):
        rng = np.random.default_rng(3)
        # 4200 columns: 16 per scan thread; 3000: 8 per thread, 64 rows x 3 KB of bins
        h, w = {"stripes": (67, 90), "wide_stripes": (40, 4200), "uncached_stripes": (150, 3000)}[pattern]
        vals = rng.integers(0, 256, size=h).astype(np.uint8)
        img = np.repeat(vals[:, None], w, axis=1)
        img[::5, ::7] = 255 - img[::5, ::7]  # a few pixels of other bins
        if pattern == "uncached_stripes":
            band_rows = 64
    else:
        img = synth.blob_scene(70, 140, 8, seed=4, n_blobs=3, margin=20).image
    plan, _buf = make_plan(img, 8, 8, ("manhattan", "euclidean", "gaussian"), (9, 9), band_rows=band_rows)
    with plan:
        check_ih(plan, img, 8, 8)
        bins = oracle_bins(img, 8, 8)
        check_windows(plan, bins, 8, "gaussian", 9, 7)


def test_rows_left_from_an_earlier_build_are_never_read():
    """A plan stores only the rows that hold each bin; the rows it skips keep
    whatever an earlier build wrote there. Build uniform noise first (every row
    of every bin stored), then stripes on the same plan: every plane through
    the row map, and maps of every tiled and direct kernel, must match the
    oracle for the second image."""
    H, W, B = 90, 150, 8
    noise = synth.uniform_image(H, W, 8, seed=11)
    rng = np.random.default_rng(12)
    stripes = np.repeat(rng.integers(0, 256, size=H).astype(np.uint8)[:, None], W, axis=1)
    stripes[::9, ::11] = 7
    kinds = ("plain", "manhattan", "euclidean", "gaussian", "wedding")
    plan, buf = make_plan(noise, 8, B, kinds, (21, 21))
    with plan:
        info = plan.info()
        assert info.d_row_map
        buf2, ptr2, _ = upload(stripes)
        plan.build_ih(ptr2)
        plan.sync_status()
        bins = check_ih(plan, stripes, 8, B)
        for kind in kinds:
            check_windows(plan, bins, B, kind, 21, 15)
        S.swih_debug_inject(plan.handle, S.SWIH_INJECT_DIRECT_GATHER)
        for kind in ("manhattan", "gaussian"):
            check_windows(plan, bins, B, kind, 9, 9)
        S.swih_debug_inject(plan.handle, 0)


def test_plans_taller_than_32767_rows_store_every_row():
    """The gathers keep stored rows as int16, so a plan of more than 32767 rows
    stores every row and has no row map; it still matches the oracle."""
    img = synth.blob_scene(32800, 24, 8, seed=13, n_blobs=40, axes=(3, 9), margin=4).image
    plan, _buf = make_plan(img, 8, 4, ("manhattan", "gaussian"), (5, 9))
    with plan:
        info = plan.info()
        assert not info.d_row_map
        bins = check_ih(plan, img, 8, 4)
        check_windows(plan, bins, 4, "manhattan", 5, 9)
        check_windows(plan, bins, 4, "gaussian", 5, 5)


def test_scales_in_one_launch_equal_single_windows():
    """swih_likelihood_scales runs the windows of a tiled kernel as one table
    launch (and the others one window at a time); every map equals the
    single-window call up to float rounding, and matches the oracle."""
    img = synth.blob_scene(160, 230, 8, seed=17, n_blobs=5, margin=20).image
    B = 16
    kinds = ("plain", "manhattan", "euclidean", "gaussian", "wedding", "exponential")
    plan, _buf = make_plan(img, 8, B, kinds, (81, 81))
    bins = oracle_bins(img, 8, B)
    windows = [(21, 21), (41, 31), (81, 81), (9, 15), (3, 3)]  # 3 x 3: the Gaussian's fitted degree drops
    with plan:
        for kind in kinds:
            targets, singles, multis = [], [], []
            for i, (w, h) in enumerate(windows):
                K = O.kernel_weights(kind, w, h)
                x0, y0, nx, ny = O.valid_centres(160, 230, w, h)
                q = O.target_hist(bins, B, K, x0 + (7 * i) % nx, y0 + (5 * i) % ny)
                targets.append(torch.tensor(q, dtype=torch.float32, device=DEV))
                singles.append(torch.empty((ny, nx), device=DEV))
                multis.append(torch.full((ny, nx), -1.0, device=DEV))
                plan.likelihood(kind, w, h, targets[i], singles[i])
            plan.likelihood_scales(kind, windows, targets, multis)
            plan.sync_status()
            for (w, h), a, b in zip(windows, singles, multis):
                assert (a - b).abs().max().item() <= 1e-6, (kind, w, h)
            K = O.kernel_weights(kind, 41, 31)
            err = np.abs(multis[1].cpu().numpy() - O.likelihood_map(bins, B, K, targets[1].cpu().numpy())).max()
            assert err <= TOL, (kind, err)
        with pytest.raises(S.SwihError):
            plan.likelihood_scales("manhattan", [(21, 21)] * 9, [targets[0]] * 9, [multis[0]] * 9)


def test_gather_counts_the_bytes_it_loads():
    """The tiled gather reports the integral-histogram bytes it requested: on
    uniform noise (every bin in every window) at least the dense bytes of its
    planes (it also loads the window halo of each column tile), on a
    constant image (one bin) far less: the one block of 4 bins that a step
    carries, a quarter of the 16 bins plus the halo."""
    H, W, B, w = 200, 300, 16, 21
    dense = 5 * B * H * 320 * 4  # Euclidean: 5 planes of 32-bit elements, rows padded to 320
    for img, lo, hi in [(synth.uniform_image(H, W, 8, seed=3), 0.9, 3.0),
                        (np.full((H, W), 77, dtype=np.uint8), 0.0, 0.5)]:
        plan, _buf = make_plan(img, 8, B, ("euclidean",), (w, w))
        with plan:
            plan.load_bytes(reset=True)
            m = torch.empty((H - w + 1, W - w + 1), device=DEV)
            plan.likelihood("euclidean", w, w, torch.full((B,), 1.0 / B, device=DEV), m)
            plan.sync_status()
            got = plan.load_bytes()
            assert lo * dense <= got <= hi * dense, (got, dense)


def test_every_gather_shape_gives_the_same_maps():
    """swih_set_gather_config picks the tiled gather's tile width, copy-ring
    depth and bins per pipeline step (2 only for 256 columns of 32-bit
    elements; any other request falls back to an automatic shape). Every shape
    gives maps equal to the oracle's within the tolerance, through single-window
    launches and the multi-window table launch, on a 32-bit plan wide enough
    for 256-column tiles with ragged tails."""
    img = synth.blob_scene(96, 610, 8, seed=23, n_blobs=6, margin=24).image
    B = 12
    kinds = ("manhattan", "euclidean")
    plan, _buf = make_plan(img, 8, B, kinds, (41, 41))
    bins = oracle_bins(img, 8, B)
    windows = [(21, 21), (41, 11), (5, 41)]
    with plan:
        assert plan.info().elem_bytes == 4
        refs = {}
        for kind in kinds:
            for i, (w, h) in enumerate(windows):
                K = O.kernel_weights(kind, w, h)
                x0, y0, nx, ny = O.valid_centres(96, 610, w, h)
                q = O.target_hist(bins, B, K, x0 + (11 * i) % nx, y0 + (3 * i) % ny)
                refs[kind, w, h] = (torch.tensor(q, dtype=torch.float32, device=DEV),
                                    O.likelihood_map(bins, B, K, q), (ny, nx))
        for kind in kinds:
            k = S.KERNELS[kind]
            for tile_cols in (0, 128, 256):
                for stages in (0, 2, 3):
                    for bps in (0, 2, 4, 8):
                        S.swih_set_gather_config(plan.handle, k, tile_cols, stages, bps)
                        targets = [refs[kind, w, h][0] for w, h in windows]
                        multis = [torch.full(refs[kind, w, h][2], -1.0, device=DEV) for w, h in windows]
                        plan.likelihood_scales(kind, windows, targets, multis)
                        w, h = windows[0]
                        single = torch.full(refs[kind, w, h][2], -1.0, device=DEV)
                        plan.likelihood(kind, w, h, targets[0], single)
                        plan.sync_status()
                        for (w, h), m in zip(windows, multis):
                            err = np.abs(m.cpu().numpy().astype(np.float64) - refs[kind, w, h][1]).max()
                            assert err <= TOL, (kind, tile_cols, stages, bps, w, h, err)
                        err = np.abs(single.cpu().numpy().astype(np.float64) - refs[kind, *windows[0]][1]).max()
                        assert err <= TOL, (kind, tile_cols, stages, bps, "single", err)
            S.swih_set_gather_config(plan.handle, k, 0, 0, 0)


def test_multi_window_call_is_captured_after_a_first_run():
    """swih_likelihood_scales reuses a job-table slot when its arguments repeat,
    enqueuing no copy: after one uncaptured call the same call is captured into
    a CUDA graph, and replays write the maps of the uncaptured call."""
    H, W, B = 300, 400, 16
    img = synth.blob_scene(H, W, 8, 41, n_blobs=5, margin=40).image
    d = torch.from_numpy(img).to(DEV)
    wins = [(21, 21), (41, 31), (61, 61)]
    q = [torch.full((B,), 1.0 / B, device=DEV) for _ in wins]
    s = torch.cuda.Stream()
    with S.Plan(S.make_desc(H, W, bins=B, kernels=("manhattan", "euclidean"), max_win=(61, 61))) as p:
        p.build_ih(d, s)
        for kernel in ("manhattan", "euclidean"):
            maps = [torch.empty((H - h + 1, W - w + 1), device=DEV) for w, h in wins]
            p.likelihood_scales(kernel, wins, q, maps, s)
            s.synchronize()
            ref = [m.clone() for m in maps]
            for m in maps:
                m.fill_(-1.0)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
                p.likelihood_scales(kernel, wins, q, maps, s)
            g.replay()
            torch.cuda.synchronize()
            for a, b in zip(ref, maps):
                assert torch.equal(a, b), kernel
        p.sync_status(s)
