"""The Gaussian approximant beyond degree 2 and beyond the 64-bit ring: plans
of degree 3 and 4, and windows whose exact Bernstein moments pass 2^64 (kept
in the ring of integers mod 2^128), against the FP64 brute-force oracle with
the same approximant. Integral histograms are bit-exact against Eq. 2 in that
ring; maps and histograms within 1e-5 (every centre on small cases, sampled
centres for windows of 151-401 px)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import swih_oracle as O  # noqa: E402
from paper_1705_03524_gb300 import swih as S  # noqa: E402
from paper_1705_03524_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5
DEV = "cuda:0"


class _View:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def scene(H, W, seed):
    return synth.blob_scene(H, W, 8, seed, n_blobs=6, axes=(12, 60), margin=40).image


def target_of(bins, B, K, cx, cy):
    return O.target_hist(bins, B, K, cx, cy)


def sampled_parity(p, img, B, w, h, degree, n=1500, seed=0):
    H, W = img.shape
    bins = O.quantize(img, 8, B)
    K = O.kernel_weights("gaussian", w, h, degree=degree)
    rx, ry = (w - 1) // 2, (h - 1) // 2
    q = target_of(bins, B, K, W // 2, H // 2)
    d_q = torch.tensor(q, dtype=torch.float32, device=DEV)
    m = torch.full((H - h + 1, W - w + 1), -1.0, device=DEV)
    p.likelihood("gaussian", w, h, d_q, m)
    p.sync_status()
    rng = np.random.default_rng(seed)
    cx = rng.integers(rx, W - rx, n)
    cy = rng.integers(ry, H - ry, n)
    ref = O.likelihood_at(bins, B, K, q, cx, cy)
    got = m.cpu().numpy()[cy - ry, cx - rx].astype(np.float64)
    assert (m >= 0).all().item(), "a centre was not written"
    return float(np.abs(got - ref).max())


def test_integral_histograms_bit_exact_in_the_128_bit_ring():
    H, W, B = 37, 70, 3
    img = scene(H, W, 3)
    bins = O.quantize(img, 8, B)
    desc = S.make_desc(H, W, bins=B, kernels=("gaussian",), max_win=(21, 21), gauss_degree=3,
                       precision=S.SWIH_PREC_RING128)
    with S.Plan(desc) as p:
        p.build_ih(torch.from_numpy(img).to(DEV))
        p.sync_status()
        info = p.info()
        assert info.elem_bytes == 16 and info.n_terms == 49
        raw = torch.as_tensor(_View(info.d_ih, (info.n_terms * B, H, info.ih_pitch * 2), "<u8"),
                              device=DEV).cpu().numpy()
        rmap = (torch.as_tensor(_View(info.d_row_map, (B, H), "<i4"), device=DEV).cpu().numpy()
                if info.d_row_map else None)
    for t in range(info.n_terms):
        pp, qq = info.term_p[t], info.term_q[t]
        for b in range(B):
            ref = O.weighted_ih(bins, b, pp, qq, 128)
            plane = raw[t * B + b]
            vals = plane[:, 0:2 * W:2].astype(object) + (plane[:, 1:2 * W:2].astype(object) << 64)
            r = rmap[b] if rmap is not None else np.arange(H)
            got = np.where((r >= 0)[:, None], vals[np.maximum(r, 0)], 0)
            assert (got == ref).all(), (pp, qq, b)


@pytest.mark.parametrize("degree,w,h", [(3, 9, 9), (3, 15, 11), (4, 15, 15), (4, 9, 21), (3, 41, 41),
                                        (3, 5, 41), (4, 3, 9)])  # the last two fit lower degrees on one axis
def test_degree_3_and_4_full_maps(degree, w, h):
    H, W, B = 140, 190, 16
    img = scene(H, W, 7 + degree)
    bins = O.quantize(img, 8, B)
    K = O.kernel_weights("gaussian", w, h, degree=degree)
    q = target_of(bins, B, K, 90, 70)
    desc = S.make_desc(H, W, bins=B, kernels=("gaussian",), max_win=(w, h), gauss_degree=degree)
    with S.Plan(desc) as p:
        p.build_ih(torch.from_numpy(img).to(DEV))
        d_q = torch.tensor(q, dtype=torch.float32, device=DEV)
        m = torch.empty((H - h + 1, W - w + 1), device=DEV)
        p.likelihood("gaussian", w, h, d_q, m)
        hist = torch.empty((20, 30, B), device=DEV)
        rx, ry = (w - 1) // 2, (h - 1) // 2
        p.local_hist("gaussian", w, h, rx + 5, ry + 3, 30, 20, hist)
        p.sync_status()
        elem = p.info().elem_bytes
    ref = O.likelihood_map(bins, B, K, q)
    assert np.abs(m.cpu().numpy() - ref).max() <= TOL, (degree, w, h, elem)
    refh = O.normalise(O.hist_rect(bins, B, K, rx + 5, ry + 3, 30, 20))
    assert np.abs(hist.cpu().numpy() - refh).max() <= TOL


@pytest.mark.parametrize("degree,w", [(3, 151), (3, 201), (3, 401), (2, 151), (2, 401), (4, 121), (4, 251)])
def test_large_windows_sampled(degree, w):
    H, W, B = 620, 700, 16
    img = scene(H, W, 11)
    desc = S.make_desc(H, W, bins=B, kernels=("gaussian",), max_win=(w, w), gauss_degree=degree)
    with S.Plan(desc) as p:
        p.build_ih(torch.from_numpy(img).to(DEV))
        assert p.info().elem_bytes == 16
        err = sampled_parity(p, img, B, w, w, degree)
    assert err <= TOL, (degree, w, err)


def test_non_square_window_and_several_scales():
    H, W, B = 400, 520, 8
    img = scene(H, W, 13)
    desc = S.make_desc(H, W, bins=B, kernels=("gaussian",), max_win=(201, 151), gauss_degree=3)
    with S.Plan(desc) as p:
        p.build_ih(torch.from_numpy(img).to(DEV))
        assert sampled_parity(p, img, B, 201, 61, 3) <= TOL
        # several windows in one call equal one call per window
        bins = O.quantize(img, 8, B)
        wins = [(151, 151), (61, 91), (201, 151)]
        qs = [torch.tensor(target_of(bins, B, O.kernel_weights("gaussian", a, b, degree=3), 260, 200),
                           dtype=torch.float32, device=DEV) for a, b in wins]
        maps = [torch.empty((H - b + 1, W - a + 1), device=DEV) for a, b in wins]
        p.likelihood_scales("gaussian", wins, qs, maps)
        for (a, b), qv, mm in zip(wins, qs, maps):
            one = torch.empty_like(mm)
            p.likelihood("gaussian", a, b, qv, one)
            p.sync_status()
            assert torch.equal(one, mm)


def test_channels_with_a_wide_gaussian():
    H, W = 200, 260
    a = scene(H, W, 17)
    b = (a.astype(np.int64) * 7 % 256).astype(np.uint8)
    chans = [S.make_channel(W, bins=8), S.make_channel(W, bins=4)]
    desc = S.make_desc(H, W, bins=1, kernels=("gaussian",), max_win=(61, 61), gauss_degree=4)
    K = O.kernel_weights("gaussian", 61, 61, degree=4)
    bins = [O.quantize(a, 8, 8), O.quantize(b, 8, 4)]
    qs = [np.full(8, 1 / 8), np.array([0.1, 0.2, 0.3, 0.4])]
    ref = O.likelihood_channels_map(bins, [8, 4], K, qs)
    da, db = torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV)
    with S.ChannelPlan(desc, chans) as p:
        p.build_ih([da.data_ptr(), db.data_ptr()])
        maps = torch.empty((2, H - 60, W - 60), device=DEV)
        p.likelihood_channels("gaussian", 61, 61, torch.tensor(np.concatenate(qs), dtype=torch.float32,
                                                               device=DEV), maps)
        p.sync_status()
    assert np.abs(maps.cpu().numpy() - ref).max() <= TOL
