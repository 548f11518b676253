"""Feature channels (swih_plan_channels): several feature images per pixel,
each quantised into its own bins, built by one scan and scored by one gather
launch into one likelihood map per channel (Sec. 4: one likelihood map per
feature). Each channel's map is compared with the FP64 brute-force oracle over
that channel alone, every valid centre, within 1e-5; the bin planes are
bit-exact."""
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


def feature_images(H, W, seed):
    """Three features of one scene: the intensity (u8), a 12-bit texture-like
    channel (u16) and a 6-bit channel stored in a pitched u8 buffer."""
    sc = synth.blob_scene(H, W, 8, seed, n_blobs=4, axes=(10, 40), margin=40).image
    tex = synth.uniform_image(H, W, 16, seed=seed + 1) >> 4  # 12 significant bits
    tex = ((tex.astype(np.int64) + 16 * sc.astype(np.int64)) % 4096).astype(np.uint16)
    six = (sc.astype(np.int64) * 3 // 4 % 64).astype(np.uint8)
    return [sc, tex, six]


def upload(img, pitch_elems=None):
    if pitch_elems is None or pitch_elems == img.shape[1]:
        t = torch.from_numpy(img if img.dtype == np.uint8 else img.view(np.int16)).to(DEV)
        return t, t.data_ptr()
    buf = np.zeros((img.shape[0], pitch_elems), dtype=img.dtype)
    buf[:, : img.shape[1]] = img
    t = torch.from_numpy(buf if buf.dtype == np.uint8 else buf.view(np.int16)).to(DEV)
    return t, t.data_ptr()


SPEC = [(S.SWIH_PIXEL_U8, 8, 16, None), (S.SWIH_PIXEL_U16, 12, 8, None), (S.SWIH_PIXEL_U8, 6, 4, 448)]


def make_plan(H, W, kernels, max_win, spec=SPEC):
    chans = [S.make_channel(W, pixel_type=pt, bitdepth=bd, bins=B,
                            pitch_bytes=(p * (1 if pt == S.SWIH_PIXEL_U8 else 2)) if p else None)
             for pt, bd, B, p in spec]
    desc = S.make_desc(H, W, bins=1, kernels=kernels, max_win=max_win)
    return S.ChannelPlan(desc, chans)


@pytest.mark.parametrize("kernel,w,h", [("manhattan", 21, 15), ("euclidean", 9, 31), ("gaussian", 25, 25),
                                        ("plain", 7, 7), ("wedding", 31, 21)])
@pytest.mark.parametrize("path", ["tiled", "direct"])
def test_channel_maps_match_the_oracle(kernel, w, h, path):
    H, W = 230, 410
    imgs = feature_images(H, W, 21)
    bins = [O.quantize(im, bd, B) for im, (_, bd, B, _) in zip(imgs, SPEC)]
    Bs = [B for _, _, B, _ in SPEC]
    K = O.kernel_weights(kernel, w, h)
    rng = np.random.default_rng(5)
    qs = []
    for B in Bs:
        q = rng.gamma(0.5, size=B) + 1e-3
        qs.append(q / q.sum())
    ref = O.likelihood_channels_map(bins, Bs, K, qs)
    bufs = [upload(im, p)[0] for im, (_, _, _, p) in zip(imgs, SPEC)]
    with make_plan(H, W, (kernel,), (w, h)) as p:
        if path == "direct":
            S.swih_debug_inject(p.handle, S.SWIH_INJECT_DIRECT_GATHER)
        p.build_ih([b.data_ptr() for b in bufs])
        q_all = torch.tensor(np.concatenate(qs), dtype=torch.float32, device=DEV)
        maps = torch.full((3, H - h + 1, W - w + 1), -1.0, device=DEV)
        p.likelihood_channels(kernel, w, h, q_all, maps)
        p.sync_status()
        info = p.info()
        assert info.n_channels == 3 and info.bins == sum(Bs)
        # bin planes: each channel's bins offset by the bins of the channels before it
        planes = torch.as_tensor(_View(info.d_bins, (3, H, info.bins_pitch), "|u1"), device=DEV).cpu().numpy()
        off = 0
        for c in range(3):
            assert np.array_equal(planes[c, :, :W], bins[c].astype(np.int64) + off), c
            off += Bs[c]
    got = maps.cpu().numpy().astype(np.float64)
    for c in range(3):
        err = np.abs(got[c] - ref[c]).max()
        assert err <= TOL, (kernel, path, c, err)


def test_channel_histograms_are_per_channel_normalised():
    H, W = 120, 150
    imgs = feature_images(H, W, 3)
    bins = [O.quantize(im, bd, B) for im, (_, bd, B, _) in zip(imgs, SPEC)]
    K = O.kernel_weights("euclidean", 15, 11)
    bufs = [upload(im, p)[0] for im, (_, _, _, p) in zip(imgs, SPEC)]
    cx0, cy0, ncx, ncy = 20, 30, 64, 17
    with make_plan(H, W, ("euclidean",), (15, 11)) as p:
        p.build_ih([b.data_ptr() for b in bufs])
        hist = torch.empty((ncy, ncx, 28), device=DEV)
        p.local_hist("euclidean", 15, 11, cx0, cy0, ncx, ncy, hist)
        p.sync_status()
    got = hist.cpu().numpy().astype(np.float64)
    off = 0
    for c, (_, _, B, _) in enumerate(SPEC):
        ref = O.normalise(O.hist_rect(bins[c], B, K, cx0, cy0, ncx, ncy))
        assert np.abs(got[..., off:off + B] - ref).max() <= TOL, c
        off += B


def test_one_channel_equals_the_single_image_plan():
    H, W = 200, 260
    img = synth.blob_scene(H, W, 8, 9, n_blobs=3, axes=(8, 30), margin=30).image
    d = torch.from_numpy(img).to(DEV)
    q = torch.full((32,), 1.0 / 32, device=DEV)
    for kernel in ("manhattan", "gaussian"):
        a = torch.empty((H - 41 + 1, W - 41 + 1), device=DEV)
        b = torch.empty_like(a)
        with S.Plan(S.make_desc(H, W, bins=32, kernels=(kernel,), max_win=(41, 41))) as p:
            p.build_ih(d)
            p.likelihood(kernel, 41, 41, q, a)
            p.sync_status()
        with make_plan(H, W, (kernel,), (41, 41), spec=[(S.SWIH_PIXEL_U8, 8, 32, None)]) as p:
            p.build_ih([d.data_ptr()])
            p.likelihood_channels(kernel, 41, 41, q, b)
            p.sync_status()
        assert torch.equal(a, b), kernel


def test_eight_channels_of_32_bins():
    # the largest bin space: 8 channels x 32 bins = 256 global bins
    H, W = 96, 130
    spec = [(S.SWIH_PIXEL_U8, 8, 32, None)] * 8
    imgs = [synth.uniform_image(H, W, 8, seed=50 + c) for c in range(8)]
    bins = [O.quantize(im, 8, 32) for im in imgs]
    K = O.kernel_weights("manhattan", 11, 13)
    qs = [np.full(32, 1.0 / 32) for _ in range(8)]
    ref = O.likelihood_channels_map(bins, [32] * 8, K, qs)
    bufs = [torch.from_numpy(im).to(DEV) for im in imgs]
    with make_plan(H, W, ("manhattan",), (11, 13), spec=spec) as p:
        p.build_ih([b.data_ptr() for b in bufs])
        maps = torch.empty((8, H - 12, W - 10), device=DEV)
        p.likelihood_channels("manhattan", 11, 13, torch.full((256,), 1.0 / 32, device=DEV), maps)
        p.sync_status()
    assert np.abs(maps.cpu().numpy() - ref).max() <= TOL


def test_channel_plan_is_not_built_by_the_single_image_call():
    with make_plan(64, 64, ("manhattan",), (9, 9), spec=[(S.SWIH_PIXEL_U8, 8, 8, None)]) as p:
        with pytest.raises(S.SwihError) as ei:
            S.swih_build_ih(p.handle, torch.zeros((64, 64), dtype=torch.uint8, device=DEV))
        assert ei.value.status == S.SWIH_ERR_INVALID_ARG
