"""The allocation-free build (swih_build_ih_noalloc) against the plan build.

swih_build_ih_noalloc serves callers that may not allocate device memory
(fixed memory pools, real-time loops that may not synchronise): it keeps the
scan's scratch in a static device array inside the library and writes the
integral histograms into memory the caller owns. This test calls it through
the C ABI twice in a row on two different frames and checks that each result
equals what a plan (swih_plan + swih_build_ih) computes for the same frame,
bit for bit (the integral histograms are exact ring integers), and that the
second call leaves free device memory unchanged. It lives in its own file
that pytest collects last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1705_03524_gb300 import swih as S  # noqa: E402
from paper_1705_03524_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


class _View:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def planes(ptr, info):
    """All integral-histogram planes as host uint arrays [T*B, H, W]; a plan's rows
    that were not stored (no pixel of the bin) are read through its row map."""
    ts = "<i4" if info.elem_bytes == 4 else "<i8"
    udt = np.uint32 if info.elem_bytes == 4 else np.uint64
    n = info.n_terms * info.bins
    t = torch.as_tensor(_View(ptr, (n, info.height, info.ih_pitch), ts), device=DEV)
    out = t.cpu().numpy()[:, :, : info.width].view(udt)
    if info.d_row_map:
        rm = torch.as_tensor(_View(info.d_row_map, (info.bins, info.height), "<i4"), device=DEV).cpu().numpy()
        for i in range(n):
            r = rm[i % info.bins]
            out[i] = np.where((r >= 0)[:, None], out[i][np.maximum(r, 0)], 0)
    return out


@pytest.mark.parametrize("kernels,shape,B", [(("manhattan", "euclidean"), (300, 500), 16),
                                              (("gaussian",), (160, 210), 8)])
def test_noalloc_build_equals_plan_build_two_calls(kernels, shape, B):
    two_calls_against_plan(kernels, shape, B)


def test_noalloc_raises_the_band_height_when_the_scratch_is_short():
    # With the default 32-row bands this frame's look-back state (5 terms, 3
    # y-exponents, 32 bins, 2048 columns, 16 bands) is far above the static
    # scratch; the entry point raises the band height until it fits. Bands
    # taller than 64 rows take the scan's path without shared-memory row copies.
    kernels, shape, B = ("manhattan", "euclidean"), (512, 2048), 32
    desc = S.make_desc(shape[0], shape[1], bins=B, kernels=kernels, max_win=(31, 31))
    with S.Plan(desc) as plan:
        assert plan.info().band_rows <= 64
    lay = two_calls_against_plan(kernels, shape, B)
    assert lay.band_rows > 64


def two_calls_against_plan(kernels, shape, B):
    H, W = shape
    desc = S.make_desc(H, W, bins=B, kernels=kernels, max_win=(31, 31))
    stream = torch.cuda.Stream()
    # size query: no device work, tells how large the output must be
    q = S.swih_build_ih_noalloc(desc, None, None, 0)
    assert q.workspace_bytes == q.n_terms * B * H * q.ih_pitch * q.elem_bytes
    d_ih = torch.empty(q.workspace_bytes, dtype=torch.uint8, device=DEV)
    d_status = torch.zeros(1, dtype=torch.int32, device=DEV)
    for call, seed in enumerate((101, 202)):
        img = synth.blob_scene(H, W, 8, seed, n_blobs=3, axes=(8, 30), margin=32).image
        d_img = torch.from_numpy(img).to(DEV)
        # reference: the existing plan entry points
        with S.Plan(desc) as plan:
            plan.build_ih(d_img, stream)
            plan.sync_status(stream)
            info = plan.info()
            ref = planes(info.d_ih, info)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        d_ih.fill_(0xA5)  # stale bytes must all be overwritten
        torch.cuda.synchronize()
        lay = S.swih_build_ih_noalloc(desc, d_img, d_ih, d_ih.numel(), d_status, stream)
        stream.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        assert int(d_status.item()) == 0
        assert (lay.elem_bytes, lay.n_terms, lay.ih_pitch, lay.plane_elems) == \
            (info.elem_bytes, info.n_terms, info.ih_pitch, info.plane_elems)
        assert list(lay.term_p)[: lay.n_terms] == list(info.term_p)[: info.n_terms]
        got = planes(d_ih.data_ptr(), lay)
        assert np.array_equal(got, ref), f"call {call}: integral histograms differ"
        if call == 1:
            assert free_after == free_before
    return lay


def test_noalloc_rejects_oversized_scratch():
    # 8192 wide, 256 bins, Gaussian terms: one band of look-back state alone
    # is far above the static scratch
    desc = S.make_desc(4096, 8192, bins=256, kernels=("gaussian",), max_win=(31, 31))
    with pytest.raises(S.SwihError) as ei:
        S.swih_build_ih_noalloc(desc, None, None, 0)
    assert ei.value.status == S.SWIH_ERR_UNSUPPORTED
    assert "static scratch" in str(ei.value)
