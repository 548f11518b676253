"""C ABI checks that need no GPU: the library loads, exports every function the
header declares, its structs match the ctypes mirrors, and host-side argument
validation answers with the documented status codes."""
import ctypes
import os
import subprocess
import tempfile

import pytest

from paper_1705_03524_gb300 import build as B
from paper_1705_03524_gb300 import swih as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_function():
    names = S.header_functions()
    assert "swih_plan" in names and "swih_likelihood" in names and len(names) >= 9
    out = subprocess.run(["nm", "-D", "--defined-only", S.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(S.LIB, n)


def test_struct_layout_matches_header():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "swih.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(swih_plan_desc), offsetof(swih_plan_desc, gauss_sigma_frac),
         offsetof(swih_plan_desc, hbm_budget_bytes), sizeof(swih_plan_info),
         offsetof(swih_plan_info, workspace_bytes), offsetof(swih_plan_desc, exp_lambda),
         offsetof(swih_plan_info, d_exp), offsetof(swih_plan_info, exp_frac_bits),
         offsetof(swih_plan_info, n_channels), sizeof(swih_channel_desc), offsetof(swih_channel_desc, bins));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True,
                                               check=True).stdout.split()]
    assert vals == [ctypes.sizeof(S.swih_plan_desc), S.swih_plan_desc.gauss_sigma_frac.offset,
                    S.swih_plan_desc.hbm_budget_bytes.offset, ctypes.sizeof(S.swih_plan_info),
                    S.swih_plan_info.workspace_bytes.offset, S.swih_plan_desc.exp_lambda.offset,
                    S.swih_plan_info.d_exp.offset, S.swih_plan_info.exp_frac_bits.offset,
                    S.swih_plan_info.n_channels.offset, ctypes.sizeof(S.swih_channel_desc),
                    S.swih_channel_desc.bins.offset]


def _desc(**kw):
    base = dict(bins=16, kernels=("manhattan",), max_win=(31, 31))
    base.update(kw)
    h = base.pop("height", 128)
    w = base.pop("width", 128)
    return S.make_desc(h, w, **base)


@pytest.mark.parametrize("kw,status", [
    (dict(width=2), S.SWIH_ERR_INVALID_ARG),
    (dict(width=9000, max_win=(31, 31)), S.SWIH_ERR_UNSUPPORTED),
    (dict(bins=0), S.SWIH_ERR_INVALID_ARG),
    (dict(bins=257), S.SWIH_ERR_INVALID_ARG),
    (dict(max_win=(30, 31)), S.SWIH_ERR_INVALID_ARG),
    (dict(max_win=(1, 1)), S.SWIH_ERR_INVALID_ARG),
    (dict(max_win=(129, 31)), S.SWIH_ERR_INVALID_ARG),
    (dict(kernels=()), S.SWIH_ERR_INVALID_ARG),
    (dict(pitch_bytes=100), S.SWIH_ERR_INVALID_ARG),
    (dict(bitdepth=9), S.SWIH_ERR_INVALID_ARG),
    (dict(gauss_degree=5, kernels=("gaussian",)), S.SWIH_ERR_UNSUPPORTED),
    (dict(precision=S.SWIH_PREC_RING32, kernels=("gaussian",)), S.SWIH_ERR_UNSUPPORTED),
    (dict(height=1024, width=1024, kernels=("gaussian",), max_win=(255, 255), precision=S.SWIH_PREC_RING64),
     S.SWIH_ERR_UNSUPPORTED),
    (dict(height=1024, width=1024, kernels=("gaussian",), max_win=(301, 301), gauss_degree=4),
     S.SWIH_ERR_UNSUPPORTED),
    (dict(hbm_budget_bytes=1000), S.SWIH_ERR_BUDGET),
    (dict(kernels=("exponential",), exp_lambda=20.0), S.SWIH_ERR_INVALID_ARG),
    (dict(kernels=("exponential",), exp_lambda=1e-4), S.SWIH_ERR_INVALID_ARG),
    (dict(kernels=("exponential",), exp_lambda=-0.5), S.SWIH_ERR_INVALID_ARG),
])
def test_plan_validation(kw, status):
    with pytest.raises(S.SwihError) as ei:
        d = _desc(**kw)
        if kw.get("hbm_budget_bytes"):
            S.swih_plan(d)  # budget is checked before any CUDA call
        else:
            S.swih_plan_workspace_bytes(d)
    assert ei.value.status == status
    assert S.swih_last_error()


def test_workspace_bytes_layout():
    # 128 x 128, B = 16, Manhattan: terms {1, x, y}, 32-bit ring
    n = S.swih_plan_workspace_bytes(_desc())
    ih = 3 * 16 * 128 * 128 * 4
    assert ih < n < ih + 2 * 1024 * 1024
    # adding the Gaussian switches the ring to 64 bits and the term set to 25
    n2 = S.swih_plan_workspace_bytes(_desc(kernels=("manhattan", "gaussian")))
    assert n2 >= 25 * 16 * 128 * 128 * 8
    # width not a multiple of 32: rows are padded to 32 elements
    n3 = S.swih_plan_workspace_bytes(_desc(width=100, max_win=(31, 31)))
    assert n3 >= 3 * 16 * 128 * 128 * 4


def test_exponential_workspace_layout():
    # four directional 8-byte planes per bin, plus band carries for two y sides;
    # the count gate keeps a plain 32-bit integral histogram (term x^0 y^0)
    n = S.swih_plan_workspace_bytes(_desc(kernels=("exponential",)))
    planes = 4 * 16 * 128 * 128 * 8
    count = 16 * 128 * 128 * 4
    assert planes + count < n < planes + count + 4 * 1024 * 1024
    # the exponential kernel alone adds nothing to the integer term set
    both = S.swih_plan_workspace_bytes(_desc(kernels=("manhattan", "exponential")))
    man = S.swih_plan_workspace_bytes(_desc())
    assert both - man >= planes


def test_scales_call_validates_on_the_host():
    assert S.LIB.swih_likelihood_scales(None, 1, 1, None, None, None, None, None) == S.SWIH_ERR_INVALID_ARG


def test_noalloc_build_refuses_the_exponential_kernel():
    # refused on the host, before any device memory is touched
    d = _desc(kernels=("exponential",))
    assert S.LIB.swih_build_ih_noalloc(ctypes.byref(d), None, None, 0, None, None, None) == S.SWIH_ERR_UNSUPPORTED
    assert "exponential" in S.swih_last_error()


def test_exponential_has_no_tiled_gather_config():
    # host-only: the configuration call is refused before anything touches a plan's memory
    assert S.LIB.swih_set_gather_config(None, S.SWIH_KERNEL_EXPONENTIAL, 0, 0, 0) == S.SWIH_ERR_INVALID_ARG


def test_null_plan_calls_fail_cleanly():
    for fn, args in [(S.LIB.swih_build_ih, (None, None, None)),
                     (S.LIB.swih_likelihood, (None, 1, 3, 3, None, None, None)),
                     (S.LIB.swih_sync_status, (None, None))]:
        assert fn(*args) == S.SWIH_ERR_INVALID_ARG
    assert S.LIB.swih_destroy(None) == S.SWIH_OK


def test_build_module_paths():
    assert B.LIB.endswith("libswih.so") and os.path.exists(B.LIB)


# --------------------------------------------------------------------------- batches
def test_batch_struct_layout_matches_header():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "swih.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(swih_batch_desc), offsetof(swih_batch_desc, gauss_sigma_frac),
         offsetof(swih_batch_desc, hbm_budget_bytes), sizeof(swih_roi_desc), offsetof(swih_roi_desc, win_h),
         offsetof(swih_roi_desc, d_target), offsetof(swih_roi_desc, d_map));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True,
                                               check=True).stdout.split()]
    assert vals == [ctypes.sizeof(S.swih_batch_desc), S.swih_batch_desc.gauss_sigma_frac.offset,
                    S.swih_batch_desc.hbm_budget_bytes.offset, ctypes.sizeof(S.swih_roi_desc),
                    S.swih_roi_desc.win_h.offset, S.swih_roi_desc.d_target.offset,
                    S.swih_roi_desc.d_map.offset]


FAKE = 1 << 20  # a non-NULL device address that host-side validation never touches


def _roi(x0=0, y0=0, w=64, h=48, kernel="manhattan", windows=((9, 9),), target=FAKE, maps=None):
    maps = maps if maps is not None else [FAKE] * len(windows)
    return S.make_roi(x0, y0, w, h, kernel, list(windows), target, maps)


def _bdesc(**kw):
    base = dict(bins=16, kernels=("manhattan", "euclidean"))
    base.update(kw)
    return S.make_batch_desc(base.pop("height", 200), base.pop("width", 300), **base)


@pytest.mark.parametrize("rois,kw,status", [
    ([_roi(x0=250)], {}, S.SWIH_ERR_INVALID_ARG),               # leaves the frame on the right
    ([_roi(y0=-1)], {}, S.SWIH_ERR_INVALID_ARG),
    ([_roi(w=2)], {}, S.SWIH_ERR_INVALID_ARG),
    ([_roi(kernel="gaussian")], {}, S.SWIH_ERR_INVALID_ARG),    # not in kernel_mask
    ([_roi(windows=((8, 9),))], {}, S.SWIH_ERR_INVALID_ARG),    # even side
    ([_roi(windows=((65, 9),))], {}, S.SWIH_ERR_INVALID_ARG),   # wider than the ROI
    ([_roi(target=0)], {}, S.SWIH_ERR_INVALID_ARG),
    ([_roi(maps=[0])], {}, S.SWIH_ERR_INVALID_ARG),
    ([_roi()], dict(bins=0), S.SWIH_ERR_INVALID_ARG),
    ([_roi()], dict(bitdepth=9), S.SWIH_ERR_INVALID_ARG),
    ([_roi()], dict(pitch_bytes=299), S.SWIH_ERR_INVALID_ARG),
    ([_roi(w=300, h=200, kernel="gaussian", windows=((255, 199),))], dict(kernels=("gaussian",)),
     S.SWIH_ERR_UNSUPPORTED),                                   # Gaussian moments beyond 2^64
    ([_roi(), "nine_scales"], {}, S.SWIH_ERR_INVALID_ARG),
])
def test_batch_validation(rois, kw, status):
    if "nine_scales" in rois:  # n_windows above SWIH_MAX_SCALES, built without make_roi's check
        r = _roi(x0=10)
        r.n_windows = S.SWIH_MAX_SCALES + 1
        rois = [rois[0], r]
    with pytest.raises(S.SwihError) as ei:
        S.swih_batch_workspace_bytes(_bdesc(**kw), rois)
    assert ei.value.status == status
    assert S.swih_last_error()


def test_batch_budget_and_null_arguments():
    rois = [_roi(), _roi(x0=100, y0=20, w=120, h=90, windows=((9, 9), (21, 15)))]
    need = S.swih_batch_workspace_bytes(_bdesc(), rois)
    with pytest.raises(S.SwihError) as ei:
        S.swih_batch_plan(_bdesc(hbm_budget_bytes=need - 1), rois, FAKE)  # before any CUDA call
    assert ei.value.status == S.SWIH_ERR_BUDGET
    with pytest.raises(S.SwihError) as ei:
        S.swih_batch_plan(_bdesc(), rois, 0)
    assert ei.value.status == S.SWIH_ERR_INVALID_ARG
    with pytest.raises(S.SwihError) as ei:
        S.swih_batch_plan(_bdesc(pixel_type=S.SWIH_PIXEL_U16, pitch_bytes=600), rois, FAKE + 1)
    assert ei.value.status == S.SWIH_ERR_INVALID_ARG  # odd address for 16-bit pixels
    for fn in (S.LIB.swih_batch_run, S.LIB.swih_batch_autotune, S.LIB.swih_batch_sync_status):
        assert fn(None, None) == S.SWIH_ERR_INVALID_ARG
    assert S.LIB.swih_batch_destroy(None) == S.SWIH_OK


def test_batch_workspace_grows_with_rois_and_terms():
    one = [_roi()]
    two = [_roi(), _roi(x0=100, y0=20, w=120, h=90)]
    n1 = S.swih_batch_workspace_bytes(_bdesc(), one)
    n2 = S.swih_batch_workspace_bytes(_bdesc(), two)
    # Manhattan + Euclidean: five terms, 32-bit ring; the second ROI adds its planes
    assert n2 - n1 >= 5 * 16 * 90 * 128 * 4
    # the Gaussian in the mask switches every ROI to 25 terms in the 64-bit ring
    g = S.swih_batch_workspace_bytes(_bdesc(kernels=("manhattan", "gaussian")), two)
    assert g >= 25 * 16 * (48 * 64 + 90 * 128) * 8


def test_channel_plan_refusals_on_the_host():
    # refused while the plan is laid out, before any device call
    desc = S.make_desc(64, 64, bins=1, kernels=("exponential",), max_win=(9, 9))
    with pytest.raises(S.SwihError) as ei:
        S.ChannelPlan(desc, [S.make_channel(64, bins=8)])
    assert ei.value.status == S.SWIH_ERR_UNSUPPORTED
    desc = S.make_desc(64, 64, bins=1, kernels=("manhattan",), max_win=(9, 9))
    for chans in ([S.make_channel(64, bins=200), S.make_channel(64, bins=57)],   # 257 bins
                  [S.make_channel(64, bins=8, bitdepth=9)],                      # u8 with 9 bits
                  [S.make_channel(64, bins=8, pitch_bytes=63)],                  # pitch below a row
                  [S.make_channel(64, bins=0)],
                  [S.make_channel(64, bins=4)] * 9):                             # more than 8 channels
        with pytest.raises(S.SwihError) as ei:
            S.ChannelPlan(desc, chans)
        assert ei.value.status == S.SWIH_ERR_INVALID_ARG


def test_gaussian_ring_choice_and_refusals():
    # the ring follows the largest Bernstein moment w h rx^2D ry^2D
    def ws(**kw):
        return S.swih_plan_workspace_bytes(_desc(kernels=("gaussian",), **kw))
    small = ws(width=1024, height=1024, max_win=(81, 81))                       # D = 2: 64-bit ring
    big = ws(width=1024, height=1024, max_win=(401, 401))                      # D = 2: 128-bit ring
    assert big > 1.9 * small
    ws(width=1024, height=1024, max_win=(401, 401), gauss_degree=3)            # 49 terms, 128-bit
    for kw, status in ((dict(max_win=(301, 301), gauss_degree=4, width=1024, height=1024), S.SWIH_ERR_UNSUPPORTED),
                       (dict(max_win=(401, 401), width=5000, height=600), S.SWIH_ERR_UNSUPPORTED),
                       (dict(gauss_degree=5), S.SWIH_ERR_UNSUPPORTED),
                       (dict(max_win=(201, 201), width=1024, height=1024, precision=S.SWIH_PREC_RING64),
                        S.SWIH_ERR_UNSUPPORTED)):
        with pytest.raises(S.SwihError) as ei:
            ws(**kw)
        assert ei.value.status == status, kw
    # the 128-bit ring serves plans of the Gaussian kernel alone
    with pytest.raises(S.SwihError) as ei:
        S.swih_plan_workspace_bytes(_desc(width=1024, height=1024, kernels=("gaussian", "manhattan"),
                                          max_win=(401, 401)))
    assert ei.value.status == S.SWIH_ERR_UNSUPPORTED
    # batches stay within degree 2 and the 64-bit ring
    with pytest.raises(S.SwihError) as ei:
        desc = S.make_batch_desc(1024, 1024, bins=16, kernels=("gaussian",), gauss_degree=3)
        roi = S.make_roi(0, 0, 300, 300, "gaussian", [(41, 41)], 256, [256])
        S.swih_batch_workspace_bytes(desc, [roi])
    assert ei.value.status == S.SWIH_ERR_UNSUPPORTED
