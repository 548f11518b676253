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
  printf("%zu %zu %zu %zu %zu\n", sizeof(swih_plan_desc), offsetof(swih_plan_desc, gauss_sigma_frac),
         offsetof(swih_plan_desc, hbm_budget_bytes), sizeof(swih_plan_info),
         offsetof(swih_plan_info, workspace_bytes));
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
                    S.swih_plan_info.workspace_bytes.offset]


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
    (dict(gauss_degree=3, kernels=("gaussian",)), S.SWIH_ERR_UNSUPPORTED),
    (dict(precision=S.SWIH_PREC_RING32, kernels=("gaussian",)), S.SWIH_ERR_UNSUPPORTED),
    (dict(height=1024, width=1024, kernels=("gaussian",), max_win=(255, 255)), S.SWIH_ERR_UNSUPPORTED),
    (dict(hbm_budget_bytes=1000), S.SWIH_ERR_BUDGET),
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


def test_null_plan_calls_fail_cleanly():
    for fn, args in [(S.LIB.swih_build_ih, (None, None, None)),
                     (S.LIB.swih_likelihood, (None, 1, 3, 3, None, None, None)),
                     (S.LIB.swih_sync_status, (None, None))]:
        assert fn(*args) == S.SWIH_ERR_INVALID_ARG
    assert S.LIB.swih_destroy(None) == S.SWIH_OK


def test_build_module_paths():
    assert B.LIB.endswith("libswih.so") and os.path.exists(B.LIB)
