"""The C ABI library loads and exports every declared symbol (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_2102_11084_gb300 as vgpkg
from paper_2102_11084_gb300 import build as vgbuild
from paper_2102_11084_gb300 import vg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    vgbuild.build()


def declared_symbols():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            names += re.findall(r"VG_API\s+[\w\s\*]+?\b(vg_\w+)\s*\(", txt)
    return names


def test_every_declared_symbol_is_exported():
    names = declared_symbols()
    assert "vg_downsample" in names
    h = ctypes.CDLL(vg.LIB_PATH)
    missing = [n for n in names if not hasattr(h, n)]
    assert not missing, missing


def test_binding_names_match_header():
    names = set(declared_symbols())
    assert set(vg._SIGS) <= names


def test_status_strings():
    assert vg.status_string(0) == "ok"
    for s in vg.Status:
        assert vg.status_string(int(s))
    assert vgpkg.version() >= 100


def test_workspace_query():
    assert vg.workspace_bytes(0) > 0
    a, b = vg.workspace_bytes(1000), vg.workspace_bytes(1_000_000)
    assert b > a > 0
    assert vg.lib().vg_downsample_workspace_bytes(-1, 0) == 0


def _call(n=0, leaf=0.1, flags=0, ws=None, wsb=0, origin=8):
    L = vg.lib()
    nv = 16
    return L.vg_downsample(None, n, origin, ctypes.c_float(leaf), None, None, None, 0, nv, None,
                           None, ws, wsb, flags, None)


def test_argument_errors_return_before_any_launch():
    assert _call(n=-1) == vg.Status.INVALID_ARG
    assert _call(leaf=0.0) == vg.Status.INVALID_ARG
    assert _call(leaf=float("nan")) == vg.Status.INVALID_ARG
    assert _call(leaf=float("inf")) == vg.Status.INVALID_ARG
    assert _call(flags=1 << 20) == vg.Status.INVALID_ARG
    assert _call(origin=None) == vg.Status.INVALID_ARG
    assert _call(n=vg.MAX_POINTS + 1) == vg.Status.INVALID_ARG
    assert _call(n=5) == vg.Status.INVALID_ARG          # xyz null with n > 0
    assert _call(origin=2) == vg.Status.ALIGN
    assert _call(ws=None, wsb=0) == vg.Status.WORKSPACE
    assert _call(ws=256, wsb=16) == vg.Status.WORKSPACE


def test_grouping_flags():
    # the grouping choices are flags of the sort method: accepted by the single-cloud call
    # and the pyramid (these calls stop at the missing workspace, before any launch), and
    # the binding's method names map onto the header's flags
    assert vg.method_flag("sort_bucket") == vg.METHOD_SORT | vg.SORT_BUCKETS
    assert vg.method_flag("sort_lsd") == vg.METHOD_SORT | vg.SORT_LSD
    assert vg.method_flag("sort") == vg.METHOD_SORT
    assert _call(flags=vg.METHOD_SORT | vg.SORT_BUCKETS) == vg.Status.WORKSPACE
    assert _call(flags=vg.METHOD_SORT | vg.SORT_LSD) == vg.Status.WORKSPACE
    assert _call(flags=vg.METHOD_SORT | 8) == vg.Status.INVALID_ARG
    assert _call(flags=vg.METHOD_SORT | vg.METHOD_HASH) == vg.Status.INVALID_ARG
    # the single-frame grouping: a flag of the sort method only, with its own workspace
    assert vg.method_flag("frame") == vg.METHOD_SORT | vg.SORT_FRAME
    assert _call(flags=vg.METHOD_SORT | vg.SORT_FRAME) == vg.Status.WORKSPACE
    assert _call(flags=vg.SORT_FRAME) == vg.Status.INVALID_ARG
    assert _call(flags=vg.METHOD_HASH | vg.SORT_FRAME) == vg.Status.INVALID_ARG
    assert vg.workspace_bytes(1000, vg.METHOD_SORT | vg.SORT_FRAME) > vg.workspace_bytes(1000)
    L = vg.lib()
    args = (None, 0, 8, ctypes.c_float(0.1), 2, None, None, None, 0, 16, None, None, None, 0)
    assert L.vg_pyramid(*args, vg.SORT_BUCKETS, None) == vg.Status.WORKSPACE
    assert L.vg_pyramid(*args, vg.SORT_LSD, None) == vg.Status.WORKSPACE
    assert L.vg_pyramid(*args, vg.METHOD_HASH, None) == vg.Status.INVALID_ARG
    assert L.vg_pyramid(*args, vg.SORT_FRAME, None) == vg.Status.INVALID_ARG


def test_no_cpu_fallback():
    import torch
    with pytest.raises(TypeError):
        vgpkg.downsample(torch.zeros((4, 3)), 0.1)


def test_frame_workspace_holds_the_one_launch_scratch():
    # the frame method's workspace holds the one-launch grouping's scratch (after the
    # call's state words: key bitmap and ranks of up to 2^26 keys and the 2^23-entry block
    # map, 48 MiB, then per point two 16-word slot bitmaps, three row sums, a slot and a
    # row key, 160 B) and the bin grouping's, growing with the frame
    frame = vg.METHOD_SORT | vg.SORT_FRAME
    for n in (1, 307_200, 2_073_600):
        assert vg.workspace_bytes(n, frame) >= (48 << 20) + 160 * n
        assert vg.workspace_bytes(n, frame) > vg.workspace_bytes(n)
    assert vg.workspace_bytes(921_600, frame) > vg.workspace_bytes(307_200, frame)


def test_one_launch_capacity_without_a_device():
    # the capacity query reads device attributes only; with no device it reports none
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert vg.frame_one_launch_points() == 0 and vg.frame_one_launch_points(posed=True) == 0
