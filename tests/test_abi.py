"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/ks.h declares; host-only queries work on the CPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ks():
    from paper_1905_13002_gb300 import _build
    _build.build()
    import paper_1905_13002_gb300 as ks
    return ks


def header_functions():
    with open(os.path.join(ROOT, "include", "ks.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ks_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("ks_build_elements", "ks_filter_scan", "ks_smooth_scan", "ks_smooth",
                     "ks_status", "ks_strerror", "ks_workspace_bytes"):
        assert required in names


def test_every_declared_symbol_is_exported(ks):
    so = ctypes.CDLL(ks.LIB_PATH)
    missing = [n for n in header_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_host_queries(ks):
    L = ks.lib()
    assert L.ks_version() >= 100
    assert L.ks_supported(4, 2) == 1
    assert L.ks_supported(5, 3) == 0
    for code in (0, -1, -2, -3, -4, -5, 7):
        assert L.ks_strerror(code)
    m = ks._KsModel(4, 2, 0, 0, 1, 0, 1, 1, 0, 1, 1, 1)   # pointers are only counted, not read
    n1 = L.ks_workspace_bytes(ctypes.byref(m), 1024, ks.KS_WS_SMOOTH)
    n2 = L.ks_workspace_bytes(ctypes.byref(m), 1024, ks.KS_WS_ELEMENTS)
    assert 0 < n1 < n2
    assert n2 >= 4 * (3 * 16 + 2 * 4) * 1024
    assert L.ks_workspace_bytes(ctypes.byref(m), 0, ks.KS_WS_SMOOTH) == 0
    bad = ks._KsModel(5, 3, 0, 0, 1, 0, 1, 1, 0, 1, 1, 1)
    assert L.ks_workspace_bytes(ctypes.byref(bad), 1024, ks.KS_WS_SMOOTH) == 0
    lay = ks._KsLayout()
    assert L.ks_elements_layout_get(ctypes.byref(m), 1000, ctypes.byref(lay)) == 0
    assert lay.ld >= 1000 and lay.ld % 64 == 0
    assert lay.offset_b - lay.offset_A == 16 * 4 * lay.ld
    assert lay.offset_J - lay.offset_eta == 4 * 4 * lay.ld


def test_argument_errors_need_no_device(ks):
    L = ks.lib()
    m = ks._KsModel(4, 2, 0, 0, 1, 0, 1, 1, 0, 1, 1, 1)
    # T out of range and null / misaligned pointers are rejected before any CUDA call
    assert L.ks_smooth(ctypes.byref(m), None, 10, None, 0, None, None, None, None, None) == ks.KS_EINVAL
    assert L.ks_smooth(ctypes.byref(m), 16, 0, 256, 1 << 20, None, None, 16, 16, None) == ks.KS_EINVAL
    # time-varying models: an unknown mode, a size without time-varying
    # support, and a misaligned y are all rejected before any launch
    tv2 = ks._KsModel(4, 2, 2, 0, 1, 0, 1, 1, 0, 1, 1, 1)
    assert L.ks_smooth(ctypes.byref(tv2), 16, 10, 256, 1 << 30, None, None, 16, 16, None) == ks.KS_EUNSUPPORTED
    tv32 = ks._KsModel(32, 8, 1, 0, 1, 0, 1, 1, 0, 1, 1, 1)
    assert L.ks_smooth(ctypes.byref(tv32), 16, 10, 256, 1 << 30, None, None, 16, 16, None) == ks.KS_EUNSUPPORTED
    assert L.ks_workspace_bytes(ctypes.byref(tv32), 10, ks.KS_WS_SMOOTH) == 0
    tv8 = ks._KsModel(8, 4, 1, 0, 1, 0, 1, 1, 0, 1, 1, 1)   # misaligned F: rejected before any launch
    assert L.ks_smooth(ctypes.byref(tv8), 16, 10, 256, 1 << 30, None, None, 16, 16, None) == ks.KS_EINVAL
    assert L.ks_workspace_bytes(ctypes.byref(tv8), 10, ks.KS_WS_SMOOTH) > 0
    tv = ks._KsModel(4, 2, 1, 0, 1, 0, 1, 1, 0, 1, 1, 1)
    assert L.ks_smooth(ctypes.byref(tv), 4, 10, 256, 1 << 30, None, None, 16, 16, None) == ks.KS_EINVAL
    assert L.ks_workspace_bytes(ctypes.byref(tv), 10, ks.KS_WS_SMOOTH) == \
        L.ks_workspace_bytes(ctypes.byref(tv), 10, ks.KS_WS_ELEMENTS) > 0
    other = ks._KsModel(5, 3, 0, 0, 1, 0, 1, 1, 0, 1, 1, 1)
    assert L.ks_smooth(ctypes.byref(other), 16, 10, 256, 1 << 30, None, None, 16, 16, None) == ks.KS_EUNSUPPORTED
    assert L.ks_filter_combine_batch(4, 10, None, None, None, 256, 256, None) == ks.KS_EINVAL
    assert L.ks_workspace_init(None, 256, None) == ks.KS_EINVAL


def test_product_path_has_no_oracle_dependency():
    """The package never imports, loads or runs anything from oracle/."""
    pkg = os.path.join(ROOT, "paper_1905_13002_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                with open(os.path.join(dirpath, f)) as fh:
                    text = fh.read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "kf_rts" not in text and "libks_oracle" not in text, f


def test_hmm_host_queries_and_argument_errors(ks):
    """The discrete-state entry points: supported sizes, workspace sizes, and
    argument errors returned before any device work."""
    L = ks.lib()
    for K in (2, 4, 8, 16, 32):
        assert L.ks_hmm_supported(K) == 1
        assert L.ks_hmm_workspace_bytes(K, 1000) > 0
    for K in (0, 3, 64):
        assert L.ks_hmm_supported(K) == 0
        assert L.ks_hmm_workspace_bytes(K, 1000) == 0
    assert L.ks_hmm_workspace_bytes(8, 0) == 0
    # bigger T, bigger workspace
    assert L.ks_hmm_workspace_bytes(32, 1 << 20) > L.ks_hmm_workspace_bytes(32, 1 << 10)
    h3 = ks._KsHmm(3, 0, 16, 16)
    assert L.ks_hmm_smooth(ctypes.byref(h3), 16, 10, 256, 1 << 20, 16, None, None, None) == ks.KS_EUNSUPPORTED
    h8 = ks._KsHmm(8, 0, 16, 16)
    assert L.ks_hmm_smooth(ctypes.byref(h8), None, 10, 256, 1 << 20, 16, None, None, None) == ks.KS_EINVAL
    assert L.ks_hmm_smooth(ctypes.byref(h8), 16, 0, 256, 1 << 20, 16, None, None, None) == ks.KS_EINVAL
    assert L.ks_hmm_smooth(ctypes.byref(h8), 16, 10, 256, 16, 16, None, None, None) == ks.KS_EINVAL   # workspace
    h32 = ks._KsHmm(32, 0, 16, 16)   # misaligned likelihood rows
    assert L.ks_hmm_smooth(ctypes.byref(h32), 4, 10, 256, 1 << 30, 16, None, None, None) == ks.KS_EINVAL
    hnull = ks._KsHmm(8, 0, 0, 16)
    assert L.ks_hmm_smooth(ctypes.byref(hnull), 16, 10, 256, 1 << 20, 16, None, None, None) == ks.KS_EINVAL


def test_mixed_batch_host_queries(ks):
    """ks_workspace_bytes_batched reads only the groups' sizes: one region per
    state size after the header, 0 for a malformed group list."""
    L = ks.lib()

    def groups(*sizes):
        arr = (ks._KsBatchGroup * len(sizes))()
        for i, (nx, ny, B, T) in enumerate(sizes):
            arr[i].models.nx, arr[i].models.ny, arr[i].models.B = nx, ny, B
            arr[i].total_T = T
        return arr

    one = L.ks_workspace_bytes_batched(1, groups((4, 2, 10, 5000)))
    three = L.ks_workspace_bytes_batched(3, groups((6, 3, 5, 3000), (4, 2, 10, 5000), (2, 1, 7, 900)))
    assert 0 < one < three
    assert one >= L.ks_workspace_bytes_batch(4, 2, 10, 5000)
    assert L.ks_workspace_bytes_batched(0, groups((4, 2, 10, 5000))) == 0
    assert L.ks_workspace_bytes_batched(2, groups((4, 2, 10, 5000), (4, 2, 3, 300))) == 0   # size twice
    assert L.ks_workspace_bytes_batched(1, groups((8, 4, 10, 5000))) == 0                  # not a register size
    assert L.ks_workspace_bytes_batched(1, groups((4, 2, 10, 5))) == 0                     # T < B
    # argument errors are returned before any CUDA call
    assert L.ks_smooth_batched(1, groups((4, 2, 10, 5000)), None, 0, None) == ks.KS_EINVAL
    assert L.ks_smooth_batched(1, groups((8, 4, 10, 5000)), None, 0, None) == ks.KS_EUNSUPPORTED
    assert L.ks_workspace_set_waits(None, 0, 0, 0, None) == ks.KS_EINVAL
    assert L.ks_refinements(None, None, None) == ks.KS_EINVAL
