"""Host-side checks of the C-ABI library that need no GPU: it builds for sm_103a, loads, and
exports every entry point that include/ogs.h declares (no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ogs_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2403_17898_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    d = _declared()
    for n in ("ogs_lod_select", "ogs_decode", "ogs_project_bin", "ogs_sort", "ogs_blend_fwd",
              "ogs_radix_sort_pairs"):
        assert n in d


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2403_17898_gb300 import abi
    assert set(_declared()) <= set(abi.exported_symbols())


def test_host_argument_checks_without_gpu(lib):
    """Invalid arguments are rejected on the host before anything is enqueued."""
    lib.ogs_lod_select_scratch_bytes.restype = ctypes.c_size_t
    lib.ogs_lod_select_scratch_bytes.argtypes = [ctypes.c_int64]
    assert lib.ogs_lod_select_scratch_bytes(4096) >= 4
    from paper_2403_17898_gb300 import abi
    L = abi.lib()
    cam = abi.Camera()
    cam.width, cam.height, cam.d_max, cam.s = 64, 64, 10.0, 1.0
    # null anchor pointers -> OGS_ERR_ARG (1), no CUDA call made
    st = L.ogs_lod_select(None, None, None, 10, 3, 10, ctypes.byref(cam), 1, None, None, 10,
                          None, None, 0, None)
    assert st == 1
    st = L.ogs_radix_sort_pairs(None, None, None, 10, 0, 32, None, 0, None)
    assert st == 1
    assert abi.version().startswith("ogs-gb300")


def test_product_path_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2403_17898_gb300 import abi
    monkeypatch.setattr(abi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(abi, "_lib", None)
    with pytest.raises(abi.OgsError):
        abi.lib()


def test_appearance_fields_checked_on_host(lib):
    """Appearance codes (Sec. 4.4): a code wider than 8 values, or codes without their arrays
    (in the decoder or, for the backward, in the gradient struct), are rejected.  The fake
    device pointers are never dereferenced: every check fails on the host first."""
    from paper_2403_17898_gb300 import abi
    L = abi.lib()
    assert ctypes.sizeof(abi.MLP) == 96 and abi.MLP.app.offset == 88
    cam = abi.Camera()
    cam.width, cam.height, cam.d_max, cam.s = 64, 64, 10.0, 1.0
    fake = 4096
    m = abi.MLP()
    for n in ("w1", "b1", "w2_op", "b2_op", "w2_col", "b2_col", "w2_cov", "b2_cov"):
        setattr(m, n, fake)
    m.F, m.H, m.k = 32, 32, 10
    g = abi.Gaussians(*([fake] * 5))

    def decode(mm):
        return L.ogs_decode(fake, fake, fake, fake, 100, ctypes.byref(mm), ctypes.byref(cam),
                            fake, fake, 0, fake, ctypes.byref(g), None)
    assert decode(m) == 0                  # valid, sel_cap = 0: nothing enqueued
    m.A = 9
    assert decode(m) == 1
    m.A = 4
    assert decode(m) == 1                  # no code arrays
    m.w1_app, m.app = fake, fake
    assert decode(m) == 0
    dm = abi.MLP()
    ctypes.memmove(ctypes.byref(dm), ctypes.byref(m), ctypes.sizeof(abi.MLP))
    dm.w1_app, dm.app = None, None          # codes in the decoder, no code gradients given
    for fn in (L.ogs_decode_bwd, L.ogs_decode_bwd_bf16):
        st = fn(fake, fake, fake, fake, 100, ctypes.byref(m), ctypes.byref(cam), fake, fake, 0,
                fake, fake, fake, fake, fake, fake, fake, fake, ctypes.byref(dm), fake, 1 << 30,
                None)
        assert st == 1


def test_counts_status_mapping(lib):
    """ogs_counts_status is host code: a read-back counter record -> a status, non-finite
    first, then expired waits, then capacity."""
    import numpy as np
    from paper_2403_17898_gb300 import abi
    c = np.zeros(8, np.uint32)
    assert abi.counts_status(c) == 0
    c[3] = 2                                    # pair capacity overflowed
    assert abi.counts_status(c) == 2
    c[6] = 1                                    # and a bounded wait expired
    assert abi.counts_status(c) == 3
    assert abi.counts_status(c, nonfinite=1) == 5
    assert abi.counts_status(np.zeros(8, np.uint32), nonfinite=4) == 5


def test_sort_bins_scratch_and_host_checks(lib):
    """ogs_sort_bins' scratch holds the tile counts behind an 8-byte chunk counter, the per
    chunk lists of long tiles and 32 deferred (Gaussian, chunk) entries of 8 bytes per tile
    (at least 4096); a scratch one byte short, a zero tile_cap or a grid of more than 65536
    tiles is refused on the host (OGS_ERR_ARG) before anything is enqueued."""
    from paper_2403_17898_gb300 import abi
    L = abi.lib()
    prev = 0
    for nt in (1, 16, 128, 2209, 8160, 65536):
        b = abi.sort_bins_scratch_bytes(nt)
        chunks = -(-nt // 1024)
        assert b >= 8 * max(4096, 32 * nt) + 4 * (nt + 2) + 4 * chunks * (1024 + 1)
        assert b >= prev
        prev = b
    fake = ctypes.c_void_p(1 << 20)                 # never dereferenced: refused first
    bins = abi.TileBins(fake, fake, 4096)
    need = abi.sort_bins_scratch_bytes(120 * 68)
    args = lambda gx, gy, sb, tb: (fake, fake, fake, 1000, -1, gx, gy, ctypes.byref(tb), fake,
                                   fake, fake, sb, None)
    assert L.ogs_sort_bins(*args(120, 68, need - 1, bins)) == 1
    assert L.ogs_sort_bins(*args(257, 256, 1 << 40, bins)) == 1
    assert L.ogs_sort_bins(*args(120, 68, need, abi.TileBins(fake, fake, 0))) == 1
