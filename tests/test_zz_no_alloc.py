"""The allocation-free sort entry point, for callers that cannot allocate device memory (an
application that owns the whole device heap, or a frame loop that must not call cudaMalloc).

Called through the C ABI twice in a row on different inputs; each result must equal the
regular entry point's (integer sort: exact).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth
from gpu_helpers import cuda, lib_ready, to_np_u32

pytestmark = pytest.mark.gpu


def _regular(abi, torch, keys, vals, n, lo, hi):
    kt, vt = cuda(keys.view(np.int32)), cuda(vals.view(np.int32))
    scr = torch.empty(abi.radix_sort_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    abi.radix_sort_pairs(kt, vt, None, n, lo, hi, scr)
    return kt, vt


def test_noalloc_sort_matches_regular_sort_twice():
    import torch
    abi = lib_ready()
    L = abi.lib()
    assert abi.radix_sort_pairs_noalloc_max_items() == 1 << 20
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed, n, lo, hi in ((11, 300_001, 0, 32), (12, 1 << 20, 0, 13)):
        keys, vals = synth.random_sort_keys(seed, n, bits=32, dup_frac=0.3)
        k_ref, v_ref = _regular(abi, torch, keys, vals, n, lo, hi)
        kt, vt = cuda(keys.view(np.int32)), cuda(vals.view(np.int32))
        st = L.ogs_radix_sort_pairs_noalloc(ctypes.c_void_p(kt.data_ptr()),
                                            ctypes.c_void_p(vt.data_ptr()), None, n, lo, hi,
                                            stream)
        assert st == 0
        torch.cuda.synchronize()
        assert np.array_equal(to_np_u32(kt), to_np_u32(k_ref))
        assert np.array_equal(to_np_u32(vt), to_np_u32(v_ref))


def test_noalloc_sort_device_count_matches_regular_sort():
    """A device-side item count below n_cap (how the renderer passes its counts): both entry
    points sort the first 123457 of 300001 entries the same way and leave the rest as it was."""
    import torch
    abi = lib_ready()
    L = abi.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n_cap, n = 300_001, 123_457
    keys, vals = synth.random_sort_keys(13, n_cap, bits=32, dup_frac=0.3)
    n_dev = cuda(np.array([n], np.int32))
    kr, vr = cuda(keys.view(np.int32)), cuda(vals.view(np.int32))
    scr = torch.empty(abi.radix_sort_scratch_bytes(n_cap), dtype=torch.uint8, device="cuda")
    abi.radix_sort_pairs(kr, vr, n_dev, n_cap, 0, 32, scr)
    for _ in range(2):
        kt, vt = cuda(keys.view(np.int32)), cuda(vals.view(np.int32))
        st = L.ogs_radix_sort_pairs_noalloc(ctypes.c_void_p(kt.data_ptr()),
                                            ctypes.c_void_p(vt.data_ptr()),
                                            ctypes.c_void_p(n_dev.data_ptr()), n_cap, 0, 32,
                                            stream)
        assert st == 0
        torch.cuda.synchronize()
        assert np.array_equal(to_np_u32(kt), to_np_u32(kr))
        assert np.array_equal(to_np_u32(vt), to_np_u32(vr))
        assert np.array_equal(to_np_u32(vt)[n:], vals[n:])
        assert np.array_equal(to_np_u32(kt)[n:], keys[n:])


def test_noalloc_sort_rejects_oversized_requests():
    import torch
    abi = lib_ready()
    kt = torch.zeros(16, dtype=torch.int32, device="cuda")
    st = abi.lib().ogs_radix_sort_pairs_noalloc(ctypes.c_void_p(kt.data_ptr()),
                                                ctypes.c_void_p(kt.data_ptr()), None,
                                                (1 << 20) + 1, 0, 32, None)
    assert st == 2   # OGS_ERR_CAPACITY, nothing enqueued
