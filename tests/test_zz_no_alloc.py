"""vgr_sort_pairs_noalloc: the pair sort for callers that may not allocate
device memory (for instance a plug-in inside a host application that owns
all device memory, or a frame loop where cudaMalloc/cudaFree are banned
because they can synchronise the device).  Its output must equal the
allocating vgr_sort_pairs bit for bit -- the bar of every integer test here --
on two calls in a row through the C ABI, since calls share one static scratch
array that keeps the previous call's contents.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2506_02774_gb300 import _abi  # noqa: E402

MAX_N = 262144


def _run(fn, keys, vals, key_bits):
    lib = _abi.load()
    k = torch.from_numpy(keys.view(np.int32)).cuda()
    v = torch.from_numpy(vals.view(np.int32)).cuda()
    ko, vo = torch.empty_like(k), torch.empty_like(v)
    s = torch.cuda.current_stream().cuda_stream
    st = getattr(lib, fn)(k.data_ptr(), v.data_ptr(), ko.data_ptr(), vo.data_ptr(), len(keys), key_bits,
                          ctypes.c_void_p(s))
    _abi.check(st)
    torch.cuda.synchronize()
    return ko.cpu().numpy().view(np.uint32), vo.cpu().numpy().view(np.uint32)


def test_noalloc_matches_allocating_sort_twice():
    rng = np.random.default_rng(2024)
    cases = [(MAX_N, 13), (100_003, 32)]  # two calls in a row, different sizes and widths
    for n, bits in cases:
        keys = rng.integers(0, 1 << bits, size=n, dtype=np.uint64).astype(np.uint32)
        vals = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
        ref_k, ref_v = _run("vgr_sort_pairs", keys, vals, bits)
        got_k, got_v = _run("vgr_sort_pairs_noalloc", keys, vals, bits)
        np.testing.assert_array_equal(got_k, ref_k)
        np.testing.assert_array_equal(got_v, ref_v)
        order = np.argsort(keys, kind="stable")
        np.testing.assert_array_equal(got_v, vals[order])


def test_noalloc_allocates_nothing_single_pass_and_second_stream():
    """After a first call on the device, further calls leave the free device
    memory (cudaMemGetInfo) unchanged -- the property the entry point exists
    for -- including a single-pass sort (key_bits = 8: no ping-pong buffer)
    and a call on a second stream made after the first call returned; both
    results equal the allocating sort's."""
    lib = _abi.load()
    rng = np.random.default_rng(7)
    n = 50_001
    keys = rng.integers(0, 1 << 8, size=n, dtype=np.uint64).astype(np.uint32)
    vals = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    keys32 = (keys.astype(np.uint64) * 2654435761 + np.arange(n, dtype=np.uint64)) % (1 << 32)
    keys32 = keys32.astype(np.uint32)
    ref8_k, ref8_v = _run("vgr_sort_pairs", keys, vals, 8)
    ref32_k, ref32_v = _run("vgr_sort_pairs", keys32, vals, 32)
    # every tensor and stream exists before the measurement
    k8 = torch.from_numpy(keys.view(np.int32)).cuda()
    k32 = torch.from_numpy(keys32.view(np.int32)).cuda()
    v = torch.from_numpy(vals.view(np.int32)).cuda()
    ko, vo, ko2, vo2 = (torch.empty_like(v) for _ in range(4))
    s1, s2 = torch.cuda.current_stream(), torch.cuda.Stream()
    _abi.check(lib.vgr_sort_pairs_noalloc(k8.data_ptr(), v.data_ptr(), ko.data_ptr(), vo.data_ptr(), n, 16,
                                          ctypes.c_void_p(s1.cuda_stream)))  # warm-up call on this device
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        _abi.check(lib.vgr_sort_pairs_noalloc(k8.data_ptr(), v.data_ptr(), ko.data_ptr(), vo.data_ptr(), n, 8,
                                              ctypes.c_void_p(s1.cuda_stream)))
        _abi.check(lib.vgr_sort_pairs_noalloc(k32.data_ptr(), v.data_ptr(), ko2.data_ptr(), vo2.data_ptr(), n, 32,
                                              ctypes.c_void_p(s2.cuda_stream)))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint32), ref8_k)
    np.testing.assert_array_equal(vo.cpu().numpy().view(np.uint32), ref8_v)
    np.testing.assert_array_equal(ko2.cpu().numpy().view(np.uint32), ref32_k)
    np.testing.assert_array_equal(vo2.cpu().numpy().view(np.uint32), ref32_v)


def test_noalloc_rejects_oversize():
    lib = _abi.load()
    x = torch.zeros(8, dtype=torch.int32, device="cuda")
    st = lib.vgr_sort_pairs_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), MAX_N + 1, 16, None)
    assert st == _abi.VGR_E_INVALID
    assert b"limit" in lib.vgr_last_error()
