"""The standalone pair sort (vgr_sort_pairs) against numpy's stable sort:
bit-exact keys and values, across tile edges (3840 keys per tile), key widths,
degenerate inputs (all equal, presorted, reversed) and arrays that do not
start on a 16-byte boundary."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2506_02774_gb300 as vgr  # noqa: E402
from paper_2506_02774_gb300 import _abi  # noqa: E402


def _sort_check(keys: np.ndarray, vals: np.ndarray, key_bits: int):
    k = torch.from_numpy(keys.view(np.int32)).cuda()
    v = torch.from_numpy(vals.view(np.int32)).cuda()
    ko, vo = vgr.sort_pairs(k, v, key_bits)
    torch.cuda.synchronize()
    mask = (1 << (8 * ((key_bits + 7) // 8))) - 1
    order = np.argsort(keys.astype(np.uint64) & mask, kind="stable")
    np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint32), keys[order])
    np.testing.assert_array_equal(vo.cpu().numpy().view(np.uint32), vals[order])
    # inputs untouched
    np.testing.assert_array_equal(k.cpu().numpy().view(np.uint32), keys)


@pytest.mark.parametrize("n", [1, 2, 100, 3839, 3840, 3841, 7681, 100_000, 1_000_003])
@pytest.mark.parametrize("key_bits", [8, 13, 32])
def test_random_keys(n, key_bits):
    rng = np.random.default_rng(n * 31 + key_bits)
    keys = rng.integers(0, 1 << key_bits, size=n, dtype=np.uint64).astype(np.uint32)
    vals = np.arange(n, dtype=np.uint32)
    _sort_check(keys, vals, key_bits)


def test_degenerate_inputs():
    n = 50_000
    vals = np.random.default_rng(1).integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    _sort_check(np.full(n, 7, np.uint32), vals, 16)           # all equal: stability only
    _sort_check(np.arange(n, dtype=np.uint32), vals, 24)       # presorted
    _sort_check(np.arange(n, dtype=np.uint32)[::-1].copy(), vals, 24)  # reversed
    few = np.random.default_rng(2).integers(0, 3, size=n).astype(np.uint32)
    _sort_check(few, np.arange(n, dtype=np.uint32), 2)         # heavy ties


@pytest.mark.parametrize("offset", [1, 2, 3])
def test_inputs_not_16_byte_aligned(offset):
    """Arrays that start 4, 8 or 12 bytes past a 16-byte boundary (views into
    a larger tensor) sort exactly like aligned ones."""
    n = 3 * 3840 + 17
    rng = np.random.default_rng(40 + offset)
    keys = rng.integers(0, 2**32, size=n + offset, dtype=np.uint64).astype(np.uint32)
    vals = np.arange(n + offset, dtype=np.uint32)
    k = torch.from_numpy(keys.view(np.int32)).cuda()[offset:]
    v = torch.from_numpy(vals.view(np.int32)).cuda()[offset:]
    assert k.data_ptr() % 16 != 0 and v.data_ptr() % 16 != 0
    ko, vo = vgr.sort_pairs(k, v, 32)
    torch.cuda.synchronize()
    order = np.argsort(keys[offset:], kind="stable")
    np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint32), keys[offset:][order])
    np.testing.assert_array_equal(vo.cpu().numpy().view(np.uint32), vals[offset:][order])


def test_large_and_wide():
    n = 5_000_000
    rng = np.random.default_rng(5)
    keys = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    _sort_check(keys, np.arange(n, dtype=np.uint32), 32)


def test_errors():
    lib = _abi.load()
    x = torch.zeros(8, dtype=torch.int32, device="cuda")
    assert lib.vgr_sort_pairs(x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), 8, 0, None) == _abi.VGR_E_INVALID
    assert lib.vgr_sort_pairs(x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), 8, 33, None) == _abi.VGR_E_INVALID
    assert lib.vgr_sort_pairs(None, None, None, None, 8, 8, None) == _abi.VGR_E_INVALID
    assert lib.vgr_sort_pairs(None, None, None, None, 0, 8, None) == _abi.VGR_OK  # n = 0: nothing to do
