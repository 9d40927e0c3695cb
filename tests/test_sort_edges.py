"""Edge cases of the single-sweep radix sort, through st_sort_keys_static (the pass kernels of
st_reorder without a handle): tile counts below, at and across the look-back window of four
tiles, ragged last tiles, one to four passes, and degenerate key distributions (all keys equal,
descending, few distinct values, long runs).  The expected result is the stable sort of the keys
on their low key_bits bits (numpy's stable argsort), compared element by element."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TILE = 4096  # keys per tile of a pass
SIZES = [1, 2, 31, 32, 33, TILE - 1, TILE, TILE + 1, 2 * TILE, 3 * TILE + 7, 4 * TILE, 4 * TILE + 1,
         5 * TILE + 4095, 9 * TILE + 1, 1 << 20]
SEEDS = {"uniform": 11, "equal": 12, "descending": 13, "few": 14, "runs": 15}


def _keys(dist, n, key_bits, rng):
    top = 1 << key_bits
    if dist == "uniform":
        return rng.integers(0, top, n, dtype=np.uint64).astype(np.uint32)
    if dist == "equal":
        return np.full(n, (top - 1) // 3, dtype=np.uint32)
    if dist == "descending":
        return ((top - 1) - (np.arange(n, dtype=np.uint64) * 7919) % top).astype(np.uint32)
    if dist == "few":
        vals = rng.integers(0, top, 3, dtype=np.uint64).astype(np.uint32)
        return vals[rng.integers(0, 3, n)]
    # runs of equal keys of random length, in random order of values
    out = np.empty(n, dtype=np.uint32)
    i = 0
    while i < n:
        m = int(rng.integers(1, 200))
        out[i:i + m] = rng.integers(0, top, dtype=np.uint64)
        i += m
    return out


def _static_sort(keys, key_bits):
    import torch

    from paper_2603_26691_gb300 import _lib

    lib = _lib.load()
    n = keys.size
    stream = torch.cuda.current_stream()
    kd = torch.as_tensor(keys.view(np.int32), device="cuda")
    sk = torch.empty(n, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    st = lib.st_sort_keys_static(C.c_void_p(kd.data_ptr()), n, key_bits, C.c_void_p(sk.data_ptr()),
                                 C.c_void_p(perm.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert st == _lib.ST_OK
    torch.cuda.synchronize()
    return sk.cpu().numpy().view(np.uint32), perm.cpu().numpy().view(np.uint32).astype(np.int64)


def _check(keys, key_bits):
    mask = np.uint64((1 << key_bits) - 1)
    want = np.argsort(keys.astype(np.uint64) & mask, kind="stable")
    sk, perm = _static_sort(keys, key_bits)
    assert np.array_equal(perm, want)
    assert np.array_equal(sk, keys[want])


@pytest.mark.parametrize("dist", list(SEEDS))
@pytest.mark.parametrize("n", SIZES)
def test_static_sort_sizes_and_distributions(n, dist):
    rng = np.random.default_rng(SEEDS[dist] * 1_000_003 + n)
    _check(_keys(dist, n, 24, rng), 24)


@pytest.mark.parametrize("key_bits", [1, 7, 8, 9, 16, 17, 24, 31, 32])
def test_static_sort_key_widths(key_bits):
    """One pass (up to 8 bits) to four passes (32 bits); bits above key_bits are ignored by the
    comparison but carried in the sorted keys."""
    rng = np.random.default_rng(100 + key_bits)
    n = 3 * TILE + 5
    keys = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    _check(keys, key_bits)
