"""st_sort_keys_static: the stable key sort for callers that cannot allocate device memory.

Such callers (code inside another framework's memory pool or arena, processes that freeze their
allocations after start-up, allocator callbacks that must not re-enter the allocator) get the
ordering sort of st_reorder without a handle and without any allocation.  This file is collected
last so that a stop at its first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2603_26691_gb300 import inputs
from tests.helpers import chunk_keys_from_cells

pytestmark = pytest.mark.gpu


def _sorted_by_reorder(Sim, N, B, seed, n):
    """Keys of a particle set and the permutation that st_reorder (the existing entry point) applies."""
    pos, vel, d, _ = inputs.particles(seed, 0, n)
    sim = Sim(N, precision="mixed_f32", chunk_edge=B)
    sim.set_params(reorder_every=0)
    sim.add_particles(pos, d, vel)
    keys = chunk_keys_from_cells(sim.cells(), (N, N, N), B)
    sim.reorder()
    ids = sim.particles()[3].astype(np.int64)
    sim.close()
    return keys, ids


def test_static_sort_matches_reorder_on_two_calls_in_a_row():
    import torch

    from paper_2603_26691_gb300 import _lib
    from paper_2603_26691_gb300.sim import Sim

    lib = _lib.load()
    stream = torch.cuda.current_stream()
    cases = [(32, 8, 5, 300_001), (64, 4, 6, 1 << 20)]
    for N, B, seed, n in cases:
        keys, want_perm = _sorted_by_reorder(Sim, N, B, seed, n)
        key_bits = int(np.ceil(np.log2((N // B) ** 3 * B ** 3)))
        kd = torch.as_tensor(keys.view(np.int32), device="cuda")
        sk = torch.empty(n, dtype=torch.int32, device="cuda")
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        st = lib.st_sort_keys_static(C.c_void_p(kd.data_ptr()), n, key_bits, C.c_void_p(sk.data_ptr()),
                                     C.c_void_p(perm.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert st == _lib.ST_OK
        torch.cuda.synchronize()
        got = perm.cpu().numpy().astype(np.int64)
        assert np.array_equal(got, want_perm)
        assert np.array_equal(sk.cpu().numpy().view(np.uint32), keys[want_perm])
        # no wait of these calls gave up
        assert lib.st_sort_keys_static_status(C.c_void_p(stream.cuda_stream)) == _lib.ST_OK


def test_static_sort_takes_no_device_memory_after_its_first_call():
    """The first call on a device may create the static array (lazy module loading); later calls take
    no device memory at all: the free device memory stays the same across them."""
    import torch

    from paper_2603_26691_gb300 import _lib

    lib = _lib.load()
    stream = torch.cuda.current_stream()
    n = 200_003
    rng = np.random.default_rng(9)
    keys = torch.as_tensor(rng.integers(0, 1 << 20, n, dtype=np.uint32).view(np.int32), device="cuda")
    sk = torch.empty(n, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")

    def call():
        st = lib.st_sort_keys_static(C.c_void_p(keys.data_ptr()), n, 20, C.c_void_p(sk.data_ptr()),
                                     C.c_void_p(perm.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert st == _lib.ST_OK
        torch.cuda.synchronize()

    call()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        call()
        assert torch.cuda.mem_get_info()[0] == free0
    want = np.argsort(keys.cpu().numpy().view(np.uint32), kind="stable")
    assert np.array_equal(perm.cpu().numpy().astype(np.int64), want)
    assert lib.st_sort_keys_static_status(C.c_void_p(stream.cuda_stream)) == _lib.ST_OK


def test_static_sort_rejects_sizes_beyond_its_maximum():
    from paper_2603_26691_gb300 import _lib

    lib = _lib.load()
    st = lib.st_sort_keys_static(C.c_void_p(1), (1 << 20) + 1, 24, C.c_void_p(1), C.c_void_p(1), None)
    assert st == _lib.ST_ERR_INVALID_ARG
    assert lib.st_sort_keys_static(None, 10, 0, None, None, None) == _lib.ST_ERR_INVALID_ARG
