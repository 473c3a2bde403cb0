"""The allocation-free sort entry point (lodge_sort_pairs_noalloc) against the
allocating one (lodge_sort_pairs), through the C ABI.

lodge_sort_pairs_noalloc exists for callers that cannot allocate device memory
at the point of the call (an application that owns all device allocations, or
a loop that cannot pay for an allocation's implicit synchronisation); its
scratch is a fixed array in the library's device memory.  The results must be
identical to the allocating sort's, bit for bit, on two calls in a row (the
array keeps the previous call's contents), and sizes beyond its limit must be
refused before any device work.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAX_PAIRS = 1 << 20


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_23158_gb300 import build
    build.build()
    from paper_2505_23158_gb300 import _capi as A
    from paper_2505_23158_gb300.api import Lodge
    ctx = Lodge(0)
    yield torch, A, ctx
    ctx.close()


def _noalloc(A, torch, keys, vals, bits):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    A.call("lodge_sort_pairs_noalloc", C.c_void_p(keys.data_ptr()), C.c_void_p(vals.data_ptr()),
           int(keys.numel()), int(bits), stream)


def test_noalloc_sort_matches_allocating_sort_twice(env):
    torch, A, ctx = env
    for call, (n, bits) in enumerate([(MAX_PAIRS, 32), (777_777, 13)]):
        rng = np.random.default_rng(1000 + call)
        keys = rng.integers(0, 1 << bits, size=n, dtype=np.uint64).astype(np.uint32)
        keys[: n // 4] = keys[1]          # long runs of equal keys: stability matters
        rng.shuffle(keys)
        vals = rng.permutation(n).astype(np.uint32)
        k_ref = torch.from_numpy(keys.view(np.int32).copy()).cuda()
        v_ref = torch.from_numpy(vals.view(np.int32).copy()).cuda()
        ctx.sort_pairs(k_ref, v_ref, bits)
        k = torch.from_numpy(keys.view(np.int32).copy()).cuda()
        v = torch.from_numpy(vals.view(np.int32).copy()).cuda()
        _noalloc(A, torch, k, v, bits)
        torch.cuda.synchronize()
        assert torch.equal(k, k_ref), f"call {call}: keys differ"
        assert torch.equal(v, v_ref), f"call {call}: values differ"


def test_noalloc_sort_refuses_oversize(env):
    torch, A, ctx = env
    k = torch.zeros(MAX_PAIRS + 1, dtype=torch.int32, device="cuda")
    v = torch.zeros(MAX_PAIRS + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(A.LodgeError) as e:
        _noalloc(A, torch, k, v, 32)
    assert e.value.status == 1 and "limit" in str(e.value)
