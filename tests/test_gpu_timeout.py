"""Bounded device-side waits: a look-back whose predecessor never publishes
gives up, the call returns LODGE_E_TIMEOUT, and the context stays usable.

The library's scans (projection, emission, the sort passes) chain per-tile
prefix sums by a decoupled look-back; each wait on a predecessor's status
word gives up after a poll limit, sets a bit in a status word and counts the
predecessor as 0, so a stalled predecessor cannot hang the GPU.
`lodge_debug_lookback` runs that look-back alone with one tile that never
publishes and a short limit; nothing here faults or hangs the device: every
wait ends after at most the given number of polls.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_23158_gb300 import build
    build.build()
    from paper_2505_23158_gb300 import _capi as A
    return torch, A


def _run(torch, A, n, missing, limit):
    out = np.zeros(n, np.uint32)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = A.lib().lodge_debug_lookback(n, missing, limit, out.ctypes.data_as(C.c_void_p), stream)
    return st, out


@pytest.mark.parametrize("n", [1, 33, 300, 1024])
def test_lookback_all_published(env, n):
    torch, A = env
    st, out = _run(torch, A, n, -1, 1 << 22)
    assert st == A.LODGE_OK
    i = np.arange(n, dtype=np.int64)
    assert np.array_equal(out.astype(np.int64), i * (i + 1) // 2)   # sum of 1..i


@pytest.mark.parametrize("n,missing", [(64, 10), (300, 0), (1024, 1000), (2, 0)])
def test_lookback_wait_gives_up(env, n, missing):
    torch, A = env
    st, out = _run(torch, A, n, missing, 1024)
    assert st == 5, A.lib().lodge_last_error()        # LODGE_E_TIMEOUT
    msg = A.lib().lodge_last_error().decode()
    assert "gave up" in msg
    i = np.arange(missing, dtype=np.int64)
    assert np.array_equal(out[:missing].astype(np.int64), i * (i + 1) // 2)
    # the context is still usable: a full run afterwards is exact
    st2, out2 = _run(torch, A, n, -1, 1 << 22)
    assert st2 == A.LODGE_OK
    j = np.arange(n, dtype=np.int64)
    assert np.array_equal(out2.astype(np.int64), j * (j + 1) // 2)
    x = torch.arange(1000, device="cuda", dtype=torch.float32)
    assert float(x.sum()) == 499500.0


def test_lookback_arguments_checked(env):
    torch, A = env
    for n, missing, limit in [(0, -1, 10), (1025, -1, 10), (10, 10, 10), (10, -1, 0), (10, -1, (1 << 22) + 1)]:
        st, _ = _run(torch, A, n, missing, limit)
        assert st == 1, (n, missing, limit)           # LODGE_E_INVALID
