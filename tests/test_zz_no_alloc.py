"""nq_count_host_noalloc: counting with no allocation, for callers that run
under a fixed device-memory budget (a serving process that reserved its memory
at start-up, or a program whose framework's allocator owns the GPU) and so
cannot let a library call cudaMalloc in mid-run.

The entry point keeps its device side in one static array inside libnq. This
test calls it through the C ABI with host arrays and checks its counts and
total against nq_count on the same prefixes -- exact equality, as every count
is an integer -- on two calls in a row (so the second call sees the first
one's leftovers in the shared array); checks every per-prefix count of the
N=16 depth-5 set against the CPU oracle's stored arrays; checks that the
device's free memory is the same before and after calls (nothing allocated);
and checks that a batch larger than the array is refused. The file is named
so that pytest collects it last.
"""
import ctypes
import json
import os

import numpy as np
import pytest

from paper_2511_12009_gb300 import nq

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
Q = {int(k): v for k, v in json.load(open(os.path.join(GOLDEN, "oeis_a000170.json")))["Q"].items()}
MAX_PREFIXES = 1 << 18


def noalloc(n, d, pre):
    fn = nq.lib().nq_count_host_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                   ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p]
    pre = np.ascontiguousarray(pre)
    counts = np.full(max(len(pre), 1), 0xDEADBEEF, dtype=np.uint64)
    total = ctypes.c_uint64(12345)
    rc = fn(n, d, pre.ctypes.data, len(pre), counts.ctypes.data, ctypes.byref(total), None)
    return rc, counts[:len(pre)], int(total.value)


def reference(n, d, pre):
    dp = nq.to_device(pre)
    cnt = torch.zeros(len(pre), dtype=torch.int64, device="cuda")
    nq.count(n, d, dp, cnt, stream=torch.cuda.current_stream())
    nq.sync(torch.cuda.current_stream())
    return cnt.cpu().numpy().view(np.uint64)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_two_calls_match_nq_count():
    for n, d in [(16, 5), (12, 3)]:   # the larger batch first: leftovers must not leak
        pre = nq.enumerate_prefixes(n, d)
        assert len(pre) <= MAX_PREFIXES
        rc, got, total = noalloc(n, d, pre)
        assert rc == nq.NQ_OK, nq.strerror(rc)
        want = reference(n, d, pre)
        assert np.array_equal(got, want)
        assert total == Q[n] == int(sum(int(m & 3) * int(c) for m, c in zip(pre["meta"], got)))


def test_same_call_twice_is_stable():
    pre = nq.enumerate_prefixes(14, 4)
    first = noalloc(14, 4, pre)
    second = noalloc(14, 4, pre)
    assert first[0] == second[0] == nq.NQ_OK
    assert np.array_equal(first[1], second[1]) and first[2] == second[2] == Q[14]


def test_batch_beyond_the_array_is_refused():
    pre = nq.enumerate_prefixes(18, 6)    # 1,199,146 records > 2^18
    assert len(pre) > MAX_PREFIXES
    rc, _, total = noalloc(18, 6, pre)
    assert rc == nq.NQ_EOVERFLOW and total == 12345


def test_counts_equal_the_oracle_arrays():
    """N=16, d=5: all 70,906 per-prefix counts against the oracle's stored arrays."""
    import numpy as np
    g = np.load(os.path.join(GOLDEN, "oracle_n16_d5.npz"))
    pre = nq.enumerate_prefixes(16, 5)
    rc, got, total = noalloc(16, 5, pre)
    assert rc == nq.NQ_OK, nq.strerror(rc)
    assert np.array_equal(got, g["counts"]) and total == Q[16]


def test_calls_allocate_no_device_memory():
    """After a first call (which commits the static array), further calls leave
    the device's free memory exactly where it was."""
    pre = nq.enumerate_prefixes(15, 4)
    assert noalloc(15, 4, pre[:0])[0] == nq.NQ_OK     # n = 0: set-up only
    assert noalloc(15, 4, pre)[0] == nq.NQ_OK         # the kernel's first launch
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        rc, _, total = noalloc(15, 4, pre)
        assert rc == nq.NQ_OK and total == Q[15]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
