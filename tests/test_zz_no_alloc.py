"""The allocation-free aggregation entry point (for callers that must not allocate
while they run) must give exactly the result of the allocating one.

Runs through the C ABI. Two calls in a row check that the shared fixed scratch
array carries nothing from one call into the next. The caller (this test) owns
and allocates the input and output buffers; the entry point itself allocates
nothing. Integer results: compared exactly, the tolerance every parity test uses.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _call(fn, vals, cnts, primes):
    np_ = len(primes)
    ov = torch.empty(1, dtype=torch.int32, device="cuda")
    oc = torch.zeros(max(np_, 1), dtype=torch.int64, device="cuda")
    pr = (C.c_uint64 * max(np_, 1))(*primes)
    stream = torch.cuda.current_stream().cuda_stream
    rc = fn(vals.numel(), vals.data_ptr(), cnts.data_ptr(), np_, pr, ov.data_ptr(), oc.data_ptr(), stream)
    torch.cuda.synchronize()
    return rc, int(ov.cpu()[0]), oc.cpu().numpy().view(np.uint64)[:np_].tolist()


def test_noalloc_matches_aggregate_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_05470_gb300 as P
    lib = P._lib.load()
    assert lib.bbtn_aggregate_noalloc_max_scratch() == 64 * 1024
    primes = P.primes(3)
    for call, (n, seed, lo) in enumerate(((70000, 1, -3), (1000, 2, -1))):
        rng = np.random.default_rng(seed)
        v = rng.integers(lo, 1, size=n).astype(np.int32)
        c = rng.integers(0, 2**61 - 1024, size=(3, n), dtype=np.uint64)
        dv = torch.from_numpy(v).cuda()
        dc = torch.from_numpy(c.view(np.int64).copy()).cuda()
        rc0, v0, c0 = _call(lib.bbtn_aggregate, dv, dc, primes)
        rc1, v1, c1 = _call(lib.bbtn_aggregate_noalloc, dv, dc, primes)
        assert rc0 == 0 and rc1 == 0, lib.bbtn_last_error()
        assert (v1, c1) == (v0, c0), f"call {call}"
