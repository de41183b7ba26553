"""zsort_pairs_noalloc: the entry point for callers that cannot allocate
device memory (hosts that forbid device allocation once they have started,
processes confined to a fixed memory pool).  Its scratch is a static device
array, so the checks here are that it sorts exactly like the CPU oracle and
like zsort_pairs on two calls in a row (the array keeps the previous call's
contents), with and without payloads and at the sizes where the executor
takes its different routes, that it reports its device status into a
caller-owned word, that free device memory does not change across its calls,
and that it rejects sizes beyond its fixed maximum.

This file is collected last on purpose: it must pass alone in a fresh
process and after every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2605_14419_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU machine
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2605_14419_gb300 as z  # noqa: E402
from paper_2605_14419_gb300 import build as zbuild  # noqa: E402

zbuild.build()
DEV = torch.device("cuda:0")


def _dev(keys, with_vals=True):
    k = torch.from_numpy(keys.view(np.int64)).to(DEV)
    v = torch.arange(keys.size, dtype=torch.int32, device=DEV) if with_vals else None
    return k, v


def _noalloc(k, v, status):
    lib = z.load()
    st = torch.cuda.current_stream()
    rc = lib.zsort_pairs_noalloc(ctypes.c_void_p(k.data_ptr()), None if v is None else ctypes.c_void_p(v.data_ptr()),
                                 k.numel(), ctypes.c_void_p(status.data_ptr()),
                                 ctypes.c_void_p(st.cuda_stream))
    assert rc == z.OK, z.strerror(rc)
    torch.cuda.synchronize()
    return int(status.item())


def _host(t, dtype):
    return t.cpu().numpy().view(dtype)


def test_noalloc_matches_oracle_and_zsort_pairs_twice_in_a_row():
    status = torch.full((1,), 12345, dtype=torch.int32, device=DEV)
    cases = [inputs.lognormal(z.NOALLOC_MAX_N, 1), inputs.zipf(300_001, 2)]
    for keys in cases:  # two calls in a row on the shared static scratch
        k1, v1 = _dev(keys)
        assert _noalloc(k1, v1, status) == z.OK
        ok_k, ok_v = oracle.zsort_pairs(keys, inputs.index_payload(keys.size))
        assert np.array_equal(_host(k1, np.uint64), ok_k) and np.array_equal(_host(v1, np.uint32), ok_v)
        k2, v2 = _dev(keys)
        z.sort_pairs(k2, v2)  # the existing entry point
        assert torch.equal(k1, k2) and torch.equal(v1, v2)


@pytest.mark.parametrize("n", [0, 1, 2, 1000, 4096, 65_536, 65_537, 1_000_003])
def test_noalloc_keys_only_and_every_route(n):
    """n <= 1 (status only), a leaf, a single-CTA partition, the first
    multi-CTA size, and a large array; keys alone (vals = NULL) and pairs,
    each called twice in a row, against the oracle."""
    status = torch.full((1,), 777, dtype=torch.int32, device=DEV)
    keys = inputs.normal(n, 40 + n) if n else np.zeros(0, dtype=np.uint64)
    ok_k, ok_v = oracle.zsort_pairs(keys, inputs.index_payload(n))
    for with_vals in (False, True):
        for _ in range(2):
            k, v = _dev(keys, with_vals)
            if n == 0:
                k = torch.empty(1, dtype=torch.int64, device=DEV)[:0]
            assert _noalloc(k, v, status) == z.OK
            assert np.array_equal(_host(k, np.uint64), ok_k)
            if with_vals:
                assert np.array_equal(_host(v, np.uint32), ok_v)


def test_noalloc_allocates_no_device_memory():
    """After one warm-up call (module load and the one-time set-up), two
    more calls leave the device's free memory and torch's allocation count
    unchanged."""
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    keys = inputs.uniform(500_000, 9)
    k, v = _dev(keys)
    kw, vw = k.clone(), v.clone()
    assert _noalloc(kw, vw, status) == z.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(DEV)
    alloc0 = torch.cuda.memory_allocated(DEV)
    for _ in range(2):
        kk, vv = k.clone(), v.clone()
        free_before, _ = torch.cuda.mem_get_info(DEV)
        assert _noalloc(kk, vv, status) == z.OK
        assert torch.cuda.mem_get_info(DEV)[0] == free_before
        assert torch.equal(kk, kw) and torch.equal(vv, vw)
        del kk, vv
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated(DEV) == alloc0
    assert torch.cuda.mem_get_info(DEV)[0] == free0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = z.load()
    rc = lib.zsort_pairs_noalloc(None, None, z.NOALLOC_MAX_N + 1, None, None)
    assert rc == z.ERR_INVALID
