"""zsort_pairs_noalloc: the entry point for callers that cannot allocate
device memory (graph capture, fixed memory pools, hosts that forbid device
allocation after start-up).  Its scratch is a static device array, so the
check here is that it sorts exactly like zsort_pairs on two calls in a row
(the array keeps the previous call's contents), reports its device status
into a caller-owned word, and rejects sizes beyond its fixed maximum.

This file is collected last on purpose: it must pass alone in a fresh
process and after every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2605_14419_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU machine
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2605_14419_gb300 as z  # noqa: E402
from paper_2605_14419_gb300 import build as zbuild  # noqa: E402

zbuild.build()
DEV = torch.device("cuda:0")


def _pairs(keys):
    k = torch.from_numpy(keys.view(np.int64)).to(DEV)
    v = torch.arange(keys.size, dtype=torch.int32, device=DEV)
    return k, v


def _noalloc(k, v, status):
    lib = z.load()
    st = torch.cuda.current_stream()
    rc = lib.zsort_pairs_noalloc(ctypes.c_void_p(k.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                 k.numel(), ctypes.c_void_p(status.data_ptr()),
                                 ctypes.c_void_p(st.cuda_stream))
    assert rc == z.OK, z.strerror(rc)
    torch.cuda.synchronize()
    return int(status.item())


def test_noalloc_matches_zsort_pairs_twice_in_a_row():
    status = torch.full((1,), 12345, dtype=torch.int32, device=DEV)
    cases = [inputs.lognormal(z.NOALLOC_MAX_N, 1), inputs.zipf(300_001, 2)]
    for keys in cases:  # two calls in a row on the shared static scratch
        k1, v1 = _pairs(keys)
        assert _noalloc(k1, v1, status) == z.OK
        k2, v2 = _pairs(keys)
        z.sort_pairs(k2, v2)  # the existing entry point
        assert torch.equal(k1, k2) and torch.equal(v1, v2)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = z.load()
    rc = lib.zsort_pairs_noalloc(None, None, z.NOALLOC_MAX_N + 1, None, None)
    assert rc == z.ERR_INVALID
