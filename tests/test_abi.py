"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/zsort.h declares (no compute calls)."""
import ctypes
import subprocess

import pytest

import paper_2605_14419_gb300 as z
from paper_2605_14419_gb300 import build as zbuild


@pytest.fixture(scope="module")
def lib():
    zbuild.build()
    return z.load()


def test_header_declares_the_boundary():
    names = z.header_functions()
    for required in ("zsort_pairs", "zsort_segmented", "zsort_pairs_i64", "zsort_pairs_f64",
                     "zsort_pairs_ex", "zsort_sync_status", "zsort_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", z.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in z.header_functions() if n not in exported]
    assert not missing, missing
    for n in z.header_functions():
        assert getattr(lib, n) is not None


def test_struct_sizes_match_header(lib):
    # zsort_default_opts writes struct_size = sizeof(zsort_opts) as compiled
    o = z.Opts()
    lib.zsort_default_opts(ctypes.byref(o))
    assert o.struct_size == ctypes.sizeof(z.Opts)
    assert o.kmax == 512 and o.mapper == z.MAP_ZSCORE and o.fallback_ratio == 4.0


def test_strerror_texts(lib):
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert lib.zsort_strerror(code)
    assert z.strerror(-5).startswith("segment offsets")


def test_host_side_argument_checks_need_no_gpu(lib):
    # rejected before any CUDA call
    assert lib.zsort_pairs_ex(None, 0, None, z.MAX_N + 1, None, None) == z.ERR_INVALID
    assert lib.zsort_pairs_ex(None, 7, None, 10, None, None) == z.ERR_INVALID
    bad = z.Opts()
    lib.zsort_default_opts(ctypes.byref(bad))
    bad.kmax = 1000  # not a power of two
    assert lib.zsort_pairs_ex(None, 0, None, 10, ctypes.byref(bad), None) == z.ERR_INVALID
    # n <= 1 and nseg == 0 are no-ops
    assert lib.zsort_pairs_ex(None, 0, None, 1, None, None) == z.OK
    assert lib.zsort_segmented_ex(None, None, 0, None, 0, None, None) == z.OK


def test_binding_refuses_cpu_tensors(lib):
    torch = pytest.importorskip("torch")
    k = torch.zeros(4, dtype=torch.int64)
    v = torch.zeros(4, dtype=torch.int32)
    with pytest.raises(ValueError):
        z.sort_pairs(k, v)
