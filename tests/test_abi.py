"""The C ABI library builds, loads and exports every symbol its header
declares; host-side argument validation answers without touching a GPU."""
import ctypes as C

import numpy as np
import pytest

from paper_2409_00876_gb300 import _native as N


@pytest.fixture(scope="module")
def lib():
    return N.load()


def test_every_declared_symbol_is_exported(lib):
    names = N.declared_symbols()
    assert "pgsgd_create" in names and "pgsgd_layout" in names and "pgsgd_stress" in names
    for name in names:
        assert hasattr(lib, name), name
    # the binding declares a signature for every exported entry point
    assert set(names) <= set(N._SIGS)


def test_status_strings(lib):
    assert lib.pgsgd_status_string(0) == b"PGSGD_OK"
    assert lib.pgsgd_status_string(1) == b"PGSGD_EINVAL"
    assert lib.pgsgd_status_string(2) == b"PGSGD_ERANGE"
    assert lib.pgsgd_status_string(99) == b"PGSGD_UNKNOWN"


def _create(lib, node_len, path_off, S=None):
    node_len = np.asarray(node_len, np.uint32)
    path_off = np.asarray(path_off, np.uint64)
    S = int(path_off[-1]) if S is None else S
    node = np.zeros(max(S, 1), np.uint32)
    rev = np.zeros(max(S, 1), np.uint8)
    pos = np.zeros(max(S, 1), np.int64)
    h = C.c_void_p()
    rc = lib.pgsgd_create(node_len.ctypes.data_as(C.c_void_p), len(node_len),
                          path_off.ctypes.data_as(C.c_void_p), len(path_off) - 1,
                          node.ctypes.data_as(C.c_void_p), rev.ctypes.data_as(C.c_void_p),
                          pos.ctypes.data_as(C.c_void_p), 0, None, C.byref(h))
    return rc, h


@pytest.mark.parametrize("node_len,path_off,status,needle", [
    ([], [0, 0], N.PGSGD_EINVAL, "n_nodes"),
    ([3], [1, 2], N.PGSGD_EINVAL, "path_off[0]"),
    ([3], [0, 4, 2], N.PGSGD_EINVAL, "decreases"),
])
def test_host_validation_rejects_bad_tables(lib, node_len, path_off, status, needle):
    rc, h = _create(lib, node_len, path_off)
    assert rc == status
    assert h.value is None
    assert needle in lib.pgsgd_last_error().decode()


def test_too_many_paths_is_a_range_error(lib):
    rc, h = _create(lib, [3], np.zeros(16386, np.uint64))
    assert rc == N.PGSGD_ERANGE
    assert h.value is None


def test_too_many_nodes_is_a_range_error(lib):
    # node ids are packed into 31 bits of the step record; the count is
    # refused before any array is read
    one = np.ones(1, np.uint32)
    off = np.zeros(2, np.uint64)
    h = C.c_void_p()
    rc = lib.pgsgd_create(one.ctypes.data_as(C.c_void_p), 1 << 31, off.ctypes.data_as(C.c_void_p), 1,
                          None, None, None, 0, None, C.byref(h))
    assert rc == N.PGSGD_ERANGE and h.value is None
    assert "2^31" in lib.pgsgd_last_error().decode()


def test_null_output_handle(lib):
    one = np.ones(1, np.uint32)
    off = np.zeros(2, np.uint64)
    rc = lib.pgsgd_create(one.ctypes.data_as(C.c_void_p), 1, off.ctypes.data_as(C.c_void_p), 1,
                          None, None, None, 0, None, None)
    assert rc == N.PGSGD_EINVAL


def test_null_handles_are_rejected(lib):
    v = C.c_int64()
    assert lib.pgsgd_get_option(None, 1, C.byref(v)) == N.PGSGD_EINVAL
    assert lib.pgsgd_layout(None, 30, None, 0.0, 0.0, 0.99, 1, 0, 30, None) == N.PGSGD_EINVAL
    assert lib.pgsgd_destroy(None) == N.PGSGD_OK


def test_product_path_has_no_cpu_fallback():
    # the CUDA package never imports the oracle or any CPU implementation
    import paper_2409_00876_gb300 as pkg
    import sys
    src = open(pkg.__file__).read() + open(N.__file__).read()
    assert "oracle" not in src.replace("oracle.", "")
    assert "oracle" not in {m.split(".")[0] for m in sys.modules if m.startswith("paper_2409")}


def test_l2_probe_rejects_bad_arguments_without_touching_the_gpu():
    import paper_2409_00876_gb300 as pg
    from paper_2409_00876_gb300 import PgsgdError
    for kw in [dict(bytes_=1 << 10), dict(bytes_=1 << 31), dict(reps=0), dict(mode=2)]:
        with pytest.raises(PgsgdError):
            pg.l2_bandwidth(**kw)

def test_hbm_gather_probe_rejects_bad_arguments_without_touching_the_gpu():
    import paper_2409_00876_gb300 as pg
    from paper_2409_00876_gb300 import PgsgdError
    for kw in [dict(bytes_=1 << 20), dict(bytes_=65 << 30), dict(reps=0), dict(reps=101), dict(mode=2),
               dict(mode=-1), dict(blocks_per_sm=0), dict(blocks_per_sm=65)]:
        with pytest.raises(PgsgdError):
            pg.hbm_gather_rate(**kw)
