"""ctypes view of libpgsgd.so (include/pgsgd.h). Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

P = C.c_void_p
u8, u32, u64, i32, i64, dbl = C.c_uint8, C.c_uint32, C.c_uint64, C.c_int, C.c_int64, C.c_double

PGSGD_OK, PGSGD_EINVAL, PGSGD_ERANGE, PGSGD_ENOMEM, PGSGD_ECUDA, PGSGD_ETIMEOUT, PGSGD_EDEVICE = range(7)

OPT = dict(coord_mode=1, updates_per_step=2, block=3, blocks_per_sm=4, updates_per_thread=5,
           atomic_updates=6, rebase=7, timing=8, max_concurrent=9,
           min_blocks=10, l2_fetch=11, store_mode=12, l2_hints=13, prefetch64=14, pipeline=15,
           warp_merge=16, drf=17, srf=18, async_depth=19, stress_async=20, stress_waves=21)


BOPT = dict(mode=1, cuda_graph=2, block=3, updates_per_thread=4, chunk=5, max_concurrent=6,
            updates_per_step=7, timeout_ms=8, timing=9, stall_test=10, blocks_per_sm=11, pipeline=12, prefetch64=13)


class StressResult(C.Structure):
    _fields_ = [("mean", dbl), ("stddev", dbl), ("ci_lo", dbl), ("ci_hi", dbl),
                ("n_valid", u64), ("n_skipped", u64)]


class Info(C.Structure):
    _fields_ = [("n_steps", u64), ("device_bytes", u64), ("max_path_steps", u64),
                ("max_path_nt", i64), ("n_nodes", u32), ("n_paths", u32), ("device", C.c_int32),
                ("sm_count", C.c_int32)]


class BatchInfo(C.Structure):
    _fields_ = [("n_steps", u64), ("device_bytes", u64), ("last_launches", u64), ("n_graphs", u32),
                ("n_nodes", u32), ("n_paths", u32), ("max_graph_paths", u32), ("last_grid", C.c_int32),
                ("reserved", C.c_int32)]


class PgsgdError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status


_SIGS = {
    "pgsgd_create": ([P, u32, P, u32, P, P, P, i32, P, P], i32),
    "pgsgd_destroy": ([P], i32),
    "pgsgd_set_option": ([P, i32, i64], i32),
    "pgsgd_get_option": ([P, i32, P], i32),
    "pgsgd_info_get": ([P, P], i32),
    "pgsgd_set_coords": ([P, P, i32, P], i32),
    "pgsgd_get_coords": ([P, P, i32, P], i32),
    "pgsgd_layout": ([P, u32, P, dbl, dbl, dbl, u64, u32, u32, P], i32),
    "pgsgd_stress": ([P, u32, u64, P, P, P], i32),
    "pgsgd_debug_sample": ([P, u32, u32, dbl, u64, u64, u64, P, P], i32),
    "pgsgd_debug_sample_reuse": ([P, u32, u32, dbl, u64, u64, u64, P, P], i32),
    "pgsgd_debug_sweep": ([P, u32, u32, dbl, dbl, u64, u64, u64, P, P], i32),
    "pgsgd_timing_read": ([P, P, P, P, i32], i32),
    "pgsgd_stress_noalloc": ([P, u32, P, u32, P, P, P, P, u32, u64, P, P], i32),
    "pgsgd_dstress": ([P, u64, u64, P, P, P], i32),
    "pgsgd_full_stress": ([P, P, P, P], i32),
    "pgsgd_dstress_backward": ([P, u64, u64, dbl, P, P], i32),
    "pgsgd_debug_pair_grad": ([P, u32, u32, dbl, u64, u64, u64, P, P], i32),
    "pgsgd_batch_create": ([u32, P, P, P, P, P, P, P, i32, P, P], i32),
    "pgsgd_batch_destroy": ([P], i32),
    "pgsgd_batch_set_option": ([P, i32, i64], i32),
    "pgsgd_batch_get_option": ([P, i32, P], i32),
    "pgsgd_batch_info_get": ([P, P], i32),
    "pgsgd_batch_set_coords": ([P, P, i32, P], i32),
    "pgsgd_batch_get_coords": ([P, P, i32, P], i32),
    "pgsgd_batch_layout": ([P, u32, P, dbl, P, u32, u32, P], i32),
    "pgsgd_batch_stress": ([P, u32, u64, P, P], i32),
    "pgsgd_batch_debug_sample": ([P, u32, u32, u32, dbl, u64, u64, u64, P, P], i32),
    "pgsgd_batch_timing_read": ([P, P, P, P, i32], i32),
    "pgsgd_batch_plan": ([u32, P, P, i32, i32, u64, i64, P, P, P, P], i32),
    "pgsgd_l2_bandwidth": ([u64, u32, i32, P, P], i32),
    "pgsgd_hbm_gather_bandwidth": ([u64, u32, i32, i32, P, P], i32),
    "pgsgd_last_error": ([], C.c_char_p),
    "pgsgd_status_string": ([i32], C.c_char_p),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpgsgd.so from the package's build folder (building it if stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libpgsgd.so not built at {path}")
            lib = C.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def status_name(status: int) -> str:
    return load().pgsgd_status_string(int(status)).decode()


def check(status: int):
    if status != PGSGD_OK:
        raise PgsgdError(status, load().pgsgd_last_error().decode())


def declared_symbols(header: str | None = None):
    """Function names the public headers (all of include/*.h, or one) declare."""
    if header is None:
        inc = os.path.join(_build.ROOT, "include")
        headers = sorted(os.path.join(inc, f) for f in os.listdir(inc) if f.endswith(".h"))
    else:
        headers = [header]
    names = set()
    for h in headers:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names.update(re.findall(r"\b(pgsgd_[a-z_]+)\s*\(", text))
    return sorted(names)
