"""GB300-native path-guided SGD (PG-SGD) pangenome graph layout.

A thin Python binding over libpgsgd.so (C ABI in include/pgsgd.h). Every step
of the layout and of the sampled path stress runs in the library's CUDA
kernels; this module only marshals arguments. PyTorch, when used, supplies
device memory and the current CUDA stream. There is no CPU fallback: without
the CUDA library or a GPU the calls raise.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native as N
from ._native import PgsgdError, StressResult

__all__ = ["Graph", "PgsgdError", "StressResult", "SAMPLE_DTYPE", "load_library", "l2_bandwidth",
           "hbm_gather_rate"]

SAMPLE_DTYPE = np.dtype([("g", "<u8"), ("i", "<u8"), ("j", "<u8"), ("d_ref", "<i8"),
                         ("path", "<u4"), ("cooling", "u1"), ("e_i", "u1"),
                         ("e_j", "u1"), ("skip", "u1")])


def load_library():
    return N.load()


def l2_bandwidth(bytes_=64 << 20, reps=20, mode=0, stream=None):
    """Measured L2 read bandwidth in GB/s (mode 0 streaming, 1 random 16-byte loads)."""
    lib = N.load()
    out = C.c_double()
    N.check(lib.pgsgd_l2_bandwidth(int(bytes_), int(reps), int(mode), C.byref(out), stream or _current_stream()))
    return out.value


def hbm_gather_rate(bytes_=4 << 30, reps=4, mode=0, blocks_per_sm=32, stream=None):
    """Random step-record-like reads per second from an HBM buffer of bytes_
    (two random 16-byte reads per unit within one of 90 "paths"; mode 1 adds
    two L2-resident 8-byte reads per unit)."""
    lib = N.load()
    out = C.c_double()
    N.check(lib.pgsgd_hbm_gather_bandwidth(int(bytes_), int(reps), int(mode), int(blocks_per_sm), C.byref(out),
                                           stream or _current_stream()))
    return out.value


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return C.c_void_p(0)


def _arg(x, dtype):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor."""
    if _is_torch(x):
        import torch
        tdt = {np.uint32: torch.uint32, np.uint8: torch.uint8, np.int64: torch.int64,
               np.uint64: torch.uint64, np.float64: torch.float64}[dtype]
        if x.dtype != tdt:
            raise TypeError(f"tensor dtype {x.dtype}, expected {tdt}")
        x = x.contiguous()
        return C.c_void_p(x.data_ptr()), int(x.is_cuda), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data_as(C.c_void_p), 0, a


def _arg_f32(x):
    if not _is_torch(x):
        raise TypeError("expected a torch tensor")
    import torch
    if x.dtype != torch.float32 or not x.is_contiguous():
        raise TypeError("expected a contiguous float32 tensor")
    return C.c_void_p(x.data_ptr()), int(x.is_cuda), x


class Graph:
    """A pangenome graph resident on the current CUDA device.

    Arrays follow ``pgsgd_create``: node lengths, path offsets and per-step
    node id, orientation and int64 nucleotide position; numpy (host) or torch
    CUDA tensors (device, all five)."""

    def __init__(self, node_len, path_off, step_node, step_rev, step_pos, stream=None):
        lib = N.load()
        self._lib = lib
        args = [_arg(node_len, np.uint32), _arg(path_off, np.uint64), _arg(step_node, np.uint32),
                _arg(step_rev, np.uint8), _arg(step_pos, np.int64)]
        on_dev = {a[1] for a in args}
        if len(on_dev) != 1:
            raise ValueError("all graph arrays must be on the host or all on the device")
        n_nodes = len(args[0][2])
        n_paths = len(args[1][2]) - 1
        h = C.c_void_p()
        N.check(lib.pgsgd_create(args[0][0], n_nodes, args[1][0], n_paths, args[2][0], args[3][0],
                                 args[4][0], on_dev.pop(), stream or _current_stream(), C.byref(h)))
        self._h = h
        self.n_nodes = n_nodes
        self.n_paths = n_paths

    @classmethod
    def from_synth(cls, g, stream=None):
        return cls(g.node_len, g.path_off, g.step_node, g.step_rev, g.step_pos, stream=stream)

    # ------------------------------------------------------------- lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._lib.pgsgd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    # ------------------------------------------------------------- options / info
    def set_option(self, name, value):
        N.check(self._lib.pgsgd_set_option(self._h, N.OPT[name], int(value)))

    def get_option(self, name):
        v = C.c_int64()
        N.check(self._lib.pgsgd_get_option(self._h, N.OPT[name], C.byref(v)))
        return v.value

    def info(self):
        out = N.Info()
        N.check(self._lib.pgsgd_info_get(self._h, C.byref(out)))
        return {f: getattr(out, f) for f, _ in out._fields_}

    # ------------------------------------------------------------- coordinates
    def set_coords(self, xy, stream=None):
        p, dev, keep = _arg(xy, np.float64)
        if tuple(keep.shape) != (self.n_nodes, 4):
            raise ValueError(f"xy must be [{self.n_nodes}, 4]")
        N.check(self._lib.pgsgd_set_coords(self._h, p, dev, stream or _current_stream()))

    def get_coords(self, out=None, stream=None):
        """Layout as float64 [n_nodes, 4]; into ``out`` (numpy or CUDA tensor) if given."""
        if out is None:
            out = np.empty((self.n_nodes, 4), dtype=np.float64)
        p, dev, keep = _arg(out, np.float64)
        N.check(self._lib.pgsgd_get_coords(self._h, p, dev, stream or _current_stream()))
        return out

    # ------------------------------------------------------------- the method
    def layout(self, iter_max=30, eta=None, eta_max=0.0, eta_min=0.0, theta=0.99, seed=1,
               iter_begin=0, iter_end=None, stream=None):
        if iter_end is None:
            iter_end = iter_max
        ep = None
        if eta is not None:
            eta = np.ascontiguousarray(eta, dtype=np.float64)
            if eta.shape != (iter_max,):
                raise ValueError("eta must hold iter_max entries")
            ep = eta.ctypes.data_as(C.c_void_p)
        N.check(self._lib.pgsgd_layout(self._h, iter_max, ep, float(eta_max), float(eta_min),
                                       float(theta), int(seed), iter_begin, iter_end,
                                       stream or _current_stream()))

    def stress(self, samples_per_step=100, seed=7, per_path=False, stream=None):
        res = N.StressResult()
        pp = np.zeros((self.n_paths, 3), dtype=np.float64) if per_path else None
        N.check(self._lib.pgsgd_stress(self._h, int(samples_per_step), int(seed), C.byref(res),
                                       pp.ctypes.data_as(C.c_void_p) if per_path else None,
                                       stream or _current_stream()))
        out = dict(mean=res.mean, std=res.stddev, ci_lo=res.ci_lo, ci_hi=res.ci_hi,
                   n_valid=int(res.n_valid), n_skipped=int(res.n_skipped))
        if per_path:
            out["per_path"] = pp
        return out

    def debug_sample(self, t, iter_max, theta, seed, u_begin, count, stream=None):
        out = np.zeros(count, dtype=SAMPLE_DTYPE)
        N.check(self._lib.pgsgd_debug_sample(self._h, t, iter_max, float(theta), int(seed),
                                             int(u_begin), int(count),
                                             out.ctypes.data_as(C.c_void_p),
                                             stream or _current_stream()))
        return out

    def debug_sample_reuse(self, t, iter_max, theta, seed, q_begin, count, stream=None):
        """With data reuse on: [count, drf] pair records of selections q_begin.. ."""
        drf = self.get_option("drf")
        out = np.zeros(count * drf, dtype=SAMPLE_DTYPE)
        N.check(self._lib.pgsgd_debug_sample_reuse(self._h, t, iter_max, float(theta), int(seed), int(q_begin),
                                                   int(count), out.ctypes.data_as(C.c_void_p),
                                                   stream or _current_stream()))
        return out.reshape(count, drf)

    def debug_sweep(self, t, iter_max, eta, theta, seed, u_begin, count, stream=None):
        out = np.zeros((count, 4), dtype=np.float32)
        N.check(self._lib.pgsgd_debug_sweep(self._h, t, iter_max, float(eta), float(theta),
                                            int(seed), int(u_begin), int(count),
                                            out.ctypes.data_as(C.c_void_p),
                                            stream or _current_stream()))
        return out

    def full_stress(self, stream=None):
        """Eq. 1 over all same-path step pairs: (value, number of pairs)."""
        v = C.c_double()
        n = C.c_uint64()
        N.check(self._lib.pgsgd_full_stress(self._h, C.byref(v), C.byref(n), stream or _current_stream()))
        return v.value, n.value

    def dstress(self, n_pairs, seed, stream=None):
        """Differentiable sampled stress: (value, n_valid)."""
        v = C.c_double()
        n = C.c_uint64()
        N.check(self._lib.pgsgd_dstress(self._h, int(n_pairs), int(seed), C.byref(v), C.byref(n),
                                        stream or _current_stream()))
        return v.value, n.value

    def dstress_backward(self, n_pairs, seed, scale, grad, stream=None):
        """grad (float32 CUDA tensor [n_nodes, 4]) <- scale * sum of per-sample gradients."""
        p, dev, keep = _arg_f32(grad)
        if not dev:
            raise ValueError("grad must be a CUDA tensor")
        N.check(self._lib.pgsgd_dstress_backward(self._h, int(n_pairs), int(seed), float(scale), p,
                                                 stream or _current_stream()))
        return grad

    def debug_pair_grad(self, t, iter_max, theta, seed, u_begin, count, stream=None):
        out = np.zeros((count, 4), dtype=np.float32)
        N.check(self._lib.pgsgd_debug_pair_grad(self._h, t, iter_max, float(theta), int(seed),
                                                int(u_begin), int(count),
                                                out.ctypes.data_as(C.c_void_p),
                                                stream or _current_stream()))
        return out

    def timing_read(self, reset=True):
        ms = C.c_double()
        launches = C.c_uint64()
        updates = C.c_uint64()
        N.check(self._lib.pgsgd_timing_read(self._h, C.byref(ms), C.byref(launches),
                                            C.byref(updates), int(reset)))
        return ms.value, launches.value, updates.value
