"""Batched layout of many independent graphs (include/pgsgd_batch.h).

Argument marshalling over libpgsgd.so, plus ``autotune``, which picks the
batch schedule (mode, pipelined loop, threads per block, updates per thread,
chunk size) by timing short layouts on the GPU. Every step of the layout runs in the
library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native as N
from . import SAMPLE_DTYPE, _arg, _current_stream

__all__ = ["Batch", "plan", "autotune", "MODES"]

MODES = {"launch": 0, "persistent": 1, "per_graph": 2}


def _u64p(a):
    return a.ctypes.data_as(C.c_void_p)


def plan(n_updates, n_nodes, block=256, updates_per_thread=2, chunk=16384, max_concurrent=-1):
    """Host-only schedule plan: (rank_to_graph, n_chunks, lanes, threads)."""
    lib = N.load()
    nu = np.ascontiguousarray(n_updates, dtype=np.uint64)
    nn = np.ascontiguousarray(n_nodes, dtype=np.uint64)
    G = len(nu)
    r2g = np.zeros(G, np.uint32)
    nch = np.zeros(G, np.uint32)
    lanes = np.zeros(G, np.uint32)
    thr = np.zeros(G, np.uint32)
    N.check(lib.pgsgd_batch_plan(G, _u64p(nu), _u64p(nn), int(block), int(updates_per_thread), int(chunk),
                                 int(max_concurrent), _u64p(r2g), _u64p(nch), _u64p(lanes), _u64p(thr)))
    return r2g, nch, lanes, thr


class Batch:
    """Graphs laid out together on the current CUDA device.

    Arrays follow ``pgsgd_batch_create``: per-graph node and path offsets
    (host), then node lengths, path offsets, LOCAL step node ids, orientations
    and positions of the concatenated graphs (numpy, or torch CUDA tensors)."""

    def __init__(self, graph_node_off, graph_path_off, node_len, path_off, step_node, step_rev, step_pos,
                 stream=None):
        lib = N.load()
        self._lib = lib
        self._gno = np.ascontiguousarray(graph_node_off, dtype=np.uint64)
        self._gpo = np.ascontiguousarray(graph_path_off, dtype=np.uint64)
        args = [_arg(node_len, np.uint32), _arg(path_off, np.uint64), _arg(step_node, np.uint32),
                _arg(step_rev, np.uint8), _arg(step_pos, np.int64)]
        on_dev = {a[1] for a in args}
        if len(on_dev) != 1:
            raise ValueError("all graph arrays must be on the host or all on the device")
        self.n_graphs = len(self._gno) - 1
        h = C.c_void_p()
        N.check(lib.pgsgd_batch_create(self.n_graphs, _u64p(self._gno), _u64p(self._gpo), args[0][0], args[1][0],
                                       args[2][0], args[3][0], args[4][0], on_dev.pop(),
                                       stream or _current_stream(), C.byref(h)))
        self._h = h
        self.n_nodes = int(self._gno[-1])

    @classmethod
    def from_arrays(cls, b, stream=None):
        """From a synth.BatchArrays."""
        return cls(b.graph_node_off, b.graph_path_off, b.node_len, b.path_off, b.step_node, b.step_rev,
                   b.step_pos, stream=stream)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pgsgd_batch_destroy(self._h)
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

    def set_option(self, name, value):
        if name == "mode" and isinstance(value, str):
            value = MODES[value]
        N.check(self._lib.pgsgd_batch_set_option(self._h, N.BOPT[name], int(value)))

    def get_option(self, name):
        v = C.c_int64()
        N.check(self._lib.pgsgd_batch_get_option(self._h, N.BOPT[name], C.byref(v)))
        return v.value

    def options(self):
        return {k: self.get_option(k) for k in N.BOPT}

    def info(self):
        out = N.BatchInfo()
        N.check(self._lib.pgsgd_batch_info_get(self._h, C.byref(out)))
        return {f: getattr(out, f) for f, _ in out._fields_}

    def node_range(self, g):
        return int(self._gno[g]), int(self._gno[g + 1])

    def set_coords(self, xy, stream=None):
        p, dev, keep = _arg(xy, np.float64)
        if tuple(keep.shape) != (self.n_nodes, 4):
            raise ValueError(f"xy must be [{self.n_nodes}, 4]")
        N.check(self._lib.pgsgd_batch_set_coords(self._h, p, dev, stream or _current_stream()))

    def get_coords(self, out=None, stream=None):
        if out is None:
            out = np.empty((self.n_nodes, 4), dtype=np.float64)
        p, dev, keep = _arg(out, np.float64)
        N.check(self._lib.pgsgd_batch_get_coords(self._h, p, dev, stream or _current_stream()))
        return out

    def _seeds(self, seeds):
        if np.isscalar(seeds):
            seeds = np.full(self.n_graphs, int(seeds), dtype=np.uint64)
        s = np.ascontiguousarray(seeds, dtype=np.uint64)
        if s.shape != (self.n_graphs,):
            raise ValueError(f"seeds must hold {self.n_graphs} values")
        return s

    def layout(self, iter_max=30, seeds=1, eta=None, theta=0.99, iter_begin=0, iter_end=None, stream=None):
        """seeds: one int for every graph or an array of n_graphs; eta: None or [n_graphs, iter_max]."""
        if iter_end is None:
            iter_end = iter_max
        s = self._seeds(seeds)
        ep = None
        if eta is not None:
            eta = np.ascontiguousarray(eta, dtype=np.float64)
            if eta.shape != (self.n_graphs, iter_max):
                raise ValueError("eta must be [n_graphs, iter_max]")
            ep = _u64p(eta)
        N.check(self._lib.pgsgd_batch_layout(self._h, iter_max, ep, float(theta), _u64p(s), iter_begin, iter_end,
                                             stream or _current_stream()))

    def stress(self, samples_per_step=100, seed=7, stream=None):
        """Eq. 2 of every graph: list of dicts as Graph.stress returns."""
        res = (N.StressResult * self.n_graphs)()
        N.check(self._lib.pgsgd_batch_stress(self._h, int(samples_per_step), int(seed), res,
                                             stream or _current_stream()))
        return [dict(mean=r.mean, std=r.stddev, ci_lo=r.ci_lo, ci_hi=r.ci_hi, n_valid=int(r.n_valid),
                     n_skipped=int(r.n_skipped)) for r in res]

    def debug_sample(self, graph, t, iter_max, theta, seed, u_begin, count, stream=None):
        out = np.zeros(count, dtype=SAMPLE_DTYPE)
        N.check(self._lib.pgsgd_batch_debug_sample(self._h, int(graph), t, iter_max, float(theta), int(seed),
                                                   int(u_begin), int(count), out.ctypes.data_as(C.c_void_p),
                                                   stream or _current_stream()))
        return out

    def timing_read(self, reset=True):
        ms = C.c_double()
        launches = C.c_uint64()
        updates = C.c_uint64()
        N.check(self._lib.pgsgd_batch_timing_read(self._h, C.byref(ms), C.byref(launches), C.byref(updates),
                                                  int(reset)))
        return ms.value, launches.value, updates.value


def _time_layout(b, xy, seeds, iter_max, theta, window, repeats):
    """Milliseconds of the window's iterations (best of repeats), from xy each
    time; an untimed first run also captures the CUDA graph."""
    b.set_option("timing", 1)
    times = []
    try:
        for i in range(repeats + 1):
            b.set_coords(xy)
            b.timing_read(reset=True)
            b.layout(iter_max, seeds=seeds, theta=theta, iter_begin=window[0], iter_end=window[1])
            ms, _, _ = b.timing_read(reset=True)
            if i:
                times.append(ms)
    finally:
        b.set_option("timing", 0)
    return min(times)


def autotune(b, xy, seeds=1, iter_max=30, theta=0.99, window=None, repeats=1, space=None, log=None):
    """Coordinate descent over the batch schedule, timing `window` (default
    the two iterations around T / 2: one before cooling is forced, one
    after) from the same layout xy each trial. Leaves the best options set on
    b and returns (best options, {options tuple: ms})."""
    if window is None:
        window = (iter_max // 2 - 1, iter_max // 2 + 1)
    space = space or dict(mode=[0, 1], pipeline=[0, 1], updates_per_thread=[2, 1, 4], block=[256, 128],
                          chunk=[16384, 4096, 32768, 65536])
    keys = list(space)
    cur = {k: b.get_option(k) for k in keys}
    for k in keys:
        if cur[k] not in space[k]:
            cur[k] = space[k][0]
    seen = {}

    def trial(opts):
        key = tuple(opts[k] for k in keys)
        if key not in seen:
            for k in keys:
                b.set_option(k, opts[k])
            seen[key] = _time_layout(b, xy, seeds, iter_max, theta, window, repeats)
            if log:
                log(f"autotune {dict(zip(keys, key))}: {seen[key]:.2f} ms")
        return seen[key]

    best = trial(cur)
    for _ in range(2):
        improved = False
        for k in keys:
            for v in space[k]:
                cand = dict(cur, **{k: v})
                ms = trial(cand)
                if ms < best:
                    best, cur, improved = ms, cand, True
        if not improved:
            break
    for k in keys:
        b.set_option(k, cur[k])
    return cur, {k: v for k, v in seen.items()}

