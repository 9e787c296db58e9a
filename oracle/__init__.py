"""CPU oracle for PG-SGD pangenome layout and path stress.

TEST INFRASTRUCTURE ONLY: a plain, slow FP64 restatement of Algorithm 1 and of
Eq. 1 / Eq. 2 of "Rapid GPU-Based Pangenome Graph Layout" (SC24), used to
check the CUDA library. Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import it. It imports nothing from the CUDA
package and the CUDA package imports nothing from it.

The arithmetic lives in ``pgsgd_oracle.c`` (each function there cites the
passage it follows); this module compiles it with gcc (no fused multiply-add,
no fast-math) and wraps it with ctypes and numpy.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
values fixed by the paper or by mathematics (worked examples, closed forms,
exact enumeration, library routines); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pgsgd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

SAMPLE_DTYPE = np.dtype([("g", "<u8"), ("i", "<u8"), ("j", "<u8"), ("d_ref", "<i8"),
                         ("path", "<u4"), ("cooling", "u1"), ("e_i", "u1"),
                         ("e_j", "u1"), ("skip", "u1")])
assert SAMPLE_DTYPE.itemsize == 40

GCC_FLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
             "-shared", "-pthread"]


def build(force: bool = False) -> str:
    """Compile the oracle library (gcc, a second or two)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *GCC_FLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            lib = C.CDLL(path)
            P = C.c_void_p
            u32, u64, dbl, i32 = C.c_uint32, C.c_uint64, C.c_double, C.c_int
            gargs = [P, u32, P, u32, P, P, P]
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_ln_f32.argtypes = [C.c_float]
            lib.orc_ln_f32.restype = C.c_float
            lib.orc_exp_f32.argtypes = [C.c_float]
            lib.orc_exp_f32.restype = C.c_float
            lib.orc_zipf_consts.argtypes = [dbl, u64, P]
            lib.orc_zipf_sample.argtypes = [dbl, u64, u64, u64, P]
            lib.orc_zipf_trials.argtypes = [dbl, u64, u32, u32, P]
            lib.orc_sample.argtypes = gargs + [u32, u32, dbl, u64, u64, u64, P]
            lib.orc_sample.restype = i32
            lib.orc_sample_wm.argtypes = gargs + [u32, u32, dbl, u64, i32, u64, u64, P]
            lib.orc_sample_wm.restype = i32
            lib.orc_sample_reuse.argtypes = gargs + [u32, u32, dbl, u64, i32, u32, u64, u64, u64, P]
            lib.orc_sample_reuse.restype = i32
            lib.orc_layout_variant.argtypes = gargs + [P, u32, P, dbl, u64, u32, u32, u64, i32, u32, P]
            lib.orc_layout_variant.restype = i32
            lib.orc_eta_schedule.argtypes = [u32, dbl, dbl, P]
            lib.orc_sweep.argtypes = gargs + [P, u32, u32, dbl, dbl, u64, u64, u64, P]
            lib.orc_sweep.restype = i32
            lib.orc_layout.argtypes = gargs + [P, u32, P, dbl, u64, u32, u32, u64, u32, P]
            lib.orc_layout.restype = i32
            lib.orc_sampled_stress.argtypes = gargs + [P, u32, u64, u32, P, P]
            lib.orc_sampled_stress.restype = i32
            lib.orc_sampled_stress_paths.argtypes = gargs + [P, u32, u64, u32, u32, u32, P, P]
            lib.orc_sampled_stress_paths.restype = i32
            lib.orc_full_stress.argtypes = gargs + [P, P]
            lib.orc_full_stress.restype = i32
            lib.orc_dstress.argtypes = gargs + [P, u64, u64, P]
            lib.orc_dstress.restype = i32
            lib.orc_dstress_grad.argtypes = gargs + [P, u64, u64, P]
            lib.orc_dstress_grad.restype = i32
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class _GraphArgs:
    """Contiguous, correctly typed views of a graph's arrays (kept alive)."""

    def __init__(self, g):
        self.node_len = np.ascontiguousarray(g.node_len, dtype=np.uint32)
        self.path_off = np.ascontiguousarray(g.path_off, dtype=np.uint64)
        self.step_node = np.ascontiguousarray(g.step_node, dtype=np.uint32)
        self.step_rev = np.ascontiguousarray(g.step_rev, dtype=np.uint8)
        self.step_pos = np.ascontiguousarray(g.step_pos, dtype=np.int64)
        self.n_paths = self.path_off.shape[0] - 1

    def args(self):
        return [_ptr(self.node_len), self.node_len.shape[0], _ptr(self.path_off), self.n_paths,
                _ptr(self.step_node), _ptr(self.step_rev), _ptr(self.step_pos)]


def _ga(g):
    cached = getattr(g, "_orc_args", None)
    if cached is None:
        cached = _GraphArgs(g)
        try:
            g._orc_args = cached
        except AttributeError:
            pass
    return cached


# ---------------------------------------------------------------- primitives

def philox4x32_10(ctr, key):
    """One Philox4x32-10 block (Salmon et al., SC'11) for counter ctr[4], key[2]."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    _L().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def ln_f32(x: float) -> np.float32:
    return np.float32(_L().orc_ln_f32(float(x)))


def exp_f32(y: float) -> np.float32:
    return np.float32(_L().orc_exp_f32(float(y)))


def zipf_consts(theta: float, N: int):
    out = np.zeros(3, dtype=np.float32)
    _L().orc_zipf_consts(float(theta), int(N), _ptr(out))
    return out


def zipf_sample(theta: float, N: int, seed: int, count: int) -> np.ndarray:
    """count Zipf(theta) draws on [1, N] by the layout's rejection-inversion."""
    out = np.zeros(count, dtype=np.uint64)
    _L().orc_zipf_sample(float(theta), int(N), int(seed), int(count), _ptr(out))
    return out


def zipf_trials(theta: float, N: int, m_begin: int = 0, count: int = 1 << 24) -> np.ndarray:
    """One rejection-inversion trial per word w = (m_begin + m) << 8: the k it
    accepts, 0 where it rejects. m over [0, 2^24) covers every trial word."""
    out = np.zeros(count, dtype=np.uint64)
    _L().orc_zipf_trials(float(theta), int(N), int(m_begin), int(count), _ptr(out))
    return out


def eta_schedule(T: int, eta_max: float, eta_min: float = 0.01) -> np.ndarray:
    out = np.zeros(T, dtype=np.float64)
    _L().orc_eta_schedule(int(T), float(eta_max), float(eta_min), _ptr(out))
    return out


def default_eta_max(g) -> float:
    """(longest path in nucleotides)^2: the annealing start of Zheng et al."""
    return float(g.path_nt_lengths().max()) ** 2


# ---------------------------------------------------------------- sampler

def sample(g, T, t, theta, seed, u_begin, count) -> np.ndarray:
    """The pair every update u in [u_begin, u_begin + count) of iteration t draws."""
    out = np.zeros(count, dtype=SAMPLE_DTYPE)
    rc = _L().orc_sample(*_ga(g).args(), int(T), int(t), float(theta), int(seed),
                         int(u_begin), int(count), _ptr(out))
    if rc:
        raise MemoryError("oracle sample")
    return out


def sample_wm(g, T, t, theta, seed, u_begin, count, wm=1) -> np.ndarray:
    """As sample, with the cooling coin of every update taken from its group of 32 (warp merging)."""
    out = np.zeros(count, dtype=SAMPLE_DTYPE)
    rc = _L().orc_sample_wm(*_ga(g).args(), int(T), int(t), float(theta), int(seed), int(wm),
                            int(u_begin), int(count), _ptr(out))
    if rc:
        raise MemoryError("oracle sample")
    return out


def sample_reuse(g, T, t, theta, seed, drf, n_sel, q_begin, count, wm=0) -> np.ndarray:
    """The drf pairs of every selection q in [q_begin, q_begin + count) under
    warp-level data reuse: [count, drf] records (round k in column k)."""
    out = np.zeros(count * drf, dtype=SAMPLE_DTYPE)
    rc = _L().orc_sample_reuse(*_ga(g).args(), int(T), int(t), float(theta), int(seed), int(wm),
                               int(drf), int(n_sel), int(q_begin), int(count), _ptr(out))
    if rc:
        raise MemoryError("oracle sample")
    return out.reshape(count, drf)


def n_selections(g, updates_per_step=10, srf=1) -> int:
    """Selections per iteration with step reduction factor srf."""
    return -(-updates_per_step * g.n_steps // srf)


def layout_variant(g, xy, T=30, eta=None, theta=0.99, seed=1, t_begin=0, t_end=None, drf=1, srf=1,
                   wm=0, updates_per_step=10, n_units=None):
    """Sequential Algorithm 1 under warp merging (wm) and data reuse (drf, srf);
    drf = srf = 1, wm = 0 is layout(..., n_threads=1). Returns (new xy, moves)."""
    xy = np.array(xy, dtype=np.float64, order="C", copy=True)
    if eta is None:
        eta = eta_schedule(T, default_eta_max(g))
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    if t_end is None:
        t_end = T
    if n_units is None:
        n_units = n_selections(g, updates_per_step, srf)
    moved = C.c_uint64()
    rc = _L().orc_layout_variant(*_ga(g).args(), _ptr(xy), int(T), _ptr(eta), float(theta), int(seed),
                                 int(t_begin), int(t_end), int(n_units), int(wm), int(drf), C.byref(moved))
    if rc:
        raise MemoryError("oracle layout")
    return xy, moved.value


def sweep(g, xy, T, t, eta, theta, seed, u_begin, count) -> np.ndarray:
    """Jacobi sweep: [count, 4] changes (dv_i, dv_j) from the frozen layout xy."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    out = np.zeros((count, 4), dtype=np.float64)
    rc = _L().orc_sweep(*_ga(g).args(), _ptr(xy), int(T), int(t), float(eta), float(theta),
                        int(seed), int(u_begin), int(count), _ptr(out))
    if rc:
        raise MemoryError("oracle sweep")
    return out


def layout(g, xy, T=30, eta=None, theta=0.99, seed=1, t_begin=0, t_end=None,
           n_updates=None, updates_per_step=10, n_threads=1, eta_max=None, eta_min=0.01):
    """Algorithm 1 on a copy of xy; returns (new xy, number of moves made)."""
    xy = np.array(xy, dtype=np.float64, order="C", copy=True)
    if eta is None:
        eta = eta_schedule(T, default_eta_max(g) if eta_max is None else eta_max, eta_min)
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    if t_end is None:
        t_end = T
    if n_updates is None:
        n_updates = updates_per_step * g.n_steps
    moved = np.zeros(1, dtype=np.uint64)
    rc = _L().orc_layout(*_ga(g).args(), _ptr(xy), int(T), _ptr(eta), float(theta), int(seed),
                         int(t_begin), int(t_end), int(n_updates), int(n_threads), _ptr(moved))
    if rc:
        raise MemoryError("oracle layout")
    return xy, int(moved[0])


def sampled_stress(g, xy, per_step=100, seed=7, n_threads=1, per_path=False, paths=None):
    """Eq. 2: dict(mean, std, ci_lo, ci_hi, n_valid, n_skipped[, per_path]).

    paths=(begin, end) restricts the sample set to those paths."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    out = np.zeros(6, dtype=np.float64)
    pp = np.zeros((g.n_paths, 3), dtype=np.float64)
    p0, p1 = (0, g.n_paths) if paths is None else paths
    rc = _L().orc_sampled_stress_paths(*_ga(g).args(), _ptr(xy), int(per_step), int(seed),
                                       int(n_threads), int(p0), int(p1), _ptr(out), _ptr(pp))
    if rc:
        raise MemoryError("oracle stress")
    res = dict(mean=out[0], std=out[1], ci_lo=out[2], ci_hi=out[3],
               n_valid=int(out[4]), n_skipped=int(out[5]))
    if per_path:
        res["per_path"] = pp
    return res


def full_stress(g, xy):
    """Eq. 1 by brute force: (path stress, number of node pairs counted)."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    out = np.zeros(2, dtype=np.float64)
    _L().orc_full_stress(*_ga(g).args(), _ptr(xy), _ptr(out))
    return float(out[0]), int(out[1])


# ---------------------------------------------------------------- differentiable stress

def dstress(g, xy, n_pairs, seed):
    """Eq. 2's estimator over a fixed set of n_pairs samples: (F, n_valid)."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    out = np.zeros(2, dtype=np.float64)
    _L().orc_dstress(*_ga(g).args(), _ptr(xy), int(n_pairs), int(seed), _ptr(out))
    return float(out[0]), int(out[1])


def dstress_grad(g, xy, n_pairs, seed):
    """dF/d(sx, sy, ex, ey) of dstress, [n_nodes, 4] float64."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    grad = np.zeros_like(xy)
    _L().orc_dstress_grad(*_ga(g).args(), _ptr(xy), int(n_pairs), int(seed), _ptr(grad))
    return grad
