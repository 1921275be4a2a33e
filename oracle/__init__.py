"""CPU oracle for the PLAS grid sort and the grid smoothness loss.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import this package.  The
product (the CUDA library under ``paper_2312_13299_gb300`` and its binding)
never imports it, and the two share no code.

The arithmetic lives in ``plas_oracle.c`` (plain C, ``-ffp-contract=off``,
explicit ``fmaf``); this module only compiles it with gcc and marshals numpy
arrays through ctypes.  Paper sections followed: Sec. 3.1 (sort, blocks,
groups of four, schedule, feature normalisation), Sec. 3.2 (smoothness loss),
supplementary "Sorting performance" (threshold 1e-4, VAD).

Parity status: every function here is pinned by tests under ``tests/``
(known-answer vectors, library routines, brute force, closed forms,
finite differences); see the test files' docstrings for which pin covers what.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "plas_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libplas_oracle.so")
_lock = threading.Lock()
_lib = None

TAG_INIT, TAG_SHIFT, TAG_GROUP = 1, 2, 3


def build(force: bool = False) -> str:
    """Compile plas_oracle.c into a shared library (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    # fmaf is correctly rounded however it is computed; on x86-64 -mfma lets
    # gcc emit the FMA instruction instead of a libm call (aarch64 always
    # does), which changes no result.  Contraction of anything else stays off.
    isa = ["-mfma"] if platform.machine() in ("x86_64", "AMD64") else []
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", *isa,
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Schedule(ctypes.Structure):
    _fields_ = [("phi0", ctypes.c_double), ("shrink", ctypes.c_double),
                ("phi_min", ctypes.c_double), ("tol", ctypes.c_double),
                ("sigma_ratio", ctypes.c_double), ("min_block", ctypes.c_int),
                ("shuffle_init", ctypes.c_int), ("normalize", ctypes.c_int),
                ("target_mode", ctypes.c_int), ("max_iters", ctypes.c_longlong),
                ("edge_blocks", ctypes.c_int), ("pad_", ctypes.c_int)]


class State(ctypes.Structure):
    _fields_ = [("it", ctypes.c_longlong), ("epoch", ctypes.c_longlong),
                ("redraws", ctypes.c_longlong), ("level", ctypes.c_int),
                ("stall", ctypes.c_int), ("has_prev", ctypes.c_int),
                ("done", ctypes.c_int), ("d_prev", ctypes.c_double),
                ("d_last", ctypes.c_double), ("scale_exp", ctypes.c_int),
                ("pad_", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


def default_schedule(**kw) -> Schedule:
    """Defaults: phi0 = w/2-1, shrink 0.95, stop below 1 (Sec. 3.1); tol 1e-4
    (supplementary); min block 16 (Sec. 3.1); sigma = 2 phi (paper silent);
    the blocks cut by the grid border take part (Sec. 3.1: the shifted
    blocks cover the whole grid, borders included)."""
    s = Schedule(phi0=0.0, shrink=0.95, phi_min=1.0, tol=1e-4, sigma_ratio=2.0,
                 min_block=16, shuffle_init=1, normalize=1, target_mode=0, max_iters=0,
                 edge_blocks=1)
    for k, v in kw.items():
        setattr(s, k, v)
    return s


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t)) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            f, d, i, u32, u64, ll = (ctypes.POINTER(ctypes.c_float), ctypes.c_double,
                                     ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64,
                                     ctypes.c_longlong)
            P = ctypes.POINTER
            L.orc_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
            L.orc_prp.argtypes = [u64, u32, u64, u32, u32]
            L.orc_prp.restype = u32
            L.orc_prp_table.argtypes = [u64, u32, u64, u32, P(u32)]
            L.orc_levels.argtypes = [P(Schedule), i, i, P(d), i]
            L.orc_levels.restype = i
            L.orc_shift.argtypes = [u64, u64, i, i, i, P(i), P(i)]
            L.orc_taps.argtypes = [i, d, f]
            L.orc_blur.argtypes = [f, i, i, i, i, i, d, f]
            L.orc_perm24_table.argtypes = [P(i)]
            L.orc_best_perm.argtypes = [f]
            L.orc_best_perm.restype = i
            L.orc_minmax.argtypes = [f, ctypes.c_long, i, f, f]
            L.orc_normalize.argtypes = [f, ctypes.c_long, i, f, i, f]
            L.orc_scale_exp.argtypes = [f, ctypes.c_long, i, f, i]
            L.orc_scale_exp.restype = i
            L.orc_sort.argtypes = [f, i, i, i, f, u64, P(Schedule), P(ctypes.c_int32), i,
                                   P(State), P(ctypes.c_int32), P(ll), P(i), ll, f]
            L.orc_sort.restype = ll
            L.orc_target.argtypes = [f, i, i, i, f, i, P(ctypes.c_int32), d, d, f]
            L.orc_target_box.argtypes = [f, i, i, i, f, i, P(ctypes.c_int32), d, f]
            L.orc_box_exp.argtypes = [f, ctypes.c_long, i, f, i]
            L.orc_box_exp.restype = i
            L.orc_gather.argtypes = [f, ctypes.c_long, i, P(ctypes.c_int32), f]
            L.orc_metrics.argtypes = [f, i, i, i, d, P(d), P(d)]
            L.orc_smooth_taps64.argtypes = [d, i, P(d)]
            L.orc_smooth_loss64.argtypes = [P(d), i, i, i, d, i, P(d), d, P(d)]
            L.orc_smooth_loss64.restype = d
            L.orc_smooth_loss64_huber.argtypes = [P(d), i, i, i, d, i, P(d), d, d, P(d)]
            L.orc_smooth_loss64_huber.restype = d
            L.orc_activate_3dgs.argtypes = [f, ctypes.c_long, i, f]
            L.orc_grid_select.argtypes = [f, ctypes.c_long, i, P(i)]
            L.orc_grid_select.restype = i
            L.orc_quantize.argtypes = [f, ctypes.c_long, i, f, f, P(i),
                                       P(ctypes.c_ushort)]
            L.orc_dequantize.argtypes = [P(ctypes.c_ushort), ctypes.c_long, i, f, f, P(i), f]
            L.orc_num_threads.restype = i
            L.orc_set_num_threads.argtypes = [i]
            _lib = L
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


# --------------------------------------------------------------------------
# random sources
# --------------------------------------------------------------------------
def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32),
                            _p(o, ctypes.c_uint32))
    return o


def prp(seed: int, tag: int, counter: int, n: int, x: int) -> int:
    return int(lib().orc_prp(seed, tag, counter, n, x))


def prp_table(seed: int, tag: int, counter: int, n: int) -> np.ndarray:
    o = np.zeros(n, np.uint32)
    lib().orc_prp_table(seed, tag, counter, n, _p(o, ctypes.c_uint32))
    return o


def shift(seed: int, epoch: int, beta: int, H: int, W: int):
    dy, dx = ctypes.c_int(), ctypes.c_int()
    lib().orc_shift(seed, epoch, beta, H, W, ctypes.byref(dy), ctypes.byref(dx))
    return dy.value, dx.value


# --------------------------------------------------------------------------
# schedule, blur, assignment pieces
# --------------------------------------------------------------------------
def levels(H: int, W: int, sched: Schedule | None = None) -> np.ndarray:
    s = sched or default_schedule()
    n = lib().orc_levels(ctypes.byref(s), H, W, None, 0)
    out = np.zeros(n, np.float64)
    lib().orc_levels(ctypes.byref(s), H, W, _p(out, ctypes.c_double), n)
    return out


def taps(r: int, sigma: float) -> np.ndarray:
    o = np.zeros(2 * r + 1, np.float32)
    lib().orc_taps(r, sigma, _p(o, ctypes.c_float))
    return o


def blur(G: np.ndarray, r: int, sigma: float) -> np.ndarray:
    """G: H x W x D float32 -> renormalised separable Gaussian target."""
    G = _f32(G)
    H, W, D = G.shape
    T = np.zeros((H, W, D), np.float32)
    lib().orc_blur(_p(G, ctypes.c_float), D, H, W, D, r, sigma, _p(T, ctypes.c_float))
    return T


def perm24() -> np.ndarray:
    o = np.zeros(96, np.int32)
    lib().orc_perm24_table(_p(o, ctypes.c_int))
    return o.reshape(24, 4)


def best_perm(C: np.ndarray) -> int:
    C = _f32(C).reshape(16)
    return int(lib().orc_best_perm(_p(C, ctypes.c_float)))


def minmax(x: np.ndarray):
    x = _f32(x)
    N, D = x.shape
    lo, hi = np.zeros(D, np.float32), np.zeros(D, np.float32)
    lib().orc_minmax(_p(x, ctypes.c_float), N, D, _p(lo, ctypes.c_float), _p(hi, ctypes.c_float))
    return lo, hi


def normalize(x: np.ndarray, w=None, normalize: bool = True) -> np.ndarray:
    x = _f32(x)
    N, D = x.shape
    w = None if w is None else _f32(w)
    F = np.zeros((N, D), np.float32)
    lib().orc_normalize(_p(x, ctypes.c_float), N, D, _p(w, ctypes.c_float), int(normalize),
                        _p(F, ctypes.c_float))
    return F


def scale_exp(x: np.ndarray, w=None, normalize: bool = True) -> int:
    x = _f32(x)
    N, D = x.shape
    w = None if w is None else _f32(w)
    return int(lib().orc_scale_exp(_p(x, ctypes.c_float), N, D, _p(w, ctypes.c_float),
                                   int(normalize)))


# --------------------------------------------------------------------------
# the sort
# --------------------------------------------------------------------------
def sort(x: np.ndarray, H: int, W: int, weights=None, seed: int = 0,
         sched: Schedule | None = None, perm_in=None, state: State | None = None,
         trace_cap: int = 1 << 16, want_target: bool = False) -> dict:
    """Run the sort (from scratch, or resumed from ``perm_in`` + ``state``).

    Returns dict(perm, state, trace_S, trace_level, iterations, T)."""
    x = _f32(x).reshape(H * W, -1)
    D = x.shape[1]
    s = sched or default_schedule()
    w = None if weights is None else _f32(weights)
    pin = None if perm_in is None else np.ascontiguousarray(perm_in, np.int32)
    st = State()
    resume = 0
    if state is not None:
        ctypes.memmove(ctypes.byref(st), ctypes.byref(state), ctypes.sizeof(State))
        resume = 1
    perm = np.zeros(H * W, np.int32)
    tS = np.full(trace_cap, -1, np.int64)
    tL = np.full(trace_cap, -1, np.int32)
    T = np.zeros((H, W, D), np.float32) if want_target else None
    ran = lib().orc_sort(_p(x, ctypes.c_float), H, W, D, _p(w, ctypes.c_float), seed,
                         ctypes.byref(s), _p(pin, ctypes.c_int32), resume, ctypes.byref(st),
                         _p(perm, ctypes.c_int32), _p(tS, ctypes.c_longlong),
                         _p(tL, ctypes.c_int), trace_cap, _p(T, ctypes.c_float))
    if ran < 0:
        raise ValueError("oracle sort rejected its arguments")
    it0 = (state.it if state is not None else 0)
    it1 = st.it
    return {"perm": perm, "state": st, "iterations": int(ran),
            "trace_S": tS[it0:min(it1, trace_cap)].copy(),
            "trace_level": tL[it0:min(it1, trace_cap)].copy(), "T": T}


def target(x: np.ndarray, H: int, W: int, perm, phi: float, weights=None,
           normalize_: bool = True, sigma_ratio: float = 2.0) -> np.ndarray:
    x = _f32(x).reshape(H * W, -1)
    D = x.shape[1]
    w = None if weights is None else _f32(weights)
    p = np.ascontiguousarray(perm, np.int32)
    T = np.zeros((H, W, D), np.float32)
    lib().orc_target(_p(x, ctypes.c_float), H, W, D, _p(w, ctypes.c_float), int(normalize_),
                     _p(p, ctypes.c_int32), phi, sigma_ratio, _p(T, ctypes.c_float))
    return T


def target_box(x: np.ndarray, H: int, W: int, perm, phi: float, weights=None,
               normalize_: bool = True) -> np.ndarray:
    """Box target (fixed-point window mean) of one arrangement -> [H, W, D]."""
    x = _f32(x).reshape(H * W, -1)
    D = x.shape[1]
    w = None if weights is None else _f32(weights)
    p = np.ascontiguousarray(perm, np.int32)
    T = np.zeros((H, W, D), np.float32)
    lib().orc_target_box(_p(x, ctypes.c_float), H, W, D, _p(w, ctypes.c_float), int(normalize_),
                         _p(p, ctypes.c_int32), phi, _p(T, ctypes.c_float))
    return T


def box_exp(x: np.ndarray, weights=None, normalize_: bool = True) -> int:
    x = _f32(x)
    n, D = x.shape
    w = None if weights is None else _f32(weights)
    return int(lib().orc_box_exp(_p(x, ctypes.c_float), n, D, _p(w, ctypes.c_float), int(normalize_)))


def gather(src: np.ndarray, perm) -> np.ndarray:
    src = _f32(src)
    N, C = src.shape
    p = np.ascontiguousarray(perm, np.int32)
    out = np.zeros((N, C), np.float32)
    lib().orc_gather(_p(src, ctypes.c_float), N, C, _p(p, ctypes.c_int32),
                     _p(out, ctypes.c_float))
    return out


def metrics(g: np.ndarray, scale: float = 1.0):
    """g: H x W x D grid -> (mean neighbour L2, VAD of values * scale)."""
    g = _f32(g)
    H, W, D = g.shape
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().orc_metrics(_p(g, ctypes.c_float), H, W, D, scale, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def smooth_taps64(sigma: float, ksize: int) -> np.ndarray:
    o = np.zeros(2 * (ksize // 2) + 1, np.float64)
    lib().orc_smooth_taps64(sigma, ksize, _p(o, ctypes.c_double))
    return o


def smooth_loss64(x: np.ndarray, sigma: float = 1.0, ksize: int = 7, lam=None,
                  grad_loss: float = 1.0, want_grad: bool = True, huber_delta: float = 0.0):
    """x: H x W x C (any float dtype, used in FP64) -> (loss, grad or None).
    huber_delta > 0 selects the Huber form of Sec. 3.2, else the squared form."""
    x = np.ascontiguousarray(x, np.float64)
    H, W, C = x.shape
    lam = None if lam is None else np.ascontiguousarray(lam, np.float64)
    g = np.zeros_like(x) if want_grad else None
    if huber_delta > 0:
        L = lib().orc_smooth_loss64_huber(_p(x, ctypes.c_double), H, W, C, sigma, ksize,
                                          _p(lam, ctypes.c_double), huber_delta, grad_loss,
                                          _p(g, ctypes.c_double))
    else:
        L = lib().orc_smooth_loss64(_p(x, ctypes.c_double), H, W, C, sigma, ksize,
                                    _p(lam, ctypes.c_double), grad_loss, _p(g, ctypes.c_double))
    return L, g


def activate_3dgs(raw: np.ndarray) -> np.ndarray:
    """Activated sort features [N, 14] of raw 3DGS parameters [N, >=14]."""
    raw = _f32(raw)
    n, stride = raw.shape
    out = np.zeros((n, 14), np.float32)
    lib().orc_activate_3dgs(_p(raw, ctypes.c_float), n, stride, _p(out, ctypes.c_float))
    return out


def grid_select(opacity_logit: np.ndarray):
    """(side, keep) of the largest square grid, keeping the highest opacities."""
    op = _f32(opacity_logit)
    n = op.shape[0]
    keep = np.zeros(max(n, 1), np.int32)
    side = lib().orc_grid_select(_p(op, ctypes.c_float), n, 1, _p(keep, ctypes.c_int))
    return side, keep[:side * side].copy()


def quantize(x: np.ndarray, lo, hi, q) -> np.ndarray:
    """Sec. 3.4 quantisation codes (uint16) of an [N, C] float32 array."""
    x = _f32(x)
    C = x.shape[-1]
    n = x.size // C
    lo_a, hi_a = _f32(lo), _f32(hi)
    q_a = np.ascontiguousarray(q, np.int32)
    out = np.zeros(x.shape, np.uint16)
    lib().orc_quantize(_p(x, ctypes.c_float), n, C, _p(lo_a, ctypes.c_float),
                       _p(hi_a, ctypes.c_float), _p(q_a, ctypes.c_int),
                       _p(out, ctypes.c_ushort))
    return out


def dequantize(codes: np.ndarray, lo, hi, q) -> np.ndarray:
    """Sec. 3.4: the float32 value of each code of an [N, C] uint16 array."""
    codes = np.ascontiguousarray(codes, np.uint16)
    C = codes.shape[-1]
    n = codes.size // C
    lo_a, hi_a = _f32(lo), _f32(hi)
    q_a = np.ascontiguousarray(q, np.int32)
    out = np.zeros(codes.shape, np.float32)
    lib().orc_dequantize(_p(codes, ctypes.c_ushort), n, C, _p(lo_a, ctypes.c_float),
                         _p(hi_a, ctypes.c_float), _p(q_a, ctypes.c_int), _p(out, ctypes.c_float))
    return out


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops (results do not depend on it)."""
    lib().orc_set_num_threads(int(n))
