"""GB300 (sm_103a) Parallel Linear Assignment Sorting and grid smoothness loss.

Python binding of the C ABI in ``include/plas.h`` (Morgenstern et al., "Compact
3D Scene Representation via Self-Organizing Gaussian Grids", arXiv 2312.13299,
Sec. 3.1 and 3.2).  This module only marshals arguments: PyTorch provides
device memory and the current CUDA stream, and every step of the sort and of
the loss runs in the library's own CUDA kernels.  There is no CPU fallback; a
missing library raises.

Main entry points
    sort(x, H, W, ...)          PLAS grid sort -> permutation (+ carried attributes)
    batch_sort(jobs, ...)       many independent grids with one schedule
    smooth_loss(x, ...)         Sec. 3.2 smoothness loss with a hand-written backward
    grid_metrics(g, scale)      mean neighbour L2 and VAD of a grid
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field, fields
from typing import Optional, Sequence

import torch

from . import _lib
from ._lib import check, load

__all__ = ["Schedule", "SortResult", "sort", "batch_sort", "Server", "gather_rows", "target",
           "group_permutation", "philox", "grid_metrics", "smooth_loss", "SmoothLoss",
           "num_levels", "sort_workspace_bytes", "check_permutation", "load"]


@dataclass
class Schedule:
    """Mirror of ``plas_schedule`` (Sec. 3.1 defaults; sigma_ratio is a reading)."""
    phi0: float = 0.0
    shrink: float = 0.95
    phi_min: float = 1.0
    tol: float = 1e-4
    sigma_ratio: float = 2.0
    min_block: int = 16
    shuffle_init: bool = True
    normalize: bool = True
    iters_per_poll: int = 8
    max_iters: int = 0
    profile: bool = False
    graphs: bool = True
    target_mode: int = 0  # 0 Gaussian target, 1 box target (fast low-pass variant)
    persistent: int = 0   # 1: one cooperative launch per batch of sweeps; 0 / -1: graph-replayed launches
    whole_blocks: bool = False  # True: only whole blocks take part (not those cut by the border)
    checked: bool = False  # guard bands around workspace regions + device bounds checks

    def to_c(self, trace_S: Optional[torch.Tensor] = None,
             trace_level: Optional[torch.Tensor] = None) -> _lib.plas_schedule:
        s = _lib.plas_schedule()
        s.phi0, s.shrink, s.phi_min, s.tol = self.phi0, self.shrink, self.phi_min, self.tol
        s.sigma_ratio, s.min_block = self.sigma_ratio, self.min_block
        s.shuffle_init, s.normalize = int(self.shuffle_init), int(self.normalize)
        s.iters_per_poll, s.max_iters, s.profile = self.iters_per_poll, self.max_iters, int(self.profile)
        s.graphs = int(self.graphs)
        s.target_mode = int(self.target_mode)
        s.persistent = int(self.persistent)
        s.checked = int(self.checked)
        s.whole_blocks = int(self.whole_blocks)
        s.trace_S = trace_S.data_ptr() if trace_S is not None else None
        s.trace_level = trace_level.data_ptr() if trace_level is not None else None
        cap = 0
        if trace_S is not None:
            cap = trace_S.numel()
        if trace_level is not None:
            cap = min(cap, trace_level.numel()) if trace_S is not None else trace_level.numel()
        s.trace_cap = cap
        return s


@dataclass
class SortResult:
    perm: torch.Tensor
    carried: Optional[torch.Tensor] = None
    sorted: Optional[torch.Tensor] = None
    state: dict = field(default_factory=dict)
    stats: Optional[dict] = None
    trace_S: Optional[torch.Tensor] = None
    trace_level: Optional[torch.Tensor] = None


def _stream(dev: torch.device) -> int:
    return torch.cuda.current_stream(dev).cuda_stream


def _need_cuda(t: torch.Tensor, name: str, dtype=torch.float32) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}")
    return t.contiguous()


def _weights(weights, D: int):
    if weights is None:
        return None
    w = [float(v) for v in (weights.tolist() if isinstance(weights, torch.Tensor) else weights)]
    if len(w) != D:
        raise ValueError(f"weights must have {D} entries")
    return (ctypes.c_float * D)(*w)


def _state_to_c(state) -> _lib.plas_state:
    st = _lib.plas_state()
    if state is None:
        return st
    if isinstance(state, _lib.plas_state):
        ctypes.memmove(ctypes.byref(st), ctypes.byref(state), ctypes.sizeof(st))
        return st
    for k, _ in _lib.plas_state._fields_:
        if k in state:
            setattr(st, k, state[k])
    return st


def _stats_to_dict(s: _lib.plas_stats) -> dict:
    d = {k: getattr(s, k) for k, _ in _lib.plas_stats._fields_ if k != "kernel"}
    d["kernels"] = {n: {"launches": s.kernel[i].launches, "ms": s.kernel[i].ms,
                        "bytes": s.kernel[i].bytes, "flops": s.kernel[i].flops}
                    for i, n in enumerate(_lib.KERNEL_NAMES)}
    return d


def num_levels(H: int, W: int, schedule: Optional[Schedule] = None) -> int:
    s = (schedule or Schedule()).to_c()
    n = load().plas_num_levels(H, W, ctypes.byref(s))
    if n < 0:
        check(n, "plas_num_levels")
    return n


def sort_workspace_bytes(H: int, W: int, D: int, schedule: Optional[Schedule] = None) -> int:
    if schedule is None:
        return int(load().plas_sort_workspace_bytes(H, W, D))
    s = schedule.to_c()
    return int(load().plas_sort_workspace_bytes_ex(H, W, D, ctypes.byref(s)))


def sort(x: torch.Tensor, H: int, W: int, weights=None, carried: Optional[torch.Tensor] = None,
         seed: int = 0, schedule: Optional[Schedule] = None,
         perm_init: Optional[torch.Tensor] = None, state=None, want_sorted: bool = False,
         want_stats: bool = False, trace_cap: int = 0,
         workspace: Optional[torch.Tensor] = None, check_perm: bool = False) -> SortResult:
    """PLAS grid sort (Sec. 3.1): x [N, D] float32 on a CUDA device, N = H*W.

    Returns the permutation (perm[p] = row of x placed at grid cell p), the
    carried attributes in grid order, optionally x in grid order, the final
    schedule state (resumable together with the permutation), statistics and
    a per-iteration trace of the fixed-point residual sum.  check_perm=True
    verifies on the device that perm is a bijection (plas_check_permutation)
    and raises PlasError with status PLAS_ERR_NOT_PERMUTATION if not."""
    lib = load()
    x = _need_cuda(x, "x")
    if x.dim() != 2 or x.shape[0] != H * W:
        raise ValueError("x must be [H*W, D]")
    N, D = x.shape
    dev = x.device
    sched = schedule or Schedule()
    perm = torch.empty(N, dtype=torch.int32, device=dev)
    C = 0
    carried_out = None
    if carried is not None:
        carried = _need_cuda(carried, "carried")
        if carried.dim() != 2 or carried.shape[0] != N:
            raise ValueError("carried must be [N, C]")
        C = carried.shape[1]
        carried_out = torch.empty_like(carried)
    sorted_out = torch.empty_like(x) if want_sorted else None
    if perm_init is not None:
        perm_init = _need_cuda(perm_init, "perm_init", torch.int32)
    tS = tL = None
    if trace_cap > 0:
        tS = torch.full((trace_cap,), -1, dtype=torch.int64, device=dev)
        tL = torch.full((trace_cap,), -1, dtype=torch.int32, device=dev)
    cs = sched.to_c(tS, tL)
    st = _state_to_c(state)
    stats = _lib.plas_stats() if want_stats else None
    ws_ptr, ws_bytes = None, 0
    if workspace is not None:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    with torch.cuda.device(dev):
        rc = lib.plas_sort(x.data_ptr(), H, W, D, _weights(weights, D),
                           carried.data_ptr() if carried is not None else None, C, seed,
                           ctypes.byref(cs), perm_init.data_ptr() if perm_init is not None else None,
                           ctypes.byref(st), perm.data_ptr(),
                           carried_out.data_ptr() if carried_out is not None else None,
                           sorted_out.data_ptr() if sorted_out is not None else None,
                           ws_ptr, ws_bytes, ctypes.byref(stats) if stats is not None else None,
                           _stream(dev))
    check(rc, "plas_sort")
    if check_perm and check_permutation(perm) >= 0:
        raise _lib.PlasError(_lib.PLAS_ERR_NOT_PERMUTATION, "plas_sort")
    res = SortResult(perm=perm, carried=carried_out, sorted=sorted_out, state=st.as_dict(),
                     stats=_stats_to_dict(stats) if stats is not None else None)
    if tS is not None:
        it0 = int(state["it"]) if isinstance(state, dict) and "it" in state else 0
        it1 = min(st.it, trace_cap)
        res.trace_S = tS[it0:it1]
        res.trace_level = tL[it0:it1]
    return res


def check_permutation(perm: torch.Tensor) -> int:
    """Bijection check on the device (Sec. 3.1: the sort places every Gaussian
    on exactly one cell).  perm: int32 CUDA tensor of N values.  Returns -1 if
    perm is a permutation of [0, N), else the smallest position whose value is
    out of range or occurs more than once."""
    lib = load()
    perm = _need_cuda(perm, "perm", torch.int32).reshape(-1)
    first = ctypes.c_int(-1)
    with torch.cuda.device(perm.device):
        rc = lib.plas_check_permutation(perm.data_ptr() if perm.numel() else None, perm.numel(),
                                        ctypes.byref(first), _stream(perm.device))
    if rc == _lib.PLAS_ERR_NOT_PERMUTATION:
        return first.value
    check(rc, "plas_check_permutation")
    return -1


def batch_sort(jobs: Sequence[dict], weights=None, schedule: Optional[Schedule] = None,
               workspace: Optional[torch.Tensor] = None) -> list:
    """Sort many independent grids (all with the same D) in one call.

    jobs: dicts with x [H*W, D], H, W, optional carried [H*W, C] and seed.
    Returns a list of SortResult (perm, carried, state)."""
    lib = load()
    if not jobs:
        return []
    D = int(jobs[0]["x"].shape[1])
    dev = jobs[0]["x"].device
    arr = (_lib.plas_job * len(jobs))()
    states = [_lib.plas_state() for _ in jobs]
    outs = []
    keep = []
    for i, j in enumerate(jobs):
        x = _need_cuda(j["x"], "x")
        H, W = int(j["H"]), int(j["W"])
        if x.shape != (H * W, D):
            raise ValueError("every job's x must be [H*W, D] with the same D")
        perm = torch.empty(H * W, dtype=torch.int32, device=dev)
        car = j.get("carried")
        cout = None
        if car is not None:
            car = _need_cuda(car, "carried")
            cout = torch.empty_like(car)
        keep += [x, car]
        arr[i].x, arr[i].H, arr[i].W = x.data_ptr(), H, W
        arr[i].carried = car.data_ptr() if car is not None else None
        arr[i].C = car.shape[1] if car is not None else 0
        arr[i].seed = int(j.get("seed", 0))
        arr[i].perm_out = perm.data_ptr()
        arr[i].carried_out = cout.data_ptr() if cout is not None else None
        arr[i].state_out = ctypes.pointer(states[i])
        outs.append((perm, cout))
    cs = (schedule or Schedule()).to_c()
    ws_ptr, ws_bytes = None, 0
    if workspace is not None:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    with torch.cuda.device(dev):
        rc = lib.plas_batch_sort(len(jobs), arr, D, _weights(weights, D), ctypes.byref(cs), ws_ptr,
                                 ws_bytes, _stream(dev))
    check(rc, "plas_batch_sort")
    return [SortResult(perm=p, carried=c, state=s.as_dict()) for (p, c), s in zip(outs, states)]


def _tuning_dict(t: "_lib.plas_tuning") -> dict:
    n = t.n_radii
    return {"fir_small_below": t.fir_small_below, "fir_medium_below": t.fir_medium_below,
            "assign_ctas_per_sm": t.assign_ctas_per_sm,
            "radius": list(t.radius[:n]), "fir_small_us": [round(v, 2) for v in t.fir_small_us[:n]],
            "fir_medium_us": [round(v, 2) for v in t.fir_medium_us[:n]],
            "fir_large_us": [round(v, 2) for v in t.fir_large_us[:n]],
            "assign_per_sm": list(t.assign_per_sm) if n else [],
            "assign_us": [round(v, 2) for v in t.assign_us] if n else [],
            "large_tma": int(t.large_tma),
            "fir_large_ring_us": [round(v, 2) for v in t.fir_large_ring_us[:n]],
            "fir_large_tma_us": [round(v, 2) for v in t.fir_large_tma_us[:n]],
            "small_fused": int(t.small_fused)}


def autotune(H: int, W: int, D: int, device=None) -> dict:
    """Time the launch-shape candidates (FIR tiling per radius, assignment CTAs
    per SM) on a synthetic H x W x D grid and install the fastest for sorts of
    this shape on this device.  Results of a sort never depend on them."""
    dev = torch.device(device) if device is not None else torch.device(
        "cuda", torch.cuda.current_device())
    t = _lib.plas_tuning()
    with torch.cuda.device(dev):
        check(load().plas_autotune(H, W, D, _stream(dev), ctypes.byref(t)), "plas_autotune")
    return _tuning_dict(t)


def set_tuning(H: int, W: int, D: int, fir_small_below: Optional[int] = None,
               assign_ctas_per_sm: Optional[int] = None,
               fir_medium_below: Optional[int] = None, large_tma: Optional[bool] = None,
               small_fused: Optional[bool] = None) -> None:
    """Install launch shapes for (H, W, D) on the current device; with every
    argument None the entry is removed (defaults apply again).  A radius r
    takes the small-radius path when r < fir_small_below (both passes in one
    launch when small_fused is set, r <= 11 and D <= 16, else the direct
    kernel), else the 64-row one when r < fir_medium_below, else the 128-row
    one (with tensor copies when large_tma is set and the grid allows it)."""
    if (fir_small_below is None and assign_ctas_per_sm is None and fir_medium_below is None
            and large_tma is None and small_fused is None):
        check(load().plas_set_tuning(H, W, D, None), "plas_set_tuning")
        return
    cur = get_tuning(H, W, D)
    t = _lib.plas_tuning()
    t.fir_small_below = cur["fir_small_below"] if fir_small_below is None else fir_small_below
    t.fir_medium_below = cur["fir_medium_below"] if fir_medium_below is None else fir_medium_below
    t.assign_ctas_per_sm = (cur["assign_ctas_per_sm"] if assign_ctas_per_sm is None
                            else assign_ctas_per_sm)
    t.large_tma = cur["large_tma"] if large_tma is None else int(bool(large_tma))
    t.small_fused = cur["small_fused"] if small_fused is None else int(bool(small_fused))
    check(load().plas_set_tuning(H, W, D, ctypes.byref(t)), "plas_set_tuning")


def get_tuning(H: int, W: int, D: int) -> dict:
    t = _lib.plas_tuning()
    check(load().plas_get_tuning(H, W, D, ctypes.byref(t)), "plas_get_tuning")
    return _tuning_dict(t)


class Server:
    """Continuous batching of sort requests (plas_server_*): requests queue up,
    are admitted while their workspaces fit the device-memory budget, and
    advance together one iteration per sweep; 'policy' picks which admitted
    grids each step advances (fifo_fill, shortest_first, all), or runs every
    admitted request on a prioritised stream of its own (concurrent).  Results equal
    sort() of each request alone under every policy.  All work runs on the
    stream current at construction."""

    POLICIES = {"fifo_fill": 0, "shortest_first": 1, "all": 2, "concurrent": 3, "adaptive": 4}

    def __init__(self, D: int, weights=None, schedule: Optional[Schedule] = None,
                 mem_budget: int = 0, device=None, policy: Optional[str] = None):
        self._lib = load()
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.D = D
        self._w = _weights(weights, D)
        self._sched = (schedule or Schedule()).to_c()
        self._stream = _stream(self.device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = self._lib.plas_server_create(D, self._w, ctypes.byref(self._sched), mem_budget,
                                              self._stream, ctypes.byref(h))
        check(rc, "plas_server_create")
        self._h = h
        self._live = {}
        self._cancelled = []  # (step number, tensors) kept until that step's work has run
        self._steps = 0
        if policy is None:  # the box target is served by one lane per request
            policy = "concurrent" if (schedule and schedule.target_mode == 1) else "fifo_fill"
        if policy not in self.POLICIES:
            self.close()
            raise ValueError(f"policy must be one of {sorted(self.POLICIES)}")
        check(self._lib.plas_server_set_policy(self._h, self.POLICIES[policy]),
              "plas_server_set_policy")

    def _lib_policy(self, policy: str) -> None:
        """Change the scheduling policy (the concurrent policy can only be
        entered or left while nothing is admitted)."""
        if policy not in self.POLICIES:
            raise ValueError(f"policy must be one of {sorted(self.POLICIES)}")
        check(self._lib.plas_server_set_policy(self._h, self.POLICIES[policy]),
              "plas_server_set_policy")

    def submit(self, x: torch.Tensor, H: int, W: int, carried: Optional[torch.Tensor] = None,
               seed: int = 0) -> int:
        x = _need_cuda(x, "x")
        if x.shape != (H * W, self.D):
            raise ValueError("x must be [H*W, D]")
        perm = torch.empty(H * W, dtype=torch.int32, device=x.device)
        cout = None
        if carried is not None:
            carried = _need_cuda(carried, "carried")
            cout = torch.empty_like(carried)
        st = _lib.plas_state()
        job = _lib.plas_job()
        job.x, job.H, job.W = x.data_ptr(), H, W
        job.carried = carried.data_ptr() if carried is not None else None
        job.C = carried.shape[1] if carried is not None else 0
        job.seed = seed
        job.perm_out = perm.data_ptr()
        job.carried_out = cout.data_ptr() if cout is not None else None
        job.state_out = ctypes.pointer(st)
        t = ctypes.c_longlong()
        with torch.cuda.device(self.device):
            rc = self._lib.plas_server_submit(self._h, ctypes.byref(job), ctypes.byref(t))
        check(rc, "plas_server_submit")
        self._live[t.value] = (x, carried, perm, cout, st)
        return t.value

    def step(self, sweeps: int = 8) -> list:
        """Run up to 'sweeps' sweeps; returns [(ticket, SortResult)] of finished requests."""
        cap = max(1, len(self._live))
        done = (ctypes.c_longlong * cap)()
        n = ctypes.c_int()
        with torch.cuda.device(self.device):
            rc = self._lib.plas_server_step(self._h, sweeps, done, cap, ctypes.byref(n))
        check(rc, "plas_server_step")
        self._steps += 1
        self._cancelled = [c for c in self._cancelled if c[0] + 2 > self._steps]
        out = []
        for i in range(n.value):
            x, car, perm, cout, st = self._live.pop(done[i])
            out.append((done[i], SortResult(perm=perm, carried=cout, state=st.as_dict())))
        return out

    def cancel(self, ticket: int) -> None:
        """Withdraw a queued or running request (plas_server_cancel); it is
        never reported by step().  Raises PlasError for a ticket that is
        unknown, finished or already cancelled."""
        check(self._lib.plas_server_cancel(self._h, ticket), "plas_server_cancel")
        # the request's tensors stay referenced until work enqueued before
        # the cancellation has run
        self._cancelled.append((self._steps, self._live.pop(ticket)))

    def status(self):
        q, a, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        check(self._lib.plas_server_status(self._h, ctypes.byref(q), ctypes.byref(a),
                                           ctypes.byref(m)), "plas_server_status")
        return q.value, a.value, m.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.plas_server_destroy(self._h)
            self._h = None
            self._live.clear()
            self._cancelled.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gather_rows(src: torch.Tensor, perm: torch.Tensor) -> torch.Tensor:
    """out[p] = src[perm[p]] on the device (every attribute follows the permutation)."""
    src = _need_cuda(src, "src")
    perm = _need_cuda(perm, "perm", torch.int32)
    src2 = src.reshape(src.shape[0], -1)
    out = torch.empty_like(src2)
    with torch.cuda.device(src.device):
        rc = load().plas_gather_rows(src2.data_ptr(), src2.shape[0], src2.shape[1], perm.data_ptr(),
                                     out.data_ptr(), _stream(src.device))
    check(rc, "plas_gather_rows")
    return out.reshape(src.shape)


def select_rows(src: torch.Tensor, idx: torch.Tensor) -> torch.Tensor:
    """out[p] = src[idx[p]] for a subset of rows (e.g. the kept Gaussians)."""
    src = _need_cuda(src, "src")
    idx = _need_cuda(idx, "idx", torch.int32)
    src2 = src.reshape(src.shape[0], -1)
    out = torch.empty((idx.numel(), src2.shape[1]), dtype=torch.float32, device=src.device)
    with torch.cuda.device(src.device):
        rc = load().plas_select_rows(src2.data_ptr(), src2.shape[0], src2.shape[1], idx.data_ptr(),
                                     idx.numel(), out.data_ptr(), _stream(src.device))
    check(rc, "plas_select_rows")
    return out.reshape((idx.numel(),) + tuple(src.shape[1:]))


def target(x: torch.Tensor, H: int, W: int, perm: torch.Tensor, phi: float, weights=None,
           normalize: bool = True, sigma_ratio: float = 2.0) -> torch.Tensor:
    """Low-pass target of one arrangement (the blur step of Sec. 3.1) -> [H, W, D]."""
    x = _need_cuda(x, "x")
    perm = _need_cuda(perm, "perm", torch.int32)
    N, D = x.shape
    T = torch.empty((H, W, D), dtype=torch.float32, device=x.device)
    with torch.cuda.device(x.device):
        rc = load().plas_target(x.data_ptr(), H, W, D, _weights(weights, D), int(normalize),
                                perm.data_ptr(), float(phi), float(sigma_ratio), T.data_ptr(),
                                _stream(x.device))
    check(rc, "plas_target")
    return T


def target_box(x: torch.Tensor, H: int, W: int, perm: torch.Tensor, phi: float, weights=None,
               normalize: bool = True) -> torch.Tensor:
    """Box target (schedule.target_mode = 1) of one arrangement -> [H, W, D]."""
    x = _need_cuda(x, "x")
    perm = _need_cuda(perm, "perm", torch.int32)
    N, D = x.shape
    T = torch.empty((H, W, D), dtype=torch.float32, device=x.device)
    with torch.cuda.device(x.device):
        rc = load().plas_target_box(x.data_ptr(), H, W, D, _weights(weights, D), int(normalize),
                                    perm.data_ptr(), float(phi), T.data_ptr(), _stream(x.device))
    check(rc, "plas_target_box")
    return T


def group_permutation(seed: int, tag: int, counter: int, n: int,
                      device="cuda") -> torch.Tensor:
    """Keyed permutation of [0, n) as int32 tensor (bits of the uint32 values)."""
    out = torch.empty(n, dtype=torch.int32, device=device)
    with torch.cuda.device(out.device):
        rc = load().plas_group_permutation(seed, tag, counter, n, out.data_ptr(),
                                           _stream(out.device))
    check(rc, "plas_group_permutation")
    return out


def philox(ctr: torch.Tensor, key0: int, key1: int) -> torch.Tensor:
    """Philox4x32-10 of n counters ([n, 4] int32 bit patterns) -> [n, 4] int32."""
    ctr = _need_cuda(ctr, "ctr", torch.int32)
    out = torch.empty_like(ctr)
    with torch.cuda.device(ctr.device):
        rc = load().plas_philox(ctr.data_ptr(), key0, key1, ctr.shape[0], out.data_ptr(),
                                _stream(ctr.device))
    check(rc, "plas_philox")
    return out


def grid_metrics(grid: torch.Tensor, scale: float = 1.0):
    """(mean neighbour L2, VAD of values*scale, mean |diff|*scale) of [H, W, D]."""
    grid = _need_cuda(grid, "grid")
    H, W, D = grid.shape
    out = (ctypes.c_double * 3)()
    with torch.cuda.device(grid.device):
        rc = load().plas_grid_metrics(grid.data_ptr(), H, W, D, float(scale), out,
                                      _stream(grid.device))
    check(rc, "plas_grid_metrics")
    return out[0], out[1], out[2]


def activate_3dgs(raw: torch.Tensor) -> torch.Tensor:
    """Raw 3DGS parameters [N, >=14] (contracted xyz, log-scale, quaternion,
    opacity logit, DC) -> activated sort features [N, 14] (Sec. 3.1)."""
    raw = _need_cuda(raw, "raw")
    if raw.dim() != 2 or raw.shape[1] < 14 or raw.stride(1) != 1:
        raise ValueError("raw must be [N, >=14] with unit column stride")
    out = torch.empty((raw.shape[0], 14), dtype=torch.float32, device=raw.device)
    with torch.cuda.device(raw.device):
        rc = load().plas_activate_3dgs(raw.data_ptr(), raw.shape[0], raw.stride(0), out.data_ptr(),
                                       _stream(raw.device))
    check(rc, "plas_activate_3dgs")
    return out


def grid_select(opacity_logit: torch.Tensor):
    """Largest square grid (Sec. 3.1): returns (side, keep) with keep the
    int32 indices of the side^2 highest-opacity Gaussians, ascending.
    opacity_logit: a 1-D CUDA float32 tensor (any element stride)."""
    op = opacity_logit
    if not isinstance(op, torch.Tensor) or not op.is_cuda or op.dtype != torch.float32 or op.dim() != 1:
        raise ValueError("opacity_logit must be a 1-D float32 CUDA tensor")
    n = op.shape[0]
    side = math.isqrt(n)
    keep = torch.empty(side * side, dtype=torch.int32, device=op.device)
    s = ctypes.c_int()
    with torch.cuda.device(op.device):
        rc = load().plas_grid_select(op.data_ptr(), n, op.stride(0), keep.data_ptr(), ctypes.byref(s),
                                     None, 0, _stream(op.device))
    check(rc, "plas_grid_select")
    assert s.value == side
    return side, keep


def _quant_args(C, lo, hi, q):
    lo_a = (ctypes.c_float * C)(*[float(v) for v in lo])
    hi_a = (ctypes.c_float * C)(*[float(v) for v in hi])
    q_a = (ctypes.c_int * C)(*[int(v) for v in q])
    return lo_a, hi_a, q_a


def quantize(x: torch.Tensor, lo, hi, q) -> torch.Tensor:
    """Sec. 3.4 quantisation of an [N, C] (or [..., C]) float32 grid: clip
    channel c to [lo[c], hi[c]] and round to the nearest of q[c] levels.
    Returns the codes as int16 storage holding uint16 values (view with
    .to(torch.int32) & 0xFFFF to read them)."""
    x = _need_cuda(x, "x")
    C = x.shape[-1]
    N = x.numel() // C
    codes = torch.empty(x.shape, dtype=torch.int16, device=x.device)
    lo_a, hi_a, q_a = _quant_args(C, lo, hi, q)
    with torch.cuda.device(x.device):
        rc = load().plas_quantize(x.data_ptr(), N, C, lo_a, hi_a, q_a, codes.data_ptr(),
                                  _stream(x.device))
    check(rc, "plas_quantize")
    return codes


def dequantize(codes: torch.Tensor, lo, hi, q) -> torch.Tensor:
    codes = _need_cuda(codes, "codes", torch.int16)
    C = codes.shape[-1]
    N = codes.numel() // C
    out = torch.empty(codes.shape, dtype=torch.float32, device=codes.device)
    lo_a, hi_a, q_a = _quant_args(C, lo, hi, q)
    with torch.cuda.device(codes.device):
        rc = load().plas_dequantize(codes.data_ptr(), N, C, lo_a, hi_a, q_a, out.data_ptr(),
                                    _stream(codes.device))
    check(rc, "plas_dequantize")
    return out


def _lam_ptr(lam: Optional[torch.Tensor]):
    return lam.data_ptr() if lam is not None else None


def smooth_loss_fwd(x: torch.Tensor, sigma: float = 1.0, ksize: int = 7,
                    lam: Optional[torch.Tensor] = None, huber_delta: float = 0.0) -> torch.Tensor:
    """Sec. 3.2 smoothness loss of an [H, W, C] grid (squared form, or the
    Huber form when huber_delta > 0)."""
    x = _need_cuda(x, "x")
    H, W, C = x.shape
    if lam is not None:
        lam = _need_cuda(lam, "lam")
    loss = torch.empty((), dtype=torch.float32, device=x.device)
    with torch.cuda.device(x.device):
        rc = load().plas_smooth_loss_fwd_ex(x.data_ptr(), H, W, C, float(sigma), int(ksize),
                                            _lam_ptr(lam), float(huber_delta), loss.data_ptr(),
                                            None, 0, _stream(x.device))
    check(rc, "plas_smooth_loss_fwd_ex")
    return loss


def smooth_loss_bwd(x: torch.Tensor, grad_loss: torch.Tensor, sigma: float = 1.0,
                    ksize: int = 7, lam: Optional[torch.Tensor] = None,
                    huber_delta: float = 0.0) -> torch.Tensor:
    x = _need_cuda(x, "x")
    H, W, C = x.shape
    if lam is not None:
        lam = _need_cuda(lam, "lam")
    g = _need_cuda(grad_loss.reshape(()).to(torch.float32), "grad_loss")
    grad = torch.empty_like(x)
    with torch.cuda.device(x.device):
        rc = load().plas_smooth_loss_bwd_ex(x.data_ptr(), H, W, C, float(sigma), int(ksize),
                                            _lam_ptr(lam), float(huber_delta), g.data_ptr(),
                                            grad.data_ptr(), None, 0, _stream(x.device))
    check(rc, "plas_smooth_loss_bwd_ex")
    return grad


class SmoothLoss(torch.autograd.Function):
    """Sec. 3.2 smoothness loss L = mean(lam_c h(x - Bx)), h the squared
    deviation or (huber_delta > 0) the Huber penalty, with a hand-written
    backward kernel.  x: [H, W, C] float32 CUDA, channel-last."""

    @staticmethod
    def forward(ctx, x, sigma=1.0, ksize=7, lam=None, huber_delta=0.0):
        ctx.sigma, ctx.ksize, ctx.huber_delta = sigma, ksize, huber_delta
        ctx.save_for_backward(x, lam) if lam is not None else ctx.save_for_backward(x)
        ctx.has_lam = lam is not None
        return smooth_loss_fwd(x, sigma, ksize, lam, huber_delta)

    @staticmethod
    def backward(ctx, g):
        if ctx.has_lam:
            x, lam = ctx.saved_tensors
        else:
            (x,), lam = ctx.saved_tensors, None
        return (smooth_loss_bwd(x, g, ctx.sigma, ctx.ksize, lam, ctx.huber_delta),
                None, None, None, None)


def smooth_loss(x: torch.Tensor, sigma: float = 1.0, ksize: int = 7,
                lam: Optional[torch.Tensor] = None, huber_delta: float = 0.0) -> torch.Tensor:
    return SmoothLoss.apply(x, sigma, ksize, lam, huber_delta)
