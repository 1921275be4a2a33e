"""Failure handling on the GPU path, with every failure made on the host.

plas_debug_inject makes the library's n-th device allocation fail as if the
device were out of memory, or freezes the sweep engine's state read-backs so
that its progress check sees grids that do not advance.  Neither touches the
GPU.  Each case checks the status the call returns, that device memory does
not leak over repeated failures, and that the next call (injection cleared)
gives the oracle's result again."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2312_13299_gb300 import synth

pytestmark = pytest.mark.gpu

PLAS_ERR_OOM, PLAS_ERR_INTERNAL = -2, -7


@pytest.fixture(autouse=True)
def _clear(plas):
    yield
    plas.load().plas_debug_inject(0, 0)


def _used():
    torch.cuda.synchronize()
    free, total = torch.cuda.mem_get_info()
    return total - free


def _status(e):
    return getattr(e, "code", None)


def test_allocation_failure_of_a_sort(plas, orc):
    """The workspace allocation of plas_sort fails: PLAS_ERR_OOM, nothing
    leaks over 30 failed calls, and the next call sorts correctly."""
    lib = plas.load()
    x = synth.rgb_uniform(40, seed=3)
    xc = torch.from_numpy(x).cuda()
    plas.sort(xc, 40, 40, seed=3)  # warm the allocator and the graph
    base = _used()
    for _ in range(30):
        assert lib.plas_debug_inject(1, 1) == 0
        with pytest.raises(RuntimeError) as e:
            plas.sort(xc, 40, 40, seed=3)
        assert _status(e.value) == PLAS_ERR_OOM
    assert _used() - base < 64 << 20
    got = plas.sort(xc, 40, 40, seed=3)
    assert np.array_equal(got.perm.cpu().numpy(), orc.sort(x, 40, 40, seed=3)["perm"])


@pytest.mark.parametrize("nth", [1, 2])
def test_allocation_failure_in_batches(plas, nth):
    """plas_batch_sort without a caller workspace: its first (workspace) or
    second (descriptor array) allocation fails with PLAS_ERR_OOM; a rerun
    gives the same results as the grids sorted alone."""
    lib = plas.load()
    jobs = []
    for i, (H, W) in enumerate([(24, 24), (17, 40)]):
        x, c = synth.gaussians_3dgs(H * W, seed=i)
        jobs.append({"x": torch.from_numpy(x).cuda(), "H": H, "W": W,
                     "carried": torch.from_numpy(c).cuda(), "seed": i})
    lib.plas_debug_inject(1, nth)
    failed = False
    try:
        plas.batch_sort(jobs)
    except RuntimeError as e:
        assert _status(e) == PLAS_ERR_OOM
        failed = True
    assert failed or nth > 1  # the first allocation always exists
    lib.plas_debug_inject(0, 0)
    res = plas.batch_sort(jobs)
    for j, r in zip(jobs, res):
        one = plas.sort(j["x"], j["H"], j["W"], carried=j["carried"], seed=j["seed"])
        assert torch.equal(r.perm, one.perm)


@pytest.mark.parametrize("policy", ["fifo_fill", "concurrent"])
def test_server_admission_allocation_failure(plas, policy):
    """With nothing running, a failed workspace allocation at admission is an
    error of that step; the queued request is admitted at a later step."""
    lib = plas.load()
    x, c = synth.gaussians_3dgs(32 * 32, seed=7)
    xc, cc = torch.from_numpy(x).cuda(), torch.from_numpy(c).cuda()
    srv = plas.Server(14, policy=policy)
    t = srv.submit(xc, 32, 32, cc, seed=7)
    lib.plas_debug_inject(1, 1)
    with pytest.raises(RuntimeError):
        srv.step(sweeps=4)
    lib.plas_debug_inject(0, 0)
    results = {}
    while t not in results:
        results.update(srv.step(sweeps=8))
    srv.close()
    one = plas.sort(xc, 32, 32, carried=cc, seed=7)
    assert torch.equal(results[t].perm, one.perm)


def test_progress_check_fires_on_frozen_read_backs(plas, orc):
    """Frozen state read-backs make a healthy grid look stalled: plas_sort
    returns PLAS_ERR_INTERNAL (the host's progress check), releases its
    memory, and the next call is correct."""
    lib = plas.load()
    x = synth.rgb_uniform(48, seed=5)
    xc = torch.from_numpy(x).cuda()
    plas.sort(xc, 48, 48, seed=5)
    base = _used()
    for _ in range(5):
        assert lib.plas_debug_inject(2, 1000) == 0
        with pytest.raises(RuntimeError) as e:
            plas.sort(xc, 48, 48, seed=5)
        assert _status(e.value) == PLAS_ERR_INTERNAL and "progress" in str(e.value)
        lib.plas_debug_inject(0, 0)
    assert _used() - base < 64 << 20
    got = plas.sort(xc, 48, 48, seed=5)
    assert np.array_equal(got.perm.cpu().numpy(), orc.sort(x, 48, 48, seed=5)["perm"])


def test_injection_arguments(plas):
    lib = plas.load()
    assert lib.plas_debug_inject(1, 0) == -1
    assert lib.plas_debug_inject(9, 1) == -1
    assert lib.plas_debug_inject(0, 0) == 0


def test_persistent_sweep_barrier_timeout(plas):
    """A zero wait limit at the persistent sweep's grid barriers (injected on
    the host): the first wait gives up, the launch ends and the call returns
    PLAS_ERR_TIMEOUT; the GPU stays usable and the next batch is correct."""
    lib = plas.load()
    jobs = []
    for i, (H, W) in enumerate([(40, 40), (33, 48), (64, 20)]):
        x, c = synth.gaussians_3dgs(H * W, seed=20 + i)
        jobs.append({"x": torch.from_numpy(x).cuda(), "H": H, "W": W,
                     "carried": torch.from_numpy(c).cuda(), "seed": i})
    sched = plas.Schedule(persistent=1)
    assert lib.plas_debug_inject(3, 1) == 0
    with pytest.raises(RuntimeError) as e:
        plas.batch_sort(jobs, schedule=sched)
    assert _status(e.value) == -4
    lib.plas_debug_inject(0, 0)
    res = plas.batch_sort(jobs, schedule=sched)
    for j, r in zip(jobs, res):
        one = plas.sort(j["x"], j["H"], j["W"], carried=j["carried"], seed=j["seed"])
        assert torch.equal(r.perm, one.perm) and torch.equal(r.carried, one.carried)


def test_checked_run_matches_oracle_and_detects_a_planted_overwrite(plas, orc):
    """schedule.checked: guard bands between the workspace regions are filled
    and verified after the sort, and the assignment checks every grouping
    entry and cell position.  A healthy run passes and equals the oracle; a
    guard byte overwritten by the host after the fill (injected) is reported
    as PLAS_ERR_INTERNAL; the next checked run passes again."""
    lib = plas.load()
    x, c = synth.gaussians_3dgs(48 * 48, seed=8)
    xc, cc = torch.from_numpy(x).cuda(), torch.from_numpy(c).cuda()
    sched = plas.Schedule(checked=True)
    got = plas.sort(xc, 48, 48, carried=cc, seed=8, schedule=sched)
    want = orc.sort(x, 48, 48, seed=8)
    assert np.array_equal(got.perm.cpu().numpy(), want["perm"])
    assert lib.plas_debug_inject(4, 1) == 0
    with pytest.raises(RuntimeError) as e:
        plas.sort(xc, 48, 48, carried=cc, seed=8, schedule=sched)
    assert _status(e.value) == PLAS_ERR_INTERNAL and "guard" in str(e.value)
    lib.plas_debug_inject(0, 0)
    again = plas.sort(xc, 48, 48, carried=cc, seed=8, schedule=sched)
    assert torch.equal(again.perm, got.perm)
