"""Batched and served sorts (continuous batching) on the GPU.

Each request's result -- permutation, carried attributes and final schedule
state -- must equal the same request sorted alone with plas_sort, bit for bit,
whether it ran in a static batch, arrived while others were running, or was
admitted later because of the memory budget (every grid keeps its own
counters and random streams)."""
import numpy as np
import pytest
import torch

from paper_2312_13299_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [(48, 48), (17, 64), (64, 17), (33, 33), (96, 80), (128, 128), (20, 200)]


def _requests(D=14, seed0=0):
    out = []
    for i, (H, W) in enumerate(SIZES):
        x, c = synth.gaussians_3dgs(H * W, seed=seed0 + i)
        out.append({"x": torch.from_numpy(x[:, :D].copy()).cuda(), "H": H, "W": W,
                    "carried": torch.from_numpy(c).cuda(), "seed": 100 + i})
    return out


def _alone(plas, r):
    return plas.sort(r["x"], r["H"], r["W"], carried=r["carried"], seed=r["seed"])


def _same(a, b):
    assert torch.equal(a.perm, b.perm)
    assert torch.equal(a.carried, b.carried)
    for k in ["it", "epoch", "redraws", "level", "done", "d_last", "d_prev"]:
        assert a.state[k] == b.state[k], k


def test_batch_sort_equals_alone(plas):
    reqs = _requests()
    res = plas.batch_sort(reqs)
    for r, got in zip(reqs, res):
        _same(got, _alone(plas, r))


def test_batch_sort_d3(plas):
    reqs = []
    for i, (H, W) in enumerate([(64, 64), (40, 72), (16, 16), (5, 9)]):
        reqs.append({"x": torch.from_numpy(synth.rgb_uniform(H, W, seed=i)).cuda(), "H": H,
                     "W": W, "seed": i})
    for r, got in zip(reqs, plas.batch_sort(reqs)):
        one = plas.sort(r["x"], r["H"], r["W"], seed=r["seed"])
        assert torch.equal(got.perm, one.perm) and got.state["it"] == one.state["it"]


@pytest.mark.parametrize("policy", ["fifo_fill", "shortest_first", "all", "concurrent", "adaptive"])
def test_server_arrivals_while_running(plas, policy):
    reqs = _requests(seed0=10)
    srv = plas.Server(14, policy=policy)
    tickets = {}
    for r in reqs[:3]:
        tickets[srv.submit(r["x"], r["H"], r["W"], r["carried"], r["seed"])] = r
    results = {}
    steps = 0
    late = list(reqs[3:])
    while len(results) < len(reqs):
        for t, res in srv.step(sweeps=4):
            results[t] = res
        steps += 1
        if late and steps % 3 == 0:  # a request arrives while others are on the GPU
            r = late.pop(0)
            tickets[srv.submit(r["x"], r["H"], r["W"], r["carried"], r["seed"])] = r
        assert steps < 100000
    srv.close()
    for t, r in tickets.items():
        _same(results[t], _alone(plas, r))


def test_server_budget_admission(plas):
    reqs = _requests(seed0=20)[:4]
    need = max(plas.sort_workspace_bytes(r["H"], r["W"], 14) for r in reqs)
    srv = plas.Server(14, mem_budget=need + 4096)
    tickets = {srv.submit(r["x"], r["H"], r["W"], r["carried"], r["seed"]): r for r in reqs}
    results, max_active = {}, 0
    while len(results) < len(reqs):
        for t, res in srv.step(sweeps=16):
            results[t] = res
        q, a, mem = srv.status()
        max_active = max(max_active, a)
        assert mem <= need + 4096
    srv.close()
    assert max_active >= 1
    for t, r in tickets.items():
        _same(results[t], _alone(plas, r))


def test_server_rejects_unknown_policy(plas):
    with pytest.raises(ValueError):
        plas.Server(3, policy="random")


def test_server_rejects_request_over_budget(plas):
    srv = plas.Server(3, mem_budget=1024)
    x = torch.rand(64 * 64, 3, device="cuda")
    with pytest.raises(RuntimeError) as e:
        srv.submit(x, 64, 64)
    assert "budget" in str(e.value)
    srv.close()


@pytest.mark.parametrize("policy", ["all", "concurrent"])
def test_server_cancel_queued_and_running(plas, policy):
    """A request cancelled while queued and one cancelled while running are
    never reported; the others give exactly their results alone, and the
    server ends with nothing queued, admitted or allocated.  Unknown,
    finished and repeated cancellations are rejected."""
    reqs = _requests(seed0=30)[:4]
    srv = plas.Server(14, policy=policy)
    t = [srv.submit(r["x"], r["H"], r["W"], r["carried"], r["seed"]) for r in reqs]
    srv.cancel(t[2])  # still queued: nothing is admitted before the first step
    with pytest.raises(RuntimeError):
        srv.cancel(t[2])
    results = dict(srv.step(sweeps=2))
    assert srv.status()[1] == 3
    srv.cancel(t[1])  # admitted and running
    steps = 0
    while len(results) < 2:
        results.update(srv.step(sweeps=8))
        steps += 1
        assert steps < 100000
    for _ in range(3):
        results.update(srv.step(sweeps=8))
    assert sorted(results) == sorted([t[0], t[3]])
    for i in (0, 3):
        _same(results[t[i]], _alone(plas, reqs[i]))
    assert srv.status() == (0, 0, 0)
    with pytest.raises(RuntimeError):
        srv.cancel(t[0])  # finished
    with pytest.raises(RuntimeError):
        srv.cancel(12345)  # unknown
    srv.close()


def test_server_cancel_frees_budget_for_the_next_request(plas):
    """With a budget for one request at a time, cancelling the running
    request admits the queued one at the next step, and that one completes
    with its result alone."""
    reqs = _requests(seed0=40)
    big, small = reqs[5], reqs[0]  # 128 x 128 and 48 x 48
    need = plas.sort_workspace_bytes(big["H"], big["W"], 14)
    srv = plas.Server(14, mem_budget=need + 4096)
    tb = srv.submit(big["x"], big["H"], big["W"], big["carried"], big["seed"])
    ts = srv.submit(small["x"], small["H"], small["W"], small["carried"], small["seed"])
    assert srv.step(sweeps=2) == []
    q, a, mem = srv.status()
    assert (q, a) == (1, 1) and mem > 0
    srv.cancel(tb)
    results = {}
    steps = 0
    while ts not in results:
        results.update(srv.step(sweeps=8))
        steps += 1
        assert steps < 100000
    assert list(results) == [ts]
    _same(results[ts], _alone(plas, small))
    assert srv.status() == (0, 0, 0)
    srv.close()


def test_server_policy_switch_needs_an_idle_server(plas):
    """The concurrent policy keeps its requests on lanes of their own, so a
    switch to or from it is refused while anything is admitted."""
    reqs = _requests(seed0=60)[:2]
    srv = plas.Server(14, policy="all")
    t = srv.submit(reqs[0]["x"], reqs[0]["H"], reqs[0]["W"], reqs[0]["carried"], reqs[0]["seed"])
    srv.step(sweeps=2)
    with pytest.raises(RuntimeError):
        srv._lib_policy("concurrent")
    results = {}
    while t not in results:
        results.update(srv.step(sweeps=8))
    srv._lib_policy("concurrent")
    t2 = srv.submit(reqs[1]["x"], reqs[1]["H"], reqs[1]["W"], reqs[1]["carried"], reqs[1]["seed"])
    while t2 not in results:
        results.update(srv.step(sweeps=8))
    srv.close()
    _same(results[t], _alone(plas, reqs[0]))
    _same(results[t2], _alone(plas, reqs[1]))
