"""The box target (schedule.target_mode = 1, a fast low-pass variant of the
target of Sec. 3.1) on the GPU: per-step targets bit-exact against the
oracle, and full and resumed sorts in box mode bit-exact (permutation and
per-iteration residual sums)."""
import numpy as np
import pytest
import torch

from paper_2312_13299_gb300 import synth

pytestmark = pytest.mark.gpu


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("H,W,D,phi,normalize", [(64, 64, 3, 31.0, True), (37, 53, 5, 7.5, True),
                                                 (128, 96, 14, 47.0, True), (20, 30, 1, 40.0, True),
                                                 (50, 40, 4, 3.0, False), (8, 200, 2, 1.0, True),
                                                 (1, 300, 15, 40.0, True), (257, 1, 2, 70.0, True),
                                                 (33, 70, 64, 12.0, True), (45, 38, 16, 9.0, False),
                                                 (4, 6144, 3, 100.0, True), (3, 7000, 3, 5.0, True),
                                                 (2, 9000, 14, 2000.0, True), (3, 2000, 14, 300.0, True),
                                                 (5, 1500, 14, 200.0, True)])
def test_box_target_bitexact(plas, orc, H, W, D, phi, normalize):
    """Ragged and degenerate shapes (single row or column, odd D, D = 64).
    Every row evaluation: one CTA per row (D <= 16, row prefix <= 200 KB,
    e.g. 5 x 1500 x 14), one CTA per row and channel pair (up to 6144 cells:
    D = 64, and 2000 x 14), and the three-launch summed-area path for wider
    rows."""
    rng = np.random.default_rng(H * W + D)
    x = (rng.standard_normal((H * W, D)) * 3).astype(np.float32)
    perm = rng.permutation(H * W).astype(np.int32)
    w = (rng.random(D) + 0.5).astype(np.float32)
    got = plas.target_box(_cuda(x), H, W, _cuda(perm), phi, weights=w, normalize=normalize).cpu().numpy()
    want = orc.target_box(x, H, W, perm, phi, weights=w, normalize_=normalize)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_box_full_sort_64x64x3(plas, orc):
    x = synth.rgb_uniform(64, seed=0)
    want = orc.sort(x, 64, 64, seed=0, sched=orc.default_schedule(target_mode=1))
    got = plas.sort(_cuda(x), 64, 64, seed=0, schedule=plas.Schedule(target_mode=1), trace_cap=1 << 15)
    assert np.array_equal(got.perm.cpu().numpy(), want["perm"])
    n = want["iterations"]
    assert got.state["it"] == n
    assert np.array_equal(got.trace_S.cpu().numpy()[:n], want["trace_S"])


def test_box_3dgs_sort_with_carried(plas, orc):
    x, c = synth.gaussians_3dgs(96 * 80, seed=2)
    want = orc.sort(x, 96, 80, seed=5, sched=orc.default_schedule(target_mode=1))
    got = plas.sort(_cuda(x), 96, 80, carried=_cuda(c), seed=5, schedule=plas.Schedule(target_mode=1))
    assert np.array_equal(got.perm.cpu().numpy(), want["perm"])
    assert np.array_equal(got.carried.cpu().numpy(), c[want["perm"]])


@pytest.mark.parametrize("side,radii", [(512, [255, 40, 4]), (1024, [511, 60, 2])])
def test_box_snapshot_parity(plas, orc, side, radii):
    x, _ = synth.gaussians_3dgs(side * side, seed=side, with_carried=False)
    xc = _cuda(x)
    phis = orc.levels(side, side)
    sched = dict(target_mode=1)
    full = plas.sort(xc, side, side, seed=side, schedule=plas.Schedule(**sched), trace_cap=200000)
    tl = full.trace_level.cpu().numpy()
    for phi in radii:
        L = int(np.argmin(np.abs(phis - phi)))
        start = int(np.nonzero(tl == L)[0][0]) + 1
        snap = plas.sort(xc, side, side, seed=side, schedule=plas.Schedule(max_iters=start, **sched))
        st = dict(snap.state)
        ost = orc.State()
        for k, v in st.items():
            if hasattr(ost, k):
                setattr(ost, k, v)
        want = orc.sort(x, side, side, seed=side, sched=orc.default_schedule(max_iters=start + 1, **sched),
                        perm_in=snap.perm.cpu().numpy(), state=ost)
        got = plas.sort(xc, side, side, seed=side, schedule=plas.Schedule(max_iters=start + 1, **sched),
                        perm_init=snap.perm, state=st)
        assert np.array_equal(got.perm.cpu().numpy(), want["perm"]), (side, phi)
        assert got.state["d_last"] == want["state"].d_last
        assert int(full.trace_S[start].item()) == int(want["trace_S"][0])


BOX_GRIDS = [(40, 40, 3), (17, 64, 3), (64, 17, 3), (48, 80, 3)]


def test_box_mode_batch_matches_oracle(plas, orc):
    """Box-target batches run one lane (stream + engine) per grid; every
    grid's permutation and final state equal the oracle's box-mode sort."""
    jobs, wants = [], []
    for i, (H, W, D) in enumerate(BOX_GRIDS):
        x = np.random.default_rng(70 + i).random((H * W, D), dtype=np.float32)
        jobs.append({"x": _cuda(x), "H": H, "W": W, "seed": 7 + i})
        wants.append(orc.sort(x, H, W, seed=7 + i, sched=orc.default_schedule(target_mode=1)))
    res = plas.batch_sort(jobs, schedule=plas.Schedule(target_mode=1))
    for r, want in zip(res, wants):
        assert np.array_equal(r.perm.cpu().numpy(), want["perm"])
        assert r.state["it"] == want["iterations"]
        assert r.state["d_last"] == want["state"].d_last


def test_box_mode_server_matches_alone(plas):
    """A box-target server takes the concurrent policy (any other is
    refused); requests arriving while others run give their results alone."""
    sched = plas.Schedule(target_mode=1)
    with pytest.raises(ValueError):
        plas.Server(3, schedule=sched, policy="bogus")
    with pytest.raises(RuntimeError):
        plas.Server(3, schedule=sched, policy="all")
    srv = plas.Server(3, schedule=sched)
    reqs, tickets, results = [], {}, {}
    for i, (H, W, D) in enumerate(BOX_GRIDS):
        x = torch.from_numpy(np.random.default_rng(90 + i).random((H * W, D), dtype=np.float32)).cuda()
        reqs.append((x, H, W, 3 + i))
    tickets[srv.submit(reqs[0][0], reqs[0][1], reqs[0][2], seed=reqs[0][3])] = reqs[0]
    steps = 0
    late = reqs[1:]
    while len(results) < len(reqs):
        results.update(srv.step(sweeps=4))
        steps += 1
        if late and steps % 2 == 0:
            r = late.pop(0)
            tickets[srv.submit(r[0], r[1], r[2], seed=r[3])] = r
        assert steps < 100000
    srv.close()
    for t, (x, H, W, seed) in tickets.items():
        one = plas.sort(x, H, W, seed=seed, schedule=sched)
        assert torch.equal(results[t].perm, one.perm)
        assert results[t].state["it"] == one.state["it"]
