"""GPU parity of the PLAS sort against the CPU oracle (through the C ABI).

Bar: bit-exact.  The permutation, the per-iteration fixed-point residual sum
and the final schedule state of the CUDA path equal the oracle's on the same
seeded inputs: Philox outputs, grouping permutations, blur targets (several
tiles, ragged tails, multi-chunk radii), full sorts of small and ragged grids,
and single iterations resumed from GPU snapshots of the full-size workloads
(512^2, 1024^2, 1448^2 x 14 channels) at large, middle and small radii.
"""
import numpy as np
import pytest
import torch

from paper_2312_13299_gb300 import synth

pytestmark = pytest.mark.gpu


def _cuda(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def test_philox_bitexact(plas, orc):
    rng = np.random.default_rng(0)
    n = 5000
    ctr = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = [0x12345678, 0x9ABCDEF0]
    got = plas.philox(_cuda(ctr.view(np.int32)), key[0], key[1]).cpu().numpy().view(np.uint32)
    for i in range(0, n, 7):
        assert np.array_equal(got[i], orc.philox(ctr[i], key))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 15, 16, 255, 256, 257, 1023, 4096, 65536, 262144])
def test_group_permutation_bitexact(plas, orc, n):
    for tag, ctr in [(3, 0), (3, 12345), (1, 0)]:
        got = plas.group_permutation(77, tag, ctr, n).cpu().numpy().view(np.uint32)
        assert np.array_equal(got, orc.prp_table(77, tag, ctr, n))


TARGET_CASES = [(64, 64, 3, 31.0), (37, 53, 3, 17.3), (80, 96, 14, 39.5), (64, 64, 14, 1.0),
                (200, 130, 3, 64.9), (17, 300, 2, 8.0), (300, 17, 5, 8.0), (1, 50, 3, 1.0),
                (50, 1, 3, 1.0), (129, 257, 14, 128.5), (400, 64, 1, 199.0), (24, 24, 16, 11.0)]


@pytest.mark.parametrize("H,W,D,phi", TARGET_CASES)
def test_target_bitexact(plas, orc, H, W, D, phi):
    rng = np.random.default_rng(H * 1000 + W)
    x = rng.random((H * W, D), dtype=np.float32)
    perm = rng.permutation(H * W).astype(np.int32)
    w = (rng.random(D) + 0.5).astype(np.float32)
    got = plas.target(_cuda(x), H, W, _cuda(perm), phi, weights=w).cpu().numpy()
    want = orc.target(x, H, W, perm, phi, weights=w)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("phi", [1.0, 6.0, 40.0])
def test_target_bitexact_wide_magnitudes(plas, orc, phi):
    """Unnormalised values spread over 2^-80 .. 2^80 (with zeros and both
    signs): the border-norm division is correctly rounded everywhere, on the
    reciprocal path and on the IEEE-division path for extreme magnitudes."""
    H, W, D = 96, 88, 3
    rng = np.random.default_rng(int(phi * 10))
    # exponent rising from -100 to +100 down the rows (identity placement), so
    # that tiny, ordinary and huge accumulators all occur
    e = np.linspace(-100, 100, H)[:, None, None] + rng.uniform(-4, 4, (H, W, D))
    sign = np.where(rng.random((H, W, D)) < 0.3, -1.0, 1.0)
    x = (np.exp2(e) * sign).astype(np.float32).reshape(H * W, D)
    x[rng.random((H * W, D)) < 0.05] = 0.0
    perm = np.arange(H * W, dtype=np.int32)
    got = plas.target(_cuda(x), H, W, _cuda(perm), phi, normalize=False).cpu().numpy()
    want = orc.target(x, H, W, perm, phi, normalize_=False)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


# tuning that forces one FIR tiling at every radius: (small_below,
# medium_below, large_tma, small_fused); "one-launch" runs both passes in one
# kernel up to r = 11 and the direct kernel above
_TILINGS = {"direct": (10 ** 6, 10 ** 6, 0, 0), "one-launch": (10 ** 6, 10 ** 6, 0, 1),
            "64-row": (0, 10 ** 6, 0, 1), "128-row": (0, 0, 0, 1),
            "128-row-tensor-copy": (0, 0, 1, 1)}


@pytest.mark.parametrize("tiling", sorted(_TILINGS))
@pytest.mark.parametrize("H,W,D,phi", [(200, 136, 14, 60.0), (131, 77, 5, 30.0), (96, 160, 3, 6.0),
                                       (1, 300, 14, 40.0), (257, 1, 2, 70.0), (68, 52, 64, 20.0),
                                       (300, 290, 14, 140.0), (150, 133, 6, 33.0),
                                       (129, 140, 10, 50.0), (77, 300, 12, 25.0), (260, 70, 16, 90.0)])
def test_target_bitexact_every_tiling(plas, orc, tiling, H, W, D, phi):
    """Each FIR tiling (the direct kernel, the ring kernel with 64 or 128 rows
    per CTA, and the persistent 128-row kernel that streams rows with tensor
    copies, for even D) gives the oracle's target bit for bit, on ragged
    grids whose sides and column counts span several tiles with partial ones
    at the end (more tiles than SMs for the persistent kernel), and on
    single-row/column grids."""
    rng = np.random.default_rng(H * 7 + W * 3 + D)
    x = rng.random((H * W, D), dtype=np.float32)
    perm = rng.permutation(H * W).astype(np.int32)
    sb, mb, tma, fused = _TILINGS[tiling]
    plas.set_tuning(H, W, D, fir_small_below=sb, fir_medium_below=mb, assign_ctas_per_sm=8,
                    large_tma=tma, small_fused=fused)
    try:
        got = plas.target(_cuda(x), H, W, _cuda(perm), phi).cpu().numpy()
    finally:
        plas.set_tuning(H, W, D)
    want = orc.target(x, H, W, perm, phi)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("fused", [1, 0])
@pytest.mark.parametrize("H,W,D,phi", [(200, 136, 14, 1.0), (200, 136, 14, 5.5), (131, 77, 5, 2.0),
                                       (131, 77, 5, 11.9), (96, 160, 3, 3.0), (96, 160, 3, 8.0),
                                       (1, 300, 14, 7.0), (257, 1, 2, 9.0), (33, 70, 16, 11.0),
                                       (50, 40, 1, 4.0), (45, 38, 15, 10.0), (64, 64, 4, 6.0),
                                       (7, 9, 13, 3.0), (40, 31, 7, 11.0), (12, 5, 11, 2.0)])
def test_target_bitexact_small_radii(plas, orc, fused, H, W, D, phi):
    """Radii 1-11 on the small-radius path: both passes in one launch (tiles
    of 32 x 32 cells with the pass along y kept in shared memory; halos cut by
    the border; odd D, where the last channel pair carries the index column)
    and the two-launch direct kernel give the oracle's target bit for bit,
    also on grids narrower than the halo and single rows or columns."""
    rng = np.random.default_rng(H * 5 + W * 11 + D + int(phi))
    x = rng.random((H * W, D), dtype=np.float32)
    perm = rng.permutation(H * W).astype(np.int32)
    plas.set_tuning(H, W, D, fir_small_below=10 ** 6, fir_medium_below=10 ** 6, small_fused=fused)
    try:
        got = plas.target(_cuda(x), H, W, _cuda(perm), phi).cpu().numpy()
    finally:
        plas.set_tuning(H, W, D)
    want = orc.target(x, H, W, perm, phi)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def _sched(plas, **kw):
    return plas.Schedule(**kw)


def _compare_full(plas, orc, x, H, W, seed, weights=None, cap=1 << 15, **kw):
    want = orc.sort(x, H, W, weights=weights, seed=seed, sched=orc.default_schedule(**kw))
    got = plas.sort(_cuda(x), H, W, weights=weights, seed=seed, schedule=_sched(plas, **kw),
                    trace_cap=cap)
    assert np.array_equal(got.perm.cpu().numpy(), want["perm"])
    n = want["iterations"]
    assert got.state["it"] == n
    assert np.array_equal(got.trace_S.cpu().numpy(), want["trace_S"])
    assert np.array_equal(got.trace_level.cpu().numpy(), want["trace_level"])
    ws = want["state"]
    for k in ["it", "epoch", "redraws", "level", "stall", "has_prev", "done", "d_prev", "d_last",
              "scale_exp"]:
        assert got.state[k] == getattr(ws, k), k
    return got, want


def test_full_sort_64x64x3(plas, orc):
    """The small workload end to end (64x64 RGB, seed 0, default schedule)."""
    x = synth.rgb_uniform(64, seed=0)
    _compare_full(plas, orc, x, 64, 64, 0)


@pytest.mark.parametrize("H,W,D,seed", [(37, 53, 3, 1), (48, 80, 14, 2), (16, 16, 1, 3),
                                        (2, 2, 3, 4), (3, 3, 3, 5), (1, 1, 3, 6), (1, 7, 3, 7),
                                        (7, 1, 3, 8), (20, 33, 5, 9), (96, 40, 4, 10)])
def test_full_sort_ragged_and_degenerate(plas, orc, H, W, D, seed):
    x = np.random.default_rng(seed).random((H * W, D), dtype=np.float32)
    _compare_full(plas, orc, x, H, W, seed)


@pytest.mark.parametrize("H,W,D,seed", [(37, 53, 3, 1), (48, 80, 14, 2), (64, 64, 3, 0)])
def test_full_sort_whole_blocks_reading(plas, orc, H, W, D, seed):
    """The alternative reading of the shifted blocks (whole blocks only, the
    blocks cut by the grid border left out) on both sides: bit-exact."""
    x = np.random.default_rng(seed + 40).random((H * W, D), dtype=np.float32)
    want = orc.sort(x, H, W, seed=seed, sched=orc.default_schedule(edge_blocks=0))
    got = plas.sort(_cuda(x), H, W, seed=seed, schedule=plas.Schedule(whole_blocks=True),
                    trace_cap=1 << 15)
    assert np.array_equal(got.perm.cpu().numpy(), want["perm"])
    n = want["iterations"]
    assert got.state["it"] == n
    assert np.array_equal(got.trace_S.cpu().numpy(), want["trace_S"])


def test_full_sort_weights_unnormalized_and_no_shuffle(plas, orc):
    rng = np.random.default_rng(11)
    x = (rng.normal(size=(40 * 44, 6)) * [1, 5, 0.1, 2, 3, 1]).astype(np.float32)
    w = np.array([1.0, 0.5, 3.0, 0.0, 2.0, -1.5], np.float32)
    _compare_full(plas, orc, x, 40, 44, 12, weights=w)
    _compare_full(plas, orc, x, 40, 44, 12, weights=w, normalize=0)
    _compare_full(plas, orc, x, 40, 44, 12, shuffle_init=0, tol=1e-3, sigma_ratio=1.0)


def test_3dgs_shaped_full_sort_with_carried(plas, orc):
    x, car = synth.gaussians_3dgs(48 * 48, seed=3)
    got, want = _compare_full(plas, orc, x, 48, 48, 3)
    res = plas.sort(_cuda(x), 48, 48, carried=_cuda(car), seed=3, want_sorted=True)
    perm = want["perm"]
    assert np.array_equal(res.perm.cpu().numpy(), perm)
    assert np.array_equal(res.carried.cpu().numpy(), orc.gather(car, perm))
    assert np.array_equal(res.sorted.cpu().numpy(), orc.gather(x, perm))


def test_empty_grid(plas):
    x = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    r = plas.sort(x, 0, 0)
    assert r.perm.numel() == 0 and r.state["done"] == 1


def test_poll_batch_size_does_not_change_result(plas):
    x = _cuda(synth.rgb_uniform(40, seed=4))
    a = plas.sort(x, 40, 40, seed=4, schedule=plas.Schedule(iters_per_poll=1)).perm
    b = plas.sort(x, 40, 40, seed=4, schedule=plas.Schedule(iters_per_poll=37)).perm
    c = plas.sort(x, 40, 40, seed=4).perm
    assert torch.equal(a, b) and torch.equal(a, c)


def test_launch_modes_give_identical_results(plas, orc):
    """Graph replay, direct launches, event-profiled launches and the
    persistent cooperative sweep run the same kernel bodies on the same work
    items: the permutation and the schedule trace match each other and the
    oracle."""
    side = 48
    x = synth.rgb_uniform(side, seed=6)
    xc = _cuda(x)
    g = plas.sort(xc, side, side, seed=6, want_stats=True, trace_cap=1 << 14,
                  schedule=plas.Schedule(persistent=-1))
    d = plas.sort(xc, side, side, seed=6, want_stats=True, trace_cap=1 << 14,
                  schedule=plas.Schedule(graphs=False, persistent=-1))
    p = plas.sort(xc, side, side, seed=6, want_stats=True, trace_cap=1 << 14,
                  schedule=plas.Schedule(profile=True, iters_per_poll=3))
    c = plas.sort(xc, side, side, seed=6, want_stats=True, trace_cap=1 << 14,
                  schedule=plas.Schedule(persistent=1, iters_per_poll=5))
    assert g.stats["graph_launches"] > 0 and g.stats["graph_captures"] >= 1
    assert d.stats["graph_launches"] == 0 and p.stats["graph_launches"] == 0
    # one cooperative launch per batch of five sweeps
    assert c.stats["graph_launches"] == 0 and c.stats["launches"] < c.state["it"]
    want = orc.sort(x, side, side, seed=6)
    for r in (g, d, p, c):
        assert np.array_equal(r.perm.cpu().numpy(), want["perm"])
        n = r.state["it"]
        assert r.trace_S[:n].cpu().numpy().tolist() == want["trace_S"][:n].tolist()


def test_autotune_and_forced_launch_shapes_give_identical_results(plas, orc):
    """The tuner measures the three FIR tilings and four assignment grid sizes;
    any installed choice (always 128-row, always 64-row, always direct, a
    mix by radius, 1 or 16 assignment CTAs per SM) gives the oracle's
    permutation and schedule trace."""
    H, W, D = 72, 56, 6
    t = plas.autotune(H, W, D)
    assert t["radius"][0] == 1 and len(t["fir_small_us"]) == len(t["radius"])
    assert len(t["fir_medium_us"]) == len(t["radius"])
    assert all(v > 0 for v in t["fir_medium_us"] + t["fir_large_us"] + t["assign_us"])
    assert all((v > 0) == (r <= 32) for v, r in zip(t["fir_small_us"], t["radius"]))
    assert t["fir_small_below"] <= t["fir_medium_below"]
    assert t["assign_ctas_per_sm"] in t["assign_per_sm"]
    assert all(v > 0 for v in t["fir_large_tma_us"] + t["fir_large_ring_us"])  # D = 6 is eligible
    rng = np.random.default_rng(11)
    x = rng.random((H * W, D), dtype=np.float32)
    want = orc.sort(x, H, W, seed=11)
    xc = _cuda(x)
    try:
        for small_below, medium_below, per_sm, tma, fused in [
                (0, 0, 1, 0, 1), (0, 0, 2, 1, 1), (10 ** 6, 10 ** 6, 16, 1, 1),
                (10 ** 6, 10 ** 6, 16, 1, 0), (0, 10 ** 6, 2, 0, 1), (3, 12, 8, 1, 1),
                (t["fir_small_below"], t["fir_medium_below"], 4, t["large_tma"], t["small_fused"])]:
            plas.set_tuning(H, W, D, fir_small_below=small_below, fir_medium_below=medium_below,
                            assign_ctas_per_sm=per_sm, large_tma=tma, small_fused=fused)
            got = plas.sort(xc, H, W, seed=11, trace_cap=1 << 14)
            assert np.array_equal(got.perm.cpu().numpy(), want["perm"]), (small_below, medium_below,
                                                                          per_sm)
            n = got.state["it"]
            assert got.trace_S[:n].cpu().numpy().tolist() == want["trace_S"][:n].tolist()
    finally:
        plas.set_tuning(H, W, D)


def _snapshot_parity(plas, orc, side, seed, radii, iters_before=2):
    """GPU runs to the first iteration of the level nearest each radius, then the
    oracle and the GPU each run one (or a few) iterations from that snapshot."""
    x, _ = synth.gaussians_3dgs(side * side, seed=seed, with_carried=False)
    xc = _cuda(x)
    phis = orc.levels(side, side)
    full = plas.sort(xc, side, side, seed=seed, trace_cap=200000)
    tl = full.trace_level.cpu().numpy()
    for phi in radii:
        L = int(np.argmin(np.abs(phis - phi)))
        start = int(np.nonzero(tl == L)[0][0]) + iters_before
        snap = plas.sort(xc, side, side, seed=seed, schedule=plas.Schedule(max_iters=start))
        st = dict(snap.state)
        perm0 = snap.perm.cpu().numpy()
        ost = orc.State()
        for k, v in st.items():
            if hasattr(ost, k):
                setattr(ost, k, v)
        want = orc.sort(x, side, side, seed=seed, sched=orc.default_schedule(max_iters=start + 1),
                        perm_in=perm0, state=ost)
        got = plas.sort(xc, side, side, seed=seed, schedule=plas.Schedule(max_iters=start + 1),
                        perm_init=snap.perm, state=st, trace_cap=start + 2)
        assert np.array_equal(got.perm.cpu().numpy(), want["perm"]), (side, phi)
        assert got.state["d_last"] == want["state"].d_last
        assert got.trace_S.cpu().numpy().tolist() == want["trace_S"].tolist()
        # the uninterrupted GPU run took the same step
        assert int(full.trace_S[start].item()) == int(want["trace_S"][0])


@pytest.mark.parametrize("side,radii", [(512, [255, 60, 10, 1]), (1024, [511, 100, 10, 1]),
                                        (1448, [723, 10, 1])])
def test_snapshot_parity_full_size(plas, orc, side, radii):
    _snapshot_parity(plas, orc, side, side, radii)


def test_nonfinite_input_rejected(plas):
    x = torch.rand(32 * 32, 3, device="cuda")
    x[100, 1] = float("nan")
    with pytest.raises(RuntimeError) as e:
        plas.sort(x, 32, 32)
    assert "NaN" in str(e.value)


def test_invalid_arguments(plas):
    x = torch.rand(32 * 32, 3, device="cuda")
    with pytest.raises(ValueError):
        plas.sort(x, 32, 31)
    with pytest.raises(RuntimeError):
        plas.sort(torch.rand(16, 17, device="cuda"), 4, 4)  # D = 17 is not supported
    with pytest.raises(RuntimeError):
        plas.sort(x, 32, 32, schedule=plas.Schedule(shrink=1.5))


def test_grid_metrics(plas, orc):
    g = np.random.default_rng(2).random((61, 47, 5), dtype=np.float32)
    nl2, vad, _ = plas.grid_metrics(_cuda(g), 255.0)
    onl2, ovad = orc.metrics(g, 255.0)
    assert abs(nl2 - onl2) <= 1e-9 * onl2 and abs(vad - ovad) <= 1e-9 * ovad


def test_gather_rows(plas, orc):
    rng = np.random.default_rng(3)
    for C in [1, 3, 4, 45, 64]:
        src = rng.random((1000, C), dtype=np.float32)
        perm = rng.permutation(1000).astype(np.int32)
        got = plas.gather_rows(_cuda(src), _cuda(perm)).cpu().numpy()
        assert np.array_equal(got, orc.gather(src, perm))


def test_batch_equals_individual(plas):
    jobs = []
    for i, (H, W) in enumerate([(40, 40), (17, 64), (64, 17), (33, 33)]):
        x, c = synth.gaussians_3dgs(H * W, seed=i)
        jobs.append({"x": _cuda(x), "H": H, "W": W, "carried": _cuda(c), "seed": 100 + i})
    res = plas.batch_sort(jobs)
    for j, r in zip(jobs, res):
        one = plas.sort(j["x"], j["H"], j["W"], carried=j["carried"], seed=j["seed"])
        assert torch.equal(r.perm, one.perm) and torch.equal(r.carried, one.carried)
        assert r.state["it"] == one.state["it"]
