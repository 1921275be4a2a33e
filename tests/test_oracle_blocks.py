"""Pins of the oracle's block reading (Sec. 3.1: the blocks are shifted at
random so that, over the iterations, the whole grid is covered).

Default reading: every block that meets the grid takes part, the blocks cut
by the grid border included; of those, each group of four whose cells all
lie inside the grid is re-assigned and the rest stay put.  The alternative
(schedule.edge_blocks = 0) re-assigns whole blocks only.

One iteration on a 37 x 29 grid with 16 x 16 blocks and a non-zero shift is
checked against properties fixed by the reading itself, computed here from
the shift and the grouping table alone (both pinned elsewhere):
- under either reading the result is a permutation, and the cells of the
  groups the reading does not re-assign keep their rows bit for bit;
- under the default reading cells outside the whole blocks do move, under
  the alternative none do;
- every re-assigned group's new arrangement is the best of its 24
  arrangements against the iteration's target (scipy's linear assignment
  on the 4 x 4 cost), so a dropped group or a shifted origin fails."""
import numpy as np
import pytest


def _groups(orc, H, W, beta, dy, dx, it, seed, edge):
    """(cells of each group, all inside the grid?) for one iteration."""
    pi = orc.prp_table(seed, orc.TAG_GROUP, it, beta * beta)
    if edge:
        oy0 = dy - beta if dy > 0 else 0
        ox0 = dx - beta if dx > 0 else 0
        nby, nbx = -(-(H - oy0) // beta), -(-(W - ox0) // beta)
    else:
        oy0, ox0 = dy, dx
        nby, nbx = (H - dy) // beta, (W - dx) // beta
    out = []
    for by in range(nby):
        for bx in range(nbx):
            oy, ox = oy0 + by * beta, ox0 + bx * beta
            for g in range(beta * beta // 4):
                cells = [(oy + int(l) // beta, ox + int(l) % beta) for l in pi[4 * g:4 * g + 4]]
                inside = all(0 <= y < H and 0 <= x < W for y, x in cells)
                out.append((cells, inside))
    return out


@pytest.mark.parametrize("edge", [1, 0])
def test_one_iteration_block_reading(orc, edge):
    from scipy.optimize import linear_sum_assignment
    H, W, D, seed = 37, 29, 3, 11
    x = np.random.default_rng(5).random((H * W, D), dtype=np.float32)
    phis = orc.levels(H, W)
    L = int(np.argmax(phis < 16))          # first level with r < 16: beta = 16
    beta = 16
    # resume at the first iteration of level L from the identity placement
    # (epoch chosen so that both shift components are non-zero)
    epoch = next(e for e in range(1, 200) if all(v > 0 for v in orc.shift(seed, e, beta, H, W)))
    dy, dx = orc.shift(seed, epoch, beta, H, W)
    st = orc.State()
    st.it, st.epoch, st.level = 40, epoch, L
    perm0 = np.arange(H * W, dtype=np.int32)
    sched = orc.default_schedule(max_iters=41, edge_blocks=edge)
    r = orc.sort(x, H, W, seed=seed, sched=sched, perm_in=perm0, state=st, want_target=True)
    perm1 = r["perm"]
    assert sorted(perm1.tolist()) == list(range(H * W))
    moved = perm1 != perm0
    groups = _groups(orc, H, W, beta, dy, dx, 40, seed, edge)
    in_group = np.zeros(H * W, bool)
    F = orc.normalize(x)
    T = r["T"].reshape(H * W, D)   # the target of the iteration (before the swap)
    for cells, inside in groups:
        if not inside:
            continue
        idx = [y * W + c for y, c in cells]
        in_group[idx] = True
        # the new arrangement is the best of the 24 (squared L2 to the target)
        src = perm1[idx]              # Gaussians now at the group's cells
        cost = ((F[perm0[idx]][:, None, :] - T[idx][None, :, :]) ** 2).sum(-1)
        ri, ci = linear_sum_assignment(cost)
        got = sum(cost[list(perm0[idx]).index(g), k] for k, g in enumerate(src))
        assert got <= cost[ri, ci].sum() + 1e-5
    assert not moved[~in_group].any()      # groups left out keep their cells
    full = np.zeros((H, W), bool)
    full[dy:dy + ((H - dy) // beta) * beta, dx:dx + ((W - dx) // beta) * beta] = True
    outside_moved = moved.reshape(H, W)[~full].any()
    assert outside_moved == bool(edge)
