"""GPU smoothness loss (Sec. 3.2) against the FP64 oracle and finite
differences.  Bar (floating point): loss within 1e-5 relative; gradient with
||g_gpu - g_64|| <= 1e-5 ||g_64|| and max|g_gpu - g_64| <= 1e-5 max|g_64|."""
import numpy as np
import pytest
import torch

from paper_2312_13299_gb300 import synth

pytestmark = pytest.mark.gpu


def _check(plas, orc, x, sigma, ksize, lam=None, g=1.0):
    xc = torch.from_numpy(x).cuda().requires_grad_(True)
    lc = torch.from_numpy(lam).cuda() if lam is not None else None
    L = plas.smooth_loss(xc, sigma, ksize, lc)
    (L * g).backward()
    L64, g64 = orc.smooth_loss64(x.astype(np.float64), sigma, ksize, lam, grad_loss=g)
    assert abs(L.item() - L64) <= 1e-5 * abs(L64)
    gg = xc.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - g64) <= 1e-5 * np.linalg.norm(g64)
    assert np.abs(gg - g64).max() <= 1e-5 * np.abs(g64).max()


@pytest.mark.parametrize("H,W,C,sigma,ksize", [(16, 16, 3, 1.0, 7), (37, 45, 5, 1.0, 7),
                                               (64, 64, 59, 1.0, 7), (33, 70, 14, 3.0, 5),
                                               (8, 200, 1, 2.0, 31), (100, 31, 2, 0.7, 3)])
def test_loss_matches_fp64(plas, orc, H, W, C, sigma, ksize):
    x = np.random.default_rng(H + W + C).random((H, W, C), dtype=np.float32)
    lam = (np.random.default_rng(1).random(C) + 0.5).astype(np.float32)
    _check(plas, orc, x, sigma, ksize)
    _check(plas, orc, x, sigma, ksize, lam, g=0.37)


def test_loss_full_size_1024x1024x59(plas, orc):
    x = synth.loss_grid(1024, 1024, seed=0).astype(np.float32)
    _check(plas, orc, x, 1.0, 7)


def test_loss_gradient_finite_differences(plas, orc):
    """Central differences of the FP64 loss at sampled points vs the GPU gradient."""
    x = np.random.default_rng(5).random((24, 24, 4), dtype=np.float32)
    xc = torch.from_numpy(x).cuda().requires_grad_(True)
    plas.smooth_loss(xc, 1.0, 7).backward()
    g = xc.grad.cpu().numpy()
    x64 = x.astype(np.float64)
    rng = np.random.default_rng(6)
    h = 1e-6
    for _ in range(30):
        i = tuple(rng.integers(0, s) for s in x.shape)
        xp, xm = x64.copy(), x64.copy()
        xp[i] += h
        xm[i] -= h
        fd = (orc.smooth_loss64(xp, 1.0, 7, want_grad=False)[0]
              - orc.smooth_loss64(xm, 1.0, 7, want_grad=False)[0]) / (2 * h)
        assert abs(g[i] - fd) <= 1e-5 * np.abs(g).max()


def test_loss_deterministic(plas):
    x = torch.rand(256, 256, 59, device="cuda")
    a = plas.smooth_loss_fwd(x)
    b = plas.smooth_loss_fwd(x)
    assert torch.equal(a, b)


def test_loss_in_training_loop_with_resorts(plas, orc):
    """The smoothness loss inside an Adam loop that re-sorts the grid every 100
    steps (Sec. 3.2 with the sort of Sec. 3.1 between steps): at every re-sort
    the GPU loss and gradient agree with the FP64 oracle, every attribute and
    both Adam moments follow the one permutation, and the loss falls."""
    H = W = 64
    x, c = synth.gaussians_3dgs(H * W, seed=3)
    grid = np.concatenate([x, c], axis=1).astype(np.float32)  # 14 sort + 45 carried
    P = torch.from_numpy(grid).cuda().requires_grad_(True)
    opt = torch.optim.Adam([P], lr=1e-3)
    losses = []
    for step in range(300):
        if step % 100 == 0:
            with torch.no_grad():
                r = plas.sort(P[:, :14].contiguous(), H, W, seed=step,
                              schedule=plas.Schedule(shuffle_init=False))
                st = opt.state[P] if P in opt.state else None
                before = {k: v.clone() for k, v in st.items() if torch.is_tensor(v) and v.dim() == 2} if st else {}
                P.copy_(plas.gather_rows(P.detach(), r.perm))
                for k, v in before.items():
                    st[k].copy_(plas.gather_rows(v, r.perm))
                    assert torch.equal(st[k], v[r.perm.long()])
            p_np = P.detach().cpu().numpy().reshape(H, W, -1).astype(np.float64)
            L64, g64 = orc.smooth_loss64(p_np, 1.0, 7, None, grad_loss=1.0)
            Pg = P.detach().clone().reshape(H, W, -1).requires_grad_(True)
            L = plas.smooth_loss(Pg, 1.0, 7)
            L.backward()
            assert abs(L.item() - L64) <= 1e-5 * abs(L64)
            gg = Pg.grad.cpu().numpy().astype(np.float64)
            assert np.linalg.norm(gg - g64) <= 1e-5 * np.linalg.norm(g64)
        opt.zero_grad()
        loss = plas.smooth_loss(P.reshape(H, W, -1), 1.0, 7)
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert losses[-1] < losses[0]


def test_loss_loop_full_size_with_resorts(plas, orc):
    """The training loop at full size (1024 x 1024 x 59, Adam lr 1e-3, a
    re-sort every 100 steps, warm-started): at each re-sort the GPU loss and
    gradient agree with the FP64 oracle within 1e-5 relative, every channel
    and both Adam moments follow the permutation, and the loss falls."""
    H = W = 1024
    P = torch.from_numpy(synth.loss_grid(H, W, seed=0).reshape(H * W, -1).astype(np.float32)).cuda()
    P.requires_grad_(True)
    opt = torch.optim.Adam([P], lr=1e-3)
    losses = []
    for step in range(201):
        if step % 100 == 0:
            with torch.no_grad():
                r = plas.sort(P[:, :14].contiguous(), H, W, seed=step,
                              schedule=plas.Schedule(shuffle_init=(step == 0)))
                st = opt.state[P] if P in opt.state else {}
                before = {k: v.clone() for k, v in st.items() if torch.is_tensor(v) and v.dim() == 2}
                P.copy_(plas.gather_rows(P.detach(), r.perm))
                for k, v in before.items():
                    st[k].copy_(plas.gather_rows(v, r.perm))
                    assert torch.equal(st[k], v[r.perm.long()])
            p_np = P.detach().cpu().numpy().reshape(H, W, -1).astype(np.float64)
            L64, g64 = orc.smooth_loss64(p_np, 1.0, 7, None, grad_loss=1.0)
            Pg = P.detach().clone().reshape(H, W, -1).requires_grad_(True)
            L = plas.smooth_loss(Pg, 1.0, 7)
            L.backward()
            assert abs(L.item() - L64) <= 1e-5 * abs(L64)
            gg = Pg.grad.cpu().numpy().astype(np.float64)
            assert np.linalg.norm(gg - g64) <= 1e-5 * np.linalg.norm(g64)
            assert np.abs(gg - g64).max() <= 1e-5 * np.abs(g64).max()
            del p_np, g64, gg
        opt.zero_grad()
        loss = plas.smooth_loss(P.reshape(H, W, -1), 1.0, 7)
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert losses[-1] < losses[0]


@pytest.mark.parametrize("H,W,C,sigma,ksize,delta", [(40, 36, 5, 1.0, 7, 0.05), (64, 64, 59, 3.0, 5, 1.0),
                                                      (33, 70, 14, 3.0, 5, 0.02), (8, 200, 2, 2.0, 31, 0.1)])
def test_huber_loss_matches_fp64(plas, orc, H, W, C, sigma, ksize, delta):
    """Huber form (Sec. 3.2) on the staged kernel and (ksize 31) the strip
    kernel: loss within 1e-5 of FP64, gradient within 1e-5 in norm and max."""
    x = (np.random.default_rng(H * W + C).random((H, W, C), dtype=np.float32) * 2.0)
    lam = (np.random.default_rng(2).random(C) + 0.5).astype(np.float32)
    xc = torch.from_numpy(x).cuda().requires_grad_(True)
    L = plas.smooth_loss(xc, sigma, ksize, torch.from_numpy(lam).cuda(), huber_delta=delta)
    (L * 0.6).backward()
    L64, g64 = orc.smooth_loss64(x, sigma, ksize, lam, grad_loss=0.6, huber_delta=delta)
    assert abs(L.item() - L64) <= 1e-5 * abs(L64)
    gg = xc.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - g64) <= 1e-5 * np.linalg.norm(g64)
    assert np.abs(gg - g64).max() <= 1e-5 * np.abs(g64).max()


def test_huber_paper_configuration_full_size(plas, orc):
    """The paper's regulariser settings (kernel 5, sigma 3, weights 0.09 on
    opacity and 0.91 on rotation, delta 1) on the 1024x1024x59 grid."""
    x = synth.loss_grid(1024, 1024, seed=1).astype(np.float32)
    lam = synth.paper_smoothness_weights()
    xc = torch.from_numpy(x).cuda().requires_grad_(True)
    L = plas.smooth_loss(xc, 3.0, 5, torch.from_numpy(lam).cuda(), huber_delta=1.0)
    L.backward()
    L64, g64 = orc.smooth_loss64(x, 3.0, 5, lam, huber_delta=1.0)
    assert abs(L.item() - L64) <= 1e-5 * abs(L64)
    gg = xc.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - g64) <= 1e-5 * np.linalg.norm(g64)
    assert np.abs(gg - g64).max() <= 1e-5 * np.abs(g64).max()
    assert np.all(gg[..., lam == 0] == 0.0)


def test_huber_rejects_bad_delta(plas):
    x = torch.rand(16, 16, 3, device="cuda")
    with pytest.raises(RuntimeError):
        plas.smooth_loss_fwd(x, 1.0, 7, huber_delta=float("nan"))
    with pytest.raises(RuntimeError):
        plas.smooth_loss_fwd(x, 1.0, 7, huber_delta=-1.0)
