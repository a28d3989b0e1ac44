"""Pins for the oracle's loss, Adam and rates (CPU only; Sec. 3.3, Sec. 4.2, Sec. 5.1)."""
import numpy as np
import pytest
import torch

from oracle import interleave as IL
from oracle import loss as LS


def setup_grid(seed=0, B=2, d=2, W=32):
    rng = np.random.default_rng(seed)
    G = rng.random((B, 4, 6, W)) < 0.3
    GT = G & (rng.random(G.shape) < 0.4)
    Gb, GTb = IL.pack_bits(G), IL.pack_bits(GT)
    coords, feats, _ = IL.interleave(Gb, W, d, 1)
    return rng, G, GT, Gb, GTb, coords


def test_perfect_and_empty_predictions_closed_form():
    rng, G, GT, Gb, GTb, coords = setup_grid()
    prm = LS.LossParams()
    y = LS.site_labels(GTb, coords, 32, 2)
    # perfect prediction: logits -> +/- infinity
    L, terms = LS.loss_terms(torch.tensor(np.where(y > 0, 1e3, -1e3)), coords, Gb, GTb, 32, 2, prm)
    for t in terms:
        assert float(t["dice"]) == pytest.approx(0.0, abs=1e-12)
        assert float(t["attr"]) == pytest.approx(0.0, abs=1e-12)
        assert float(t["rep"]) == pytest.approx(0.0, abs=1e-12)
    # empty prediction
    L, terms = LS.loss_terms(torch.full(y.shape, -1e3, dtype=torch.float64), coords, Gb, GTb, 32, 2, prm)
    for b, t in enumerate(terms):
        gtp = GT[b].sum()
        assert t["gtp"] == gtp
        assert float(t["dice"]) == pytest.approx(1 - prm.eps / (prm.alpha * gtp + prm.eps), rel=1e-12)
        assert float(t["attr"]) == pytest.approx(gtp / (gtp + prm.eps), rel=1e-12)
        assert float(t["rep"]) == 0.0


def test_hand_computed_example():
    """Two froxels in one site, GT = (1, 0), p = (0.8, 0.3), both occupied: TP = 0.8, FN = 0.2,
    FP = 0.3, GTP = 1; alpha = 0.9, eps = 1, lambda = 0.99."""
    G = np.zeros((1, 1, 1, 32), bool)
    G[0, 0, 0, :2] = True
    GT = np.zeros_like(G)
    GT[0, 0, 0, 0] = True
    coords, _, _ = IL.interleave(IL.pack_bits(G), 32, 1, 1)
    p = np.array([0.8, 0.3])
    logits = torch.tensor(np.log(p / (1 - p))[:, None])
    L, (t,) = LS.loss_terms(logits, coords, IL.pack_bits(G), IL.pack_bits(GT), 32, 1)
    dice = 1 - (1.6 + 1) / (1.6 + 0.9 * 0.2 + 0.1 * 0.3 + 1)
    attr, rep = 0.2 / 2, 0.3 / 2
    assert float(t["dice"]) == pytest.approx(dice, rel=1e-12)
    assert float(t["attr"]) == pytest.approx(attr, rel=1e-12)
    assert float(t["rep"]) == pytest.approx(rep, rel=1e-12)
    assert float(L) == pytest.approx(0.99 * dice + 0.01 * (attr + rep), rel=1e-12)


def test_layout_invariance():
    """The loss on the interleaved sparse layout equals the same sums on the dense froxel grid."""
    rng, G, GT, Gb, GTb, coords = setup_grid(seed=4)
    logits = rng.normal(size=(len(coords), 8))
    L, terms = LS.loss_terms(torch.tensor(logits), coords, Gb, GTb, 32, 2)
    p = IL.deinterleave(coords, 1 / (1 + np.exp(-logits)), *G.shape, 2) * G
    for b, t in enumerate(terms):
        y = GT[b].astype(np.float64)
        tp = (y * p[b]).sum()
        fp = ((1 - y) * p[b]).sum()
        assert float(t["tp"]) == pytest.approx(tp, rel=1e-12)
        assert float(t["fp"]) == pytest.approx(fp, rel=1e-12)


def test_loss_gradient_matches_central_differences():
    rng, G, GT, Gb, GTb, coords = setup_grid(seed=5)
    prm = LS.LossParams(w_bce=0.7)
    z = torch.tensor(rng.normal(size=(len(coords), 8)), requires_grad=True)
    L, _ = LS.loss_terms(z, coords, Gb, GTb, 32, 2, prm)
    L.backward()
    flat = z.detach().view(-1)
    for idx in rng.choice(flat.numel(), 20, replace=False):
        h = 1e-6
        old = float(flat[idx])
        flat[idx] = old + h
        lp = float(LS.loss_terms(z.detach(), coords, Gb, GTb, 32, 2, prm)[0])
        flat[idx] = old - h
        lm = float(LS.loss_terms(z.detach(), coords, Gb, GTb, 32, 2, prm)[0])
        flat[idx] = old
        fd = (lp - lm) / (2 * h)
        g = float(z.grad.view(-1)[idx])
        assert abs(g - fd) <= 1e-6 * max(abs(g), 1e-4)


def test_adam_matches_torch_optim():
    rng = np.random.default_rng(0)
    theta0 = rng.normal(size=50)
    grads = [rng.normal(size=50) for _ in range(5)]
    p = torch.tensor(theta0.copy(), requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-3, betas=(0.9, 0.999), eps=1e-8, weight_decay=1e-10)
    th, m, v = theta0.copy(), np.zeros(50), np.zeros(50)
    for t, g in enumerate(grads, 1):
        p.grad = torch.tensor(g)
        opt.step()
        th, m, v = LS.adam_step(th, g, m, v, t)
        np.testing.assert_allclose(th, p.detach().numpy(), rtol=1e-13, atol=1e-15)
    # first step closed form: theta - lr * g / (|g| + eps)
    th1, _, _ = LS.adam_step(theta0, grads[0], np.zeros(50), np.zeros(50), 1, wd=0.0)
    np.testing.assert_allclose(th1, theta0 - 1e-3 * grads[0] / (np.abs(grads[0]) + 1e-8), rtol=1e-12)


def test_rates():
    gt = IL.pack_bits(np.array([[1, 1, 1, 1, 0, 0] + [0] * 26], bool))
    pv = IL.pack_bits(np.array([[1, 1, 0, 0, 1, 0] + [0] * 26], bool))
    fnr, fpr = LS.rates(pv, gt)
    assert fnr == 0.5 and fpr == 0.25
