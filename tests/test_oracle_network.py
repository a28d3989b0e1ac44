"""Pins for the oracle's sparse convolutions, networks and gradients (CPU only).

Sparse SubM3 / down2 / up2 equal the library's dense conv3d / conv_transpose3d on the zero-filled
grid, read at the active sites (the masked-dense definition, Sec. 2.3); SubM3 also equals a direct
loop; the analytic gradients equal central finite differences in float64.
"""
import itertools

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import npvs_inputs as I
from oracle import network as N



@pytest.fixture(autouse=True)
def _float64_default():
    """These pins build their tensors in float64; the default is restored after each test so that
    other test modules in the same process keep float32."""
    old = torch.get_default_dtype()
    torch.set_default_dtype(torch.float64)
    yield
    torch.set_default_dtype(old)


def random_level(rng, dims, frac):
    B, Dz, Hy, Wx = dims
    m = rng.random(dims) < frac
    m[0, 0, 0, 0] = True
    return N.Level(np.argwhere(m), dims), m


def dense_of(level, x):
    B, Dz, Hy, Wx = level.dims
    g = torch.zeros(B, x.shape[1], Dz, Hy, Wx)
    c = level.coords
    g[c[:, 0], :, c[:, 1], c[:, 2], c[:, 3]] = x
    return g


def test_subm3_equals_masked_conv3d_and_loops():
    rng = np.random.default_rng(0)
    lv, _ = random_level(rng, (2, 4, 5, 6), 0.3)
    cin, cout = 3, 5
    x = torch.tensor(rng.normal(size=(lv.n, cin)))
    W = torch.tensor(rng.normal(size=(27, cin, cout)))
    b = torch.tensor(rng.normal(size=cout))
    y = N.subm3(lv, x, W, b)
    wt = W.reshape(3, 3, 3, cin, cout).permute(4, 3, 0, 1, 2)     # out, in, kz, ky, kx
    ref = F.conv3d(dense_of(lv, x), wt, b, padding=1)
    c = lv.coords
    torch.testing.assert_close(y, ref[c[:, 0], :, c[:, 1], c[:, 2], c[:, 3]], rtol=1e-12, atol=1e-12)
    # direct loops on a few sites
    pos = {tuple(cc.tolist()): i for i, cc in enumerate(c)}
    for n in range(0, lv.n, max(1, lv.n // 7)):
        bb, z, yy, xx = c[n].tolist()
        acc = b.clone()
        for k, (dz, dy, dx) in enumerate(itertools.product((-1, 0, 1), repeat=3)):
            m = pos.get((bb, z + dz, yy + dy, xx + dx))
            if m is not None:
                acc = acc + x[m] @ W[k]
        torch.testing.assert_close(y[n], acc, rtol=1e-12, atol=1e-12)


def test_down2_and_up2_equal_strided_convs():
    rng = np.random.default_rng(1)
    fine, _ = random_level(rng, (2, 4, 6, 8), 0.25)
    coarse = fine.parent()
    cin, cout = 4, 3
    x = torch.tensor(rng.normal(size=(fine.n, cin)))
    W = torch.tensor(rng.normal(size=(8, cin, cout)))
    b = torch.tensor(rng.normal(size=cout))
    y = N.down2(fine, coarse, x, W, b)
    wt = W.reshape(2, 2, 2, cin, cout).permute(4, 3, 0, 1, 2)
    ref = F.conv3d(dense_of(fine, x), wt, b, stride=2)
    P = coarse.coords
    torch.testing.assert_close(y, ref[P[:, 0], :, P[:, 1], P[:, 2], P[:, 3]], rtol=1e-12, atol=1e-12)
    # the parent set is exactly the set of floor(p / 2)
    exp = sorted({(b_, z // 2, y_ // 2, x_ // 2) for b_, z, y_, x_ in fine.coords.tolist()})
    assert [tuple(p) for p in P.tolist()] == exp
    # up2: transposed conv onto the fine set
    z = torch.tensor(rng.normal(size=(coarse.n, cout)))
    Wu = torch.tensor(rng.normal(size=(8, cout, cin)))
    bu = torch.tensor(rng.normal(size=cin))
    yu = N.up2(coarse, fine, z, Wu, bu)
    wtu = Wu.reshape(2, 2, 2, cout, cin).permute(3, 4, 0, 1, 2)   # in, out, kz, ky, kx
    refu = F.conv_transpose3d(dense_of(coarse, z), wtu, bu, stride=2)
    c = fine.coords
    torch.testing.assert_close(yu, refu[c[:, 0], :, c[:, 1], c[:, 2], c[:, 3]], rtol=1e-12, atol=1e-12)


def small_unet():
    return I.unet_layers(8, [4, 6, 8], 8)


@pytest.mark.parametrize("which", ["plain", "unet"])
def test_gradients_match_central_differences(which):
    rng = np.random.default_rng(2)
    layers = I.plain_layers([8, 6, 5, 8]) if which == "plain" else small_unet()
    n_levels = 1 if which == "plain" else 3
    lv0, _ = random_level(rng, (1, 4, 8, 8), 0.3)
    levels = [lv0]
    for _ in range(n_levels - 1):
        levels.append(levels[-1].parent())
    ws, bs = I.kaiming_uniform(layers, seed=0, bias_scale=0.1)
    W, B = N.to_torch_params(ws, bs, requires_grad=True)
    x = torch.tensor(rng.random((lv0.n, 8)))
    tgt = torch.tensor(rng.normal(size=(lv0.n, 8)))

    def loss_fn():
        return ((N.forward(layers, W, B, levels, x) - tgt) ** 2).sum()

    L = loss_fn()
    L.backward()
    for li in range(len(layers)):
        for P in (W[li], B[li]):
            flat = P.detach().view(-1)
            for idx in rng.choice(flat.numel(), size=min(4, flat.numel()), replace=False):
                h = 1e-6 * max(1.0, abs(float(flat[idx])))
                old = float(flat[idx])
                with torch.no_grad():
                    flat[idx] = old + h
                    lp = float(loss_fn())
                    flat[idx] = old - h
                    lm = float(loss_fn())
                    flat[idx] = old
                fd = (lp - lm) / (2 * h)
                g = float(P.grad.view(-1)[idx])
                # central-difference rounding error ~ eps * L / h
                assert abs(g - fd) <= 1e-5 * max(abs(g), abs(fd)) + 1e-8 * abs(float(L.detach())), (layers[li].name, g, fd)


def test_rulebook_oracle_by_brute_force():
    """nbr[n][k] = m exactly when coords[m] - coords[n] is offset k (all pairs); parents equal
    the unique floor(p/2) set computed independently; down/up maps invert each other."""
    from oracle import rulebook as RB
    rng = np.random.default_rng(4)
    lv, _ = random_level(rng, (2, 4, 6, 6), 0.3)
    c = lv.coords.numpy()
    nbr = RB.neighbour_map(c)
    exp = np.full_like(nbr, -1)
    for n in range(len(c)):
        for m in range(len(c)):
            dlt = c[m] - c[n]
            if dlt[0] == 0 and np.all(np.abs(dlt[1:]) <= 1):
                exp[n, ((dlt[1] + 1) * 3 + dlt[2] + 1) * 3 + dlt[3] + 1] = m
    np.testing.assert_array_equal(nbr, exp)
    parents, down, up = RB.parent_level(c)
    np.testing.assert_array_equal(parents, lv.parent().coords.numpy())
    for n in range(len(c)):
        assert down[up[n] // 8, up[n] % 8] == n
    assert (down >= 0).sum() == len(c)


def test_down3_and_up3_equal_strided_convs_with_padding():
    """k = 3, stride 2, padding 1 and its transpose equal conv3d / conv_transpose3d (output_padding
    1 restores the even fine size) read at the active sites; the dilated output set is exactly the
    support of the dense strided conv of a positive input with positive weights."""
    rng = np.random.default_rng(5)
    fine, _ = random_level(rng, (2, 6, 4, 8), 0.15)
    coarse = fine.strided3()
    cin, cout = 3, 4
    x = torch.tensor(rng.normal(size=(fine.n, cin)))
    W = torch.tensor(rng.normal(size=(27, cin, cout)))
    b = torch.tensor(rng.normal(size=cout))
    y = N.down3(fine, coarse, x, W, b)
    wt = W.reshape(3, 3, 3, cin, cout).permute(4, 3, 0, 1, 2)        # out, in, kz, ky, kx
    ref = F.conv3d(dense_of(fine, x), wt, b, stride=2, padding=1)
    Q = coarse.coords
    torch.testing.assert_close(y, ref[Q[:, 0], :, Q[:, 1], Q[:, 2], Q[:, 3]], rtol=1e-12, atol=1e-12)
    pos = F.conv3d(dense_of(fine, torch.ones(fine.n, 1)), torch.ones(1, 1, 3, 3, 3), stride=2, padding=1)[:, 0]
    np.testing.assert_array_equal(Q.numpy(), torch.nonzero(pos > 0).numpy())
    # the dilated set holds the parent set and, where an odd coordinate p has p + 1 < the fine size,
    # the site (p + 1) / 2 as well
    assert {tuple(p) for p in fine.parent().coords.tolist()} <= {tuple(q) for q in Q.tolist()}
    assert coarse.n > fine.parent().n
    z = torch.tensor(rng.normal(size=(coarse.n, cout)))
    Wu = torch.tensor(rng.normal(size=(27, cout, cin)))
    bu = torch.tensor(rng.normal(size=cin))
    yu = N.up3(coarse, fine, z, Wu, bu)
    wtu = Wu.reshape(3, 3, 3, cout, cin).permute(3, 4, 0, 1, 2)      # in, out, kz, ky, kx
    refu = F.conv_transpose3d(dense_of(coarse, z), wtu, bu, stride=2, padding=1, output_padding=1)
    c = fine.coords
    torch.testing.assert_close(yu, refu[c[:, 0], :, c[:, 1], c[:, 2], c[:, 3]], rtol=1e-12, atol=1e-12)


def test_strided3_rulebook_oracle_by_brute_force():
    """The dict-built output set equals the max-pool one; down[q][k] and up[p][k] are the rows of
    every (q, p, k) with p = 2q + k - 1 found by a search over all pairs, and gathering through
    them reproduces down3 / up3."""
    from oracle import rulebook as RB
    rng = np.random.default_rng(6)
    fine, _ = random_level(rng, (2, 4, 6, 4), 0.2)
    c = fine.coords.numpy()
    outs, down, up = RB.strided3_level(c, fine.dims)
    coarse = fine.strided3()
    np.testing.assert_array_equal(outs, coarse.coords.numpy())
    exp_d = np.full_like(down, -1)
    exp_u = np.full_like(up, -1)
    for i, q in enumerate(outs):
        for n, p in enumerate(c):
            if q[0] != p[0]:
                continue
            k = p[1:] - 2 * q[1:] + 1
            if np.all((k >= 0) & (k <= 2)):
                t = (k[0] * 3 + k[1]) * 3 + k[2]
                exp_d[i, t] = n
                exp_u[n, t] = i
    np.testing.assert_array_equal(down, exp_d)
    np.testing.assert_array_equal(up, exp_u)
    cin, cout = 2, 3
    x = torch.tensor(rng.normal(size=(fine.n, cin)))
    W = torch.tensor(rng.normal(size=(27, cin, cout)))
    b = torch.tensor(rng.normal(size=cout))
    xz = torch.cat([x, torch.zeros(1, cin)])                            # row -1 -> zeros
    y = b + sum(xz[torch.tensor(down[:, k])] @ W[k] for k in range(27))
    torch.testing.assert_close(y, N.down3(fine, coarse, x, W, b), rtol=1e-12, atol=1e-12)
    z = torch.tensor(rng.normal(size=(coarse.n, cout)))
    Wu = torch.tensor(rng.normal(size=(27, cout, cin)))
    zz = torch.cat([z, torch.zeros(1, cout)])
    yu = b[:cin] + sum(zz[torch.tensor(up[:, k])] @ Wu[k] for k in range(27))
    torch.testing.assert_close(yu, N.up3(coarse, fine, z, Wu, b[:cin]), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("strided", [False, True])
def test_unet_wiring_equals_dense_straight_line_composition(strided):
    """Pin of the U-Net composition in `forward` (Sec. 3.3 f_theta on the interleaved grid; the
    U-Net reading: stem, per level two SubM3 then a stride-2 down conv, per decoder level the
    transposed up conv with ReLU, the encoder level's output added after that ReLU, two SubM3, a
    1x1 head without ReLU). The same network is written out a second way: dense conv3d /
    conv_transpose3d on the zero-filled grid, every layer's output multiplied by its level's
    active mask, the level masks from max-pooling the level-0 indicator (not from Level.parent),
    and the skip wiring as straight-line code. Every layer output kept by `forward` must equal
    the dense one at the active sites. A skip taken one layer early, a level pairing off by one
    or a ReLU on the head would fail here. strided: the same with k = 3, stride 2, padding 1 down convs
    (dense conv3d, levels from 3x3x3 max-pooling with stride 2 and padding 1) and their transposes
    (conv_transpose3d with output padding 1)."""
    rng = np.random.default_rng(11)
    dims = (2, 8, 8, 8)
    lv0, m = random_level(rng, dims, 0.3)
    layers = I.unet_layers(5, [4, 6, 8], 8, k3=strided)
    ws, bs = I.kaiming_uniform(layers, seed=3, bias_scale=0.2)
    W, B = N.to_torch_params(ws, bs)
    x = torch.tensor(rng.normal(size=(lv0.n, 5)))
    levels = N.build_levels(lv0.coords.numpy(), dims, 3, strided3=strided)
    keep = {}
    out = N.forward(layers, W, B, levels, x, keep=keep)

    P = {l.name: (W[i], B[i]) for i, l in enumerate(layers)}
    m0 = torch.tensor(m, dtype=torch.float64).unsqueeze(1)                  # B, 1, D, H, W
    pool = (lambda a: F.max_pool3d(a, kernel_size=3, stride=2, padding=1)) if strided else \
        (lambda a: F.max_pool3d(a, kernel_size=2, stride=2))
    m1 = pool(m0)
    m2 = pool(m1)

    def k3(name):
        w, b = P[name]
        return w.reshape(3, 3, 3, w.shape[1], w.shape[2]).permute(4, 3, 0, 1, 2), b

    def sub(name, a, mask, relu=True):
        w, b = k3(name)
        y = F.conv3d(a, w, b, padding=1)
        return (torch.relu(y) if relu else y) * mask

    kk = 3 if strided else 2
    pad = dict(padding=1) if strided else {}

    def down(name, a, mask):
        w, b = P[name]
        wt = w.reshape(kk, kk, kk, w.shape[1], w.shape[2]).permute(4, 3, 0, 1, 2)
        return torch.relu(F.conv3d(a, wt, b, stride=2, **pad)) * mask

    def up(name, a, mask):
        w, b = P[name]
        wt = w.reshape(kk, kk, kk, w.shape[1], w.shape[2]).permute(3, 4, 0, 1, 2)
        extra = dict(padding=1, output_padding=1) if strided else {}
        return torch.relu(F.conv_transpose3d(a, wt, b, stride=2, **extra)) * mask

    x0 = dense_of(lv0, x)
    D = {}
    D["stem"] = sub("stem", x0, m0)
    D["enc0a"] = sub("enc0a", D["stem"], m0)
    D["enc0b"] = sub("enc0b", D["enc0a"], m0)
    D["down0"] = down("down0", D["enc0b"], m1)
    D["enc1a"] = sub("enc1a", D["down0"], m1)
    D["enc1b"] = sub("enc1b", D["enc1a"], m1)
    D["down1"] = down("down1", D["enc1b"], m2)
    D["enc2a"] = sub("enc2a", D["down1"], m2)
    D["enc2b"] = sub("enc2b", D["enc2a"], m2)
    D["up1"] = up("up1", D["enc2b"], m1)
    D["up1+skip"] = D["up1"] + D["enc1b"]
    D["dec1a"] = sub("dec1a", D["up1+skip"], m1)
    D["dec1b"] = sub("dec1b", D["dec1a"], m1)
    D["up0"] = up("up0", D["dec1b"], m0)
    D["up0+skip"] = D["up0"] + D["enc0b"]
    D["dec0a"] = sub("dec0a", D["up0+skip"], m0)
    D["dec0b"] = sub("dec0b", D["dec0a"], m0)
    wh, bh = P["head"]
    D["head"] = F.conv3d(D["dec0b"], wh.reshape(1, 1, 1, wh.shape[1], wh.shape[2]).permute(4, 3, 0, 1, 2), bh) * m0

    lvl = {n: 0 for n in ("stem", "enc0a", "enc0b", "up0", "up0+skip", "dec0a", "dec0b", "head")}
    lvl.update({n: 1 for n in ("down0", "enc1a", "enc1b", "up1", "up1+skip", "dec1a", "dec1b")})
    lvl.update({n: 2 for n in ("down1", "enc2a", "enc2b")})
    assert set(keep) == set(D) == set(lvl)
    for i, mk in enumerate((m0, m1, m2)):          # the level sets themselves
        np.testing.assert_array_equal(levels[i].coords.numpy(), torch.nonzero(mk[:, 0] > 0).numpy())
    for name, dense in D.items():
        c = levels[lvl[name]].coords
        ref = dense[c[:, 0], :, c[:, 1], c[:, 2], c[:, 3]]
        assert keep[name].shape == ref.shape, name
        assert float(ref.abs().max()) > 0, name
        torch.testing.assert_close(keep[name], ref, rtol=1e-12, atol=1e-12, msg=name)
    torch.testing.assert_close(out, D["head"][lv0.coords[:, 0], :, lv0.coords[:, 1], lv0.coords[:, 2],
                                              lv0.coords[:, 3]], rtol=1e-12, atol=1e-12)
    # the dense composition gives zero outside the level-0 set
    assert float((D["head"] * (1 - m0)).abs().max()) == 0.0
