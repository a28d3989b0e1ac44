"""k = 3, stride 2, padding 1 sparse convolutions and their transposes (DOWN3 / UP3, the strided
sparse convolution of Sec. 2.3 with a 3^3 kernel and a dilated output set): the DOWN3 rulebook
bit-exact against the oracle's brute force, and the convolutions (FP64, FP32, BF16; gather and
product forms) and their backward against the oracle's masked dense definition."""
import numpy as np
import pytest
import torch

import npvs_inputs as I
from oracle import network as onet
from oracle import rulebook as orb
from test_gpu_parity import DEV, bf16_round, lib, normwise

pytestmark = pytest.mark.gpu


def strided3_levels(occ, coarse_cap=None):
    """Fine level of the active set `occ` ([B][Z][Y][X] bool), its SUBM3 table, and the DOWN3
    rulebook onto the halved grid. Returns (fine, coarse, down map, up map, fine coords, status)."""
    L, ops, P = lib()
    B, Z, Y, X = occ.shape
    fine = P.SparseLevel.alloc(X, Y, Z, B, X * Y * Z * B, DEV)
    cap = coarse_cap if coarse_cap is not None else (X // 2) * (Y // 2) * (Z // 2) * B
    coarse = P.SparseLevel.alloc(X // 2, Y // 2, Z // 2, B, cap, DEV)
    c0 = np.argwhere(occ).astype(np.int32)
    if len(c0):
        fine.coords[:len(c0)] = torch.from_numpy(c0).to(DEV)
    fine.n_rows.fill_(len(c0))
    down = torch.full((coarse.capacity, 27), -7, dtype=torch.int32, device=DEV)
    up = torch.full((fine.capacity, 27), -7, dtype=torch.int32, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    ops.npvs_build_rulebook(L.RB_SUBM3, fine, None, fine.nbr)
    ops.npvs_build_rulebook(L.RB_DOWN3, fine, coarse, down, up, status=status)
    return fine, coarse, down, up, c0, status


@pytest.mark.parametrize("shape,frac", [((2, 6, 8, 10), 0.12), ((1, 4, 4, 6), 1.0), ((1, 8, 6, 4), 0.0),
                                        ((2, 4, 6, 8), 0.03)])
def test_rulebook_down3_bit_exact(shape, frac):
    L, ops, _ = lib()
    occ = np.random.default_rng(int(frac * 100) + shape[1]).random(shape) < frac
    fine, coarse, down, up, c0, status = strided3_levels(occ)
    assert ops.npvs_check_status(status) == 0
    outs, down_ref, up_ref = orb.strided3_level(c0.astype(np.int64), shape)
    n = int(coarse.n_rows.item())
    assert n == len(outs)
    np.testing.assert_array_equal(coarse.coords[:n].cpu().numpy(), outs)
    np.testing.assert_array_equal(down[:n].cpu().numpy(), down_ref)
    np.testing.assert_array_equal(up[:len(c0)].cpu().numpy(), up_ref)
    assert (down[n:] == -7).all() and (up[len(c0):] == -7).all()      # rows past the counts untouched
    B, Z, Y, X = shape
    table = np.full(B * (Z // 2) * (Y // 2) * (X // 2), -1)
    for i, (b, z, y, x) in enumerate(outs.tolist()):
        table[((b * (Z // 2) + z) * (Y // 2) + y) * (X // 2) + x] = i
    np.testing.assert_array_equal(coarse.table.cpu().numpy(), table)


def test_rulebook_down3_capacity_overflow():
    L, ops, _ = lib()
    occ = np.random.default_rng(9).random((2, 6, 8, 10)) < 0.12
    outs, down_ref, _ = orb.strided3_level(np.argwhere(occ).astype(np.int64), occ.shape)
    cap = len(outs) - 5
    fine, coarse, down, up, c0, status = strided3_levels(occ, coarse_cap=cap)
    assert ops.npvs_check_status(status) == L.ERR_CAPACITY
    assert int(coarse.n_rows.item()) == cap
    np.testing.assert_array_equal(coarse.coords[:cap].cpu().numpy(), outs[:cap])
    np.testing.assert_array_equal(down[:cap].cpu().numpy(), down_ref[:cap])


CASES = [("down3", 16, 32), ("down3", 32, 64), ("down3", 64, 32), ("down3", 128, 128), ("up3", 32, 16),
         ("up3", 64, 64), ("up3", 128, 32), ("down3", 2, 16), ("up3", 16, 3)]


@pytest.mark.parametrize("dt,mode", [("f64", None), ("f32", None), ("f32", "product"), ("bf16", "gather"),
                                     ("bf16", "product"), ("bf16", "gather-split")])
@pytest.mark.parametrize("kind,cin,cout", CASES)
def test_strided3_conv_parity(kind, cin, cout, dt, mode):
    L, ops, P = lib()
    rng = np.random.default_rng(cin * 101 + cout * 7 + (kind == "up3"))
    occ = rng.random((2, 6, 8, 10)) < 0.15
    fine, coarse, down, up, c0, status = strided3_levels(occ)
    assert ops.npvs_check_status(status) == 0
    flv = onet.Level(c0, occ.shape)
    clv = flv.strided3()
    lv_in, lv_out, mp = (fine, coarse, down) if kind == "down3" else (coarse, fine, up)
    n_in, n_out = (flv.n, clv.n) if kind == "down3" else (clv.n, flv.n)
    assert int(lv_out.n_rows.item()) == n_out and int(lv_in.n_rows.item()) == n_in
    layer = I.Layer("t", kind, cin, cout, True)
    w = I.kaiming_uniform([layer], seed=11)[0][0]
    b = rng.normal(size=cout).astype(np.float32) * 0.1
    x = rng.normal(size=(n_in, cin)).astype(np.float32)
    skip = rng.normal(size=(n_out, cout)).astype(np.float32) if kind == "up3" else None
    if dt == "bf16":
        x_ref, w_ref, s_ref = bf16_round(x), bf16_round(w), (bf16_round(skip) if skip is not None else None)
    else:
        x_ref, w_ref, s_ref = x.astype(np.float64), w.astype(np.float64), skip
    T = lambda a: torch.tensor(np.asarray(a, np.float64))
    fn = onet.down3 if kind == "down3" else onet.up3
    args = (flv, clv) if kind == "down3" else (clv, flv)
    ref = torch.relu(fn(*args, T(x_ref), T(w_ref), T(b))).numpy()
    if s_ref is not None:
        ref = ref + s_ref
    tdt = {"bf16": torch.bfloat16, "f32": torch.float32, "f64": torch.float64}[dt]
    dtype = {"bf16": L.BF16, "f32": L.F32, "f64": L.F64}[dt]
    xin = torch.zeros(lv_in.capacity, cin, dtype=tdt, device=DEV)
    xin[:n_in] = torch.from_numpy(x).to(DEV).to(tdt)
    y = torch.full((lv_out.capacity, cout), float("nan"), dtype=tdt, device=DEV)
    sk = None
    if skip is not None:
        sk = torch.zeros(lv_out.capacity, cout, dtype=tdt, device=DEV)
        sk[:n_out] = torch.from_numpy(skip).to(DEV).to(tdt)
    kid = P.KIND[kind]
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    desc = ops.conv_desc(kid, dtype, cin, cout, True, mp, lv_out.n_rows, lv_out.capacity, n_in=lv_in.n_rows,
                         cap_in=lv_in.capacity, status=st, form={"gather": 1, "gather-split": 1, "product": 2}.get(mode, 0),
                         max_split=1 if mode == "gather" else 0)
    if mode in ("product", "gather-split"):
        ws = ops.conv_workspace(ops.npvs_conv_workspace_bytes(desc), DEV)
        desc.workspace, desc.workspace_bytes = ws.data_ptr(), ws.numel()
    w_dev = torch.from_numpy(w).to(DEV).contiguous()
    if dt == "bf16":
        wp = torch.empty(ops.npvs_packed_weight_bytes(kid, cin, cout), dtype=torch.uint8, device=DEV)
        ops.npvs_pack_weights(kid, cin, cout, w_dev, wp)
        w_dev = wp
    elif dt == "f64":
        w_dev = w_dev.double()
    bias = torch.from_numpy(b).to(DEV)
    if dt == "f64":
        bias = bias.double()
    ops.npvs_sparse_conv_fwd(desc, xin, w_dev, bias, sk, y)
    assert ops.npvs_check_status(st) == 0
    got = y[:n_out].double().cpu().numpy()
    assert not np.isnan(got).any()
    assert torch.isnan(y[n_out:].double()).all()
    tol = {"bf16": 8e-3, "f32": 1e-5, "f64": 1e-12}[dt]
    assert normwise(got, ref) <= tol


BWD_CASES = [("down3", 16, 32), ("down3", 32, 64), ("down3", 64, 32), ("up3", 32, 16), ("up3", 64, 64),
             ("up3", 128, 32)]


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("kind,cin,cout", BWD_CASES)
def test_strided3_conv_backward_parity(kind, cin, cout, dt):
    """Backward of the k = 3, stride 2 pair against the oracle's autograd of its masked dense
    definition: g = dy * 1[y > 0], db = sum g, dW_k = sum x[in]^T g[out] over the tap's pairs, and dx
    by the transposed conv on the same rulebook (DOWN3's is UP3 with W_k^T, and the other way
    round), plus a gradient dx_add from another path; rows past n_in untouched; bitwise
    reproducible."""
    L, ops, P = lib()
    rng = np.random.default_rng(cin * 31 + cout * 3 + (kind == "up3"))
    occ = rng.random((2, 6, 8, 10)) < 0.15
    fine, coarse, down, up, c0, status = strided3_levels(occ)
    assert ops.npvs_check_status(status) == 0
    flv = onet.Level(c0, occ.shape)
    clv = flv.strided3()
    if kind == "down3":
        lv_in, lv_out, mp, mp2, n_in, n_out = fine, coarse, down, up, flv.n, clv.n
    else:
        lv_in, lv_out, mp, mp2, n_in, n_out = coarse, fine, up, down, clv.n, flv.n
    w = I.kaiming_uniform([I.Layer("t", kind, cin, cout, True)], seed=13)[0][0]
    b = (rng.normal(size=cout) * 0.1).astype(np.float32)
    x = rng.normal(size=(n_in, cin)).astype(np.float32)
    dy = rng.normal(size=(n_out, cout)).astype(np.float32)
    add = rng.normal(size=(n_in, cin)).astype(np.float32)
    rnd = bf16_round if dt == "bf16" else (lambda a: np.asarray(a, np.float64))
    x_r, dy_r, add_r = rnd(x), rnd(dy), rnd(add)
    xt = torch.tensor(x_r, requires_grad=True)
    wt = torch.tensor(w.astype(np.float64), requires_grad=True)
    bt = torch.tensor(b.astype(np.float64), requires_grad=True)
    pre = onet.down3(flv, clv, xt, wt, bt) if kind == "down3" else onet.up3(clv, flv, xt, wt, bt)
    y_ref = torch.relu(pre)
    g = torch.tensor(dy_r) * (y_ref > 0).double()
    gx, gw, gb = torch.autograd.grad(pre, (xt, wt, bt), grad_outputs=g)
    dtype = {"f32": L.F32, "bf16": L.BF16, "f64": L.F64}[dt]
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f64": torch.float64}[dt]
    mdt = torch.float64 if dt == "f64" else torch.float32

    def dev_rows(a, cap):
        t = torch.zeros(cap, a.shape[1], dtype=tdt, device=DEV)
        t[:len(a)] = torch.from_numpy(np.asarray(a, np.float64)).to(DEV).to(tdt)
        return t

    xin, dyd = dev_rows(x, lv_in.capacity), dev_rows(dy, lv_out.capacity)
    yd, addd = dev_rows(y_ref.detach().numpy(), lv_out.capacity), dev_rows(add, lv_in.capacity)
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    desc = ops.conv_desc(P.KIND[kind], dtype, cin, cout, True, mp, lv_out.n_rows, lv_out.capacity, map2=mp2,
                         n_in=lv_in.n_rows, cap_in=lv_in.capacity, status=st)
    ws = ops.conv_workspace(ops.npvs_conv_bwd_workspace_bytes(desc), DEV)
    w_dev = torch.from_numpy(w).to(DEV).to(mdt).contiguous()
    results = []
    reps = 2
    if dt == "bf16":   # a third call reads the dgrad image packed beforehand (npvs_pack_weights_many)
        reps = 3
        wt_img = torch.empty(ops.npvs_packed_weight_bytes_transposed(P.KIND[kind], cin, cout), dtype=torch.uint8,
                             device=DEV)
        ops.npvs_pack_weights_many([(P.KIND[kind], cin, cout, 1, w_dev, wt_img)])
    for rep in range(reps):
        dx = torch.full((lv_in.capacity, cin), float("nan"), dtype=tdt, device=DEV)
        dw = torch.full(w.shape, float("nan"), dtype=mdt, device=DEV)
        db = torch.full((cout,), float("nan"), dtype=mdt, device=DEV)
        desc.w_transposed = wt_img.data_ptr() if rep == 2 else None
        ops.npvs_sparse_conv_bwd(desc, xin, w_dev, yd, dyd, dx, addd, dw, db, ws)
        assert ops.npvs_check_status(st) == 0
        results.append((dx, dw, db))
    dx, dw, db = results[0]
    tol_dx = {"f32": 1e-5, "bf16": 2e-2, "f64": 1e-12}[dt]
    tol_w = {"f32": 1e-5, "bf16": 1e-5, "f64": 1e-12}[dt]
    assert normwise(dw.cpu().numpy(), gw.numpy()) <= tol_w
    assert normwise(db.cpu().numpy(), gb.numpy()) <= tol_w
    got = dx[:n_in].double().cpu().numpy()
    assert normwise(got - add_r, gx.numpy()) <= tol_dx, normwise(got - add_r, gx.numpy())
    assert torch.isnan(dx[n_in:].float()).all()
    for other in results[1:]:
        for a, b2 in zip(results[0], other):
            assert torch.equal(torch.nan_to_num(a.float(), 7.0), torch.nan_to_num(b2.float(), 7.0))


def test_strided3_argument_errors():
    """DOWN3 / UP3 need n_in and cap_in, and their dgrad needs the rulebook's other map."""
    L, ops, P = lib()
    occ = np.ones((1, 4, 4, 4), bool)
    fine, coarse, down, up, c0, _ = strided3_levels(occ)
    z = torch.zeros(64, 16, device=DEV)
    w = torch.zeros(27, 16, 16, device=DEV)
    d = ops.conv_desc(L.CONV_DOWN3, L.F32, 16, 16, True, down, coarse.n_rows, coarse.capacity)
    with pytest.raises(L.NpvsError) as e:
        ops.npvs_sparse_conv_fwd(d, z, w, None, None, z[:8])
    assert e.value.status == L.ERR_INVALID_ARG
    d = ops.conv_desc(L.CONV_DOWN3, L.F32, 16, 16, True, down, coarse.n_rows, coarse.capacity,
                      n_in=fine.n_rows, cap_in=fine.capacity)
    nb = ops.npvs_conv_bwd_workspace_bytes(d)
    assert nb > 0
    ws = torch.zeros(nb, dtype=torch.uint8, device=DEV)
    with pytest.raises(L.NpvsError) as e:     # dx without map2
        ops.npvs_sparse_conv_bwd(d, z, w, z[:8], z[:8], z, None, torch.zeros_like(w), None, ws)
    assert e.value.status == L.ERR_INVALID_ARG
