"""k = 3, stride 2, padding 1 sparse convolutions and their transposes (DOWN3 / UP3, the strided
sparse convolution of Sec. 2.3 with a 3^3 kernel and a dilated output set): the DOWN3 rulebook
bit-exact against the oracle's brute force, and the convolutions (FP64, FP32, BF16; gather and
product forms) against the oracle's masked dense definition."""
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


def test_strided3_argument_errors():
    """DOWN3 / UP3 need n_in and cap_in, and have no backward."""
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
    assert ops.npvs_conv_bwd_workspace_bytes(d) == 0
    ws = torch.zeros(1024, dtype=torch.uint8, device=DEV)
    with pytest.raises(L.NpvsError) as e:
        ops.npvs_sparse_conv_bwd(d, z, w, z[:8], z[:8], None, None, torch.zeros_like(w), None, ws)
    assert e.value.status == L.ERR_UNSUPPORTED
