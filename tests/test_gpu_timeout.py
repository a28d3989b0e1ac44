"""The bounded waits of the tensor-core kernels, made to run out (GPU).

Every mbarrier wait in the tcgen05 kernels is bounded; on expiry the CTA stops issuing copies and
MMAs, waits for those in flight, frees its tensor memory, returns, and NPVS_ERR_TIMEOUT reaches the
caller through the status word. Here the bound is lowered with npvs_set_wait_limit to one SM cycle,
so that every wait that is not already satisfied when it is first tested expires (a bulk copy from L2
takes a few hundred cycles, and the epilogue always waits for copies and MMAs): the kernels must
return and report the timeout, and with the default bound restored the same calls on the same
context must give correct results again. Only kernel forms whose in-flight work is drained by the
threads that issued it run here: the product form (one thread issues every TMA copy), the cp.async
gather (each thread waits for its own copies) and the weight-gradient kernel (cp.async).
"""
import numpy as np
import pytest
import torch

import npvs_inputs as I
from oracle import network as onet
from test_gpu_parity import DEV, bf16_round, build_rulebooks, lib, make_levels, normwise

pytestmark = pytest.mark.gpu

SHORT = 1  # SM cycles: any wait not satisfied at its first test expires


def conv_case(cin, cout, form, seed):
    """A BF16 submanifold conv on ~800 coarse sites: device buffers, its descriptor and the FP64
    oracle's output on the BF16-rounded operands."""
    L, ops, P = lib()
    rng = np.random.default_rng(seed)
    occ = rng.random((2, 10, 12, 14)) < 0.12
    lvs, c0 = make_levels(occ, 1)
    build_rulebooks(lvs)
    torch.cuda.synchronize()
    fine = onet.Level(c0, occ.shape)
    w = I.kaiming_uniform([I.Layer("t", "subm3", cin, cout, True)], seed=5)[0][0]
    b = (rng.normal(size=cout) * 0.1).astype(np.float32)
    x = rng.normal(size=(fine.n, cin)).astype(np.float32)
    T = lambda a: torch.tensor(np.asarray(a, np.float64))
    ref = torch.relu(onet.subm3(fine, T(bf16_round(x)), T(bf16_round(w)), T(b))).numpy()
    lv = lvs[0]
    xin = torch.zeros(lv.capacity, cin, dtype=torch.bfloat16, device=DEV)
    xin[:fine.n] = torch.from_numpy(x).to(DEV).to(torch.bfloat16)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    desc = ops.conv_desc(P.KIND["subm3"], L.BF16, cin, cout, True, lv.nbr, lv.n_rows, lv.capacity,
                         n_in=lv.n_rows, cap_in=lv.capacity, status=status, form=form)
    wp = torch.empty(ops.npvs_packed_weight_bytes(P.KIND["subm3"], cin, cout), dtype=torch.uint8, device=DEV)
    ops.npvs_pack_weights(P.KIND["subm3"], cin, cout, torch.from_numpy(w).to(DEV), wp)
    # the levels are returned too: the descriptor holds raw pointers into them
    return desc, status, xin, wp, torch.from_numpy(b).to(DEV), ref, fine.n, lv.capacity, lvs


def run_fwd(case, with_workspace):
    L, ops, _ = lib()
    desc, status, xin, wp, b, ref, n, cap, _ = case
    ws = None
    if with_workspace:   # a fresh zero-filled workspace each call
        ws = ops.conv_workspace(ops.npvs_conv_workspace_bytes(desc), DEV)
        desc.workspace, desc.workspace_bytes = ws.data_ptr(), ws.numel()
    y = torch.zeros(cap, desc.cout, dtype=torch.bfloat16, device=DEV)
    ops.npvs_sparse_conv_fwd(desc, xin, wp, b, None, y)
    return ops.npvs_check_status(status), y[:n].float().cpu().numpy()


@pytest.fixture
def short_waits():
    _, ops, _ = lib()
    prev = ops.npvs_set_wait_limit(SHORT)
    try:
        yield
    finally:
        ops.npvs_set_wait_limit(0)
    assert prev in (0, 4_000_000_000)


@pytest.mark.parametrize("cin,cout,form,workspace", [(32, 32, 2, True),     # product form: one TMA issuer
                                                     (16, 16, 1, False)])   # cp.async gather
def test_conv_wait_timeout_is_reported_and_recoverable(cin, cout, form, workspace):
    L, ops, _ = lib()
    case = conv_case(cin, cout, form, seed=cin * 13 + form)
    prev = ops.npvs_set_wait_limit(SHORT)
    try:
        st, _ = run_fwd(case, workspace)
    finally:
        assert ops.npvs_set_wait_limit(0) == SHORT
    assert st == L.ERR_TIMEOUT       # the kernels returned (the status read synchronises) and said why
    assert prev == 4_000_000_000
    st, got = run_fwd(case, workspace)           # default bound: the same call is correct again
    assert st == 0
    assert normwise(got, case[5]) <= 8e-3


def test_wgrad_wait_timeout_is_reported(short_waits):
    """The BF16 backward (dgrad on the cp.async gather, weight gradient on tcgen05) under the short
    bound reports the timeout; the default bound is restored by the fixture."""
    L, ops, P = lib()
    desc, status, xin, wp, b, ref, n, cap, lvs = conv_case(16, 16, 0, seed=3)
    cin = cout = 16
    w = torch.from_numpy(I.kaiming_uniform([I.Layer("t", "subm3", cin, cout, True)], seed=5)[0][0]).to(DEV)
    y = torch.zeros(cap, cout, dtype=torch.bfloat16, device=DEV)
    y[:n] = torch.from_numpy(ref).to(DEV).to(torch.bfloat16)
    dy = torch.randn(cap, cout, device=DEV).to(torch.bfloat16)
    ws = ops.conv_workspace(ops.npvs_conv_bwd_workspace_bytes(desc), DEV)
    dx = torch.zeros(cap, cin, dtype=torch.bfloat16, device=DEV)
    dw = torch.zeros(27, cin, cout, device=DEV)
    db = torch.zeros(cout, device=DEV)
    ops.npvs_sparse_conv_bwd(desc, xin, w, y, dy, dx, None, dw, db, ws)
    assert ops.npvs_check_status(status) == L.ERR_TIMEOUT

