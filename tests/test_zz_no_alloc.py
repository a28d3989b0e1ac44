"""npvs_interleave_noalloc: the interleave for callers that cannot allocate device memory.

Such callers (an engine that reserves its whole GPU heap at start-up, or code on a frame's critical
path where cudaMalloc / cudaFree may not be called) cannot hand the library a workspace; this entry
point keeps its scratch in a fixed array inside the library instead. Its results must equal those of
npvs_interleave with a caller-provided workspace, call after call (the array is shared and keeps the
previous call's contents), and grids beyond the fixed limit must be refused with a clear error.

The file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

DEV = "cuda"


def random_bits(seed, B, D, H, W, frac):
    rng = np.random.default_rng(seed)
    occ = np.zeros((B, D, H, W), bool)
    n = int(frac * B * D * H * W / 6)
    b, z, y, x = (rng.integers(0, s, n) for s in (B, D, H, W))
    for dz in range(2):
        for dy in range(3):
            occ[b, np.minimum(z + dz, D - 1), np.minimum(y + dy, H - 1), x] = True
    words = np.packbits(occ.astype(np.uint8), axis=-1, bitorder="little")
    return np.ascontiguousarray(words).view("<u4").astype(np.uint32)


def run(fn, bits, grid_args, d, in_ch, dtype, capacity=None, expect_status=0, **kw):
    from paper_2509_24677_gb300 import ops
    W, H, D, B = grid_args
    sites = B * (W // d) * (H // d) * (D // d)
    cap = sites if capacity is None else capacity
    C = in_ch * d ** 3
    tdt = torch.bfloat16 if dtype == 1 else torch.float32
    coords = torch.full((max(cap, 1), 4), -5, dtype=torch.int32, device=DEV)
    feats = torch.full((max(cap, 1), C), 7.0, dtype=tdt, device=DEV)
    n = torch.full((1,), -3, dtype=torch.int32, device=DEV)
    table = torch.full((sites,), -9, dtype=torch.int32, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    fn(torch.from_numpy(bits.view(np.int32)).to(DEV), ops.grid(W, H, D, B), d, in_ch, dtype, cap, coords, feats, n,
       table=table, status=status, **kw)
    assert ops.npvs_check_status(status) == expect_status
    N = int(n.item())
    return N, coords[:N].cpu(), feats[:N].float().cpu(), table.cpu()


def assert_same(got, ref):
    assert got[0] == ref[0]
    for a, b in zip(got[1:], ref[1:]):
        assert torch.equal(a, b)


def test_noalloc_interleave_matches_workspace_entry_point():
    from paper_2509_24677_gb300 import _lib as L
    from paper_2509_24677_gb300 import ops
    cases = [  # two calls in a row with different inputs and shapes share the fixed scratch
        (random_bits(1, 2, 32, 40, 96, 0.04), (96, 40, 32, 2), 4, 2, L.BF16),
        (random_bits(2, 1, 64, 64, 64, 0.02), (64, 64, 64, 1), 2, 1, L.F32),
    ]
    for bits, g, d, in_ch, dtype in cases:
        ref = run(ops.npvs_interleave, bits, g, d, in_ch, dtype)
        got = run(ops.npvs_interleave_noalloc, bits, g, d, in_ch, dtype)
        assert ref[0] > 0 and got[0] == ref[0]
        for a, b in zip(got[1:], ref[1:]):
            assert torch.equal(a, b)
    # and the first case again after the second one
    bits, g, d, in_ch, dtype = cases[0]
    ref = run(ops.npvs_interleave, bits, g, d, in_ch, dtype)
    got = run(ops.npvs_interleave_noalloc, bits, g, d, in_ch, dtype)
    assert got[0] == ref[0] and all(torch.equal(a, b) for a, b in zip(got[1:], ref[1:]))


def test_noalloc_interleave_refuses_grids_beyond_its_limit():
    from paper_2509_24677_gb300 import _lib as L
    from paper_2509_24677_gb300 import ops
    # 2048 x 2048 x 64 froxels at d = 1: 268 M coarse sites, far above the 4,194,304 limit
    dummy = torch.zeros(16, dtype=torch.int32, device=DEV)
    with pytest.raises(L.NpvsError) as e:
        ops.npvs_interleave_noalloc(dummy, ops.grid(2048, 2048, 64, 1), 1, 1, L.F32, 1, dummy, dummy, dummy)
    assert e.value.status == L.ERR_UNSUPPORTED
    assert "limit" in str(e.value)


def test_noalloc_interleave_d16_and_capacity_overflow():
    """The d >= 16 path (features written by a separate pass over (row, slab) pairs) and a capacity
    below the active count (status NPVS_ERR_CAPACITY, n_active clamped to the capacity, the rows
    that fit written) give the same results through both entry points."""
    from paper_2509_24677_gb300 import _lib as L
    from paper_2509_24677_gb300 import ops
    bits = random_bits(3, 1, 64, 64, 64, 0.05)
    ref = run(ops.npvs_interleave, bits, (64, 64, 64, 1), 16, 2, L.BF16)
    got = run(ops.npvs_interleave_noalloc, bits, (64, 64, 64, 1), 16, 2, L.BF16)
    assert ref[0] > 8
    assert_same(got, ref)
    bits = random_bits(4, 2, 32, 40, 96, 0.04)
    full = run(ops.npvs_interleave, bits, (96, 40, 32, 2), 4, 1, L.F32)
    cap = full[0] // 3
    for _ in range(2):      # twice in a row: the shared scratch keeps the previous call's contents
        ref = run(ops.npvs_interleave, bits, (96, 40, 32, 2), 4, 1, L.F32, capacity=cap, expect_status=L.ERR_CAPACITY)
        got = run(ops.npvs_interleave_noalloc, bits, (96, 40, 32, 2), 4, 1, L.F32, capacity=cap,
                  expect_status=L.ERR_CAPACITY)
        assert ref[0] == cap
        assert_same(got, ref)
        assert torch.equal(got[1], full[1][:cap]) and torch.equal(got[2], full[2][:cap])


def test_noalloc_interleave_at_its_site_limit():
    """Exactly 4,194,304 coarse sites (256 x 256 x 64 froxels at d = 1: every CTA slot of the fixed
    scratch in use) equals the workspace entry point; one more column of 32 is refused."""
    from paper_2509_24677_gb300 import _lib as L
    from paper_2509_24677_gb300 import ops
    bits = random_bits(5, 1, 64, 256, 256, 0.01)
    ref = run(ops.npvs_interleave, bits, (256, 256, 64, 1), 1, 1, L.F32)
    got = run(ops.npvs_interleave_noalloc, bits, (256, 256, 64, 1), 1, 1, L.F32)
    assert ref[0] > 1000 and int((ref[3] >= 0).sum()) == ref[0]
    assert_same(got, ref)
    dummy = torch.zeros(16, dtype=torch.int32, device=DEV)
    with pytest.raises(L.NpvsError) as e:
        ops.npvs_interleave_noalloc(dummy, ops.grid(288, 256, 64, 1), 1, 1, L.F32, 1, dummy, dummy, dummy)
    assert e.value.status == L.ERR_UNSUPPORTED
