"""GPU parity: every hot-path step through the C ABI against the FP64 / binary32-mirror oracle.

Bit-exact: froxelization, interleave (coords, table, features incl. BF16 rounding), rulebooks.
Floating point: single convolutions (FP32 normwise 1e-5, BF16 8e-3 on BF16-rounded operands),
whole networks per layer output (FP32 1e-4, BF16 2e-2 normwise) and thresholded PVS agreement
>= 99.9% of occupied froxels. Sizes span several tiles with ragged tails; the full 256x256x128
workload runs in the bench's launch configuration.
"""
import dataclasses

import numpy as np
import pytest
import torch

import npvs_inputs as I
from oracle import camera as ocam
from oracle import froxel as ofx
from oracle import interleave as oil
from oracle import network as onet
from oracle import rulebook as orb

pytestmark = pytest.mark.gpu

DEV = "cuda"


def lib():
    from paper_2509_24677_gb300 import _lib, ops, pipeline
    return _lib, ops, pipeline


def u32(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def popcount(a):
    return int(np.unpackbits(np.ascontiguousarray(a).view(np.uint8)).sum())


def normwise(y, ref):
    y = np.asarray(y, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.abs(y - ref).max() / max(np.abs(ref).max(), 1e-30))


def gpu_froxelize(scenes, vcs, W, H, D, s):
    L, ops, _ = lib()
    cams = [ops.npvs_camera_setup(v, D) for v in vcs]
    boxes = np.concatenate(scenes, 0)
    off = np.cumsum([0] + [len(b) for b in scenes]).astype(np.int32)
    occ = torch.empty(len(vcs) * D * H * (W // 32), dtype=torch.int32, device=DEV)
    ops.npvs_froxelize(torch.from_numpy(boxes).to(DEV), torch.from_numpy(off).to(DEV),
                       ops.cameras_to_device(cams), ops.grid(W, H, D, len(vcs)), s, occ)
    torch.cuda.synchronize()
    return u32(occ).reshape(len(vcs), D, H, W // 32)


# ------------------------------------------------------------------------------------------
# a2 froxelization
# ------------------------------------------------------------------------------------------

def test_froxelize_plain64_bit_exact():
    boxes, vc = I.plain64_scene()
    got = gpu_froxelize([boxes], [vc], 64, 64, 32, 8)[0]
    ref = ofx.froxelize(ocam.frustum(vc, 32), boxes, 64, 64, 32, 8)
    assert popcount(ref) > 1000
    assert popcount(got ^ ref) == 0


def test_froxelize_batched_ragged_bit_exact():
    """Three viewcells from two small cities in one launch; H, D not powers of two."""
    p = dataclasses.replace(I.CityParams(), n_buildings=400)
    scenes = [I.city_boxes(0, p), I.city_boxes(1, p), I.city_boxes(0, p)]
    vcs = I.city_viewcells(0, 2, p) + I.city_viewcells(5, 1, p)
    W, H, D, s = 96, 40, 24, 3
    got = gpu_froxelize(scenes, vcs, W, H, D, s)
    for b in range(3):
        ref = ofx.froxelize(ocam.frustum(vcs[b], D), scenes[b], W, H, D, s)
        assert popcount(ref) > 100
        assert popcount(got[b] ^ ref) == 0, b


def test_froxelize_empty_and_culled():
    vc = I.Viewcell(centre=(0.0, 0.0, 0.0), half=0.5, yaw=0.0)
    behind = np.array([[-5, -5, -30, 5, 5, -10]], np.float32)
    got = gpu_froxelize([behind], [vc], 32, 32, 16, 2)
    assert popcount(got) == 0
    got = gpu_froxelize([np.zeros((0, 6), np.float32)], [vc], 32, 32, 16, 2)
    assert popcount(got) == 0


def test_froxelize_city256_full_size_sampled_columns():
    """Full 256x256x128, s=8 grid of the benchmark workload; 800 sampled froxel columns recomputed
    by the oracle ray by ray."""
    wl = I.workload("city256")
    boxes = I.city_boxes(0)
    vc = I.city_viewcells(0, 1)[0]
    got = gpu_froxelize([boxes], [vc], wl.W, wl.H, wl.D, wl.supersample)[0]
    dense = oil.unpack_bits(got, wl.W)                  # D, H, W
    occ_cols = np.argwhere(dense.any(0))                # (y, x) with geometry
    rng = np.random.default_rng(0)
    pick = np.concatenate([occ_cols[rng.choice(len(occ_cols), 600, replace=False)],
                           np.stack([rng.integers(0, wl.H, 200), rng.integers(0, wl.W, 200)], 1)])
    cols = np.stack([pick[:, 1], pick[:, 0]], 1)       # (x, y)
    ref = ofx.froxel_columns(ocam.frustum(vc, wl.D), boxes, wl.W, wl.H, wl.D, wl.supersample, cols)
    for (x, y), w in zip(cols, ref):
        exp = [k for k in range(wl.D) if (w[k >> 5] >> (k & 31)) & 1]
        assert list(np.nonzero(dense[:, y, x])[0]) == exp, (x, y)
    occ = dense.mean()
    assert 0.02 <= occ <= 0.08, occ


@pytest.mark.parametrize("vc_index,height,s", [(3, (2.0, 2.0), 8), (1, (30.0, 60.0), 4)])
def test_froxelize_city256_whole_frame_bit_exact(vc_index, height, s):
    """Whole 256x256x128 frames of the 2,001-box city against the oracle's full grid: a street-level
    viewcell at s = 8 (the ground at grazing angles, walls edge-on) and one 30-60 units up at s = 4
    (roofs from above). Every column the kernel settles from interval bounds must give the same bits
    as casting its rays."""
    wl = I.workload("city256")
    boxes = I.city_boxes(0)
    vc = I.city_viewcells(0, vc_index + 1, height=height)[vc_index]
    got = gpu_froxelize([boxes], [vc], wl.W, wl.H, wl.D, s)[0]
    ref = ofx.froxelize(ocam.frustum(vc, wl.D), boxes, wl.W, wl.H, wl.D, s)
    assert popcount(ref) > 20000
    assert popcount(got ^ ref) == 0


def test_froxelize_more_faces_than_the_fused_offsets_bit_exact():
    """A batch of two viewcells of the 12,000-building city (144,012 faces, more than the 65,536 whose
    offsets the item kernel adds itself): the chunked scan path, bit for bit against the oracle."""
    p = dataclasses.replace(I.CityParams(), n_buildings=12000, mu=2.3, sigma=0.7)
    boxes = I.city_boxes(2, p)
    vcs = I.city_viewcells(2, 2, p, height=(2.0, 60.0))
    W, H, D, s = 32, 32, 16, 2
    assert 2 * 6 * len(boxes) > 65536
    got = gpu_froxelize([boxes, boxes], vcs, W, H, D, s)
    for b in range(2):
        ref = ofx.froxelize(ocam.frustum(vcs[b], D), boxes, W, H, D, s)
        assert popcount(ref) > 100
        assert popcount(got[b] ^ ref) == 0, b


# ------------------------------------------------------------------------------------------
# a3 interleave, a7 de-interleave
# ------------------------------------------------------------------------------------------

def clustered_bits(rng, B, D, H, W, frac=0.04):
    occ = np.zeros((B, D, H, W), bool)
    for b in range(B):
        n = int(frac * D * H * W / 20)
        z, y, x = rng.integers(0, D, n), rng.integers(0, H, n), rng.integers(0, W, n)
        for dz in range(2):
            for dy in range(3):
                occ[b, np.minimum(z + dz, D - 1), np.minimum(y + dy, H - 1), x] = True
    return occ


@pytest.mark.parametrize("d,in_ch,dt", [(2, 1, "f32"), (4, 2, "bf16"), (4, 2, "f32"), (8, 2, "bf16"), (2, 2, "bf16"),
                                        (16, 1, "bf16"), (16, 2, "f32"), (1, 1, "bf16"), (1, 2, "f32"),
                                        (8, 1, "f32"), (32, 1, "bf16"), (32, 1, "f32")])
def test_interleave_bit_exact(d, in_ch, dt):
    L, ops, _ = lib()
    rng = np.random.default_rng(d * 10 + in_ch)
    B, D, H, W = 2, 6 * d, 5 * d, 96 if d != 8 else 64
    occ = clustered_bits(rng, B, D, H, W)
    bits = oil.pack_bits(occ)
    coords_ref, feats_ref, active = oil.interleave(bits, W, d, in_ch)
    C = in_ch * d ** 3
    cap = active.size
    g = ops.grid(W, H, D, B)
    tdt = torch.bfloat16 if dt == "bf16" else torch.float32
    coords = torch.zeros(cap, 4, dtype=torch.int32, device=DEV)
    feats = torch.zeros(cap, C, dtype=tdt, device=DEV)
    n = torch.zeros(1, dtype=torch.int32, device=DEV)
    table = torch.zeros(active.size, dtype=torch.int32, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    ops.npvs_interleave(torch.from_numpy(bits.view(np.int32)).to(DEV), g, d, in_ch,
                        L.BF16 if dt == "bf16" else L.F32, cap, coords, feats, n, table=table, status=status)
    assert ops.npvs_check_status(status) == 0
    N = int(n.item())
    assert N == len(coords_ref)
    np.testing.assert_array_equal(coords.cpu().numpy()[:N], coords_ref)
    exp_table = np.full(active.size, -1)
    exp_table[np.flatnonzero(active.ravel())] = np.arange(N)
    np.testing.assert_array_equal(table.cpu().numpy(), exp_table)
    if dt == "bf16":
        got = feats[:N].view(torch.int16).cpu().numpy().view(np.uint16)
        exp = oil.to_bf16_bits(feats_ref.astype(np.float32))
    else:
        got = feats[:N].cpu().numpy()
        exp = feats_ref.astype(np.float32)
    np.testing.assert_array_equal(got, exp)


@pytest.mark.parametrize("cap_frac", [1.0, 0.5])
def test_interleave_large_grid_scan_path(cap_frac):
    """524,288 coarse sites at d = 1 (2,048 CTAs, more than the 1,024 whose offsets the write kernel
    sums itself): the single-CTA scan path, bit-exact against the oracle; with half the needed
    capacity, the capacity status and the clamped row count."""
    L, ops, _ = lib()
    rng = np.random.default_rng(11)
    B, D, H, W = 1, 64, 64, 128
    occ = clustered_bits(rng, B, D, H, W, frac=0.03)
    bits = oil.pack_bits(occ)
    coords_ref, feats_ref, active = oil.interleave(bits, W, 1, 2)
    N = len(coords_ref)
    cap = max(1, int(cap_frac * N))
    g = ops.grid(W, H, D, B)
    coords = torch.zeros(cap, 4, dtype=torch.int32, device=DEV)
    feats = torch.zeros(cap, 2, dtype=torch.float32, device=DEV)
    n = torch.zeros(1, dtype=torch.int32, device=DEV)
    table = torch.zeros(active.size, dtype=torch.int32, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    ops.npvs_interleave(torch.from_numpy(bits.view(np.int32)).to(DEV), g, 1, 2, L.F32, cap, coords, feats, n,
                        table=table, status=status)
    st = ops.npvs_check_status(status)
    m = min(cap, N)
    assert int(n.item()) == m
    assert st == (0 if cap >= N else L.ERR_CAPACITY)
    np.testing.assert_array_equal(coords.cpu().numpy()[:m], coords_ref[:m])
    np.testing.assert_array_equal(feats.cpu().numpy()[:m], feats_ref[:m].astype(np.float32))
    exp_table = np.full(active.size, -1)
    idx = np.flatnonzero(active.ravel())[:m]
    exp_table[idx] = np.arange(m)
    np.testing.assert_array_equal(table.cpu().numpy(), exp_table)


def test_interleave_empty_full_and_overflow():
    L, ops, _ = lib()
    d, B, D, H, W = 4, 1, 8, 8, 32
    g = ops.grid(W, H, D, B)
    sites = (D // d) * (H // d) * (W // d)
    for fill, exp_n in ((0, 0), (1, sites)):
        bits = np.full((B, D, H, W // 32), 0xFFFFFFFF if fill else 0, np.uint32)
        coords = torch.zeros(sites, 4, dtype=torch.int32, device=DEV)
        feats = torch.zeros(sites, 2 * d ** 3, dtype=torch.float32, device=DEV)
        n = torch.full((1,), -7, dtype=torch.int32, device=DEV)
        ops.npvs_interleave(torch.from_numpy(bits.view(np.int32)).to(DEV), g, d, 2, L.F32, sites, coords, feats, n)
        assert int(n.item()) == exp_n
    # capacity overflow: flagged, count clamped, nothing written past capacity
    bits = np.full((B, D, H, W // 32), 0xFFFFFFFF, np.uint32)
    cap = 5
    coords = torch.full((cap + 3, 4), -9, dtype=torch.int32, device=DEV)
    feats = torch.zeros(cap + 3, 2 * d ** 3, dtype=torch.float32, device=DEV)
    n = torch.zeros(1, dtype=torch.int32, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    ops.npvs_interleave(torch.from_numpy(bits.view(np.int32)).to(DEV), g, d, 2, L.F32, cap, coords, feats, n,
                        status=status)
    assert ops.npvs_check_status(status) == L.ERR_CAPACITY
    assert int(n.item()) == cap
    assert (coords[cap:].cpu().numpy() == -9).all()


def test_deinterleave_threshold_and_mask():
    L, ops, _ = lib()
    rng = np.random.default_rng(11)
    d, B, D, H, W = 4, 2, 16, 20, 64
    occ = clustered_bits(rng, B, D, H, W, 0.08)
    bits = oil.pack_bits(occ)
    coords_ref, _, active = oil.interleave(bits, W, d, 1)
    N = len(coords_ref)
    logits = rng.normal(size=(N, d ** 3)).astype(np.float32)
    logits[np.abs(logits) < 1e-5] = 0.5          # keep clear of the p = 0.5 tie
    table = np.full(active.size, -1, np.int32)
    table[np.flatnonzero(active.ravel())] = np.arange(N)
    pvs = torch.zeros(bits.size, dtype=torch.int32, device=DEV)
    probs = torch.zeros(N + 7, d ** 3, dtype=torch.float32, device=DEV)
    n = torch.tensor([N], dtype=torch.int32, device=DEV)
    ops.npvs_deinterleave(torch.from_numpy(logits).to(DEV), torch.from_numpy(table).to(DEV), n,
                          ops.grid(W, H, D, B), d, 0.5, torch.from_numpy(bits.view(np.int32)).to(DEV), pvs,
                          probs_out=probs, capacity=N + 7)
    ref_bits, ref_dense = oil.pvs_from_logits(coords_ref, logits.astype(np.float64), bits, W, d)
    assert popcount(u32(pvs).reshape(bits.shape) ^ ref_bits) == 0
    np.testing.assert_allclose(probs[:N].cpu().numpy(), 1 / (1 + np.exp(-logits.astype(np.float64))), rtol=2e-7)


# ------------------------------------------------------------------------------------------
# a4 rulebooks
# ------------------------------------------------------------------------------------------

def make_levels(occ_coarse, n_levels):
    """Device levels for a given active set of the finest coarse grid (numpy bool [B][Z][Y][X])."""
    _, ops, P = lib()
    B, Z, Y, X = occ_coarse.shape
    lvs = []
    for li in range(n_levels):
        cap = X * Y * Z * B
        lvs.append(P.SparseLevel.alloc(X, Y, Z, B, cap, DEV))
        X, Y, Z = X // 2, Y // 2, Z // 2
    c0 = np.argwhere(occ_coarse).astype(np.int32)
    lvs[0].coords[:len(c0)] = torch.from_numpy(c0).to(DEV)
    lvs[0].n_rows.fill_(len(c0))
    for li in range(n_levels - 1):
        lvs[li].down = torch.zeros(lvs[li + 1].capacity, 8, dtype=torch.int32, device=DEV)
        lvs[li].up = torch.zeros(lvs[li].capacity, 1, dtype=torch.int32, device=DEV)
    return lvs, c0


def build_rulebooks(lvs, prebuilt=False):
    L, ops, _ = lib()
    for li, lv in enumerate(lvs):
        ops.npvs_build_rulebook(L.RB_SUBM3_TABLE if (prebuilt and li > 0) else L.RB_SUBM3, lv, None, lv.nbr)
        if li + 1 < len(lvs):
            ops.npvs_build_rulebook(L.RB_DOWN2, lv, lvs[li + 1], lv.down, lv.up)


@pytest.mark.parametrize("prebuilt", [False, True])
def test_rulebooks_bit_exact(prebuilt):
    rng = np.random.default_rng(3)
    occ = rng.random((2, 8, 12, 16)) < 0.15
    lvs, c0 = make_levels(occ, 3)
    build_rulebooks(lvs, prebuilt)
    torch.cuda.synchronize()
    coords = c0
    for li in range(3):
        lv = lvs[li]
        n = int(lv.n_rows.item())
        assert n == len(coords)
        np.testing.assert_array_equal(lv.coords[:n].cpu().numpy(), coords)
        np.testing.assert_array_equal(lv.nbr[:n].cpu().numpy(), orb.neighbour_map(coords))
        if li < 2:
            parents, down, up = orb.parent_level(coords)
            npar = int(lvs[li + 1].n_rows.item())
            assert npar == len(parents)
            np.testing.assert_array_equal(lv.down[:npar].cpu().numpy(), down)
            np.testing.assert_array_equal(lv.up[:n, 0].cpu().numpy(), up)
            coords = parents


# ------------------------------------------------------------------------------------------
# a5/a6 single convolutions
# ------------------------------------------------------------------------------------------

def bf16_round(a):
    return oil.bf16_bits_to_f64(oil.to_bf16_bits(np.asarray(a, np.float32)))


CONV_CASES = [
    ("subm3", 8, 16), ("subm3", 16, 16), ("subm3", 32, 32), ("subm3", 64, 64), ("subm3", 128, 32),
    ("subm3", 128, 16), ("subm3", 256, 256), ("subm3", 1024, 64), ("subm3", 16, 8), ("down2", 16, 32),
    ("down2", 32, 64), ("down2", 256, 512), ("up2", 512, 256),
    ("down2", 128, 256), ("up2", 32, 16), ("up2", 64, 32), ("up2", 256, 128), ("head1", 16, 64),
    ("head1", 32, 64), ("head1", 64, 512),
    # channel counts off the tensor-core tiles (BF16 SIMT kernel): the stem and head of a network
    # without interleave (d = 1) and odd shapes of every kind
    ("subm3", 1, 16), ("subm3", 2, 192), ("subm3", 3, 5), ("down2", 2, 8), ("up2", 8, 3), ("head1", 16, 1),
    ("head1", 192, 1), ("head1", 64, 5), ("down2", 3, 64), ("up2", 4, 32), ("head1", 8, 17), ("subm3", 1, 256),
]


WINDOW_MODES = ("window", "window-split", "window-s2", "window3", "window3-split", "window3-s2")


@pytest.mark.parametrize("dt,mode", [("f32", None), ("bf16", "gather"), ("bf16", "gather-split"),
                                     ("bf16", "product"), ("bf16", "product-split"), ("bf16", "window"),
                                     ("bf16", "window-split"),
                                     ("bf16", "window3"), ("bf16", "window3-s2"), ("bf16", "gather-s4"),
                                     ("f32", "product"), ("f32", "gather")])
@pytest.mark.parametrize("kind,cin,cout", CONV_CASES)
def test_single_conv_parity(kind, cin, cout, dt, mode):
    if dt == "bf16" and kind == "up2" and cout % 16 and cin % 8 == 0 and cout % 8 == 0:
        pytest.skip("BF16 up conv on the tensor cores needs cout % 16 == 0")
    if mode in ("product", "product-split") and kind not in ("subm3", "down2", "up2"):
        pytest.skip("the product form applies to submanifold, strided and transposed convs")
    if mode in WINDOW_MODES and (kind != "subm3" or cin % 32):
        pytest.skip("the window gather applies to submanifold convs with cin % 32 == 0")
    rng = np.random.default_rng(sum(map(ord, kind)) * 100003 + cin * 1009 + cout)
    occ = rng.random((2, 10, 12, 14)) < 0.12          # ~ 800 fine sites: several 128-row tiles
    got, ref, _ = single_conv(kind, cin, cout, dt, mode, occ, rng)
    err = normwise(got, ref)
    assert err <= (8e-3 if dt == "bf16" else 1e-5), err


def dense_next_plane_occupancy():
    """Coarse occupancy where the window gather's windows overflow: in each batch element, plane
    z = 1 holds every 9th site of a 32 x 32 plane and plane z = 2 is full, so a 128-row tile of
    plane 1 has its dz = +1 neighbours spread over ~1,000 rows of plane 2 (far more than one
    window); the other planes are sparse, and the last tile is ragged."""
    rng = np.random.default_rng(77)
    occ = rng.random((2, 6, 32, 32)) < 0.05
    occ[:, 1] = False
    occ[:, 1].reshape(2, -1)[:, ::9] = True
    occ[:, 2] = True
    occ[1, 4, 5, :7] = True
    return occ


@pytest.mark.parametrize("cin,cout", [(32, 32), (64, 64), (128, 32), (256, 256)])
@pytest.mark.parametrize("mode", WINDOW_MODES)
def test_window_gather_window_overflow(cin, cout, mode):
    """Neighbours past the end of a tile's window are read from global memory: results equal the
    oracle, and (one channel block, same k order, no k-split) bitwise the gather form's."""
    rng = np.random.default_rng(cin * 7 + cout)
    occ = dense_next_plane_occupancy()
    got, ref, y = single_conv("subm3", cin, cout, "bf16", mode, occ, rng)
    assert normwise(got, ref) <= 8e-3
    got_g, _, _ = single_conv("subm3", cin, cout, "bf16", "gather", occ, np.random.default_rng(cin * 7 + cout),
                              want_ref=False)
    if cin <= 64 and not mode.endswith("-split"):
        np.testing.assert_array_equal(got, got_g)
    else:   # another summation order of the FP32 accumulators: BF16 outputs may differ by an ulp
        assert normwise(got, got_g) <= 2.0 ** -7


def single_conv(kind, cin, cout, dt, mode, occ, rng, want_ref=True):
    """One convolution of `kind` on the levels of coarse occupancy `occ` through the C ABI and the
    oracle's masked dense convolution on the same (BF16-rounded where BF16) operands. Returns the
    device output rows, the oracle's and the device output buffer (rows past n_out are NaN)."""
    L, ops, P = lib()
    lvs, c0 = make_levels(occ, 2)
    build_rulebooks(lvs)
    torch.cuda.synchronize()
    fine = onet.Level(c0, occ.shape)
    coarse = fine.parent()
    layer = I.Layer("t", kind, cin, cout, True)
    ws, _ = I.kaiming_uniform([layer], seed=5)
    w = ws[0]
    b = rng.normal(size=cout).astype(np.float32) * 0.1
    n_in = {"subm3": fine.n, "down2": fine.n, "up2": coarse.n, "head1": fine.n}[kind]
    n_out = {"subm3": fine.n, "down2": coarse.n, "up2": fine.n, "head1": fine.n}[kind]
    x = rng.normal(size=(n_in, cin)).astype(np.float32)
    skip = rng.normal(size=(n_out, cout)).astype(np.float32) if kind == "up2" else None
    if dt == "bf16":
        x_ref, w_ref, s_ref = bf16_round(x), bf16_round(w), (bf16_round(skip) if skip is not None else None)
    else:
        x_ref, w_ref, s_ref = x.astype(np.float64), w.astype(np.float64), skip
    T = lambda a: torch.tensor(np.asarray(a, np.float64))
    fn = {"subm3": lambda: onet.subm3(fine, T(x_ref), T(w_ref), T(b)),
          "down2": lambda: onet.down2(fine, coarse, T(x_ref), T(w_ref), T(b)),
          "up2": lambda: onet.up2(coarse, fine, T(x_ref), T(w_ref), T(b)),
          "head1": lambda: onet.head1(fine, T(x_ref), T(w_ref), T(b))}[kind]
    ref = None
    if want_ref:
        ref = torch.relu(fn()).numpy()
        if s_ref is not None:
            ref = ref + s_ref
    # device side
    lv_out = lvs[1] if kind == "down2" else lvs[0]
    dtype = L.BF16 if dt == "bf16" else L.F32
    tdt = torch.bfloat16 if dt == "bf16" else torch.float32
    xin = torch.zeros(lvs[1 if kind == "up2" else 0].capacity, cin, dtype=tdt, device=DEV)
    xin[:n_in] = torch.from_numpy(x).to(DEV).to(tdt)
    out_f32 = kind == "head1"
    y = torch.full((lv_out.capacity, cout), float("nan"), dtype=torch.float32 if (out_f32 or dt == "f32") else tdt,
                   device=DEV)
    sk = None
    if skip is not None:
        sk = torch.zeros(lv_out.capacity, cout, dtype=tdt, device=DEV)
        sk[:n_out] = torch.from_numpy(skip).to(DEV).to(tdt)
    kid = P.KIND[kind]
    mp = {"subm3": lvs[0].nbr, "down2": lvs[0].down, "up2": lvs[0].up, "head1": None}[kind]
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    lv_in = lvs[1] if kind == "up2" else lvs[0]
    desc = ops.conv_desc(kid, dtype, cin, cout, True, mp, lv_out.n_rows, lv_out.capacity, out_f32=out_f32,
                         map2=lvs[0].down if kind == "up2" else None, n_in=lv_in.n_rows, cap_in=lv_in.capacity,
                         status=status, form={"gather": 1, "gather-split": 1, "product": 2,
                                              "product-split": 2, "gather-s4": 1}.get(mode, 0),
                         gather=(4 if mode.startswith("window3") else 3) if mode in WINDOW_MODES else 0,
                         max_split=1 if mode in ("window", "window-s2", "window3") else
                         (8 if mode == "product-split" else 0),
                         stages=2 if mode in ("window-s2", "window3-s2") else (4 if mode == "gather-s4" else 0))
    if mode in ("gather-split", "product", "product-split", "window-split", "window3-split"):
        ws = ops.conv_workspace(ops.npvs_conv_workspace_bytes(desc), DEV)
        desc.workspace, desc.workspace_bytes = ws.data_ptr(), ws.numel()
    w_dev = torch.from_numpy(w).to(DEV).contiguous()
    if dt == "bf16":
        wp = torch.empty(ops.npvs_packed_weight_bytes(kid, cin, cout), dtype=torch.uint8, device=DEV)
        ops.npvs_pack_weights(kid, cin, cout, w_dev, wp)
        w_dev = wp
    ops.npvs_sparse_conv_fwd(desc, xin, w_dev, torch.from_numpy(b).to(DEV), sk, y)
    assert ops.npvs_check_status(status) == 0
    got = y[:n_out].float().cpu().numpy()
    assert not np.isnan(got).any()
    assert torch.isnan(y[n_out:].float()).all()       # rows past n_out untouched
    return got, ref, y


# ------------------------------------------------------------------------------------------
# whole frames
# ------------------------------------------------------------------------------------------

def oracle_frame(wl, boxes, vc, ws, bs, keep):
    cam = ocam.frustum(vc, wl.D)
    G = ofx.froxelize(cam, boxes, wl.W, wl.H, wl.D, wl.supersample)[None]
    coords, feats, _ = oil.interleave(G, wl.W, wl.d, wl.in_ch)
    n_levels = 1 + sum(1 for l in wl.layers if l.kind in ("down2", "down3"))
    levels = onet.build_levels(coords, (1, wl.D // wl.d, wl.H // wl.d, wl.W // wl.d), n_levels,
                               strided3=onet.unet_is_k3(wl.layers))
    W_, B_ = onet.to_torch_params(ws, bs)
    with torch.no_grad():
        logits = onet.forward(list(wl.layers), W_, B_, levels, torch.tensor(feats), keep=keep).numpy()
    pvs, _ = oil.pvs_from_logits(coords, logits, G, wl.W, wl.d)
    return G, coords, logits, pvs


def gpu_frame(wl, boxes, vc, ws, bs, dtype, tune=False):
    L, ops, P = lib()
    net = P.Net(wl.layers, ws, bs, DEV)
    fp = P.FramePipeline(wl, net, 1, dtype)
    cams = ops.cameras_to_device([ops.npvs_camera_setup(vc, wl.D)])
    bx = torch.from_numpy(boxes).to(DEV)
    off = torch.tensor([0, len(boxes)], dtype=torch.int32, device=DEV)
    if tune:
        fp.autotune(bx, off, cams, reps=2)
    fp.run(bx, off, cams)
    assert ops.npvs_check_status(fp.status) == 0
    return fp


@pytest.mark.parametrize("name,dt", [("plain64", "f32"), ("plain64", "bf16"), ("city256", "bf16"), ("city256", "f32"),
                                     ("city256", "bf16-tuned"), ("paper64", "bf16"), ("paper64", "f32"),
                                     ("paper64", "bf16-tuned"), ("nointerleave64", "bf16"), ("nointerleave64", "f32"),
                                     ("nointerleave64", "bf16-tuned"), ("paper64_d8", "bf16"), ("paper64_d8", "f32"),
                                     ("paper64_d8", "bf16-tuned"), ("paper64_d32", "bf16"), ("paper64_d32", "f32"),
                                     ("city256_k3", "bf16"), ("city256_k3", "f32"), ("city256_k3", "bf16-tuned")])
def test_frame_parity(name, dt):
    L, ops, P = lib()
    wl = I.workload(name)
    if name == "plain64":
        boxes, vc = I.plain64_scene()
    else:
        boxes, vc = I.city_boxes(0), I.city_viewcells(0, 1)[0]
    ws, bs = I.kaiming_uniform(wl.layers, seed=0, bias_scale=0.05)
    keep = {}
    G, coords, logits, pvs_ref = oracle_frame(wl, boxes, vc, ws, bs, keep)
    fp = gpu_frame(wl, boxes, vc, ws, bs, L.F32 if dt == "f32" else L.BF16, tune=dt == "bf16-tuned")
    dt = "f32" if dt == "f32" else "bf16"
    assert popcount(u32(fp.occ).reshape(G.shape) ^ G) == 0
    n0 = int(fp.levels[0].n_rows.item())
    np.testing.assert_array_equal(fp.levels[0].coords[:n0].cpu().numpy(), coords)
    tol = 2e-2 if dt == "bf16" else 1e-4
    lv_of = fp._level_of_layers()
    for l in wl.layers:
        n = int(fp.levels[lv_of[l.name]].n_rows.item())
        ref = keep[l.name + "+skip"] if l.kind in ("up2", "up3") else keep[l.name]   # skip add is fused
        err = normwise(fp.acts[l.name][:n].float().cpu().numpy(), ref.numpy())
        assert err <= tol, (l.name, err)
    # thresholded PVS: disagreements are allowed only at ties, i.e. froxels whose oracle logit is
    # within the measured logit error of the threshold (tau = 0.5 <=> logit 0)
    n0 = len(coords)
    z_gpu = fp.logits[:n0].float().cpu().numpy()
    zerr = float(np.abs(z_gpu - logits).max())
    zref = oil.deinterleave(coords, logits, 1, wl.D, wl.H, wl.W, wl.d)
    occ = oil.unpack_bits(G, wl.W)
    diff = oil.unpack_bits(u32(fp.pvs).reshape(G.shape) ^ pvs_ref, wl.W)
    assert not (diff & ~occ).any()
    ties = occ & (np.abs(zref) <= zerr)
    assert not (diff & ~ties).any(), int((diff & ~ties).sum())
    # spec criterion on froxels that are not ties; the overall figure (ties counted as
    # disagreements) is reported and must stay close
    agree_non_tie = 1 - (diff & ~ties).sum() / (occ & ~ties).sum()
    agree = 1 - diff.sum() / occ.sum()
    print(f"PVS agreement {agree:.6f} overall, {agree_non_tie:.6f} outside {int(ties.sum())} ties")
    assert agree_non_tie >= 0.999
    assert agree >= 0.995, (agree, int(ties.sum()))
