"""Planted mistakes: each test runs one pin with a plausible error put into the oracle, and the pin
must fail (CPU only).

A pin that still passes with a dropped term, a mirrored kernel, a transposed channel order or an
off-by-one slice in place would not be evidence that the oracle is right. Here every mistake is
planted in the oracle on the CPU for the length of one test: a Python function is swapped for a
copy with the error (pytest's monkeypatch restores it), and the C froxelizer is rebuilt from a
copy of its source with one expression changed, into a temporary folder. Nothing here touches the
CUDA path. Each test names the passage of the paper, or the reading of it, that the mistake breaks.
"""
import dataclasses
import math

import numpy as np
import pytest
import torch

import test_oracle_froxel as PF
import test_oracle_interleave as PI
import test_oracle_loss as PL
import test_oracle_network as PN
from oracle import camera, froxel
from oracle import interleave as IL
from oracle import loss as LS
from oracle import network as N
from oracle import rulebook as RB


@pytest.fixture(autouse=True)
def _float64_default():
    """The network pins build their tensors in float64 (their module sets this by a fixture)."""
    old = torch.get_default_dtype()
    torch.set_default_dtype(torch.float64)
    yield
    torch.set_default_dtype(old)


def must_fail(pin, *args, **kw):
    with pytest.raises(AssertionError):
        pin(*args, **kw)


# ------------------------------------------------------------------------------------------
# sparse convolutions and the U-Net (Sec. 2.3, Sec. 3.3)
# ------------------------------------------------------------------------------------------

def test_subm3_with_mirrored_taps(monkeypatch):
    """Tap k applied at offset -k (correlation read as convolution)."""
    orig = N.subm3
    monkeypatch.setattr(N, "subm3", lambda lv, x, W, b: orig(lv, x, W.flip(0), b))
    must_fail(PN.test_subm3_equals_masked_conv3d_and_loops)


def test_down2_with_x_major_children(monkeypatch):
    """The eight children of a parent enumerated x-major instead of z-major."""
    orig = N.down2
    xm = lambda W: W.reshape(2, 2, 2, W.shape[1], W.shape[2]).permute(2, 1, 0, 3, 4).reshape(W.shape)
    monkeypatch.setattr(N, "down2", lambda f, c, x, W, b: orig(f, c, x, xm(W), b))
    must_fail(PN.test_down2_and_up2_equal_strided_convs)


def test_up2_with_x_major_children(monkeypatch):
    orig = N.up2
    xm = lambda W: W.reshape(2, 2, 2, W.shape[1], W.shape[2]).permute(2, 1, 0, 3, 4).reshape(W.shape)
    monkeypatch.setattr(N, "up2", lambda c, f, z, W, b: orig(c, f, z, xm(W), b))
    must_fail(PN.test_down2_and_up2_equal_strided_convs)


def test_parent_level_out_of_linear_order(monkeypatch):
    """Parents listed in reverse linear order (active sites are kept in (b, z, y, x) order)."""
    orig = N.Level.parent
    monkeypatch.setattr(N.Level, "parent", lambda self: N.Level(orig(self).coords.flip(0), orig(self).dims))
    must_fail(PN.test_down2_and_up2_equal_strided_convs)


def test_down3_without_padding(monkeypatch):
    """k = 3 stride-2 down conv reading input 2q + k (padding 0) instead of 2q + k - 1."""
    def down3(fine, coarse, x, W, b):
        g = N._dense(fine, x, 1)
        Q = coarse.coords
        y = b.expand(coarse.n, W.shape[2])
        for k, (kz, ky, kx) in enumerate(N.K27):
            y = y + g[Q[:, 0], 2 * Q[:, 1] + kz + 1, 2 * Q[:, 2] + ky + 1, 2 * Q[:, 3] + kx + 1] @ W[k]
        return y
    monkeypatch.setattr(N, "down3", down3)
    must_fail(PN.test_down3_and_up3_equal_strided_convs_with_padding)


def test_up3_without_output_shift(monkeypatch):
    """The transposed k = 3 conv writing output 2q + k instead of 2q + k - 1."""
    def up3(coarse, fine, z, W, b):
        zd = N._dense(coarse, z, 0)
        B, Dc, Hc, Wc, _ = zd.shape
        out = torch.zeros((B, 2 * Dc + 1, 2 * Hc + 1, 2 * Wc + 1, W.shape[2]), dtype=zd.dtype)
        for k, (kz, ky, kx) in enumerate(N.K27):
            out[:, kz:kz + 2 * Dc:2, ky:ky + 2 * Hc:2, kx:kx + 2 * Wc:2] += zd @ W[k]
        c = fine.coords
        return b + out[c[:, 0], c[:, 1], c[:, 2], c[:, 3]]
    monkeypatch.setattr(N, "up3", up3)
    must_fail(PN.test_down3_and_up3_equal_strided_convs_with_padding)


def test_strided3_output_set_taken_as_parents(monkeypatch):
    """The output set of the k = 3, stride 2, padding 1 conv taken as the 2x2x2 parent set (the
    dilation by the padded window dropped)."""
    monkeypatch.setattr(N.Level, "strided3", N.Level.parent)
    must_fail(PN.test_down3_and_up3_equal_strided_convs_with_padding)


def unet_copy(skip_after="b", detach_skip=False):
    """A copy of the oracle's U-Net forward in which a mistake can be planted: skip_after "a" takes
    the skip of encoder level i after enc{i}a instead of after enc{i}b; detach_skip adds a detached
    copy of it (the forward values unchanged, its gradient path cut). The defaults are the
    oracle's own wiring."""
    def forward(layers, weights, biases, levels, x, keep=None):
        wi = {l.name: i for i, l in enumerate(layers)}

        def run(name, fn, *args):
            i = wi[name]
            y = fn(*args, weights[i], biases[i])
            y = torch.relu(y) if layers[i].relu else y
            if keep is not None:
                keep[name] = y
            return y

        nl = sum(1 for l in layers if l.kind in ("down2", "down3")) + 1
        dn, upf = (N.down3, N.up3) if N.unet_is_k3(layers) else (N.down2, N.up2)
        a = run("stem", N.subm3, levels[0], x)
        skips = []
        for i in range(nl):
            a = run(f"enc{i}a", N.subm3, levels[i], a)
            if skip_after == "a":
                skips.append(a)
            a = run(f"enc{i}b", N.subm3, levels[i], a)
            if skip_after == "b":
                skips.append(a)
            if i + 1 < nl:
                a = run(f"down{i}", lambda x_, W, b, i=i: dn(levels[i], levels[i + 1], x_, W, b), a)
        for i in range(nl - 2, -1, -1):
            a = run(f"up{i}", lambda x_, W, b, i=i: upf(levels[i + 1], levels[i], x_, W, b), a)
            a = a + (skips[i].detach() if detach_skip else skips[i])
            if keep is not None:
                keep[f"up{i}+skip"] = a
            a = run(f"dec{i}a", N.subm3, levels[i], a)
            a = run(f"dec{i}b", N.subm3, levels[i], a)
        return run("head", N.head1, levels[0], a)
    return forward


@pytest.mark.parametrize("strided", [False, True])
def test_unet_copy_without_a_plant_passes(monkeypatch, strided):
    """Control: the copy with the oracle's own wiring passes the wiring and gradient pins, so what
    fails below is the planted line."""
    monkeypatch.setattr(N, "forward", unet_copy())
    PN.test_unet_wiring_equals_dense_straight_line_composition(strided)
    if not strided:
        PN.test_gradients_match_central_differences("unet")


@pytest.mark.parametrize("strided", [False, True])
def test_unet_skip_taken_one_layer_early(monkeypatch, strided):
    monkeypatch.setattr(N, "forward", unet_copy(skip_after="a"))
    must_fail(PN.test_unet_wiring_equals_dense_straight_line_composition, strided)


def test_unet_gradient_with_a_detached_skip(monkeypatch):
    """The skip added as a detached copy: the forward values are those of the oracle, the analytic
    gradient misses the skip path, and central differences see it."""
    monkeypatch.setattr(N, "forward", unet_copy(detach_skip=True))
    PN.test_unet_wiring_equals_dense_straight_line_composition(False)
    must_fail(PN.test_gradients_match_central_differences, "unet")


def test_unet_head_with_relu(monkeypatch):
    """A ReLU on the 1x1 head (the logits are signed)."""
    orig = N.forward

    def forward(layers, weights, biases, levels, x, keep=None):
        y = torch.relu(orig(layers, weights, biases, levels, x, keep))
        if keep is not None:
            keep["head"] = y
        return y
    monkeypatch.setattr(N, "forward", forward)
    must_fail(PN.test_unet_wiring_equals_dense_straight_line_composition, False)


def test_neighbour_map_with_x_major_offsets(monkeypatch):
    """Rulebook offsets enumerated x-major while the weights are z-major."""
    orig = RB.neighbour_map
    monkeypatch.setattr(RB, "neighbour_map",
                        lambda c: orig(c).reshape(-1, 3, 3, 3).transpose(0, 3, 2, 1).reshape(-1, 27))
    must_fail(PN.test_rulebook_oracle_by_brute_force)


def test_strided3_up_map_with_mirrored_taps(monkeypatch):
    """The transposed conv's map indexed by the mirrored tap 26 - k."""
    orig = RB.strided3_level

    def strided3_level(c, dims):
        outs, down, up = orig(c, dims)
        return outs, down, np.ascontiguousarray(up[:, ::-1])
    monkeypatch.setattr(RB, "strided3_level", strided3_level)
    must_fail(PN.test_strided3_rulebook_oracle_by_brute_force)


# ------------------------------------------------------------------------------------------
# interleave g_d, depth channel, threshold, bit layout, BF16 rounding (Sec. 3.1, Sec. 3.3)
# ------------------------------------------------------------------------------------------

def test_interleave_with_x_major_channels(monkeypatch):
    """Channels of a site ordered (dx, dy, dz) instead of (dz, dy, dx)."""
    def g_d(dense, d):
        B, D, H, W = dense.shape
        t = dense.reshape(B, D // d, d, H // d, d, W // d, d).transpose(0, 1, 3, 5, 6, 4, 2)
        return t.reshape(B, D // d, H // d, W // d, d ** 3)
    monkeypatch.setattr(IL, "g_d", g_d)
    must_fail(PI.test_channel_order_by_loops)


def test_depth_channel_at_slice_start(monkeypatch):
    """Normalised depth k / D (slice start) instead of the slice centre (k + 1/2) / D."""
    monkeypatch.setattr(IL, "depth_channel", lambda D: (np.arange(D) / D).astype(np.float32))
    must_fail(PI.test_depth_channel_exact)
    must_fail(PI.test_channel_order_by_loops)


def test_pvs_not_masked_by_geometry(monkeypatch):
    """V = 1[sigmoid(f) >= tau] without the AND with G (supp(V) within supp(G), Sec. 3.2)."""
    def pvs_from_logits(coords, logits, G_bits, W, d, tau=0.5):
        B, D, H, _ = G_bits.shape
        p = 1.0 / (1.0 + np.exp(-np.asarray(logits, dtype=np.float64)))
        dense = IL.deinterleave(coords, p, B, D, H, W, d)
        return IL.pack_bits(dense >= tau), dense
    monkeypatch.setattr(IL, "pvs_from_logits", pvs_from_logits)
    must_fail(PI.test_pvs_threshold_and_mask)


def test_bf16_by_truncation(monkeypatch):
    """binary32 -> bfloat16 by dropping the low 16 bits instead of rounding to nearest even."""
    monkeypatch.setattr(IL, "to_bf16_bits",
                        lambda x: (np.ascontiguousarray(x, np.float32).view(np.uint32) >> 16).astype(np.uint16))
    must_fail(PI.test_bf16_rounding_matches_torch)


def test_bits_in_big_endian_order(monkeypatch):
    """Bit x of a row stored as bit 31 - (x & 31) of its word."""
    def pack_bits(dense):
        by = np.packbits(dense.astype(np.uint8), axis=-1, bitorder="big")
        return np.ascontiguousarray(by).view("<u4").astype(np.uint32)

    def unpack_bits(bits, W):
        b = np.ascontiguousarray(bits, dtype="<u4").view(np.uint8)
        return np.unpackbits(b, axis=-1, bitorder="big")[..., :W].astype(bool)
    monkeypatch.setattr(IL, "pack_bits", pack_bits)
    monkeypatch.setattr(IL, "unpack_bits", unpack_bits)
    must_fail(PI.test_bit_layout)


# ------------------------------------------------------------------------------------------
# loss, Adam, rates (Sec. 3.3, Sec. 4.2, Sec. 5.1)
# ------------------------------------------------------------------------------------------

def test_dice_alpha_on_false_positives(monkeypatch):
    """alpha weighing FP instead of FN in the weighted Dice denominator (the paper's naming of FN
    and FP read the other way round)."""
    orig = LS.loss_terms
    monkeypatch.setattr(LS, "loss_terms", lambda z, c, G, GT, W, d, prm=LS.LossParams():
                        orig(z, c, G, GT, W, d, dataclasses.replace(prm, alpha=1 - prm.alpha)))
    must_fail(PL.test_hand_computed_example)


def test_loss_without_repulsion(monkeypatch):
    """L = lambda L_dice + (1 - lambda) L_attr: the repulsive term dropped."""
    orig = LS.loss_terms

    def loss_terms(z, c, G, GT, W, d, prm=LS.LossParams()):
        _, terms = orig(z, c, G, GT, W, d, prm)
        for t in terms:
            t["L"] = prm.lam * t["dice"] + (1 - prm.lam) * t["attr"] + prm.w_bce * t["bce"]
        return sum(t["L"] for t in terms) / len(terms), terms
    monkeypatch.setattr(LS, "loss_terms", loss_terms)
    must_fail(PL.test_hand_computed_example)


def test_attraction_as_printed(monkeypatch):
    """L_attr = 1 - FN / (GTP + eps), the printed form that rewards misses: a perfect prediction
    would cost 1."""
    orig = LS.loss_terms

    def loss_terms(z, c, G, GT, W, d, prm=LS.LossParams()):
        L, terms = orig(z, c, G, GT, W, d, prm)
        for t in terms:
            t["attr"] = 1.0 - t["fn"] / (t["gtp"] + prm.eps)
        return L, terms
    monkeypatch.setattr(LS, "loss_terms", loss_terms)
    must_fail(PL.test_perfect_and_empty_predictions_closed_form)


def test_adam_without_bias_correction(monkeypatch):
    def adam_step(theta, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, wd=1e-10):
        g = grad + wd * theta
        m = b1 * m + (1.0 - b1) * g
        v = b2 * v + (1.0 - b2) * g * g
        return theta - lr * m / (np.sqrt(v) + eps), m, v
    monkeypatch.setattr(LS, "adam_step", adam_step)
    must_fail(PL.test_adam_matches_torch_optim)


def test_fpr_over_negatives(monkeypatch):
    """FPR = FP / (froxels - GTP) (the usual false-positive rate) instead of FP / GTP (Sec. 5.1)."""
    def rates(pvs_bits, gt_bits):
        pc = lambda a: int(np.unpackbits(np.ascontiguousarray(a).view(np.uint8)).sum())
        gtp, n = pc(gt_bits), 32 * gt_bits.size
        return pc(gt_bits & ~pvs_bits) / gtp, pc(pvs_bits & ~gt_bits) / (n - gtp)
    monkeypatch.setattr(LS, "rates", rates)
    must_fail(PL.test_rates)


# ------------------------------------------------------------------------------------------
# frustum, froxelization and ground truth (Sec. 3.1, Sec. 3.2)
# ------------------------------------------------------------------------------------------

def test_frustum_apex_without_depth_margin(monkeypatch):
    """Apex moved back by h / tan(theta / 2) only (the cube's own depth extent not covered)."""
    orig = camera.frustum

    def frustum(vc, D):
        cam = orig(vc, D)
        h = vc.half
        return dataclasses.replace(cam, origin=(cam.origin + np.float32(h) * cam.fwd).astype(np.float32))
    monkeypatch.setattr(camera, "frustum", frustum)
    must_fail(PF.test_frustum_basis_and_slices)


def test_frustum_without_rotation_margin(monkeypatch):
    """Half-angle theta / 2 instead of (theta + 2 beta) / 2."""
    orig = camera.frustum
    monkeypatch.setattr(camera, "frustum", lambda vc, D: dataclasses.replace(
        orig(vc, D), tan_half=np.float32(math.tan(0.5 * math.radians(vc.fov_deg)))))
    must_fail(PF.test_frustum_basis_and_slices)


def plant_c(monkeypatch, tmp_path, old, new):
    """Rebuild the C froxelizer from a copy of its source with `old` replaced by `new` (every
    occurrence) into tmp_path, and load that library for the rest of the test."""
    with open(froxel._SRC) as f:
        src = f.read()
    assert src.count(old) >= 1, old
    path = tmp_path / "froxel.c"
    path.write_text(src.replace(old, new))
    monkeypatch.setattr(froxel, "_SRC", str(path))
    monkeypatch.setattr(froxel, "_LIB_PATH", str(tmp_path / "_build" / "liboracle_froxel.so"))
    monkeypatch.setattr(froxel, "_lib", None)


def test_froxel_rays_through_pixel_corners(monkeypatch, tmp_path):
    """Sub-pixel rays through the corner (2a - sW) / sW instead of the centre (2a + 1 - sW) / sW."""
    plant_c(monkeypatch, tmp_path, "(2 * a + 1 - sW)", "(2 * a - sW)")
    must_fail(PF.test_froxelize_matches_slab_method, 0.45)


def test_froxel_column_one_sub_pixel_too_wide(monkeypatch, tmp_path):
    """Froxel column x gathering sub-pixel rays x s .. (x + 1) s inclusive."""
    plant_c(monkeypatch, tmp_path, "a < (x + 1) * s", "a <= (x + 1) * s")
    must_fail(PF.test_froxelize_matches_slab_method, 0.45)


def test_slice_lookup_with_strict_bound(monkeypatch, tmp_path):
    """Slice k = max{k : z_k < t} instead of z_k <= t (a depth on a boundary goes one slice down)."""
    plant_c(monkeypatch, tmp_path, "if (z[i] <= t) k = i;", "if (z[i] < t) k = i;")
    must_fail(PF.test_slice_lookup_matches_searchsorted)


def test_ground_truth_last_face_instead_of_first(monkeypatch, tmp_path):
    """The binary64 ground truth keeping the last face hit found instead of the nearest."""
    plant_c(monkeypatch, tmp_path, "if (!(t > 0.0) || !(t < best)) continue;", "if (!(t > 0.0)) continue;")
    must_fail(PF.test_point_viewcell_is_zbuffer_visibility, 64)


def test_ground_truth_mirror_with_slab_exit(monkeypatch, tmp_path):
    """The binary32 mirror entering each slab at max(t0, t1) instead of min(t0, t1)."""
    plant_c(monkeypatch, tmp_path, "tn = fmaxf(tn, fminf(t0, t1));", "tn = fmaxf(tn, fmaxf(t0, t1));")
    must_fail(PF.test_point_viewcell_is_zbuffer_visibility, 32)
