"""C-ABI boundary checks that need no GPU: the library builds and loads, exports every entry point
include/npvs.h declares, and its host-side frustum setup (Sec. 3.2) equals the oracle's."""
import math
import os
import re

import numpy as np
import pytest

import npvs_inputs as I
from oracle import camera as ocam

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(npvs_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    from paper_2509_24677_gb300 import _lib
    lib = _lib.load()
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(_lib.SIGNATURES), set(names) - set(_lib.SIGNATURES)
    assert lib.npvs_version().decode().startswith("npvs")


@pytest.mark.parametrize("vc", [
    I.plain64_scene()[1],
    *I.city_viewcells(0, 3),
    I.Viewcell(centre=(1.5, -2.0, 3.25), half=1.0, yaw=4.0, near=0.3, far=1000.0),
])
@pytest.mark.parametrize("D", [32, 128, 192])
def test_camera_setup_matches_oracle(vc, D):
    from paper_2509_24677_gb300 import ops
    cam = ops.npvs_camera_setup(vc, D)
    ref = ocam.frustum(vc, D)
    np.testing.assert_array_equal(np.array(cam.origin[:], np.float32), ref.origin)
    np.testing.assert_array_equal(np.array(cam.right[:], np.float32), ref.right)
    np.testing.assert_array_equal(np.array(cam.up[:], np.float32), ref.up)
    np.testing.assert_array_equal(np.array(cam.fwd[:], np.float32), ref.fwd)
    assert np.float32(cam.tan_half) == ref.tan_half
    assert cam.n_slices == D
    np.testing.assert_array_equal(np.array(cam.slices[:D + 1], np.float32), ref.slices)


def test_camera_setup_rejects_bad_arguments():
    from paper_2509_24677_gb300 import ops
    from paper_2509_24677_gb300._lib import NpvsError
    vc = I.Viewcell(centre=(0.0, 0.0, 0.0), half=0.5, yaw=0.0)
    with pytest.raises(NpvsError):
        ops.npvs_camera_setup(vc, 0)
    with pytest.raises(NpvsError):
        ops.npvs_camera_setup(vc, 257)
    with pytest.raises(NpvsError):
        ops.npvs_camera_setup(I.Viewcell(centre=(0.0, 0.0, 0.0), half=0.5, yaw=0.0, near=1.0, far=0.5), 8)


def test_forward_plan_validation_on_host():
    """npvs_forward_workspace_bytes validates a plan without touching a device: a network that does
    not end in d^3 logits, or whose widths do not chain, has no workspace (0)."""
    from paper_2509_24677_gb300 import _lib as L
    lib = L.load()
    lay = (L.NetLayer * 2)()
    lay[0].kind, lay[0].cin, lay[0].cout, lay[0].relu, lay[0].w = L.CONV_SUBM3, 8, 16, 1, 1
    lay[1].kind, lay[1].cin, lay[1].cout, lay[1].relu, lay[1].w = L.CONV_SUBM3, 16, 8, 0, 1
    desc = L.NetDesc(L.Grid(64, 64, 32, 1), 2, 1, 8, L.F32, 0.5, 40, 0, 2, lay)
    good = lib.npvs_forward_workspace_bytes(desc)
    assert good > 64 * 64 * 32 // 8
    lay[1].cout = 4
    assert lib.npvs_forward_workspace_bytes(desc) == 0
    lay[1].cout, lay[1].cin = 8, 12
    assert lib.npvs_forward_workspace_bytes(desc) == 0


def test_packed_weight_and_workspace_sizes_of_narrow_bf16_convs():
    """BF16 convolutions with cin or cout off the tensor-core tiles (the stem and head of a network
    without interleave) keep plain BF16 weights [taps][cin][cout] and need no product tiles; the
    tensor-core shapes keep their larger tiled images."""
    from paper_2509_24677_gb300 import _lib as L
    from paper_2509_24677_gb300 import ops
    rnd = lambda b: (b + 255) // 256 * 256
    for kind, taps in ((L.CONV_SUBM3, 27), (L.CONV_DOWN2, 8), (L.CONV_UP2, 8), (L.CONV_HEAD1, 1), (L.CONV_DOWN3, 27),
                       (L.CONV_UP3, 27)):
        for cin, cout in ((1, 16), (2, 192), (3, 5), (192, 1), (16, 1)):
            assert ops.npvs_packed_weight_bytes(kind, cin, cout) == rnd(taps * cin * cout * 2), (kind, cin, cout)
        assert ops.npvs_packed_weight_bytes(kind, 16, 16) >= taps * 16 * 16 * 2
    base = ops.npvs_conv_workspace_bytes(None)
    narrow = ops.conv_desc(L.CONV_SUBM3, L.BF16, 1, 192, True, None, None, 1000)
    wide = ops.conv_desc(L.CONV_SUBM3, L.BF16, 16, 192, True, None, None, 1000)
    assert ops.npvs_conv_workspace_bytes(narrow) == base
    assert ops.npvs_conv_workspace_bytes(wide) >= base + 1000 * 27 * 192 * 4


def test_strided3_sizes_on_host():
    """DOWN3 / UP3 keep product tiles of 27 taps and a tiled BF16 image at least as large as the
    plain one; their backward's workspace holds the dgrad image (the transposed pair's)."""
    from paper_2509_24677_gb300 import _lib as L
    from paper_2509_24677_gb300 import ops
    base = ops.npvs_conv_workspace_bytes(None)
    for kind in (L.CONV_DOWN3, L.CONV_UP3):
        d = ops.conv_desc(kind, L.BF16, 32, 64, True, None, None, 500, cap_in=700)
        assert ops.npvs_conv_workspace_bytes(d) >= base + 700 * 27 * 64 * 4
        assert ops.npvs_packed_weight_bytes(kind, 32, 64) >= 2 * 27 * 32 * 64 * 2
        other = L.CONV_UP3 if kind == L.CONV_DOWN3 else L.CONV_DOWN3
        assert ops.npvs_packed_weight_bytes_transposed(kind, 32, 64) == ops.npvs_packed_weight_bytes(other, 64, 32)
        assert ops.npvs_conv_bwd_workspace_bytes(d) >= ops.npvs_packed_weight_bytes_transposed(kind, 32, 64)
    assert ops.npvs_packed_weight_bytes(6, 32, 64) == 0


def test_argument_errors_of_the_strided3_entry_points_on_host():
    """The DOWN3 rulebook and the DOWN3 / UP3 convolutions validate their arguments before touching
    the device: the documented status comes back (with a message) on a machine without a GPU. The
    pointers are placeholders that the library must not dereference on these paths."""
    import ctypes
    from paper_2509_24677_gb300 import _lib as L
    lib = L.load()
    fake = ctypes.c_void_p(256)

    def level(X, Y, Z, B, cap):
        return L.Level(L.Dims(X, Y, Z, B), cap, fake, fake, fake)

    fine, coarse = level(8, 6, 4, 1, 192), level(4, 3, 2, 1, 24)
    ws = lib.npvs_rulebook_workspace_bytes(coarse.dims)
    rb = lambda kind, a, b, m2, nbytes: lib.npvs_build_rulebook(kind, ctypes.byref(a), ctypes.byref(b), fake, m2,
                                                                  None, fake, nbytes, None)
    assert rb(L.RB_DOWN3, fine, coarse, None, ws) == L.ERR_INVALID_ARG          # no transposed map
    assert lib.npvs_last_error().decode().startswith("npvs_build_rulebook")
    assert rb(L.RB_DOWN3, fine, level(4, 3, 3, 1, 36), fake, ws) == L.ERR_UNSUPPORTED   # not halved
    assert rb(L.RB_DOWN3, fine, coarse, fake, ws - 1) == L.ERR_WORKSPACE
    assert rb(7, fine, coarse, fake, ws) == L.ERR_UNSUPPORTED
    n = ctypes.c_void_p(512)
    for kind in (L.CONV_DOWN3, L.CONV_UP3):
        d = L.ConvDesc(kind, L.F32, 16, 16, 1, 0, fake, None, n, 24, None, 0)   # no n_in / cap_in
        assert lib.npvs_sparse_conv_fwd(ctypes.byref(d), fake, fake, None, None, fake, None) == L.ERR_INVALID_ARG
        d.n_in, d.cap_in = n, 192
        # the dgrad of a strided conv runs the transposed pair over the other map: map2 is required
        assert lib.npvs_sparse_conv_bwd(ctypes.byref(d), fake, fake, fake, fake, fake, None, fake, None, fake,
                                        1 << 20, None) == L.ERR_INVALID_ARG
        assert "map2" in lib.npvs_last_error().decode()
        d.map2 = fake
        d.w_transposed = fake   # a prepacked dgrad image is a BF16 operand
        assert lib.npvs_sparse_conv_bwd(ctypes.byref(d), fake, fake, fake, fake, fake, None, fake, None, fake,
                                        1 << 20, None) == L.ERR_INVALID_ARG
        assert "w_transposed" in lib.npvs_last_error().decode()
    d = L.ConvDesc(9, L.F32, 16, 16, 1, 0, fake, None, n, 24, n, 24)
    assert lib.npvs_sparse_conv_fwd(ctypes.byref(d), fake, fake, None, None, fake, None) == L.ERR_UNSUPPORTED


def test_wait_limit_setter_is_host_only_and_checks_its_argument():
    """npvs_set_wait_limit changes a host-side setting only (no GPU needed): it returns the previous
    bound, 0 restores the default of 4e9 SM cycles, and a negative bound is refused."""
    from paper_2509_24677_gb300 import _lib as L
    from paper_2509_24677_gb300 import ops
    assert ops.npvs_set_wait_limit(0) == 4_000_000_000
    assert ops.npvs_set_wait_limit(12345) == 4_000_000_000
    assert ops.npvs_set_wait_limit(0) == 12345
    with pytest.raises(L.NpvsError) as e:
        ops.npvs_set_wait_limit(-1)
    assert e.value.status == L.ERR_INVALID_ARG
    assert ops.npvs_set_wait_limit(0) == 4_000_000_000


def test_pack_weights_many_checks_every_job_on_host():
    """npvs_pack_weights_many validates all jobs before any launch (placeholder pointers are never
    dereferenced), n = 0 is a no-op, and the dgrad image of each kind has the size of the forward
    image of its transposed convolution."""
    import ctypes
    from paper_2509_24677_gb300 import _lib as L
    from paper_2509_24677_gb300 import ops
    lib = L.load()
    fake = ctypes.c_void_p(256).value
    ok = L.PackJob(L.CONV_SUBM3, 32, 64, 0, fake, fake)
    arr = (L.PackJob * 3)(ok, ok, L.PackJob(L.CONV_SUBM3, 32, 64, 0, None, fake))
    assert lib.npvs_pack_weights_many(3, arr, None) == L.ERR_INVALID_ARG
    assert "job 2" in lib.npvs_last_error().decode()
    arr[2] = L.PackJob(L.CONV_SUBM3, 1, 64, 1, fake, fake)        # transposed image of a narrow conv
    assert lib.npvs_pack_weights_many(3, arr, None) == L.ERR_UNSUPPORTED
    arr[2] = L.PackJob(11, 32, 64, 0, fake, fake)
    assert lib.npvs_pack_weights_many(3, arr, None) == L.ERR_UNSUPPORTED
    arr[2] = L.PackJob(L.CONV_SUBM3, 32, 64, 2, fake, fake)        # transposed is 0 or 1
    assert lib.npvs_pack_weights_many(3, arr, None) == L.ERR_INVALID_ARG
    assert lib.npvs_pack_weights_many(-1, arr, None) == L.ERR_INVALID_ARG
    assert lib.npvs_pack_weights_many(0, None, None) == L.OK
    pairs = {L.CONV_SUBM3: L.CONV_SUBM3, L.CONV_DOWN2: L.CONV_UP2, L.CONV_UP2: L.CONV_DOWN2,
             L.CONV_HEAD1: L.CONV_HEAD1, L.CONV_DOWN3: L.CONV_UP3, L.CONV_UP3: L.CONV_DOWN3}
    for k, t in pairs.items():
        for cin, cout in ((32, 64), (192, 256), (64, 48)):
            assert ops.npvs_packed_weight_bytes_transposed(k, cin, cout) == ops.npvs_packed_weight_bytes(t, cout, cin)
        assert ops.npvs_packed_weight_bytes_transposed(k, 1, 64) == 0
