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
