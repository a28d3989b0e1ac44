"""Oracle regression fixtures (CPU): the oracle's outputs on the seeded 64x64x32 scene equal the
values stored in tests/golden/oracle_plain64.json by tests/golden/make_golden.py (integers exactly,
FP64 values to 1e-9 relative: FP64 library convolutions may sum in another order on another host).
These are regression guards on the oracle, not pins: the paper prints no worked example of the
per-frame computation; the pins are in test_oracle_*.py."""
import json
import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))


def test_oracle_matches_stored_plain64_outputs():
    import make_golden
    with open(os.path.join(HERE, "golden", "oracle_plain64.json")) as f:
        want = json.load(f)
    got = make_golden.compute()
    for key in ("occupied_per_slice", "occupied", "active_sites", "coords_checksum", "pvs_froxels"):
        assert got[key] == want[key], key
    for key in ("logits_sum", "logits_abs_sum", "loss_total"):
        assert got[key] == pytest.approx(want[key], rel=1e-9, abs=1e-12), key
    assert got["logits_first"] == pytest.approx(want["logits_first"], rel=1e-9, abs=1e-12)
    for k, v in want["loss"].items():
        assert got["loss"][k] == pytest.approx(v, rel=1e-9, abs=1e-12), k
