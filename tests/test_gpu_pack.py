"""Weight packing in one launch (npvs_pack_weights_many): the forward images are byte for byte
those of npvs_pack_weights, and the dgrad images it packs after an optimizer step give bitwise the
gradients of the backward that packs them itself."""
import numpy as np
import pytest
import torch

import npvs_inputs as I
from test_gpu_parity import DEV, lib

pytestmark = pytest.mark.gpu

# (kind, cin, cout): every kind, BKE 32 and 64, padded and exact column blocks, narrow layers
SHAPES = [("subm3", 16, 32), ("subm3", 32, 32), ("subm3", 64, 192), ("subm3", 96, 48), ("subm3", 1, 192),
          ("down2", 32, 64), ("down2", 192, 256), ("up2", 64, 32), ("up2", 256, 192), ("head1", 32, 64),
          ("head1", 192, 4096), ("head1", 256, 1), ("down3", 32, 64), ("up3", 64, 32), ("subm3", 8, 24)]


def rand_w(kind, cin, cout, seed):
    L, ops, P = lib()
    taps = {0: 27, 1: 8, 2: 8, 3: 1, 4: 27, 5: 27}[P.KIND[kind]]
    g = torch.Generator().manual_seed(seed)
    return (torch.rand(taps, cin, cout, generator=g) * 2 - 1).to(DEV).contiguous()


def test_pack_many_equals_one_by_one():
    """32 jobs (two launches of images): each forward image equals npvs_pack_weights' bytes."""
    L, ops, P = lib()
    jobs, refs = [], []
    for i in range(32):
        kind, cin, cout = SHAPES[i % len(SHAPES)]
        k = P.KIND[kind]
        w = rand_w(kind, cin, cout, i)
        # both buffers start with the same fill: bytes past an image (allocation padding) are not written
        ref = torch.full((ops.npvs_packed_weight_bytes(k, cin, cout),), 0xA5, dtype=torch.uint8, device=DEV)
        ops.npvs_pack_weights(k, cin, cout, w, ref)
        out = torch.full_like(ref, 0xA5)
        jobs.append((k, cin, cout, 0, w, out))
        refs.append(ref)
    ops.npvs_pack_weights_many(jobs)
    torch.cuda.synchronize()
    for (k, cin, cout, _, _, out), ref in zip(jobs, refs):
        assert torch.equal(out, ref), (k, cin, cout)
    ops.npvs_pack_weights_many([])          # nothing to do


def test_pack_many_argument_errors():
    L, ops, P = lib()
    w = rand_w("subm3", 1, 192, 0)
    buf = torch.zeros(ops.npvs_packed_weight_bytes(P.KIND["subm3"], 1, 192), dtype=torch.uint8, device=DEV)
    assert ops.npvs_packed_weight_bytes_transposed(P.KIND["subm3"], 1, 192) == 0
    with pytest.raises(L.NpvsError) as e:       # no transposed image of a narrow convolution
        ops.npvs_pack_weights_many([(P.KIND["subm3"], 1, 192, 1, w, buf)])
    assert e.value.status == L.ERR_UNSUPPORTED
    with pytest.raises(L.NpvsError) as e:
        ops.npvs_pack_weights_many([(9, 1, 192, 0, w, buf)])
    assert e.value.status == L.ERR_UNSUPPORTED


@pytest.mark.parametrize("dt", ["bf16"])
def test_trainer_dgrad_images_are_the_in_call_packs(dt):
    """The Trainer packs every layer's dgrad image with the forward images after Adam; its backward
    then gives bitwise the gradients of a backward that packs each dgrad image in the call."""
    L, ops, P = lib()
    from test_gpu_train import UNET_SMALL, make_trainer
    tr, inp, *_ = make_trainer(UNET_SMALL, L.BF16)
    tr.loss_forward()
    tr.backward()
    tr.optimizer_step()                      # new weights, repacked (forward and dgrad images)
    tr.forward(*inp)
    tr.loss_forward()
    tr.backward()
    torch.cuda.synchronize()
    got = ([g.clone() for g in tr.params.gw], [g.clone() for g in tr.params.gb],
           {k: v.clone() for k, v in tr.dacts.items()})
    assert tr.packed_t[0] is None and all(t is not None for t in tr.packed_t[1:])
    tr.packed_t = [None] * len(tr.layers)   # every dgrad image packed inside the call instead
    tr.backward()
    torch.cuda.synchronize()
    assert ops.npvs_check_status(tr.pipe.status) == 0
    for a, b in zip(got[0], tr.params.gw):
        assert torch.equal(a, b)
    for a, b in zip(got[1], tr.params.gb):
        assert torch.equal(a, b)
    for k, v in got[2].items():
        assert torch.equal(v, tr.dacts[k]), k
