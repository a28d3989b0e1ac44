"""Trainer checkpoints on the host (no GPU): the state round-trips through torch.save with every
tensor, the sampler-independent fields and the kernel forms intact, and loading refuses another
network, another dtype, a tensor of another shape and a foreign file."""
import copy
import types

import pytest
import torch

import npvs_inputs as I
from paper_2509_24677_gb300 import _lib as L
from paper_2509_24677_gb300 import train as T


class FakePipe:
    def __init__(self, layers, form):
        self.cfg = {l.name: {"tune_form": form, "tune_gather": 0} for l in layers}

    def tuned_configs(self):
        return copy.deepcopy(self.cfg)

    def apply_tuned(self, cfg):
        self.cfg = copy.deepcopy(cfg)


def fake_trainer(seed, form=0, layers=None):
    g = torch.Generator().manual_seed(seed)
    layers = layers or I.plain_layers([8, 16, 8])
    n = 1000
    return types.SimpleNamespace(
        layers=layers, dtype=L.F32, params=types.SimpleNamespace(theta=torch.randn(n, generator=g)),
        m=torch.randn(n, generator=g), v=torch.rand(n, generator=g),
        adam_state=torch.tensor([seed, 0], dtype=torch.int32), pipe=FakePipe(layers, form))


def test_trainer_state_round_trip(tmp_path):
    a, b = fake_trainer(3, form=2), fake_trainer(5, form=1)
    path = tmp_path / "ck.pt"
    torch.save(T.trainer_state(a), path)
    T.load_trainer_state(b, torch.load(path, weights_only=False))
    for name in ("m", "v", "adam_state"):
        assert torch.equal(getattr(a, name), getattr(b, name))
    assert torch.equal(a.params.theta, b.params.theta)
    assert b.pipe.cfg == a.pipe.cfg
    b.params.theta.add_(1.0)                      # the state holds copies, not views
    assert not torch.equal(a.params.theta, b.params.theta)


def test_trainer_state_refuses_mismatches():
    a = fake_trainer(1)
    sd = T.trainer_state(a)
    with pytest.raises(ValueError):
        T.load_trainer_state(fake_trainer(2, layers=I.plain_layers([8, 16, 16, 8])), sd)
    other = fake_trainer(2)
    other.dtype = L.F64
    with pytest.raises(ValueError):
        T.load_trainer_state(other, sd)
    with pytest.raises(ValueError):
        T.load_trainer_state(fake_trainer(2), dict(sd, theta=sd["theta"][:-1]))
    with pytest.raises(ValueError):
        T.load_trainer_state(fake_trainer(2), dict(sd, format="something else"))
