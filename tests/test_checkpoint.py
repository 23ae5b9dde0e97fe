"""Checkpoint / resume of the learned proposal's training state (host side,
no GPU): the FP32 master weights, the AdamW moments and the step count
survive a save and a load bit for bit."""
import torch

from paper_2506_00970_gb300 import proposal


def test_trainer_state_round_trip(tmp_path):
    a = proposal.Trainer(seed=3, batch=4, device="cpu")
    a.m.copy_(torch.randn_like(a.m))
    a.v.copy_(torch.rand_like(a.v))
    a.step = 17
    path = str(tmp_path / "net.pt")
    a.save(path)
    b = proposal.Trainer(seed=9, batch=4, device="cpu")
    assert not torch.equal(a.params, b.params)
    b.load(path)
    assert torch.equal(a.params, b.params) and torch.equal(a.m, b.m) and torch.equal(a.v, b.v)
    assert b.step == 17
