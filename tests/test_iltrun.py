"""ILT run checkpoint and resume (host logic, CPU): a run stopped after k
steps and resumed from its files reaches the same theta and losses, bit for
bit, as a run that never stopped.  The gradient is a stand-in with the shape
of the ILT step (a per-clip quadratic), so no GPU is needed."""
import numpy as np
import torch

from paper_2602_15036_gb300.iltrun import IltRun


def _grad_fn(theta, target):
    d = theta - target
    return 2.0 * d * (1.0 + 0.1 * torch.sin(theta)), (d * d).sum(dim=(1, 2)).double().numpy()


def _start(seed=3):
    g = torch.Generator().manual_seed(seed)
    theta = torch.rand((2, 16, 16), generator=g) * 2 - 1
    target = (torch.rand((2, 16, 16), generator=g) > 0.5).float()
    return theta, target


def test_resume_is_bit_identical(tmp_path):
    theta, target = _start()
    full = IltRun(theta.clone(), target, _grad_fn, step_size=0.3)
    full.run(12)
    part = IltRun(theta.clone(), target, _grad_fn, step_size=0.3)
    prefix = str(tmp_path / "run")
    part.run(5, checkpoint_prefix=prefix, every=2)
    again = IltRun.load(prefix, target, _grad_fn)
    assert again.step_index == 5 and again.step_size == 0.3 and again.losses == part.losses
    again.run(7)
    assert torch.equal(again.theta, full.theta)
    assert again.losses == full.losses and again.step_index == 12
    assert full.losses[-1] < full.losses[0]


def test_checkpoint_files_are_replaced_whole(tmp_path):
    theta, target = _start(5)
    r = IltRun(theta.clone(), target, _grad_fn)
    prefix = str(tmp_path / "ck")
    r.run(3, checkpoint_prefix=prefix, every=1)
    assert sorted(p.name for p in tmp_path.iterdir()) == ["ck_state.npy", "ck_theta.npy"]
    state = np.load(prefix + "_state.npy")
    assert state[0] == 3 and len(state) == 2 + 3
