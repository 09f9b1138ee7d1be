"""ILT run state with checkpoint and resume.

A run is normalised gradient descent on the ILT loss of litho_ilt_grad:
theta <- theta - step_size * g / max|g| per clip.  Its state is theta, the
step index and the per-step loss history; `save` writes them to host files
(`<prefix>_theta.npy`, float32 [b][n][n], and `<prefix>_state.npy`, float64
[step, step_size, losses...]), each through a temporary file and a rename, so
a run stopped at any point resumes from its last complete checkpoint with
`IltRun.load`, bit-identically to a run that never stopped.
"""
from __future__ import annotations

import os

import numpy as np


class IltRun:
    def __init__(self, theta, target, grad_fn, step_size: float = 0.5, step: int = 0, losses=None):
        """theta, target: torch float32 [b][n][n] on the gradients' device.
        grad_fn(theta, target) -> (grad [b][n][n], per-clip losses [b])."""
        self.theta = theta
        self.target = target
        self.grad_fn = grad_fn
        self.step_size = float(step_size)
        self.step_index = int(step)
        self.losses = list(losses or [])

    @staticmethod
    def litho_grad_fn(kern, precision: str = "fft32/coarse", **loss_kw):
        """The gradient of litho_ilt_grad (loss parameters as its keywords), with a reused workspace."""
        import torch
        from . import litho as L
        cache = {}

        def fn(theta, target):
            b = theta.shape[0]
            if cache.get("b") != b:
                cache["b"] = b
                cache["ws"] = torch.empty(L.litho_ilt_workspace_size(kern, b)[0], dtype=torch.uint8,
                                          device=theta.device)
                cache["grad"] = torch.empty_like(theta)
            grad, loss = L.litho_ilt_grad(kern, theta, target, precision=precision, grad=cache["grad"],
                                          workspace=cache["ws"], **loss_kw)
            return grad, loss
        return fn

    def step(self) -> float:
        grad, loss = self.grad_fn(self.theta, self.target)
        scale = grad.abs().amax(dim=(1, 2), keepdim=True).clamp_min(1e-30)
        self.theta.sub_(self.step_size * grad / scale)
        self.step_index += 1
        total = float(np.sum(np.asarray(loss, dtype=np.float64)))
        self.losses.append(total)
        return total

    def run(self, steps: int, checkpoint_prefix: str | None = None, every: int = 0):
        """`steps` more steps; with a prefix, a checkpoint every `every` steps and at the end."""
        for i in range(steps):
            self.step()
            if checkpoint_prefix and every > 0 and (i + 1) % every == 0:
                self.save(checkpoint_prefix)
        if checkpoint_prefix:
            self.save(checkpoint_prefix)
        return self.losses

    def save(self, prefix: str):
        theta = self.theta.detach().cpu().numpy().astype(np.float32)
        state = np.array([self.step_index, self.step_size] + self.losses, dtype=np.float64)
        for suffix, arr in (("_theta.npy", theta), ("_state.npy", state)):
            path = prefix + suffix
            tmp = path + ".tmp.npy"
            np.save(tmp, arr)
            os.replace(tmp, path)

    @classmethod
    def load(cls, prefix: str, target, grad_fn, device=None):
        import torch
        theta = torch.from_numpy(np.load(prefix + "_theta.npy"))
        state = np.load(prefix + "_state.npy")
        if device is not None:
            theta = theta.to(device)
        return cls(theta, target, grad_fn, step_size=float(state[1]), step=int(state[0]),
                   losses=[float(v) for v in state[2:]])
