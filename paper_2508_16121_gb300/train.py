"""Teacher-student training of the factor generator on synthetic pairs.

The paper trains the generator end to end through the fused transform with
Adam (Sec. 4.2; loss Eq. 11, whose MSE term is used here).  Its photo datasets
are not available, so the training pairs are made by the transform itself:
a frozen, seeded teacher generator (identity-biased output layer, final
weights N(0, teacher_scale)) predicts image-dependent parameters, svdlut_apply
renders the target.  The loss is Eq. 11 without its LPIPS term: MSE plus
lambda_c = 0.005 times the CIE94 colour difference.  Every step runs in the
library's kernels:
  student forward (svdlut_generator_forward, dropout on)
  -> svdlut_apply -> svdlut_mse + svdlut_cie94 (loss and dy)
  -> svdlut_backward (parameter gradients)
  -> svdlut_generator_backward -> svdlut_generator_adam.
Data and dropout are seeded per step, so a run resumed from a checkpoint
reproduces the uninterrupted run bit for bit.
"""
from __future__ import annotations

import math
import os

import numpy as np

import svdlut_inputs as si

from . import CIE94_WEIGHT, Generator, PARAM_NAMES, adam_step, apply, backward, cie94, mse


def _torch():
    import torch
    return torch


def step_decay_lr(base_lr: float, step: int, every: int | None, factor: float = 0.1) -> float:
    """Learning rate of optimizer step `step` (1-based) under the paper's
    schedule (Sec. 4.2: Adam at 1e-4, multiplied by 0.1 every 100 epochs):
    base_lr * factor ** floor((step - 1) / every); constant when every is
    None or 0."""
    if not every:
        return float(base_lr)
    if step < 1:
        raise ValueError("steps are counted from 1")
    return float(base_lr) * float(factor) ** ((step - 1) // int(every))


class Trainer:
    def __init__(self, K=8, batch=64, size=256, lr=1e-3, seed=0, teacher_seed=1, teacher_scale=0.1,
                 data_seed=2, device="cuda", cie94_weight=CIE94_WEIGHT, lr_decay_every=None, lr_decay=0.1):
        """lr_decay_every: multiply the learning rate by lr_decay every that
        many steps (the paper's step decay, Sec. 4.2); None keeps it constant."""
        torch = _torch()
        self.K, self.batch, self.size, self.lr = K, batch, size, lr
        self.lr_decay_every, self.lr_decay = lr_decay_every, float(lr_decay)
        self.cie94_weight = float(cie94_weight)
        self.device = torch.device(device)
        self.data_seed = data_seed
        w0 = si.generator_init(K, np.random.default_rng(seed), 0.0)
        tw = si.generator_init(K, np.random.default_rng(teacher_seed), teacher_scale)
        self.student = Generator(K, torch.tensor(w0, dtype=torch.float32, device=self.device), max_batch=batch)
        self.teacher = Generator(K, torch.tensor(tw, dtype=torch.float32, device=self.device), max_batch=batch)
        n = self.student.n
        self.m = torch.zeros(n, dtype=torch.float32, device=self.device)
        self.v = torch.zeros(n, dtype=torch.float32, device=self.device)
        self.dw = torch.empty(n, dtype=torch.float32, device=self.device)
        self.step = 0
        self.dy = torch.empty(batch, 3, size, size, dtype=torch.float32, device=self.device)
        self.bwd_ws = None
        self.losses = []

    def batch_images(self, step):
        torch = _torch()
        g = torch.Generator(device=self.device)
        g.manual_seed(self.data_seed * 1_000_003 + step)
        return si.torch_photos(g, self.batch, self.size, self.size, self.device)

    def pair(self, step):
        x = self.batch_images(step)
        tp = self.teacher.forward(x)
        return x, apply(x, tp)

    def train_step(self):
        torch = _torch()
        self.step += 1
        x, yt = self.pair(self.step)
        sp = self.student.forward(x, training=True, seed=self.step)
        y = apply(x, sp)
        loss = mse(y, yt, self.dy)
        if self.cie94_weight:
            loss = loss + self.cie94_weight * cie94(y, yt, self.cie94_weight, dy=self.dy, accumulate=True)
        g = backward(x, sp, self.dy, want=tuple("d" + n for n in PARAM_NAMES), workspace=self.bwd_ws)
        self.student.backward({n: g["d" + n] for n in PARAM_NAMES}, dweights=self.dw)
        adam_step(self.student.weights, self.dw, self.m, self.v, self.step, lr=self.current_lr())
        self.losses.append(loss)
        return loss

    def current_lr(self):
        """learning rate of the step being taken (self.step, 1-based)"""
        return step_decay_lr(self.lr, max(self.step, 1), self.lr_decay_every, self.lr_decay)

    def run(self, steps):
        for _ in range(steps):
            self.train_step()
        torch = _torch()
        torch.cuda.synchronize()
        return [float(l) for l in self.losses[-steps:]]

    # ---- checkpoint / resume ----
    def save(self, path):
        torch = _torch()
        torch.save({"K": self.K, "batch": self.batch, "size": self.size, "lr": self.lr, "step": self.step,
                    "data_seed": self.data_seed, "cie94_weight": self.cie94_weight, "lr_decay_every": self.lr_decay_every,
                    "lr_decay": self.lr_decay, "weights": self.student.weights.cpu(), "m": self.m.cpu(),
                    "v": self.v.cpu(), "teacher": self.teacher.weights.cpu(), "version": 1}, path)

    def load(self, path):
        torch = _torch()
        ck = torch.load(path, map_location="cpu")
        if ck["version"] != 1 or ck["K"] != self.K or ck["batch"] != self.batch or ck["size"] != self.size:
            raise ValueError("checkpoint does not match this trainer")
        self.student.weights.copy_(ck["weights"].to(self.device))
        self.teacher.weights.copy_(ck["teacher"].to(self.device))
        self.m.copy_(ck["m"].to(self.device))
        self.v.copy_(ck["v"].to(self.device))
        self.step, self.lr, self.data_seed = ck["step"], ck["lr"], ck["data_seed"]
        self.cie94_weight = ck.get("cie94_weight", self.cie94_weight)
        self.lr_decay_every = ck.get("lr_decay_every", self.lr_decay_every)
        self.lr_decay = ck.get("lr_decay", self.lr_decay)


def psnr(y, t):
    """PSNR (dB) over [0,1] images through the library's MSE kernel."""
    return 10.0 * math.log10(1.0 / max(float(mse(y, t)), 1e-20))


def evaluate(trainer: Trainer, n_batches=4, eval_seed=99, mean_batches=8):
    """Held-out PSNR against the teacher's rendering of: the trained student,
    the identity transform, and the teacher's parameters averaged over
    training images (one fixed, non-adaptive transform)."""
    torch = _torch()
    ev = Trainer.__new__(Trainer)
    ev.__dict__.update(trainer.__dict__)
    ev.data_seed = eval_seed
    mean_p = None
    for b in range(mean_batches):
        x = trainer.batch_images(10_000 + b)
        tp = trainer.teacher.forward(x)
        s = {k: v.mean(dim=0, keepdim=True) for k, v in tp.items()}
        mean_p = s if mean_p is None else {k: mean_p[k] + s[k] for k in s}
    mean_p = {k: (v / mean_batches).expand(trainer.batch, *v.shape[1:]).contiguous() for k, v in mean_p.items()}
    out = {"student": [], "identity": [], "mean_teacher": []}
    for b in range(n_batches):
        x, yt = ev.pair(b)
        out["student"].append(psnr(apply(x, trainer.student.forward(x)), yt))
        out["identity"].append(psnr(x, yt))
        out["mean_teacher"].append(psnr(apply(x, mean_p), yt))
    torch.cuda.synchronize()
    return {k: float(np.mean(v)) for k, v in out.items()}


def main(argv=None):
    """Command line: train the generator for a number of steps on the GPU and
    report the loss and held-out PSNR, e.g.
    ``python -m paper_2508_16121_gb300.train --steps 320 --batch 64 --size 256``."""
    import argparse
    ap = argparse.ArgumentParser(description="teacher-student training of the SVDLUT factor generator")
    ap.add_argument("--steps", type=int, default=320)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--K", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-decay-every", type=int, default=0,
                    help="multiply the learning rate by --lr-decay every N steps (0: constant)")
    ap.add_argument("--lr-decay", type=float, default=0.1)
    ap.add_argument("--cie94", type=float, default=CIE94_WEIGHT, help="weight of the CIE94 term (0: MSE only)")
    ap.add_argument("--eval", action="store_true", help="held-out PSNR before and after")
    ap.add_argument("--save", default=None, help="checkpoint path")
    args = ap.parse_args(argv)
    tr = Trainer(K=args.K, batch=args.batch, size=args.size, lr=args.lr, cie94_weight=args.cie94,
                 lr_decay_every=args.lr_decay_every or None, lr_decay=args.lr_decay)
    if args.eval:
        print("before:", evaluate(tr))
    losses = tr.run(args.steps)
    print(f"steps {args.steps}: loss first {losses[0]:.5f} last {losses[-1]:.5f}")
    if args.eval:
        print("after:", evaluate(tr))
    if args.save:
        tr.save(args.save)


if __name__ == "__main__":
    main()
