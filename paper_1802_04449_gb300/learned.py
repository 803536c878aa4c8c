"""Learned initial guess of the primitive root solve (not in the paper):
sample collection from the solver's own states and training on the GPU,
both through the C ABI (the samples, gradient and Adam kernels live in
libclv).  The network and its features are defined in include/clv.h."""
from __future__ import annotations

import numpy as np

from . import clv

NIN, NHID, NOUT = 10, 64, 4
SHAPES = [(NHID, NIN), (NHID,), (NHID, NHID), (NHID,), (NOUT, NHID), (NOUT,)]


def init_params(seed=0):
    """Packed W1|b1|W2|b2|W3|b3 (float32): weights uniform in +-1/sqrt(fan in),
    biases zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for shape in SHAPES:
        if len(shape) == 2:
            lim = 1.0 / np.sqrt(shape[1])
            parts.append(rng.uniform(-lim, lim, shape).ravel())
        else:
            parts.append(np.zeros(shape))
    out = np.concatenate(parts).astype(np.float32)
    assert out.size == clv.MLP_NPARAM
    return out


def collect_samples(hydro, nsteps, every, buf=None):
    """Evolve `hydro` for nsteps, appending the samples of its state to `buf`
    (a SampleBuffer; a new one sized for the dumps if None) before the first
    step and after every `every` steps.  Returns the buffer."""
    if buf is None:
        buf = SampleBuffer(hydro.torch, hydro.device, (nsteps // every + 1) * hydro.N)
    done = 0
    while True:
        buf.append(hydro)
        if done + every > nsteps:
            break
        hydro.step(every)
        done += every
    return buf


class SampleBuffer:
    """Device buffer of training rows filled by successive dumps."""

    def __init__(self, torch, device, capacity):
        self.X = torch.empty((capacity, NIN), dtype=torch.float32, device=device)
        self.Y = torch.empty((capacity, NOUT), dtype=torch.float32, device=device)
        self.rows = 0

    def append(self, hydro):
        if self.rows + hydro.N > self.X.shape[0]:
            raise ValueError("sample buffer full")
        x, _ = hydro.mlp_samples(self.X[self.rows:], self.Y[self.rows:])
        self.rows += x.shape[0]

    def data(self):
        return self.X[:self.rows], self.Y[:self.rows]


def train(X, Y, iters, batch=32768, lr=2e-3, seed=1, params=None, lr_final=None, final_frac=0.25):
    """Adam on mini-batches drawn on the device; the last `final_frac` of the
    iterations run at lr_final (default lr / 4).  Returns (params, losses)
    as device tensors."""
    import torch
    dev = X.device
    p = torch.as_tensor(init_params(seed) if params is None else np.asarray(params, np.float32),
                        device=dev).contiguous()
    work = torch.zeros(clv.MLP_TRAIN_WORK_FLOATS, dtype=torch.float32, device=dev)
    n2 = int(iters * final_frac)
    n1 = iters - n2
    l1 = clv.mlp_train(p, work, X, Y, n1, batch, lr, seed, 0)
    l2 = clv.mlp_train(p, work, X, Y, n2, batch, lr_final or lr / 4, seed, n1)
    return p, torch.cat([l1, l2])
