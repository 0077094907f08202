"""Training driver of the learned implicit guess.

Generates samples from the plain hybrid pusher itself (fpic_learn_sample:
features, the converged implicit step and the plain test's verdict for
every particle, without moving them), advances the particles with the plain
push, and trains the network with the tensor-core training step
(fpic_mlp_train_step).  Two forms (see fpic_learned_cfg): the skip form
learns from every alive particle, the corrector form from the particles the
plain test rejects (the rows it is applied to).  Dataset statistics and minibatch selection are host
plumbing; every network evaluation and gradient runs in the library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import fpic as F

LOSS_W = (1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 0.0, 0.1, 0.0)


def _alive_rows(p):
    return p.alive.bool()


def _rows(p, cfg, S):
    """Valid sample rows: particle rows of alive particles (skip form), or
    the queue slots of the particles the plain test rejected (corrector form:
    the only rows the network sees in the push)."""
    if cfg is not None and cfg.mode == F.FPIC_LEARN_CORRECT:
        m = torch.zeros_like(S, dtype=torch.bool)
        m[: int(p.alive.sum().item())] = True
        return m & (S > 0.5)
    return _alive_rows(p)


def fit_cfg(ctx, p, fields, prm, p_skip=0.5, mode=F.FPIC_LEARN_SKIP, restart_after=0):
    """Standardisation of features (and, skip form, increments) from one raw sample."""
    raw = F.learned_cfg(mode=mode) if mode == F.FPIC_LEARN_CORRECT else None
    X, T, S = F.fpic_learn_sample(ctx, p, fields, prm, raw)
    a = _rows(p, raw, S)
    Xa, Ta = X[a][:, :14].double(), T[a][:, :6].double()
    mean = Xa.mean(0).cpu().numpy()
    std = Xa.std(0).cpu().numpy()
    std[std < 1e-30] = 1.0
    inc = Ta.std(0).cpu().numpy()
    inc[inc < 1e-300] = 1.0
    return F.learned_cfg(mean, std, inc, p_skip, mode, restart_after)


def generate(ctx, p, fields, prm, cfg, steps):
    """Samples from `steps` plain steps (the particles advance with the plain push)."""
    xs, ts, ss = [], [], []
    for _ in range(steps):
        X, T, S = F.fpic_learn_sample(ctx, p, fields, prm, cfg)
        a = _rows(p, cfg, S)
        xs.append(X[a]); ts.append(T[a]); ss.append(S[a])
        F.fpic_push(ctx, p, fields, prm)
    return torch.cat(xs), torch.cat(ts), torch.cat(ss)


def init_params(seed=0, device="cuda"):
    rng = np.random.default_rng(seed)
    dims = (14, 128, 128, 128, 9)
    parts = []
    for l in range(4):
        ni, no = dims[l], dims[l + 1]
        parts.append(rng.normal(0, np.sqrt(2.0 / ni), (no, ni)).ravel())
        parts.append(np.zeros(no))
    return torch.tensor(np.concatenate(parts), dtype=torch.float32, device=device)


def train(X, T, S, steps=1000, batch=8192, lr=2e-3, seed=0, log_every=0):
    """Adam on the tensor-core gradient; returns (net, params, loss history)."""
    net = F.MLP()
    P = init_params(seed, X.device)
    net.set_params(P)
    mom = torch.zeros_like(P)
    vel = torch.zeros_like(P)
    g = torch.Generator(device=X.device)
    g.manual_seed(seed)
    hist = []
    n = X.shape[0]
    for step in range(1, steps + 1):
        idx = torch.randint(0, n, (batch,), device=X.device, generator=g)
        xb, tb, sb = X[idx].contiguous(), T[idx].contiguous(), S[idx].contiguous()
        want = log_every and (step % log_every == 0 or step == 1)
        lr_t = lr * (0.1 ** (step / steps))
        L = net.train_step(P, mom, vel, xb, tb, sb, LOSS_W, step, lr=lr_t, want_loss=bool(want))
        if want:
            hist.append((step, L))
    return net, P, hist
