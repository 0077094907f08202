"""Autotuner of the launch shapes the library leaves open (fpic_set_tuning).

Each candidate is timed on the caller's own particles and fields with CUDA
events around the push, starting every trial from the same saved state, and
the fastest is kept in the context.  The particles are restored afterwards.
"""
from __future__ import annotations

import torch

from . import fpic as F

_STATE = ("r", "th", "ph", "ur", "uth", "uph", "H0", "D0", "Hn", "alive", "scheme", "iters", "cell")


def _save(p):
    return {k: getattr(p, k).clone() for k in _STATE if getattr(p, k, None) is not None}


def _load(p, snap):
    for k, v in snap.items():
        getattr(p, k).copy_(v)


def tune_imr_blocks(ctx, p, fields, prm, candidates=(1, 2, 3, 4), reps=3, push=None):
    """Pick FPIC_TUNE_IMR_BLOCKS_PER_SM by timing `reps` pushes per candidate
    (push(ctx, p, fields, prm) defaults to fpic_push).  Returns
    {candidate: mean ms} and leaves the best value set in ctx."""
    return _tune_push(ctx, p, fields, prm, F.FPIC_TUNE_IMR_BLOCKS_PER_SM, candidates, reps, push)


def tune_stage_fields(ctx, p, fields, prm, reps=3, push=None):
    """Pick FPIC_TUNE_STAGE_FIELDS (TMA staging of the field tiles of each
    block of cell-sorted particles: 0 off, 1 on) by timing `reps` pushes of
    each on the caller's particles.  Returns {0: ms, 1: ms} and leaves the
    faster set in ctx (the results are the same either way)."""
    times = _tune_push(ctx, p, fields, prm, F.FPIC_TUNE_STAGE_FIELDS, (0, 1), reps, push)
    return times


def staged_fraction(ctx, p, fields, prm):
    """Share of the explicit pass's blocks that staged their field tile in
    one push with staging on, from the same saved state (restored after)."""
    snap = _save(p)
    old = F.fpic_get_tuning(ctx, F.FPIC_TUNE_STAGE_FIELDS)
    F.fpic_set_tuning(ctx, F.FPIC_TUNE_STAGE_FIELDS, 1)
    st = F.fpic_push(ctx, p, fields, prm, stats=True)
    F.fpic_set_tuning(ctx, F.FPIC_TUNE_STAGE_FIELDS, old)
    _load(p, snap)
    torch.cuda.synchronize()
    return st["n_tiles_staged"] / max(1, (p.n + 127) // 128)


def _tune_push(ctx, p, fields, prm, key, candidates, reps, push):
    push = push or (lambda c, q, f, m: F.fpic_push(c, q, f, m))
    snap = _save(p)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = {}
    for v in candidates:
        F.fpic_set_tuning(ctx, key, v)
        _load(p, snap)
        push(ctx, p, fields, prm)          # warm-up at this shape
        tot = 0.0
        for _ in range(reps):
            _load(p, snap)
            torch.cuda.synchronize()
            e0.record()
            push(ctx, p, fields, prm)
            e1.record()
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        times[v] = tot / reps
    best = min(times, key=times.get)
    F.fpic_set_tuning(ctx, key, best)
    _load(p, snap)
    torch.cuda.synchronize()
    return times


def tune_deposit_threads(ctx, p, size, candidates=(64, 128, 256), reps=3):
    """Pick FPIC_TUNE_DEP_THREADS by timing `reps` deposits (sort included)
    per candidate on the caller's particles.  The deposit's output does not
    depend on the choice; the particles end up sorted by cell either way.
    Returns {candidate: mean ms} and leaves the best value set in ctx."""
    out = tuple(torch.zeros(size, dtype=torch.float64, device=p.r.device) for _ in range(4))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = {}
    for v in candidates:
        F.fpic_set_tuning(ctx, F.FPIC_TUNE_DEP_THREADS, v)
        F.fpic_deposit(ctx, p, size, out=out)      # warm-up at this shape
        tot = 0.0
        for _ in range(reps):
            torch.cuda.synchronize()
            e0.record()
            F.fpic_deposit(ctx, p, size, out=out)
            e1.record()
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        times[v] = tot / reps
    best = min(times, key=times.get)
    F.fpic_set_tuning(ctx, F.FPIC_TUNE_DEP_THREADS, best)
    return times
