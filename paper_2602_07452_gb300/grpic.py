"""One GRPIC step in the order of Sec. 2.1, driving the C ABI.

`GRPIC.step()` runs: [divergence cleaning, Sec. 2.4] -> FDTD sub-steps 1-4
-> [pair injection, Sec. 3.3] -> push with D^{n+3/2}, B^{n+3/2} -> deposit
at n+2 (the Sec. 2.3 deposit, or the charge-conserving variant with the
FDTD in its conserving mode) -> [sum of the sources over ranks] -> FDTD
sub-steps 7-10 -> swap of the leapfrog levels.  Every step of it is a
library call; this class only sequences them and holds the buffers.
"""
from __future__ import annotations

import torch

from . import fpic as F
from . import parallel as par


class GRPIC:
    """Plasma + fields on one grid, stepped in the paper's order.

    ctx, grid : a context with the grid set (fpic_set_grid)
    fields    : F.Fields holding the leapfrog levels (filled by the caller)
    store     : F.Particles with room for injected pairs; the first n in use
    n         : particles in use
    push_prm  : F.push_params(...) of the push (its dt is the step)
    fdtd_prm  : F.fdtd_params(...) (its `conserving` flag is set here)
    conserving: use fpic_deposit_conserving instead of fpic_deposit; the
                push writes the state it starts from into a second store
                (fpic_push_params.before), which the deposit reads as the
                move's start
    clean     : (every, sweeps) or None
    inject    : (every, F.fpic_inject_params, draws tensor) or None
    """

    def __init__(self, ctx, grid, fields, store, n, push_prm, fdtd_prm, conserving=False, clean=None,
                 inject=None):
        self.ctx, self.grid, self.fields, self.store, self.n = ctx, grid, fields, store, int(n)
        self.push_prm, self.fdtd_prm = push_prm, fdtd_prm
        self.fdtd_prm.conserving = 1 if conserving else 0
        self.conserving, self.clean, self.inject = conserving, clean, inject
        self.k = 0
        self.pairs = 0
        self.cleanings = 0
        self.prev_store = None
        if conserving:
            self.prev_store = F.Particles(*[getattr(store, f).clone() for f in store.__dataclass_fields__])
        self.out = (fields.rho1, fields.j1[0], fields.j1[1], fields.j1[2])

    @property
    def particles(self):
        return self.store.head(self.n)

    def deposit_initial(self):
        """Sources of the starting state (rho^{n+1}, J) before the first step."""
        p = self.particles
        if self.conserving:
            F.fpic_deposit_conserving(self.ctx, p, p, self.push_prm.dt, out=self.out)
        else:
            F.fpic_deposit(self.ctx, p, self.grid.size, out=self.out)
        par.allreduce_sources(self.out)

    def step(self, events=None):
        """One step; events: optional 5 CUDA events recorded between phases
        (start, after FDTD 1-4 / injection, after the push, after the
        deposit, after FDTD 7-10)."""
        fl = self.fields
        rec = (lambda i: events[i].record()) if events is not None else (lambda i: None)
        rec(0)
        if self.clean is not None and self.k % self.clean[0] == 0:
            F.fpic_div_clean(self.ctx, fl.D1, fl.rho0, self.clean[1])
            self.cleanings += 1
        F.fpic_fdtd_step(self.ctx, fl, self.fdtd_prm, 1)
        if self.inject is not None and self.k % self.inject[0] == 0:
            n_new, wanted, _ = F.fpic_inject_pairs(self.ctx, self.store, self.n, fl.B1[0], fl.B1[1],
                                                   self.inject[1], self.inject[2])
            self.pairs += wanted
            self.n = n_new
        self.k += 1
        p = self.particles
        prev = None
        if self.conserving:
            prev = self.prev_store.head(self.n)
            F.set_push_before(self.push_prm, prev)
        rec(1)
        F.fpic_push(self.ctx, p, fl.push_fields(), self.push_prm)
        rec(2)
        if self.conserving:
            F.fpic_deposit_conserving(self.ctx, prev, p, self.push_prm.dt, out=self.out)
        else:
            F.fpic_deposit(self.ctx, p, self.grid.size, out=self.out)
        par.allreduce_sources(self.out)
        rec(3)
        F.fpic_fdtd_step(self.ctx, fl, self.fdtd_prm, 2)
        rec(4)
        fl.swap()
        self.out = (fl.rho1, fl.j1[0], fl.j1[1], fl.j1[2])
