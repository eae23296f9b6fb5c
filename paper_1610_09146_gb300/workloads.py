"""Seeded synthetic workloads: the batched ensemble and the serving request stream.

Both are Taylor-Green solves (Section 3) with parameters drawn from fixed
distributions; nothing here is arithmetic of the method.

* ensemble(): 64 instances, cubic grids drawn uniformly from {32, 48, 64, 96, 128}^3,
  Re uniform in [400, 3200], Mach uniform in [0.1, 0.4], 100 RK3 steps each,
  numpy default_rng(1610).
* requests(): a Poisson stream with mean rate 20 requests/s, grids drawn uniformly
  from the multiples of 16 in [48, 192], step counts uniform in {50..500}, Re
  uniform in [400, 3200], Mach uniform in [0.1, 0.4], binary32 or binary64 with
  equal probability, numpy default_rng(9146).
The time step of every solve follows the rule of Section 3 (dt_for_grid).
"""
from __future__ import annotations

import numpy as np

ENSEMBLE_GRIDS = (32, 48, 64, 96, 128)


def dt_for_grid(n: int) -> float:
    """Time step of the paper's validation runs for an n^3 grid (Section 3: 3.385e-3 at
    64^3, halved for each doubling of n); grids below 64^3 keep the 64^3 value."""
    return 3.385e-3 * 64.0 / max(int(n), 64)


def ensemble(count: int = 64, steps: int = 100, seed: int = 1610):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.choice(ENSEMBLE_GRIDS))
        out.append(dict(n=n, Re=float(rng.uniform(400, 3200)), Mach=float(rng.uniform(0.1, 0.4)), Pr=0.71,
                        gamma=1.4, dt=dt_for_grid(n), steps=steps))
    return out


def requests(count: int = 400, rate: float = 20.0, seed: int = 9146, grids=None, steps_range=(50, 500)):
    """List of dicts with arrival time `t` (seconds from 0), grid n, steps, Re, Mach, dtype."""
    rng = np.random.default_rng(seed)
    grids = list(grids) if grids is not None else list(range(48, 193, 16))
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        n = int(rng.choice(grids))
        out.append(dict(id=i, t=t, n=n, steps=int(rng.integers(steps_range[0], steps_range[1] + 1)),
                        Re=float(rng.uniform(400, 3200)), Mach=float(rng.uniform(0.1, 0.4)), Pr=0.71, gamma=1.4,
                        dt=dt_for_grid(n), dtype="f32" if rng.random() < 0.5 else "f64"))
    return out
