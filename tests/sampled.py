"""The oracle's one-step result at sample points of a large grid (test helper).

A full-size grid is beyond what the oracle finishes in seconds, but one RK3
step at a point depends only on the points within 6 of it (2 per stage), so
each sample is computed on a small periodic block cut around it.
"""
import numpy as np

import oracle as O


def _block(Q, z, y, x, r):
    nz, ny, nx = Q.shape[1:]
    iz = (np.arange(z - r, z + r + 1)) % nz
    iy = (np.arange(y - r, y + r + 1)) % ny
    ix = (np.arange(x - r, x + r + 1)) % nx
    return np.ascontiguousarray(Q[:, iz][:, :, iy][:, :, :, ix])


def oracle_one_step_at(Q0, pts, dt, h):
    """The oracle's one-step result at sample points, each computed on a periodic
    17^3 block cut around the point with the parent grid spacing.  The scheme's
    dependency radius is 2 points per stage (6 per step), so the centre of the
    block is unaffected by the block's own wrap-around."""
    r = 8
    out = []
    for (z, y, x) in pts:
        B = _block(Q0, z, y, x, r)
        B1 = O.run(B, 1, dt=dt, h=h)
        out.append(B1[:, r, r, r])
    return np.array(out)
