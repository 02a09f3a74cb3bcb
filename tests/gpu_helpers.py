"""Helpers shared by the GPU tests: move seeded inputs to the device, run the
library through its C ABI, compare against the CPU oracle."""
import numpy as np
import torch

import oracle
from paper_1711_06203_b300 import binding as hb
from paper_1711_06203_b300 import inputs

I3 = (slice(None), slice(4, -4), slice(4, -4), slice(4, -4))
I2 = (slice(None), 0, slice(4, -4), slice(4, -4))


def interior(U, dim):
    return U[I3] if dim == 3 else U[I2]


def to_dev(U):
    return torch.from_numpy(np.ascontiguousarray(U)).to("cuda")


def oracle_params(dim, n, dx, bc, gamma, cfl=0.5, grav=(0.0, 0.0, 0.0), flatten=True):
    return oracle.params(dim, n, dx=dx, bc=bc, gamma=gamma, cfl=cfl, grav=grav, flatten=flatten)


def gpu_steps(U, dim, n, dx, bc, gamma, dts, grav=(0.0, 0.0, 0.0), flatten=True, variant="default", ctx=None,
              cfl=0.5):
    """Advance U with the library by each dt in dts (ghosts derived from bc).
    Returns (U_final numpy with interior updated, list of dt_next from the library)."""
    n3 = tuple(n) + (1,) * (3 - len(n))
    own = ctx is None
    ctx = ctx or hb.Context(0, variant)
    p = hb.params(dim, gamma=gamma, cfl=cfl, grav=grav, flatten=flatten)
    a = to_dev(U)
    b = torch.empty_like(a)
    nexts = []
    for dt in dts:
        ba, bb = hb.box(a, n3, dx, bc), hb.box(b, n3, dx, bc)
        nexts.append(ctx.hydro_advance_box(ba, bb, p, dt, want_dt_next=True))
        a, b = b, a
    torch.cuda.synchronize()
    out = np.array(U, copy=True)
    res = a.cpu().numpy()
    if dim == 3:
        out[I3] = res[I3]
    else:
        out[I2] = res[I2]
    if own:
        ctx.close()
    return out, nexts


def rel_linf(a, b):
    """Normwise relative L-infinity per field: max|a-b| / max|b| (0 where b is identically 0)."""
    a = a.reshape(5, -1)
    b = b.reshape(5, -1)
    den = np.abs(b).max(axis=1)
    num = np.abs(a - b).max(axis=1)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def blocky_state(rng, n, dim, gamma):
    """Piecewise-constant blocks of 3 zones: a few shared states (so neighbouring
    blocks are often equal bit for bit, and zones sit at rest), velocities
    drawn from +0, -0 and +-0.3, densities and pressures lognormal."""
    shape = inputs.grown_shape(tuple(n) + (1,) * (3 - len(n)), dim)
    pal = []
    for _ in range(4):
        vel = [rng.choice([0.0, -0.0, 0.3, -0.3]) for _ in range(3)]
        pal.append((rng.lognormal(0, 0.6), *vel, rng.lognormal(0, 0.6)))
    blocks = [(s + 2) // 3 for s in shape]
    pick = rng.integers(0, len(pal), size=blocks)
    idx = np.indices(shape)
    ids = pick[tuple(i // 3 for i in idx)]
    q = np.array(pal)[ids]  # (..., 5): rho, u, v, w, p
    if dim == 2:
        q[..., 3] = 0.0
    return inputs.conserved(q[..., 0], q[..., 1], q[..., 2], q[..., 3], q[..., 4], gamma)
