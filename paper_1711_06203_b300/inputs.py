"""Seeded synthetic initial data for the CTU-PPM hydro step.

Problem set-up only: this module builds initial conditions from their
primitive definitions (density, velocity, pressure) and converts them to the
conserved fields with the ideal-gas relation rho*E = p/(gamma-1) + rho|u|^2/2.
It holds none of the scheme's arithmetic and serves the CUDA path and the CPU
oracle alike, so both always see the same bits.

Arrays are float64, shape (5, gz, gy, gx): components (rho, rho*u, rho*v,
rho*w, rho*E), x fastest, over the grown box (interior plus NG = 4 ghost zones
per side of each active axis; 2-D boxes have gz = 1).  The shapes mirror the
paper's workloads: Sedov blasts and stratified stellar atmospheres on
block-structured boxes of uneven sizes (Sec. 4, Figs. 1, 3, 4), plus the
textbook Sod shock tube.
"""
import numpy as np

NG = 4
BC_OUTFLOW, BC_REFLECT, BC_PERIODIC, BC_PREFILLED = 0, 1, 2, 3


def grown_shape(n, dim):
    """(gz, gy, gx) of a box with interior n = (nx, ny, nz)."""
    nx, ny, nz = n
    gz = nz + 2 * NG if dim == 3 else 1
    return (gz, ny + 2 * NG, nx + 2 * NG)


def conserved(rho, u, v, w, p, gamma):
    """Conserved fields from primitive ones (ideal gas)."""
    rho = np.asarray(rho, dtype=np.float64)
    U = np.empty((5,) + rho.shape, dtype=np.float64)
    U[0] = rho
    U[1] = rho * u
    U[2] = rho * v
    U[3] = rho * w
    U[4] = p / (gamma - 1.0) + 0.5 * rho * ((u * u + v * v) + w * w)
    return U


def zone_centres(n, dim, dx, lo=(0.0, 0.0, 0.0)):
    """Zone-centre coordinates on the grown box (ghosts included)."""
    gz, gy, gx = grown_shape(n, dim)
    x = lo[0] + (np.arange(gx) - NG + 0.5) * dx[0]
    y = lo[1] + (np.arange(gy) - NG + 0.5) * dx[1]
    if dim == 3:
        z = lo[2] + (np.arange(gz) - NG + 0.5) * dx[2]
    else:
        z = np.zeros(1)
    return np.meshgrid(z, y, x, indexing="ij")[::-1]  # x, y, z arrays of shape (gz, gy, gx)


def sod(n=64, dim=2, axis=0, gamma=1.4, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1), x0=0.5):
    """Sod shock tube along `axis` on the unit square/cube: (rho, u_n, p) left/right of x0."""
    nn = (n, n, n if dim == 3 else 1)
    dx = (1.0 / n,) * 3
    X = zone_centres(nn, dim, dx)[axis]
    L = X < x0
    rho = np.where(L, left[0], right[0])
    un = np.where(L, left[1], right[1])
    p = np.where(L, left[2], right[2])
    vel = [np.zeros_like(rho) for _ in range(3)]
    vel[axis] = un
    return conserved(rho, vel[0], vel[1], vel[2], p, gamma)


def sedov_deposit_mask(n, dim=3, radius_zones=4.0):
    """Zones whose centre lies strictly within radius_zones * dx of the domain centre.

    Decided in units of dx on half-integer offsets, so the set is exact."""
    gz, gy, gx = grown_shape((n, n, n if dim == 3 else 1), dim)
    ox = np.arange(gx) - NG + 0.5 - n / 2.0
    oy = np.arange(gy) - NG + 0.5 - n / 2.0
    oz = (np.arange(gz) - NG + 0.5 - n / 2.0) if dim == 3 else np.zeros(1)
    Z, Y, X = np.meshgrid(oz, oy, ox, indexing="ij")
    return (X * X + Y * Y + Z * Z) < radius_zones * radius_zones


def sedov(n=128, dim=3, gamma=1.4, E=1.0, rho0=1.0, p_amb=1e-5, radius_zones=4.0):
    """Sedov blast: energy E deposited uniformly as pressure in the zones within
    radius_zones*dx of the centre of the unit cube; the deposit replaces the
    ambient pressure there.  Returns (U, number of deposit zones)."""
    dx = 1.0 / n
    mask = sedov_deposit_mask(n, dim, radius_zones)
    ndep = int(mask[:, NG:-NG, NG:-NG].sum()) if dim == 2 else int(mask[NG:-NG, NG:-NG, NG:-NG].sum())
    vol = dx * dx * dx if dim == 3 else dx * dx
    p_dep = (gamma - 1.0) * E / (ndep * vol)
    rho = np.full(mask.shape, rho0)
    p = np.where(mask, p_dep, p_amb)
    z = np.zeros_like(rho)
    return conserved(rho, z, z, z, p, gamma), ndep


def random_box(rng, n, dim=3, gamma=5.0 / 3.0, sigma_rho=0.5, sigma_u=0.1, sigma_p=0.3):
    """Every zone (ghosts included): rho ~ LogNormal(0, sigma_rho), each velocity
    component ~ N(0, sigma_u), p ~ LogNormal(0, sigma_p)."""
    shape = grown_shape(n, dim)
    rho = rng.lognormal(0.0, sigma_rho, shape)
    u = rng.normal(0.0, sigma_u, shape)
    v = rng.normal(0.0, sigma_u, shape)
    w = rng.normal(0.0, sigma_u, shape) if dim == 3 else np.zeros(shape)
    p = rng.lognormal(0.0, sigma_p, shape)
    return conserved(rho, u, v, w, p, gamma)


def stratified(n, dim=3, gamma=5.0 / 3.0, g=1.0, H=0.1, perturb=0.0, rng=None):
    """Isothermal atmosphere in hydrostatic balance under gravity -g along the
    last active axis: rho = exp(-z/H), p = rho g H at zone centres, optional
    seeded relative pressure perturbation p *= 1 + perturb N(0,1)."""
    nn = (n, n, n if dim == 3 else 1)
    dx = (1.0 / n,) * 3
    X = zone_centres(nn, dim, dx)
    z = X[dim - 1]
    rho = np.exp(-z / H)
    p = rho * g * H
    if perturb:
        p = p * (1.0 + perturb * rng.normal(0.0, 1.0, p.shape))
    zero = np.zeros_like(rho)
    return conserved(rho, zero, zero, zero, p, gamma)


def uniform_flow(rho, vel, p, dim, gamma):
    """A density field carried by a uniform velocity `vel` at uniform pressure
    `p` (w = 0 in 2-D)."""
    z = np.zeros_like(rho)
    w = vel[2] if dim == 3 else 0.0
    return conserved(rho, vel[0] + z, vel[1] + z, w + z, p + z, gamma)


def product_profile(n, dim, dx, vel, t=0.0, amp=0.3, gamma=1.4):
    """rho = 2 + amp * prod_a (x_a - vel_a t + 1) over the active axes (bilinear
    in 2-D, trilinear in 3-D), uniform velocity `vel` and p = 1, sampled at
    zone centres (equal to the zone averages: the profile is linear in each
    coordinate separately).  At t > 0 it is the exact solution translated by
    vel * t."""
    X = zone_centres(n, dim, dx)
    r = 1.0
    for a in range(dim):
        r = r * (X[a] - vel[a] * t + 1.0)
    return uniform_flow(2.0 + amp * r, vel, 1.0, dim, gamma)


def translation_box(rng, n, dim, dx, dt, signs, gamma=1.4, sigma_rho=0.5):
    """Random density rho ~ LogNormal(0, sigma_rho) on every zone (ghosts
    included), carried at uniform pressure 1 by the uniform velocity whose
    component a is signs[a] * dx[a] / dt: in one step of length dt the exact
    solution moves every zone average by exactly one zone along each active
    axis.  Returns (U, U_translated), the second the exact answer on the
    interior."""
    shape = grown_shape(n, dim)
    rho = rng.lognormal(0.0, sigma_rho, shape)
    vel = tuple(signs[a] * dx[a] / dt for a in range(3))
    moved = rho
    for a in range(dim):
        moved = np.roll(moved, signs[a], axis=2 - a)
    return uniform_flow(rho, vel, 1.0, dim, gamma), uniform_flow(moved, vel, 1.0, dim, gamma)


LEVEL_SIDES = (16, 24, 32, 48, 64)


def level_box_sizes(nbox=512, seed=1711, sides=LEVEL_SIDES):
    """Interior sizes (nx, ny, nz) of an AMR level of uneven boxes: each side drawn
    independently and uniformly from `sides`."""
    rng = np.random.default_rng(seed)
    return [tuple(int(s) for s in rng.choice(sides, 3)) for _ in range(nbox)]


def level_boxes(nbox=512, seed=1711, gamma=5.0 / 3.0, sides=LEVEL_SIDES):
    """The batched-level workload: sizes plus random prefilled states for every box."""
    sizes = level_box_sizes(nbox, seed, sides)
    rng = np.random.default_rng(seed + 1)
    return sizes, [random_box(rng, s, 3, gamma) for s in sizes]


def two_state(n, dim=3, gamma=1.4, rhoL=1.0, pL=1.0, rhoR=0.125, pR=0.1, x0=0.5):
    """Planar two-state Riemann problem along x at rest (the served 'two-state' kind)."""
    return sod(n, dim, 0, gamma, (rhoL, 0.0, pL), (rhoR, 0.0, pR), x0)


SERVE_SIDES = (32, 64, 96, 128, 192, 256)


def serve_requests(count, seed=1711, sides=SERVE_SIDES):
    """Seeded stream of independent problems for the server: kind uniform over
    {Sod (gamma 1.4), Sedov (gamma 1.4, E = 1, ambient p = 1e-5), two-state
    (rho_L, rho_R, p_L, p_R ~ LogNormal(0, 1), gamma from {1.4, 5/3})}, cubic
    side uniform over `sides`, steps uniform in [10, 100].  Returns a list of
    keyword dicts (kind 0 = Sod, 1 = Sedov, 2 = two-state)."""
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(count):
        kind = int(rng.integers(0, 3))
        n = int(rng.choice(sides))
        steps = int(rng.integers(10, 101))
        r = dict(kind=kind, n=n, steps=steps, gamma=1.4)
        if kind == 2:
            rl, rr, pl, pr = rng.lognormal(0.0, 1.0, 4)
            r.update(gamma=float(rng.choice((1.4, 5.0 / 3.0))), rho_l=float(rl), p_l=float(pl), rho_r=float(rr),
                     p_r=float(pr))
        reqs.append(r)
    return reqs


def poisson_arrivals(count, rate, seed=1711):
    """Arrival times (seconds from 0) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed + 7)
    return np.cumsum(rng.exponential(1.0 / rate, count))


def level_tiling(domain, sides=LEVEL_SIDES, seed=1711):
    """Cut a rectangular domain into a level of uneven boxes: along each axis
    the domain is split into consecutive pieces with lengths drawn from `sides`
    (the last piece takes the remainder, which must be a multiple of 8).
    Returns (lo corners, sizes) of the product tiling, x fastest."""
    rng = np.random.default_rng(seed)
    cuts = []
    for n in domain:
        pieces, pos = [], 0
        while pos < n:
            s = int(rng.choice(sides))
            if pos + s > n:
                s = n - pos
            pieces.append((pos, s))
            pos += s
        cuts.append(pieces)
    lo, sizes = [], []
    for (z0, nz) in (cuts[2] if len(domain) == 3 else [(0, 1)]):
        for (y0, ny) in cuts[1]:
            for (x0, nx) in cuts[0]:
                lo.append((x0, y0, z0))
                sizes.append((nx, ny, nz))
    return lo, sizes


def amr_field(x, y, z, dim, gamma, p_amp=4.0, r0=0.12, centre=(0.5, 0.5, 0.5)):
    """Smooth periodic background on the unit domain with a Gaussian pressure
    bump: rho = 1 + 0.3 sin(2 pi x) cos(2 pi y) [cos(2 pi z)],
    u = 0.2 sin(2 pi y), v = 0.2 cos(2 pi x), w = 0.1 sin(2 pi x) (3-D),
    p = 1 + p_amp exp(-(r / r0)^2), r the distance to `centre`."""
    tp = 2.0 * np.pi
    cz = np.cos(tp * z) if dim == 3 else 1.0
    rho = 1.0 + 0.3 * np.sin(tp * x) * np.cos(tp * y) * cz
    u = 0.2 * np.sin(tp * y)
    v = 0.2 * np.cos(tp * x)
    w = 0.1 * np.sin(tp * x) if dim == 3 else np.zeros_like(x)
    r2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 + ((z - centre[2]) ** 2 if dim == 3 else 0.0)
    p = 1.0 + p_amp * np.exp(-r2 / (r0 * r0))
    return conserved(rho, u + 0.0 * x, v + 0.0 * x, w + 0.0 * x, p + 0.0 * x, gamma)


def amr_two_level(domain, dim, fine_lo, fine_n, gamma=1.4, **kw):
    """A two-level hierarchy on the unit-width domain (coarse spacing
    1/domain[0] on every axis, fine spacing half of it), both levels sampled
    from amr_field at their zone centres (ghosts included).
    fine_lo / fine_n: corners and sizes of the fine boxes in the fine index
    space.  Returns (coarse grown array, [fine grown arrays], coarse dx)."""
    n = tuple(domain) + (1,) * (3 - len(domain))
    dx = (1.0 / n[0],) * 3
    X = zone_centres(n, dim, dx)
    Uc = amr_field(X[0], X[1], X[2], dim, gamma, **kw)
    fines = []
    dxf = tuple(v / 2 for v in dx)
    for lo, s in zip(fine_lo, fine_n):
        s = tuple(s) + (1,) * (3 - len(s))
        org = tuple(lo[a] * dxf[a] if a < dim else 0.0 for a in range(3))
        Xf = zone_centres(s, dim, dxf, org)
        fines.append(amr_field(Xf[0], Xf[1], Xf[2], dim, gamma, **kw))
    return Uc, fines, dx


def species_fractions(rng, shape, nspec, concentration=1.0):
    """Mass fractions of nspec species at every zone of `shape`: a
    Dirichlet(concentration) draw per zone (non-negative, summing to one)."""
    g = rng.gamma(concentration, 1.0, (nspec,) + tuple(shape))
    return g / g.sum(axis=0)


def with_species(U, X):
    """The conserved state U (5, ...) extended by the species densities
    rho X_k (X: (nspec, ...) mass fractions on the same zones)."""
    return np.concatenate([U, U[0][None] * X], axis=0)
