"""Two-level subcycled advance with refluxing -- TEST INFRASTRUCTURE ONLY (oracle).

Sec. 3 says the codes sit on block-structured AMR with subcycling in time, and
Sec. 4 says how Castro integrates on the hierarchy: a coarse level advances
first, the finer level then takes several smaller steps to reach the same
time, and the levels are synchronised.  The paper gives no formulas for the
pieces; this module takes the Berger-Colella reading that block-structured
AMR codes of this family use, for a refinement ratio of 2 in space and time:

  1. coarse step: one CTU-PPM step of dt on the whole coarse level (one box
     over the domain here; its fluxes through every face are kept);
  2. fine steps: two steps of dt/2 on every fine box.  Before each, every
     fine ghost zone is copied from the fine box whose interior holds it, or
     else interpolated from the coarse level: first in time (the coarse state
     at t for the first step, the mean 0.5*U(t) + 0.5*U(t+dt) for the second),
     then in space (linear, with a monotonised-central slope per axis);
  3. reflux: a coarse zone outside the fine region that shares a face with a
     covered coarse zone has that face's coarse flux replaced by the fine
     fluxes through it, averaged over the 2^(dim-1) fine faces and the two
     fine steps;
  4. average down: a covered coarse zone becomes the mean of its 2^dim fine
     children.

The readings (interpolation, time centring, nesting rules and summation orders)
are stated where they are used.  Everything is plain loops or whole-array
numpy on the grown arrays of the single-box oracle (layout (5, gz, ny+8, nx+8),
gz = nz+8 in 3-D, 1 in 2-D); the step itself is `oracle.step`.
"""
import numpy as np

from . import BC_PREFILLED, dt as box_dt, params, step

NG = 4
RATIO = 2


def _at(U, dim, i, j, k):
    """Conserved vector (5,) of zone (i, j, k) of a grown array (i, j, k may be arrays)."""
    if dim == 3:
        return U[:, k + NG, j + NG, i + NG]
    return U[:, 0, j + NG, i + NG]


def _set(U, dim, i, j, k, v):
    if dim == 3:
        U[:, k + NG, j + NG, i + NG] = v
    else:
        U[:, 0, j + NG, i + NG] = v


def _grown_coords(n, dim):
    """Local zone coordinates (i, j, k) of every zone of a grown box, flattened."""
    zr = np.arange(-NG, n[2] + NG) if dim == 3 else np.array([0])
    k, j, i = np.meshgrid(zr, np.arange(-NG, n[1] + NG), np.arange(-NG, n[0] + NG), indexing="ij")
    return i.ravel(), j.ravel(), k.ravel()


class FineBox:
    """A fine box: lower corner `lo` in the fine index space (twice the coarse
    one), interior size `n`, grown conserved array `U`."""

    def __init__(self, lo, n, U):
        self.lo = tuple(int(v) for v in lo) + (0,) * (3 - len(lo))
        self.n = tuple(int(v) for v in n) + (1,) * (3 - len(n))
        self.U = np.array(U, dtype=np.float64)

    def contains(self, gi, gj, gk, dim):
        c = (gi >= self.lo[0]) & (gi < self.lo[0] + self.n[0]) & (gj >= self.lo[1]) & (gj < self.lo[1] + self.n[1])
        if dim == 3:
            c &= (gk >= self.lo[2]) & (gk < self.lo[2] + self.n[2])
        return c


def check_nesting(domain, fines, dim):
    """The hierarchy this module (and the kernels it checks) accepts: fine
    boxes with even corners and sizes, no two overlapping, and every fine box,
    coarsened and grown by 3 coarse zones (2 for its 4 fine ghost layers, 1 for
    the interpolation slope), inside the coarse domain -- so fine ghost zones
    never need a domain boundary condition and every coarse zone the
    interpolation reads is an interior zone."""
    for b in fines:
        for a in range(dim):
            if b.lo[a] % RATIO or b.n[a] % RATIO:
                raise ValueError("fine box corners and sizes must be even")
            if b.lo[a] // RATIO - 3 < 0 or (b.lo[a] + b.n[a]) // RATIO + 3 > domain[a]:
                raise ValueError("fine box too close to the domain boundary")
    for x in range(len(fines)):
        for y in range(x + 1, len(fines)):
            A, B = fines[x], fines[y]
            if all(A.lo[a] < B.lo[a] + B.n[a] and B.lo[a] < A.lo[a] + A.n[a] for a in range(dim)):
                raise ValueError("fine boxes overlap")


def mc_slope(ul, u0, ur):
    """Monotonised-central slope of u0 between its neighbours (whole arrays):
    zero unless both one-sided differences are non-zero with the same sign,
    else the smallest of twice either one-sided difference and the central
    difference, with their common sign."""
    dl = u0 - ul
    dr = ur - u0
    same = ((dl > 0) & (dr > 0)) | ((dl < 0) & (dr < 0))
    m = np.minimum(np.minimum(2.0 * np.abs(dl), 2.0 * np.abs(dr)), 0.5 * np.abs(dl + dr))
    return np.where(same, np.copysign(m, dl), 0.0)


def prolong(T, dim, gi, gj, gk):
    """Conservative linear interpolation of the coarse grown array T at fine
    zones (gi, gj, gk) (arrays, fine index space).  The parent coarse zone is
    g // 2; the child's centre sits a quarter of a coarse zone below or above
    the parent's along each axis.  Value = parent + s_x*o_x + s_y*o_y + s_z*o_z
    (in that order) with s the MC slope of the parent along each axis.  The
    offsets of the 2^dim children sum to zero, so their mean is the parent."""
    g = [gi, gj, gk]
    P = [v // RATIO for v in g]
    o = [np.where(v % RATIO == 0, -0.25, 0.25) for v in g]
    u0 = _at(T, dim, P[0], P[1], P[2])
    val = u0.copy()
    for d in range(dim):
        lo = list(P)
        hi = list(P)
        lo[d] = P[d] - 1
        hi[d] = P[d] + 1
        s = mc_slope(_at(T, dim, *lo), u0, _at(T, dim, *hi))
        val = val + s * o[d]
    return val


def coarse_at_time(Uc_old, Uc_new, half):
    """Coarse state at the fine step's start: U(t), or 0.5*U(t) + 0.5*U(t+dt)."""
    if not half:
        return Uc_old
    return 0.5 * Uc_old + 0.5 * Uc_new


def fill_fine(fines, T, dim):
    """Fill every ghost zone of every fine box (in place): a copy from the fine
    box whose interior holds the zone, else prolong(T)."""
    new = []
    for A in fines:
        i, j, k = _grown_coords(A.n, dim)
        ghost = (i < 0) | (i >= A.n[0]) | (j < 0) | (j >= A.n[1])
        if dim == 3:
            ghost |= (k < 0) | (k >= A.n[2])
        i, j, k = i[ghost], j[ghost], k[ghost]
        gi, gj, gk = i + A.lo[0], j + A.lo[1], (k + A.lo[2]) if dim == 3 else np.zeros_like(i)
        V = np.empty((5, i.size))
        done = np.zeros(i.size, dtype=bool)
        for B in fines:
            if B is A:
                continue
            m = B.contains(gi, gj, gk, dim)
            if m.any():
                V[:, m] = _at(B.U, dim, gi[m] - B.lo[0], gj[m] - B.lo[1], (gk[m] - B.lo[2]) if dim == 3 else 0)
                done |= m
        u = ~done
        V[:, u] = prolong(T, dim, gi[u], gj[u], gk[u])
        W = A.U.copy()
        _set(W, dim, i, j, k, V)
        new.append(W)
    for A, W in zip(fines, new):  # every box filled from the states before any write
        A.U = W


def covered_mask(domain, fines, dim):
    """Coarse zones covered by the fine level (array [nz][ny][nx], 2-D: nz = 1)."""
    nz = domain[2] if dim == 3 else 1
    M = np.zeros((nz, domain[1], domain[0]), dtype=bool)
    for B in fines:
        c0 = [B.lo[a] // RATIO for a in range(3)]
        c1 = [(B.lo[a] + B.n[a]) // RATIO for a in range(3)]
        if dim == 3:
            M[c0[2]:c1[2], c0[1]:c1[1], c0[0]:c1[0]] = True
        else:
            M[0, c0[1]:c1[1], c0[0]:c1[0]] = True
    return M


def interface_faces(domain, fines, dim):
    """Coarse-fine interface faces, grouped by the uncovered coarse zone they
    bound: [(zone (i, j, k), [(d, side), ...])] with side -1 for the zone's low
    face and +1 for its high face, faces in the order x-low, x-high, y-low,
    y-high, z-low, z-high; zones in row-major order (x fastest)."""
    M = covered_mask(domain, fines, dim)
    nz = M.shape[0]
    out = []
    for k in range(nz):
        for j in range(domain[1]):
            for i in range(domain[0]):
                if M[k, j, i]:
                    continue
                faces = []
                for d in range(dim):
                    for side in (-1, 1):
                        z = [i, j, k]
                        z[d] += side
                        if 0 <= z[d] < domain[d] and M[z[2], z[1], z[0]]:
                            faces.append((d, side))
                if faces:
                    out.append(((i, j, k), faces))
    return out


def _fine_box_of(fines, g, dim):
    for B in fines:
        if all(B.lo[a] <= g[a] < B.lo[a] + B.n[a] for a in range(dim)):
            return B
    raise AssertionError("fine zone not covered")


def fine_face_sum(fines, fluxes, zone, d, side, dim, acc):
    """Add to acc (5,) the final fluxes through the 2^(dim-1) fine faces under
    the coarse face (zone, d, side) of one fine step, fluxes[b][d] being box
    b's flux array (a face f along d is stored at the position of zone f).
    Order: the second transverse axis outer, the first inner (each offset 0
    then 1), transverse axes in increasing order."""
    face = zone[d] + (1 if side > 0 else 0)       # coarse face position along d
    gf = RATIO * face                             # the same face in the fine index space
    inside = gf if side > 0 else gf - 1           # the covered fine zone next to it
    t = [a for a in range(dim) if a != d]
    offs = [(0,), (0,)]
    if len(t) >= 1:
        offs[0] = (0, 1)
    if len(t) == 2:
        offs[1] = (0, 1)
    for o2 in offs[1]:
        for o1 in offs[0]:
            g = [0, 0, 0]
            g[d] = inside
            if len(t) >= 1:
                g[t[0]] = RATIO * zone[t[0]] + o1
            if len(t) == 2:
                g[t[1]] = RATIO * zone[t[1]] + o2
            b = _fine_box_of(fines, g, dim)
            F = fluxes[fines.index(b)][d]
            loc = [g[a] - b.lo[a] for a in range(3)]
            loc[d] = gf - b.lo[d]
            acc = acc + _at(F, dim, loc[0], loc[1], loc[2] if dim == 3 else 0)
    return acc


def average_down(Uc, fines, dim):
    """Covered coarse zones become the mean of their children: the children
    summed z-offset outer, then y, then x (each 0 then 1), times 2^-dim."""
    w = 0.5 ** dim
    for B in fines:
        c0 = [B.lo[a] // RATIO for a in range(3)]
        c1 = [(B.lo[a] + B.n[a]) // RATIO for a in range(3)]
        if dim == 2:
            c0[2], c1[2] = 0, 1
        for K in range(c0[2], c1[2]):
            for J in range(c0[1], c1[1]):
                for I in range(c0[0], c1[0]):
                    s = np.zeros(5)
                    for oz in ((0, 1) if dim == 3 else (0,)):
                        for oy in (0, 1):
                            for ox in (0, 1):
                                fi = RATIO * I + ox - B.lo[0]
                                fj = RATIO * J + oy - B.lo[1]
                                fk = (RATIO * K + oz - B.lo[2]) if dim == 3 else 0
                                s = s + _at(B.U, dim, fi, fj, fk)
                    _set(Uc, dim, I, J, K, s * w)


def advance(Uc, fines, dt, dim, domain, domain_bc, dx, gamma=1.4, cfl=0.5, grav=(0.0, 0.0, 0.0),
            reflux=True, **kw):
    """One coarse step dt of the two-level hierarchy.

    Uc: coarse grown array over the whole domain (domain boundary kinds
    domain_bc, coarse spacing dx); fines: list of FineBox (fine spacing dx/2);
    dt: the coarse step.  Returns (Uc_new, fines_new, dt_next, bad) where
    dt_next = min(CFL step of the synchronised coarse level, 2 * CFL step of
    each fine box) and bad is True if any step met a non-physical state.
    `reflux=False` skips step 3 (used only to show that the conservation pin
    depends on it)."""
    check_nesting(domain, fines, dim)
    n = tuple(domain[:dim])
    Pc = params(dim, n, dx=dx, bc=domain_bc, gamma=gamma, cfl=cfl, grav=grav, **kw)
    dxf = tuple(v / RATIO for v in dx)
    bad = False
    # 1. coarse step, its final fluxes kept
    Uc_new, rc, dbg = step(Uc, Pc, dt, debug=True)
    bad |= rc != 0
    Fc = dbg["flux_final"]
    # 2. two fine steps of dt/2
    fines = [FineBox(b.lo, b.n, b.U) for b in fines]
    fine_fluxes = []
    for half in (False, True):
        fill_fine(fines, coarse_at_time(Uc, Uc_new, half), dim)
        fl = []
        for B in fines:
            Pf = params(dim, B.n[:dim], dx=dxf, bc=BC_PREFILLED, gamma=gamma, cfl=cfl, grav=grav, **kw)
            B.U, rc, dbg = step(B.U, Pf, dt / RATIO, debug=True)
            bad |= rc != 0
            fl.append(dbg["flux_final"])
        fine_fluxes.append(fl)
    # 3. reflux the uncovered coarse zones at the coarse-fine interface
    if reflux:
        w = 0.5 ** dim  # 1 / (2^(dim-1) fine faces * 2 fine steps)
        for zone, faces in interface_faces(domain, fines, dim):
            u = _at(Uc_new, dim, *zone).copy()
            for d, side in faces:
                face = list(zone)
                if side > 0:
                    face[d] += 1
                fc = _at(Fc[d], dim, *face)
                acc = np.zeros(5)
                for fl in fine_fluxes:
                    acc = fine_face_sum(fines, fl, zone, d, side, dim, acc)
                sgn = -1.0 if side > 0 else 1.0
                u = u + (sgn * (dt / dx[d])) * (acc * w - fc)
            _set(Uc_new, dim, *zone, u)
    # 4. average down
    average_down(Uc_new, fines, dim)
    # the next step: the CFL limit of both levels on the coarse clock
    d_c, rc = box_dt(Uc_new, Pc)
    bad |= rc != 0
    dt_next = d_c
    for B in fines:
        Pf = params(dim, B.n[:dim], dx=dxf, bc=BC_PREFILLED, gamma=gamma, cfl=cfl, grav=grav, **kw)
        d_f, rc = box_dt(B.U, Pf)
        bad |= rc != 0
        dt_next = min(dt_next, RATIO * d_f)
    return Uc_new, fines, dt_next, bad
