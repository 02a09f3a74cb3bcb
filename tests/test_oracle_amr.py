"""Pins of the two-level subcycled oracle (oracle/amr.py) against what the
mathematics fixes, independent of the oracle's own formulas:

  * interpolation: the mean of a parent's children is the parent (the
    conservation the scheme needs), linear data are reproduced exactly, the
    slope vanishes at an extremum and is the textbook MC value elsewhere;
  * conservation: on a periodic domain without gravity the composite total
    (uncovered coarse zones plus fine zones, each times its volume) of every
    conserved quantity is unchanged by a step to rounding, and the same
    check fails by many orders of magnitude when the reflux is left out;
  * exactness: a density profile linear in space, advected by a uniform
    velocity at uniform pressure, is advanced exactly by the single-level
    step, and so by the two-level advance -- which needs the fine steps to
    take dt/2, the fine ghosts to be interpolated correctly in space and at
    the right time, and the averaging down to be the mean; the check fails
    when the second fine step's ghosts are taken at the old time;
  * structure: cutting a fine box in two changes nothing (fine ghosts are
    copied from fine neighbours, not interpolated), and with no fine boxes
    the advance is the single-level step.
"""
import numpy as np
import pytest

import oracle
from oracle import amr
from paper_1711_06203_b300 import inputs

PER, PRE = oracle.BC_PERIODIC, oracle.BC_PREFILLED


def _interior(U, dim):
    return U[:, 4:-4, 4:-4, 4:-4] if dim == 3 else U[:, 0, 4:-4, 4:-4]


def _boxes(fine_lo, fine_n, arrays):
    return [amr.FineBox(lo, n, U) for lo, n, U in zip(fine_lo, fine_n, arrays)]


def test_mc_slope_textbook_values():
    s = amr.mc_slope(np.array([1.0, 0.0, 1.0, 0.0, 3.0, 5.0]),
                     np.array([2.0, 1.0, 2.0, 0.0, 2.0, 3.0]),
                     np.array([3.0, 1.25, 1.0, 1.0, 0.0, 2.75]))
    # smooth: central; steep on one side: twice the gentle side; extremum: 0;
    # flat on one side: 0; decreasing: negative central; decreasing, one side gentle
    assert np.array_equal(s, [1.0, 0.5, 0.0, 0.0, -1.5, -0.5])


@pytest.mark.parametrize("dim", [2, 3])
def test_prolong_children_mean_is_parent(dim):
    rng = np.random.default_rng(5 + dim)
    n = (10, 9, 8 if dim == 3 else 1)
    T = inputs.random_box(rng, n, dim)
    for I, J, K in [(1, 1, 1), (4, 5, 3), (8, 7, 6), (2, 6, 1)]:
        K = K if dim == 3 else 0
        kids = []
        for oz in ((0, 1) if dim == 3 else (0,)):
            for oy in (0, 1):
                for ox in (0, 1):
                    kids.append(amr.prolong(T, dim, np.array([2 * I + ox]), np.array([2 * J + oy]),
                                            np.array([2 * K + oz]))[:, 0])
        kids = np.array(kids)
        parent = T[:, K + 4, J + 4, I + 4] if dim == 3 else T[:, 0, J + 4, I + 4]
        scale = np.abs(kids).max(axis=0)
        assert np.all(np.abs(kids.mean(axis=0) - parent) <= 4e-16 * scale)
        # the interpolant adds no new extremum along any single axis
        assert np.all(kids.max(axis=0) >= parent) and np.all(kids.min(axis=0) <= parent)


@pytest.mark.parametrize("dim", [2, 3])
def test_prolong_reproduces_linear_data(dim):
    n = (8, 8, 8 if dim == 3 else 1)
    X = inputs.zone_centres(n, dim, (1.0, 1.0, 1.0))
    coef = np.array([[0.3, -1.7, 2.2], [1.1, 0.5, -0.25], [-2.0, 0.0, 1.0], [0.7, 0.7, 0.7], [5.0, -3.0, 0.125]])
    T = np.array([10.0 + c[0] * X[0] + c[1] * X[1] + (c[2] * X[2] if dim == 3 else 0.0) for c in coef])
    g = np.arange(2, 14)
    gi, gj = np.meshgrid(g, g, indexing="ij")
    gk = (gi + gj) % 12 + 2 if dim == 3 else np.zeros_like(gi)
    gi, gj, gk = gi.ravel(), gj.ravel(), gk.ravel()
    got = amr.prolong(T, dim, gi, gj, gk)
    xc = [(gi + 0.5) / 2, (gj + 0.5) / 2, (gk + 0.5) / 2]  # child centres in coarse units
    want = np.array([10.0 + c[0] * xc[0] + c[1] * xc[1] + (c[2] * xc[2] if dim == 3 else 0.0) for c in coef])
    assert np.max(np.abs(got - want)) <= 1e-13


def test_prolong_flat_at_extremum():
    n = (6, 6, 1)
    T = np.ones((5, 1, 14, 14))
    T[:, 0, 4 + 3, 4 + 3] = 2.0   # a peak at coarse zone (3, 3)
    v = amr.prolong(T, 2, np.array([6, 7, 6, 7]), np.array([6, 6, 7, 7]), np.zeros(4, dtype=int))
    assert np.array_equal(v, np.full((5, 4), 2.0))


def _hier3():
    # two fine boxes side by side in x, of different heights in y: the union
    # has a concave corner (a coarse zone with two interface faces)
    return (24, 24, 24), [(12, 12, 12), (24, 12, 12)], [(12, 12, 12), (12, 8, 12)]


def _hier2():
    return (32, 32), [(20, 20, 0), (36, 20, 0), (20, 32, 0)], [(16, 12, 1), (8, 20, 1), (12, 8, 1)]


def _composite_total(Uc, fines, domain, dim, dx):
    dvc = np.prod(dx[:dim])
    dvf = dvc / 2 ** dim
    I = _interior(Uc, dim)
    M = amr.covered_mask(domain, fines, dim).reshape(I[0].shape)
    tot = np.array([np.sum(I[c][~M]) for c in range(5)]) * dvc
    tot = tot + sum(_interior(B.U, dim).reshape(5, -1).sum(axis=1) for B in fines) * dvf
    scale = np.abs(I).reshape(5, -1).sum(axis=1) * dvc
    return tot, np.where(scale > 0, scale, 1.0)  # w = 0 in 2-D: compare its total absolutely


@pytest.mark.parametrize("dim", [3, 2])
def test_two_level_advance_conserves(dim):
    domain, flo, fn = _hier3() if dim == 3 else _hier2()
    Uc, Uf, dx = inputs.amr_two_level(domain, dim, flo, fn)
    bc = ((PER, PER),) * 3
    errs = {}
    for reflux in (True, False):
        C, F = Uc, _boxes(flo, fn, Uf)
        t0, scale = _composite_total(C, F, domain, dim, dx)
        d = 0.3 * dx[0] / 4.0
        for _ in range(2):
            C, F, d_next, bad = amr.advance(C, F, d, dim, domain, bc, dx, reflux=reflux)
            assert not bad
            d = d_next
        t1, _ = _composite_total(C, F, domain, dim, dx)
        errs[reflux] = np.max(np.abs(t1 - t0) / scale)
        if reflux:
            # after the average down the coarse level alone carries the same totals
            tc = _interior(C, dim).reshape(5, -1).sum(axis=1) * np.prod(dx[:dim])
            assert np.max(np.abs(tc - t1) / scale) <= 1e-13
    assert errs[True] <= 1e-13, errs
    assert errs[False] > 1e-9, errs


def _linear_state(n, dim, dx, lo, t, gamma, b=(0.8, -0.6, 0.4), vel=(0.7, 0.4, -0.3)):
    """rho = 2 + b.(x - vel t) with uniform velocity and pressure: the exact
    solution of the Euler equations (a contact wave), sampled at zone centres
    (equal to the zone averages of a linear function)."""
    X = inputs.zone_centres(n, dim, dx, lo)
    rho = 2.0 + sum(b[a] * (X[a] - vel[a] * t) for a in range(dim))
    w = vel[2] if dim == 3 else 0.0
    return inputs.conserved(rho, vel[0] + 0.0 * rho, vel[1] + 0.0 * rho, w + 0.0 * rho, 1.0 + 0.0 * rho, gamma)


def _linear_hierarchy(dim, t):
    domain, flo, fn = _hier3() if dim == 3 else _hier2()
    n = tuple(domain) + (1,) * (3 - len(domain))
    dx = (1.0 / n[0],) * 3
    Uc = _linear_state(n, dim, dx, (0.0, 0.0, 0.0), t, 1.4)
    fines = []
    for lo, s in zip(flo, fn):
        s = tuple(s) + (1,) * (3 - len(s))
        org = tuple(lo[a] * dx[a] / 2 if a < dim else 0.0 for a in range(3))
        fines.append(amr.FineBox(lo, s, _linear_state(s, dim, tuple(v / 2 for v in dx), org, t, 1.4)))
    return domain, fines, Uc, dx


@pytest.mark.parametrize("dim", [3, 2])
def test_linear_advection_is_exact(dim, monkeypatch):
    domain, F0, U0, dx = _linear_hierarchy(dim, 0.0)
    dt = 0.4 * dx[0] / (1.0 + np.sqrt(1.4 * 1.0 / 1.5))
    _, F1, U1, _ = _linear_hierarchy(dim, dt)
    # the single-level step alone is exact on this profile (the premise)
    P = oracle.params(dim, domain, dx=dx, bc=PRE, gamma=1.4)
    S, rc = oracle.step(U0, P, dt)
    assert rc == 0
    assert np.max(np.abs(_interior(S, dim) - _interior(U1, dim))) <= 1e-13

    def err(C, F):
        e = np.max(np.abs(_interior(C, dim) - _interior(U1, dim)))
        for A, B in zip(F, F1):
            e = max(e, np.max(np.abs(_interior(A.U, dim) - _interior(B.U, dim))))
        return e

    C, F, _, bad = amr.advance(U0, F0, dt, dim, domain, PRE, dx, gamma=1.4)
    assert not bad
    assert err(C, F) <= 1e-13
    # planted mistake: the second fine step's ghosts taken at the old time
    monkeypatch.setattr(amr, "coarse_at_time", lambda old, new, half: old)
    C, F, _, _ = amr.advance(U0, F0, dt, dim, domain, PRE, dx, gamma=1.4)
    assert err(C, F) > 1e-6


def test_cutting_a_fine_box_changes_nothing():
    dim = 3
    domain = (20, 20, 20)
    whole = ([(12, 12, 12)], [(16, 12, 12)])
    cut = ([(12, 12, 12), (20, 12, 12)], [(8, 12, 12), (8, 12, 12)])
    Uc, Uw, dx = inputs.amr_two_level(domain, dim, *whole)
    # the two halves hold the same interior values; their ghosts start as NaN
    # (the fill must overwrite every one)
    Ucut = [np.full((5, 20, 20, 16), np.nan) for _ in range(2)]
    for h in range(2):
        Ucut[h][:, 4:-4, 4:-4, 4:-4] = Uw[0][:, 4:-4, 4:-4, 4 + 8 * h:12 + 8 * h]
    bc = ((PER, PER),) * 3
    d = 0.3 * dx[0] / 4.0
    Cw, Fw, dw, _ = amr.advance(Uc, _boxes(*whole, Uw), d, dim, domain, bc, dx)
    Cc, Fc, dc, _ = amr.advance(Uc, _boxes(*cut, Ucut), d, dim, domain, bc, dx)
    assert np.array_equal(_interior(Cw, dim), _interior(Cc, dim))
    W = _interior(Fw[0].U, dim)
    assert np.array_equal(W[:, :, :, :8], _interior(Fc[0].U, dim))
    assert np.array_equal(W[:, :, :, 8:], _interior(Fc[1].U, dim))
    assert dw == dc


def test_no_fine_boxes_is_the_single_level_step():
    domain = (16, 12, 10)
    rng = np.random.default_rng(3)
    U = inputs.random_box(rng, domain, 3)
    dx = (0.1, 0.1, 0.1)
    C, F, dn, bad = amr.advance(U, [], 1e-3, 3, domain, ((PER, PER),) * 3, dx, gamma=5 / 3)
    P = oracle.params(3, domain, dx=dx, bc=PER, gamma=5 / 3)
    S, rc = oracle.step(U, P, 1e-3)
    assert np.array_equal(_interior(C, 3), _interior(S, 3)) and F == []
    assert dn == oracle.dt(S, P)[0]


def test_nesting_rules_enforced():
    z = np.zeros((5, 28, 28, 28))
    with pytest.raises(ValueError):   # odd corner
        amr.check_nesting((20, 20, 20), [amr.FineBox((13, 12, 12), (8, 8, 8), z)], 3)
    with pytest.raises(ValueError):   # within 3 coarse zones of the domain boundary
        amr.check_nesting((20, 20, 20), [amr.FineBox((4, 12, 12), (8, 8, 8), z)], 3)
    with pytest.raises(ValueError):   # overlap
        amr.check_nesting((20, 20, 20), [amr.FineBox((12, 12, 12), (8, 8, 8), z),
                                         amr.FineBox((16, 12, 12), (8, 8, 8), z)], 3)
    amr.check_nesting((20, 20, 20), [amr.FineBox((6, 6, 6), (28, 28, 28), z)], 3)
