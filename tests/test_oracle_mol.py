"""Pins of the method-of-lines oracle step (oracle_mol_step: SSP-RK2 in time,
flattened PPM edge values, HLLC, passive species carried by the upwind mass
flux) against what the mathematics fixes:

  * conservation of mass, momentum, energy and every species on a periodic
    domain (rounding level);
  * a uniform mass fraction stays uniform (the species flux is the mass flux
    times the upwind fraction), and species never change the hydrodynamics;
  * a linear density and fraction profile advected at uniform velocity and
    pressure is advanced exactly (zones whose stencil does not reach the
    caller-held ghosts);
  * second-order convergence on a smooth periodic wave, first order on Sod
    against the exact Riemann solution;
  * free fall of a uniform state: the momentum changes by exactly rho g dt
    and the internal energy does not change (the two-stage scheme is exact
    for a linear-in-time velocity);
  * a 1-D problem gives the same numbers in 2-D, in 3-D and along every axis.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1711_06203_b300 import inputs

PER, PRE, OUT = oracle.BC_PERIODIC, oracle.BC_PREFILLED, oracle.BC_OUTFLOW


def _int3(U):
    return U[:, 4:-4, 4:-4, 4:-4]


def test_conservation_periodic_with_species():
    rng = np.random.default_rng(21)
    n = (16, 12, 10)
    U = inputs.with_species(inputs.random_box(rng, n, 3), inputs.species_fractions(rng, inputs.grown_shape(n, 3), 4))
    P = oracle.params(3, n, dx=(0.1, 0.1, 0.1), bc=PER, gamma=5 / 3)
    V = U
    for _ in range(3):
        V, rc = oracle.mol_step(V, P, 2e-3)
        assert rc == 0
    t0 = _int3(U).reshape(9, -1).sum(axis=1)
    t1 = _int3(V).reshape(9, -1).sum(axis=1)
    scale = np.abs(_int3(U)).reshape(9, -1).sum(axis=1)
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale)


def test_uniform_fraction_stays_uniform_and_species_are_passive():
    rng = np.random.default_rng(22)
    n = (14, 10, 12)
    U = inputs.random_box(rng, n, 3)
    X = np.stack([np.full(U.shape[1:], 0.25), np.full(U.shape[1:], 0.75)])
    W = inputs.with_species(U, X)
    P = oracle.params(3, n, dx=(0.1, 0.1, 0.1), bc=((PER, PER), (OUT, OUT), (oracle.BC_REFLECT,) * 2), gamma=5 / 3)
    V, rc = oracle.mol_step(W, P, 2e-3)
    assert rc == 0
    rho = _int3(V)[0]
    assert np.all(np.abs(_int3(V)[5] - 0.25 * rho) <= 1e-14 * rho)
    assert np.all(np.abs(_int3(V)[6] - 0.75 * rho) <= 1e-14 * rho)
    # the hydrodynamic fields do not see the species (bitwise)
    H, rc = oracle.mol_step(U, P, 2e-3)
    assert np.array_equal(_int3(H), _int3(V)[:5])


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("which", ["density", "fraction"])
def test_linear_profile_is_advected_exactly(dim, which):
    """density: rho linear, one uniform species; fraction: rho uniform, the
    mass fraction linear (so rho X stays linear too)."""
    n = (20, 18, 16 if dim == 3 else 1)
    dx = (1.0 / 20,) * 3
    vel = (0.7, -0.4, 0.3)
    b = (0.8, -0.6, 0.4)

    def state(t):
        X = inputs.zone_centres(n, dim, dx)
        s = sum(b[a] * (X[a] - vel[a] * t) for a in range(dim))
        one = 0.0 * s + 1.0
        rho = 2.0 + s if which == "density" else 2.0 * one
        frac = 0.5 * one if which == "density" else 0.5 + 0.25 * s
        U = inputs.conserved(rho, vel[0] * one, vel[1] * one, (vel[2] if dim == 3 else 0.0) * one, one, 1.4)
        return inputs.with_species(U, frac[None])

    dt = 0.3 * dx[0] / (1.0 + math.sqrt(1.4 / 1.4))
    U0, U1 = state(0.0), state(dt)
    P = oracle.params(dim, n[:dim], dx=dx, bc=PRE, gamma=1.4)
    V, rc = oracle.mol_step(U0, P, dt)
    assert rc == 0
    # prefilled ghosts hold t^n data for both stages: zones within 4 of a face
    # see them in the second stage, the rest must be exact
    core = (slice(None),) + ((slice(8, -8),) * 3 if dim == 3 else (0, slice(8, -8), slice(8, -8)))
    assert np.max(np.abs(V[core] - U1[core])) <= 1e-13


def _wave_error(n, tend=0.2, cfl=0.4):
    """L1 density error of a periodic sine wave advected at u = 1 (2-D run, 4 rows)."""
    f = lambda x: 1.0 + 0.2 * np.sin(2 * np.pi * x)
    gx, gw = np.polynomial.legendre.leggauss(5)

    def avg(t):
        xc = (np.arange(n + 8) - 4 + 0.5) / n
        return sum(0.5 * w_ * f(xc + 0.5 / n * x_ - t) for x_, w_ in zip(gx, gw))

    R = np.repeat(avg(0.0)[None, :], 12, axis=0)[None]
    U = inputs.conserved(R, 1.0 + 0 * R, 0 * R, 0 * R, 1.0 + 0 * R, 1.4)
    P = oracle.params(2, (n, 4), dx=(1.0 / n,) * 3, bc=PER, gamma=1.4)
    nst = math.ceil(tend / (cfl / n / (1.0 + math.sqrt(1.4 / 0.8))))
    for _ in range(nst):
        U, rc = oracle.mol_step(U, P, tend / nst)
        assert rc == 0
    return np.abs(U[0, 0, 4, 4:-4] - avg(tend)[4:-4]).mean()


def test_second_order_on_a_smooth_wave():
    e = [_wave_error(n) for n in (32, 64, 128)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert min(orders) >= 1.85, (e, orders)


def test_sod_first_order_against_exact():
    errs = []
    for n in (64, 128):
        U = inputs.sod(n, 2, 0, 1.4)
        P = oracle.params(2, (n, n), bc=OUT, gamma=1.4, cfl=0.4)
        t = 0.0
        while t < 0.2 - 1e-14:
            d, _ = oracle.dt(U, P)
            d = min(d, 0.2 - t)
            U, rc = oracle.mol_step(U, P, d)
            assert rc == 0
            t += d
        assert np.array_equal(U[:, 0, 4:-4, 4:-4], np.repeat(U[:, 0, 4:5, 4:-4], n, axis=1))  # rows identical
        x = (np.arange(n) + 0.5) / n
        W = oracle.exact_sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4, (x - 0.5) / 0.2)
        errs.append(np.abs(U[0, 0, 4, 4:-4] - W[:, 0]).mean())
    assert errs[1] <= 5e-3
    assert math.log2(errs[0] / errs[1]) >= 0.8


def test_free_fall_of_a_uniform_state():
    n = (8, 8, 8)
    rho, w0, p = 1.3, 0.2, 0.9
    shape = inputs.grown_shape(n, 3)
    one = np.ones(shape)
    U = inputs.conserved(rho * one, 0 * one, 0 * one, w0 * one, p * one, 1.4)
    P = oracle.params(3, n, dx=(0.1,) * 3, bc=PER, gamma=1.4, grav=(0.0, 0.0, -1.0))
    dt = 0.01
    V, rc = oracle.mol_step(U, P, dt)
    assert rc == 0
    I = _int3(V)
    assert np.all(np.abs(I[3] / I[0] - (w0 - dt)) <= 1e-14)
    pres = 0.4 * (I[4] - 0.5 * I[3] ** 2 / I[0])
    assert np.all(np.abs(pres - p) <= 1e-14)


def test_one_dimensional_problem_in_every_orientation():
    """x-problem in 2-D == in 3-D; the same problem along y and z is its transpose."""
    rng = np.random.default_rng(23)
    nx = 24
    rho = rng.lognormal(0.0, 0.5, nx + 8)
    un = rng.normal(0.0, 0.3, nx + 8)
    p = rng.lognormal(0.0, 0.3, nx + 8)
    X = rng.uniform(0.0, 1.0, nx + 8)
    dt = 1e-3
    res = {}
    for ax in range(3):
        shape = [8 + 8, 8 + 8, 8 + 8]  # 8 zones across
        shape[2 - ax] = nx + 8
        bshape = [1, 1, 1]
        bshape[2 - ax] = nx + 8
        R = np.broadcast_to(rho.reshape(bshape), shape)
        vel = [np.broadcast_to(un.reshape(bshape), shape) if a == ax else np.zeros(shape) for a in range(3)]
        U = inputs.with_species(inputs.conserved(R, vel[0], vel[1], vel[2], np.broadcast_to(p.reshape(bshape), shape), 1.4),
                                np.broadcast_to(X.reshape(bshape), shape)[None])
        n = [8, 8, 8]
        n[ax] = nx
        P = oracle.params(3, n, dx=(0.05,) * 3, bc=OUT, gamma=1.4)
        V, rc = oracle.mol_step(U, P, dt)
        assert rc == 0
        idx = [8, 8, 8]
        idx[2 - ax] = slice(4, -4)
        res[ax] = np.array([V[c][tuple(idx)] for c in (0, 1 + ax, 4, 5)])
    assert np.array_equal(res[0], res[1]) and np.array_equal(res[0], res[2])
    # the x-problem in 2-D
    R = np.broadcast_to(rho[None, None, :], (1, 16, nx + 8))
    U2 = inputs.with_species(inputs.conserved(R, np.broadcast_to(un[None, None, :], R.shape), 0 * R, 0 * R,
                                              np.broadcast_to(p[None, None, :], R.shape), 1.4),
                             np.broadcast_to(X[None, None, :], R.shape)[None])
    P2 = oracle.params(2, (nx, 8), dx=(0.05,) * 3, bc=OUT, gamma=1.4)
    V2, rc = oracle.mol_step(U2, P2, dt)
    assert np.array_equal(np.array([V2[c][0, 8, 4:-4] for c in (0, 1, 4, 5)]), res[0])


def test_passive_step_keeps_its_bounds():
    """A species step carried by a uniform flow stays within its initial
    range [0, 1] (upwind transport with limited edges); a downwind species
    flux would not."""
    n = 64
    x = (np.arange(n + 8) - 4 + 0.5) / n
    X = np.where((x > 0.25) & (x < 0.5), 1.0, 0.0)
    R = np.ones((1, 12, n + 8))
    U = inputs.with_species(inputs.conserved(R, 1.0 + 0 * R, 0 * R, 0 * R, 1.0 + 0 * R, 1.4),
                            np.broadcast_to(X, R.shape)[None])
    P = oracle.params(2, (n, 4), bc=PER, gamma=1.4)
    dt = 0.4 / n / (1.0 + math.sqrt(1.4))
    for _ in range(40):
        U, rc = oracle.mol_step(U, P, dt)
        assert rc == 0
    f = U[5, 0, 4:-4, 4:-4] / U[0, 0, 4:-4, 4:-4]
    assert f.min() >= 0.0 and f.max() <= 1.0
    assert f.max() > 0.99  # still a step, not smeared away


def test_flattening_acts_only_near_the_shock():
    """Flattening changes the result, and only within a few zones of the
    shock and contact of a strong two-state problem (its detector needs
    compression and a large pressure jump)."""
    n = 128
    res = {}
    for fl in (True, False):
        U = inputs.two_state(n, 2, 1.4, 1.0, 100.0, 1.0, 0.1)
        P = oracle.params(2, (n, 4), bc=((OUT, OUT), (PER, PER), (OUT, OUT)), gamma=1.4, cfl=0.4, flatten=fl)
        U = U[:, :, :12, :]
        d, _ = oracle.dt(U, P)
        for _ in range(12):
            U, rc = oracle.mol_step(U, P, d)
            assert rc == 0
        res[fl] = U[0, 0, 4, 4:-4]
    diff = np.nonzero(res[True] != res[False])[0]
    assert diff.size > 0
    assert diff.min() >= n // 2 - 20 and diff.max() <= n // 2 + 20
