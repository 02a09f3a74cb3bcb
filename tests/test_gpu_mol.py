"""Method-of-lines step with passive species on the GPU (hydro_mol_advance_box)
against the oracle's oracle_mol_step, through the C ABI:

  * one step on ragged 2-D/3-D boxes with periodic, reflecting, outflow and
    prefilled faces, gravity, Einfeldt speeds, flattening off, 0..13 species:
    bitwise for the contraction-free build (all 5 + nspec fields and the next
    dt), within 1e-10 for the product build;
  * 20 steps of the product build within 1e-8;
  * the bench workload (Sedov 128^3 with 13 species): a full-box comparison
    after GPU steps, and conservation of every species on a periodic 128^3 box;
  * argument checks.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import rel_linf
from paper_1711_06203_b300 import binding as hb
from paper_1711_06203_b300 import inputs

pytestmark = pytest.mark.gpu

O, R, PER, PRE = hb.BC_OUTFLOW, hb.BC_REFLECT, hb.BC_PERIODIC, hb.BC_PREFILLED


def _interior(U, dim):
    return U[:, 4:-4, 4:-4, 4:-4] if dim == 3 else U[:, 0, 4:-4, 4:-4]


def _rel(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    den = np.abs(b).max(axis=1)
    num = np.abs(a - b).max(axis=1)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


SEEDS = {"random3d_periodic": 31, "sod2d_species": 32, "mixed3d_gravity_13": 33, "sedov24_13": 34,
         "einfeldt_noflat_2d": 35, "hydro_only": 36, "wide_x_3d": 37}


def _case(name):
    rng = np.random.default_rng(SEEDS[name])
    if name == "random3d_periodic":
        n, dim, bc, kw = (13, 10, 11), 3, PER, {}
        U = inputs.random_box(rng, n, 3)
        nspec = 3
    elif name == "sod2d_species":
        n, dim, bc, kw = (40, 6, 1), 2, O, dict(gamma=1.4)
        U = inputs.sod(40, 2, 0, 1.4)[:, :, :14, :]
        nspec = 2
    elif name == "mixed3d_gravity_13":
        n, dim = (12, 9, 14), 3
        bc = ((PER, PER), (R, O), (PRE, R))
        kw = dict(grav=(0.0, 0.3, -1.0))
        U = inputs.random_box(rng, n, 3)
        nspec = 13
    elif name == "sedov24_13":
        n, dim, bc, kw = (24, 24, 24), 3, O, dict(gamma=1.4)
        U, _ = inputs.sedov(24)
        nspec = 13
    elif name == "einfeldt_noflat_2d":
        n, dim, bc, kw = (17, 15, 1), 2, ((O, R), (PER, PER), (O, O)), dict(einfeldt=True, flatten=False)
        U = inputs.random_box(rng, n, 2)
        nspec = 1
    elif name == "hydro_only":
        n, dim, bc, kw = (10, 12, 9), 3, R, {}
        U = inputs.random_box(rng, n, 3)
        nspec = 0
    elif name == "wide_x_3d":
        # 63 x-zones (-1..61) span three 28-zone warps of the x reconstruction, the last one ragged
        n, dim = (61, 7, 6), 3
        bc = ((PER, PER), (R, O), (O, R))
        kw = {}
        U = inputs.random_box(rng, n, 3)
        nspec = 2
    X = inputs.species_fractions(rng, U.shape[1:], max(nspec, 1))[:nspec]
    return inputs.with_species(U, X), n, dim, bc, kw, nspec


CASES = ["random3d_periodic", "sod2d_species", "mixed3d_gravity_13", "sedov24_13", "einfeldt_noflat_2d",
         "hydro_only", "wide_x_3d"]


def _gpu(U, n, dim, bc, kw, nspec, dts, variant, dx=0.05):
    ctx = hb.Context(0, variant)
    gamma = kw.get("gamma", 5 / 3)
    p = hb.params(dim, gamma=gamma, cfl=0.4, grav=kw.get("grav", (0.0, 0.0, 0.0)),
                  flatten=kw.get("flatten", True), einfeldt=kw.get("einfeldt", False))
    a = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    # one step: an all-NaN output shows that only its interior is written;
    # several steps: both buffers keep the caller's prefilled ghost layers
    b = torch.full_like(a, float("nan")) if len(dts) == 1 else a.clone()
    nexts = []
    for d in dts:
        nexts.append(ctx.hydro_mol_advance_box(hb.box(a, n, (dx,) * 3, bc), hb.box(b, n, (dx,) * 3, bc), p, nspec, d,
                                               want_dt_next=True))
        a, b = b, a
    out = a.cpu().numpy()
    ctx.close()
    return out, nexts


def _oracle_params(n, dim, bc, kw, dx=0.05):
    return oracle.params(dim, n[:dim], dx=(dx,) * 3, bc=bc, gamma=kw.get("gamma", 5 / 3), cfl=0.4,
                         grav=kw.get("grav", (0.0, 0.0, 0.0)), flatten=kw.get("flatten", True),
                         einfeldt=kw.get("einfeldt", False))


@pytest.mark.parametrize("variant", ["exact", "default"])
@pytest.mark.parametrize("name", CASES)
def test_one_step_matches_oracle(name, variant):
    U, n, dim, bc, kw, nspec = _case(name)
    P = _oracle_params(n, dim, bc, kw)
    dt, rc = oracle.dt(U, P)
    assert rc == 0
    ref, rc = oracle.mol_step(U, P, dt)
    assert rc == 0
    dref, _ = oracle.dt(ref, P)
    got, nexts = _gpu(U, n, dim, bc, kw, nspec, [dt], variant)
    g, w = _interior(got, dim), _interior(ref, dim)
    if variant == "exact":
        assert np.array_equal(g, w)
        assert nexts[0] == dref
    else:
        assert np.all(_rel(g, w) <= 1e-10)
        assert abs(nexts[0] - dref) <= 1e-13 * dref


def test_twenty_steps_within_tolerance():
    U, n, dim, bc, kw, nspec = _case("mixed3d_gravity_13")
    P = _oracle_params(n, dim, bc, kw)
    ref, dts = U, []
    for _ in range(20):
        d, rc = oracle.dt(ref, P)
        dts.append(d)
        ref, rc = oracle.mol_step(ref, P, d)
        assert rc == 0
    got, _ = _gpu(U, n, dim, bc, kw, nspec, dts, "default")
    assert np.all(_rel(_interior(got, dim), _interior(ref, dim)) <= 1e-8)


def _sedov_species(n, nspec=13, seed=1711):
    U, _ = inputs.sedov(n)
    X = inputs.species_fractions(np.random.default_rng(seed), U.shape[1:], nspec)
    return inputs.with_species(U, X)


def test_sedov_128_13_species_full_box():
    n, nspec = 128, 13
    U = _sedov_species(n, nspec)
    ctx = hb.Context(0)
    p = hb.params(3, gamma=1.4, cfl=0.4)
    a = torch.from_numpy(U).cuda()
    b = torch.empty_like(a)
    box = lambda t: hb.box(t, (n, n, n), (1.0 / n,) * 3, O)
    dt = ctx.hydro_dt(box(a), p)
    for _ in range(6):
        dt = ctx.hydro_mol_advance_box(box(a), box(b), p, nspec, dt, want_dt_next=True)
        a, b = b, a
    state = a.cpu().numpy()
    dn = ctx.hydro_mol_advance_box(box(a), box(b), p, nspec, dt, want_dt_next=True)
    got = b.cpu().numpy()
    ctx.close()
    del a, b
    torch.cuda.empty_cache()
    P = oracle.params(3, (n, n, n), gamma=1.4, cfl=0.4)
    ref, rc = oracle.mol_step(state, P, dt)
    assert rc == 0
    assert np.all(_rel(_interior(got, 3), _interior(ref, 3)) <= 1e-10)
    dref, _ = oracle.dt(ref, P)
    assert abs(dn - dref) <= 1e-10 * dref


def test_species_conserved_at_bench_size():
    n, nspec = 128, 13
    rng = np.random.default_rng(5)
    U = inputs.random_box(rng, (n, n, n), 3)
    U = inputs.with_species(U, inputs.species_fractions(rng, U.shape[1:], nspec))
    ctx = hb.Context(0)
    p = hb.params(3, gamma=5 / 3, cfl=0.4)
    a = torch.from_numpy(U).cuda()
    b = torch.empty_like(a)
    box = lambda t: hb.box(t, (n, n, n), (1.0 / n,) * 3, PER)
    t0 = a[:, 4:-4, 4:-4, 4:-4].sum(dim=(1, 2, 3))
    scale = a[:, 4:-4, 4:-4, 4:-4].abs().sum(dim=(1, 2, 3))
    dt = ctx.hydro_dt(box(a), p)
    for _ in range(3):
        dt = ctx.hydro_mol_advance_box(box(a), box(b), p, nspec, dt, want_dt_next=True)
        a, b = b, a
    t1 = a[:, 4:-4, 4:-4, 4:-4].sum(dim=(1, 2, 3))
    err = ((t1 - t0).abs() / scale).cpu().numpy()
    ctx.close()
    del a, b
    torch.cuda.empty_cache()
    assert np.all(err <= 1e-13), err


def test_argument_checks():
    U, n, dim, bc, kw, nspec = _case("random3d_periodic")
    ctx = hb.Context(0)
    p = hb.params(3)
    a = torch.from_numpy(U).cuda()
    b = torch.empty_like(a)
    ba, bb = hb.box(a, n, (0.1,) * 3, bc), hb.box(b, n, (0.1,) * 3, bc)
    for ns in (-1, hb.MOL_MAX_SPECIES + 1):
        rc, _ = ctx.hydro_mol_advance_box(ba, bb, p, ns, 1e-3, raise_on_error=False)
        assert rc == hb.HYDRO_EINVAL
    # output overlapping the input's species fields
    alias = hb.box(a[1:], n, (0.1,) * 3, bc)
    rc, _ = ctx.hydro_mol_advance_box(ba, alias, p, nspec, 1e-3, raise_on_error=False)
    assert rc == hb.HYDRO_EINVAL
    rc, _ = ctx.hydro_mol_advance_box(ba, bb, hb.params(3, grav=(0, 0, -1), flux_grav_energy=True), nspec, 1e-3,
                                      raise_on_error=False)
    assert rc == hb.HYDRO_ENOTIMPL
    assert ctx.hydro_mol_advance_box(ba, bb, p, nspec, 1e-3) is None
    ctx.close()
