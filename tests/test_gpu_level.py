"""A level of uneven boxes tiling a domain: device ghost fill (hydro_fill_boundary)
plus the batched step advance the level exactly like one box covering the
whole domain with the same boundary kinds.

  * after the fill, every box's ghost zones equal the corresponding zones of
    the single box with its ghosts filled by the oracle (bitwise);
  * K steps of fill + batched step + level dt reduction (all on the device)
    equal K steps of the single box: bitwise for the contraction-free build,
    to the parity tolerance for the product build (whose batched and
    single-box kernels may fuse multiply-adds differently);
  * two level steps equal two steps of the CPU oracle on the single box over
    the domain: bitwise (contraction-free build), within 1e-10 (product).
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import rel_linf
from paper_1711_06203_b300 import binding as hb
from paper_1711_06203_b300 import inputs

pytestmark = pytest.mark.gpu

O, R, PER = hb.BC_OUTFLOW, hb.BC_REFLECT, hb.BC_PERIODIC


def _split(U, lo, sizes, dim):
    """Copy each box's interior out of the big grown array (ghosts left NaN)."""
    out = []
    for c, s in zip(lo, sizes):
        gz = s[2] + 8 if dim == 3 else 1
        B = np.full((5, gz, s[1] + 8, s[0] + 8), np.nan)
        if dim == 3:
            B[:, 4:-4, 4:-4, 4:-4] = U[:, 4 + c[2]:4 + c[2] + s[2], 4 + c[1]:4 + c[1] + s[1], 4 + c[0]:4 + c[0] + s[0]]
        else:
            B[:, 0, 4:-4, 4:-4] = U[:, 0, 4 + c[1]:4 + c[1] + s[1], 4 + c[0]:4 + c[0] + s[0]]
        out.append(B)
    return out


def _region(U, c, s, dim, ghosts=0):
    g = ghosts
    if dim == 3:
        return U[:, 4 + c[2] - g:4 + c[2] + s[2] + g, 4 + c[1] - g:4 + c[1] + s[1] + g, 4 + c[0] - g:4 + c[0] + s[0] + g]
    return U[:, 0, 4 + c[1] - g:4 + c[1] + s[1] + g, 4 + c[0] - g:4 + c[0] + s[0] + g]


def _setup(dim):
    domain = (96, 64, 48) if dim == 3 else (96, 80, 1)
    lo, sizes = inputs.level_tiling(domain[:dim], seed=7)
    if dim == 2:
        lo = [(x, y, 0) for x, y, _ in lo]
    rng = np.random.default_rng(11 + dim)
    U = inputs.random_box(rng, domain, dim)
    bc = ((PER, PER), (R, R), (O, O))
    dx = (1.0 / 96,) * 3
    return domain, lo, sizes, U, bc, dx


@pytest.mark.parametrize("dim", [3, 2])
def test_fill_boundary_matches_single_box_ghosts(dim):
    domain, lo, sizes, U, bc, dx = _setup(dim)
    P = oracle.params(dim, domain[:dim], dx=dx, bc=bc, gamma=5 / 3)
    W = oracle.fill_ghosts(U, P)
    ctx = hb.Context(0)
    boxes = [torch.from_numpy(B).cuda() for B in _split(U, lo, sizes, dim)]
    descs = [hb.box(t, s, dx, hb.BC_PREFILLED) for t, s in zip(boxes, sizes)]
    ctx.hydro_fill_boundary(descs, lo, dim, domain[:dim], bc[:dim])
    ctx.close()
    for t, c, s in zip(boxes, lo, sizes):
        got = t.cpu().numpy()
        got = got[:, 0] if dim == 2 else got
        want = _region(W, c, s, dim, ghosts=4)
        if dim == 3:
            assert np.array_equal(got, want)
        else:
            assert np.array_equal(got, want)


@pytest.mark.parametrize("variant,dim", [("exact", 3), ("default", 3), ("exact", 2)])
def test_level_advance_equals_single_box(variant, dim):
    domain, lo, sizes, U, bc, dx = _setup(dim)
    steps = 5
    p = hb.params(dim, gamma=5 / 3, cfl=0.5)
    ctx = hb.Context(0, variant)
    # the single box over the whole domain
    big = torch.from_numpy(U).cuda()
    big2 = torch.empty_like(big)
    bbox = lambda t: hb.box(t, domain, dx, bc)
    dt = ctx.hydro_dt(bbox(big), p)
    dts = []
    for _ in range(steps):
        dts.append(dt)
        dt = ctx.hydro_advance_box(bbox(big), bbox(big2), p, dt, want_dt_next=True)
        big, big2 = big2, big
    ref = big.cpu().numpy()
    # the tiled level: fill, batched step, level dt, all on the device
    a = [torch.from_numpy(B).cuda() for B in _split(U, lo, sizes, dim)]
    b = [torch.full_like(x, float("nan")) for x in a]
    da = [hb.box(t, s, dx, hb.BC_PREFILLED) for t, s in zip(a, sizes)]
    db = [hb.box(t, s, dx, hb.BC_PREFILLED) for t, s in zip(b, sizes)]
    nbox = len(sizes)
    dt_dev = torch.full((nbox,), dts[0], dtype=torch.float64, device="cuda")
    dt_next = torch.empty_like(dt_dev)
    level_dts = []
    for _ in range(steps):
        ctx.hydro_fill_boundary(da, lo, dim, domain[:dim], bc[:dim])
        level_dts.append(dt_dev[0].item())
        ctx.hydro_advance_batch(da, db, p, dt_dev, dt_next)
        ctx.hydro_level_min_dt(dt_next, dt_dev)
        da, db = db, da
        a, b = b, a
    torch.cuda.synchronize()
    ctx.close()
    if variant == "exact":
        assert level_dts == dts
    else:
        assert np.allclose(level_dts, dts, rtol=1e-13, atol=0)
    for t, c, s in zip(a, lo, sizes):
        got = t.cpu().numpy()
        got = got[:, 4:-4, 4:-4, 4:-4] if dim == 3 else got[:, 0, 4:-4, 4:-4]
        want = _region(ref, c, s, dim)
        if variant == "exact":
            assert np.array_equal(got, want)
        else:
            assert np.all(rel_linf(got, want) <= 1e-10)


def test_fill_boundary_rejects_bad_tilings():
    ctx = hb.Context(0)
    U = inputs.random_box(np.random.default_rng(0), (16, 16, 16), 3)
    t = torch.from_numpy(U).cuda()
    d = hb.box(t, (16, 16, 16), (0.1,) * 3, hb.BC_PREFILLED)
    with pytest.raises(hb.HydroError):  # does not cover a 32^3 domain
        ctx.hydro_fill_boundary([d], [(0, 0, 0)], 3, (32, 32, 32), ((O, O),) * 3)
    with pytest.raises(hb.HydroError):  # overlapping boxes
        ctx.hydro_fill_boundary([d, d], [(0, 0, 0), (0, 0, 0)], 3, (16, 16, 16), ((O, O),) * 3)
    with pytest.raises(hb.HydroError):  # periodic on one face only
        ctx.hydro_fill_boundary([d], [(0, 0, 0)], 3, (16, 16, 16), ((PER, O), (O, O), (O, O)))
    ctx.close()


@pytest.mark.parametrize("variant,dim", [("exact", 3), ("default", 3), ("default", 2)])
def test_level_two_steps_against_oracle(variant, dim):
    """Two level steps (device ghost fill, batched step, level dt reduction)
    against the CPU oracle's single box over the whole domain, each side
    taking its own CFL steps: bitwise for the contraction-free build, within
    1e-10 for the product build."""
    domain, lo, sizes, U, bc, dx = _setup(dim)
    P = oracle.params(dim, domain[:dim], dx=dx, bc=bc, gamma=5 / 3, cfl=0.5)
    ref, _, odts = oracle.run(U, P, 2)
    p = hb.params(dim, gamma=5 / 3, cfl=0.5)
    ctx = hb.Context(0, variant)
    a = [torch.from_numpy(B).cuda() for B in _split(U, lo, sizes, dim)]
    b = [torch.full_like(x, float("nan")) for x in a]
    da = [hb.box(t, s, dx, hb.BC_PREFILLED) for t, s in zip(a, sizes)]
    db = [hb.box(t, s, dx, hb.BC_PREFILLED) for t, s in zip(b, sizes)]
    big = torch.from_numpy(U).cuda()
    dt_dev = torch.full((len(sizes),), ctx.hydro_dt(hb.box(big, domain, dx, bc), p), dtype=torch.float64,
                        device="cuda")
    dt_next = torch.empty_like(dt_dev)
    level_dts = []
    for _ in range(2):
        ctx.hydro_fill_boundary(da, lo, dim, domain[:dim], bc[:dim])
        level_dts.append(dt_dev[0].item())
        ctx.hydro_advance_batch(da, db, p, dt_dev, dt_next)
        ctx.hydro_level_min_dt(dt_next, dt_dev)
        da, db = db, da
        a, b = b, a
    torch.cuda.synchronize()
    ctx.close()
    if variant == "exact":
        assert level_dts == odts
    else:
        assert np.allclose(level_dts, odts, rtol=1e-13, atol=0)
    for t, c, s in zip(a, lo, sizes):
        got = t.cpu().numpy()
        got = got[:, 4:-4, 4:-4, 4:-4] if dim == 3 else got[:, 0, 4:-4, 4:-4]
        want = _region(ref, c, s, dim)
        if variant == "exact":
            assert np.array_equal(got, want)
        else:
            assert np.all(rel_linf(got, want) <= 1e-10)
