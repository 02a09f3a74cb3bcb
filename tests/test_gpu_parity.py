"""Parity of the CUDA CTU-PPM step (through the C ABI) with the CPU oracle.

Tolerances (normwise relative L-infinity per conserved field, max|g-o|/max|o|):
  * contraction-free build (libhydro_exact.so): bitwise equal to the oracle —
    both evaluate the same FP64 operations in the same order;
  * product build (multiply-add contraction on): <= 1e-10 after one step and
    <= 1e-8 after 100 steps; conserved totals to 1e-13 relative.
Boxes span several thread blocks and ragged sizes (not multiples of 32 or 128).
"""
import zlib

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import blocky_state, gpu_steps, interior, oracle_params, rel_linf, to_dev
from paper_1711_06203_b300 import binding as hb
from paper_1711_06203_b300 import inputs

pytestmark = pytest.mark.gpu

O, R, PER, PRE = hb.BC_OUTFLOW, hb.BC_REFLECT, hb.BC_PERIODIC, hb.BC_PREFILLED


def _case(name):
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    if name == "sod2d":
        n, dim = (64, 64), 2
        return inputs.sod(64, 2, 0), dim, n, (1 / 64,) * 3, O, 1.4, (0, 0, 0), True
    if name == "random2d_periodic":
        n, dim = (37, 29), 2
        return inputs.random_box(rng, (37, 29, 1), 2), dim, n, (1 / 37, 1 / 29, 1.0), PER, 5 / 3, (0, 0, 0), True
    if name == "random3d_prefilled":
        n, dim = (21, 13, 10), 3
        return inputs.random_box(rng, n, 3), dim, n, (1 / 21, 1 / 13, 1 / 10), PRE, 5 / 3, (0, 0, 0), True
    if name == "random3d_periodic_noflat":
        n, dim = (16, 12, 9), 3
        return inputs.random_box(rng, n, 3), dim, n, (1 / 16,) * 3, PER, 5 / 3, (0, 0, 0), False
    if name == "sedov3d":
        U, _ = inputs.sedov(24)
        return U, 3, (24, 24, 24), (1 / 24,) * 3, O, 1.4, (0, 0, 0), True
    if name == "sedov3d_64":
        U, _ = inputs.sedov(64)
        return U, 3, (64, 64, 64), (1 / 64,) * 3, O, 1.4, (0, 0, 0), True
    if name == "stratified3d_gravity":
        U = inputs.stratified(16, 3, 5 / 3, 1.0, 0.1, perturb=1e-3, rng=rng)
        bc = ((PER, PER), (PER, PER), (R, R))
        return U, 3, (16, 16, 16), (1 / 16,) * 3, bc, 5 / 3, (0.0, 0.0, -1.0), True
    if name == "mixed_bc3d":
        n = (18, 11, 13)
        bc = ((O, R), (R, O), (PRE, O))
        return inputs.random_box(rng, n, 3), 3, n, (0.05, 0.07, 0.06), bc, 1.4, (0.3, -0.2, 0.1), True
    raise KeyError(name)


CASES = ["sod2d", "random2d_periodic", "random3d_prefilled", "random3d_periodic_noflat", "sedov3d",
         "stratified3d_gravity", "mixed_bc3d"]


def _oracle_dt(U, dim, n, dx, bc, gamma, grav, flat):
    P = oracle_params(dim, n, dx, bc, gamma, grav=grav, flatten=flat)
    d, rc = oracle.dt(U, P)
    assert rc == 0
    return P, d


@pytest.mark.parametrize("name", CASES)
def test_exact_build_is_bitwise_equal_to_oracle(name):
    U, dim, n, dx, bc, gamma, grav, flat = _case(name)
    P, d = _oracle_dt(U, dim, n, dx, bc, gamma, grav, flat)
    ref, rc = oracle.step(U, P, d)
    assert rc == 0
    got, nxt = gpu_steps(U, dim, n, dx, bc, gamma, [d], grav=grav, flatten=flat, variant="exact")
    gi, ri = interior(got, dim), interior(ref, dim)
    bad = np.argwhere(gi != ri)
    assert bad.size == 0, f"{len(bad)} zones differ; first {bad[:5].tolist()} max {np.abs(gi - ri).max()}"
    dref, _ = oracle.dt(ref, P)
    assert nxt[0] == dref


@pytest.mark.parametrize("name", CASES)
def test_one_step_parity(name):
    U, dim, n, dx, bc, gamma, grav, flat = _case(name)
    P, d = _oracle_dt(U, dim, n, dx, bc, gamma, grav, flat)
    ref, _ = oracle.step(U, P, d)
    got, nxt = gpu_steps(U, dim, n, dx, bc, gamma, [d], grav=grav, flatten=flat)
    err = rel_linf(interior(got, dim), interior(ref, dim))
    assert np.all(err <= 1e-10), err
    dref, _ = oracle.dt(ref, P)
    assert abs(nxt[0] - dref) <= 1e-10 * dref


@pytest.mark.parametrize("seed", range(8))
def test_exact_build_bitwise_on_blocky_states(seed):
    """Adversarial inputs for the kernels' exact-zero paths (flat parabolas,
    vanishing slopes, equal fluxes, signed zeros, reflected momenta): the
    contraction-free build equals the oracle bit for bit over 3 steps."""
    rng = np.random.default_rng(900 + seed)
    dim = 3 if seed % 4 else 2
    n = (13, 11, 9) if dim == 3 else (17, 15)
    kinds = (O, R, PER)
    bc = []
    for a in range(3):
        k = kinds[rng.integers(0, 3)]
        bc.append((k, k) if k == PER else (k, kinds[rng.integers(0, 2)]))
    bc = tuple(bc)
    grav = (0.0, 0.0, 0.0) if seed % 2 else (0.2, -0.3, 0.1 if dim == 3 else 0.0)
    gamma = 1.4
    dx = (1 / 13, 1 / 11, 1 / 9)
    U = blocky_state(rng, n, dim, gamma)
    P = oracle_params(dim, n, dx, bc, gamma, grav=grav)
    ref, got = U, U
    ctx = hb.Context(0, "exact")
    for _ in range(3):
        d, rc = oracle.dt(ref, P)
        assert rc == 0
        ref, rc = oracle.step(ref, P, d)
        assert rc == 0
        got, nxt = gpu_steps(got, dim, n, dx, bc, gamma, [d], grav=grav, ctx=ctx)
        assert np.array_equal(interior(got, dim), interior(ref, dim)), (seed, bc, grav)
        assert nxt[0] == oracle.dt(ref, P)[0]
    ctx.close()


@pytest.mark.parametrize("name,steps", [("sedov3d", 40), ("sod2d", 40)])
def test_exact_build_many_steps_bitwise(name, steps):
    """Many steps of a blast in gas at rest, in the contraction-free build:
    bit for bit the oracle's run after every step.  The front between moving
    and resting gas sweeps through the box, so zones switch between the
    kernels' at-rest paths (flat data, equal fluxes) and the general ones."""
    U, dim, n, dx, bc, gamma, grav, flat = _case(name)
    P = oracle_params(dim, n, dx, bc, gamma, grav=grav, flatten=flat)
    ref = U
    got = U
    ctx = hb.Context(0, "exact")
    for _ in range(steps):
        d, rc = oracle.dt(ref, P)
        assert rc == 0
        ref, rc = oracle.step(ref, P, d)
        assert rc == 0
        got, _ = gpu_steps(got, dim, n, dx, bc, gamma, [d], grav=grav, flatten=flat, ctx=ctx)
        assert np.array_equal(interior(got, dim), interior(ref, dim))
    ctx.close()


@pytest.mark.parametrize("name,steps", [("sod2d", 100), ("random3d_periodic_noflat", 100), ("sedov3d", 100),
                                        ("sedov3d_64", 100)])
def test_many_step_parity(name, steps):
    U, dim, n, dx, bc, gamma, grav, flat = _case(name)
    P = oracle_params(dim, n, dx, bc, gamma, grav=grav, flatten=flat)
    # both sides take the same time steps (the oracle's), so only the arithmetic differs
    ref, t, dts = oracle.run(U, P, steps)
    got, _ = gpu_steps(U, dim, n, dx, bc, gamma, dts, grav=grav, flatten=flat)
    err = rel_linf(interior(got, dim), interior(ref, dim))
    assert np.all(err <= 1e-8), err


@pytest.mark.parametrize("dim", [2, 3])
def test_periodic_conservation_on_gpu(dim):
    rng = np.random.default_rng(7 + dim)
    n = (33, 17, 11) if dim == 3 else (45, 23, 1)
    U = inputs.random_box(rng, n, dim)
    dx = (1 / 33, 1 / 17, 1 / 11)
    P = oracle_params(dim, n, dx, PER, 5 / 3)
    U0 = oracle.fill_ghosts(U, P)
    d, _ = oracle.dt(U, P)
    got, _ = gpu_steps(U, dim, n, dx, PER, 5 / 3, [d, d, d])
    g, u0 = interior(got, dim), interior(U0, dim)
    tot0, tot = u0.reshape(5, -1).sum(1), g.reshape(5, -1).sum(1)
    mag = np.abs(u0).reshape(5, -1).sum(1)
    rel = np.abs(tot - tot0) / np.where(mag > 0, mag, 1.0)
    assert np.all(rel <= 1e-13), rel


@pytest.mark.parametrize("variant", ["exact", "default"])
def test_conservation_against_boundary_fluxes(variant):
    """Non-periodic boxes (outflow, reflecting, prefilled faces; g = 0): the
    change of every conserved total over one step equals what crosses the
    box's outer faces, -dt * sum_d (1/dx_d) sum_faces (F_hi - F_lo), with the
    fluxes the library records for its own step; the recorded fluxes equal
    the oracle's final fluxes (bitwise in the contraction-free build)."""
    import math
    rng = np.random.default_rng(31)
    for dim, n, bc in ((3, (21, 14, 11), ((O, R), (PRE, O), (R, R))), (2, (33, 19, 1), ((R, O), (O, PRE)))):
        U = inputs.random_box(rng, n, dim)
        dx = (1 / 21, 1 / 14, 1 / 11)
        bc3 = tuple(bc) + ((O, O),) * (3 - len(bc))
        P = oracle_params(dim, n[:dim], dx, bc3, 5 / 3)
        d, _ = oracle.dt(U, P)
        ref, rc, dbg = oracle.step(U, P, d, debug=True)
        assert rc == 0
        ctx = hb.Context(0, variant)
        ctx.hydro_ctx_record_face_fluxes(True)
        a = to_dev(U)
        b = torch.empty_like(a)
        ctx.hydro_advance_box(hb.box(a, n, dx, bc3), hb.box(b, n, dx, bc3), hb.params(dim, gamma=5 / 3), d)
        faces = {}
        for ax in range(dim):
            t = [x for x in range(3) if x != ax]
            shape = (5, n[t[1]] if t[1] < dim else 1, n[t[0]])
            for side in (0, 1):
                f = torch.empty(shape, dtype=torch.float64, device="cuda")
                ctx.hydro_ctx_face_flux(ax, side, f)
                faces[ax, side] = f.cpu().numpy()
        got = b.cpu().numpy()
        ctx.close()
        U0, U1 = interior(oracle.fill_ghosts(U, P), dim), interior(got, dim)
        for c in range(5):
            if dim == 2 and c == 3:
                continue
            change = math.fsum(U1[c].ravel()) - math.fsum(U0[c].ravel())
            through = -math.fsum(d / dx[ax] * (math.fsum(faces[ax, 1][c].ravel()) - math.fsum(faces[ax, 0][c].ravel()))
                                 for ax in range(dim))
            scale = math.fsum(np.abs(U0[c]).ravel())
            assert abs(change - through) <= 1e-13 * scale, (dim, c, change, through)
        # the recorded planes are the oracle's final fluxes on the outer faces
        for ax in range(dim):
            F = dbg["flux_final"][ax]
            for side in (0, 1):
                sl = [slice(None), slice(4, -4), slice(4, -4), slice(4, -4)] if dim == 3 else \
                     [slice(None), slice(0, 1), slice(4, -4), slice(4, -4)]
                sl[3 - ax] = 4 + (n[ax] if side else 0)
                want = F[tuple(sl)].reshape(faces[ax, side].shape)
                if variant == "exact":
                    assert np.array_equal(faces[ax, side], want)
                else:
                    # per field, relative to that flux over the whole box (a
                    # reflecting wall's mass flux is exactly 0 in the oracle)
                    scale = np.abs(F.reshape(5, -1)).max(axis=1)[:, None, None]
                    assert np.all(np.abs(faces[ax, side] - want) <= 1e-10 * scale)


def test_hydro_dt_matches_oracle():
    rng = np.random.default_rng(3)
    n = (19, 23, 7)
    U = inputs.random_box(rng, n, 3)
    dx = (0.1, 0.07, 0.13)
    P = oracle_params(3, n, dx, PRE, 5 / 3, cfl=0.8)
    dref, _ = oracle.dt(U, P)
    for variant in ("exact", "default"):
        ctx = hb.Context(0, variant)
        a = to_dev(U)
        d = ctx.hydro_dt(hb.box(a, n, dx, PRE), hb.params(3, gamma=5 / 3, cfl=0.8))
        ctx.close()
        if variant == "exact":
            assert d == dref
        else:
            assert abs(d - dref) <= 1e-14 * dref


def test_bad_state_is_reported():
    rng = np.random.default_rng(1)
    n = (12, 12, 12)
    U = inputs.random_box(rng, n, 3)
    U[0, 8, 8, 8] = -1.0  # negative density in the interior
    ctx = hb.Context(0)
    a = to_dev(U)
    b = torch.empty_like(a)
    p = hb.params(3, gamma=5 / 3)
    rc, _ = ctx.hydro_advance_box(hb.box(a, n, (0.1,) * 3, PRE), hb.box(b, n, (0.1,) * 3, PRE), p, 1e-3,
                                  want_dt_next=True, raise_on_error=False)
    assert rc == hb.HYDRO_EBADSTATE
    # asynchronous form: recorded in the context, reported by hydro_ctx_check, then cleared
    ctx.hydro_advance_box(hb.box(a, n, (0.1,) * 3, PRE), hb.box(b, n, (0.1,) * 3, PRE), p, 1e-3)
    assert ctx.hydro_ctx_check() == hb.HYDRO_EBADSTATE
    assert ctx.hydro_ctx_check() == hb.HYDRO_OK
    with pytest.raises(hb.HydroError) as e:
        ctx.hydro_dt(hb.box(a, n, (0.1,) * 3, PRE), p)
    assert e.value.status == hb.HYDRO_EBADSTATE
    ctx.close()


def test_injected_allocation_failure_is_reported_and_recoverable():
    """Fault injection on the host: with the context's allocations made to
    fail, a step that needs scratch (single box, host buffers, a batched
    level) returns HYDRO_ENOMEM and writes nothing; with allocation restored
    the same context steps, bitwise as a fresh one."""
    rng = np.random.default_rng(5)
    n, dx, bc = (20, 18, 16), (0.05,) * 3, ((O, O), (R, R), (PER, PER))
    U = inputs.random_box(rng, n, 3)
    p = hb.params(3, gamma=5 / 3)
    d, _ = oracle.dt(U, oracle_params(3, n, dx, bc, 5 / 3))
    ctx = hb.Context(0)
    ctx.hydro_ctx_fail_allocations(True)
    a = to_dev(U)
    b = torch.full_like(a, float("nan"))
    rc, _ = ctx.hydro_advance_box(hb.box(a, n, dx, bc), hb.box(b, n, dx, bc), p, d, want_dt_next=True,
                                  raise_on_error=False)
    assert rc == hb.HYDRO_ENOMEM
    torch.cuda.synchronize()
    assert torch.isnan(b).all()
    hin = torch.from_numpy(U.copy()).pin_memory()
    hout = torch.full_like(hin, float("nan")).pin_memory()
    with pytest.raises(hb.HydroError) as e:
        ctx.hydro_advance_box_host(hb.box(hin, n, dx, bc), hb.box(hout, n, dx, bc), p, d)
    assert e.value.status == hb.HYDRO_ENOMEM
    assert torch.isnan(hout).all()
    dt_dev = torch.full((1,), d, dtype=torch.float64, device="cuda")
    with pytest.raises(hb.HydroError) as e:
        ctx.hydro_advance_batch([hb.box(a, n, dx, PRE)], [hb.box(b, n, dx, PRE)], p, dt_dev)
    assert e.value.status == hb.HYDRO_ENOMEM
    ctx.hydro_ctx_fail_allocations(False)
    got = ctx.hydro_advance_box(hb.box(a, n, dx, bc), hb.box(b, n, dx, bc), p, d, want_dt_next=True)
    ctx.close()
    ref, ref_dt = gpu_steps(U, 3, n, dx, bc, 5 / 3, [d])
    assert np.array_equal(interior(b.cpu().numpy(), 3), interior(ref, 3))
    assert got == ref_dt[0]


def test_invalid_arguments_are_rejected():
    ctx = hb.Context(0)
    U = inputs.random_box(np.random.default_rng(0), (8, 8, 8), 3)
    a = to_dev(U)
    b = torch.empty_like(a)
    p = hb.params(3, gamma=5 / 3)
    good_in, good_out = hb.box(a, (8, 8, 8), (0.1,) * 3, PRE), hb.box(b, (8, 8, 8), (0.1,) * 3, PRE)
    cases = []
    x = hb.box(a, (8, 8, 8), (0.1,) * 3, PRE); x.ng = 3; cases.append((x, good_out, p, 1e-3))
    x = hb.box(a, (8, 8, 8), (0.0, 0.1, 0.1), PRE); cases.append((x, good_out, p, 1e-3))
    x = hb.box(a, (8, 8, 8), (0.1,) * 3, PRE); x.bc[0][0] = hb.BC_PERIODIC; cases.append((x, good_out, p, 1e-3))
    x = hb.box(a, (8, 8, 8), (0.1,) * 3, PRE); x.stride[0] = 4; cases.append((x, good_out, p, 1e-3))
    cases.append((good_in, good_in, p, 1e-3))  # in == out overlaps
    cases.append((good_in, good_out, p, -1.0))  # negative dt
    bad_p = hb.params(3, gamma=1.0); cases.append((good_in, good_out, bad_p, 1e-3))
    bad_p = hb.params(4, gamma=1.4); cases.append((good_in, good_out, bad_p, 1e-3))
    o2 = hb.box(b, (8, 8, 7), (0.1,) * 3, PRE); cases.append((good_in, o2, p, 1e-3))
    for bi, bo, pp, dt in cases:
        rc, _ = ctx.hydro_advance_box(bi, bo, pp, dt, want_dt_next=True, raise_on_error=False)
        assert rc == hb.HYDRO_EINVAL
    ctx.close()


def test_strided_boxes_and_streams():
    """Input and output with different padded strides, on a side stream."""
    rng = np.random.default_rng(12)
    n = (14, 10, 9)
    U = inputs.random_box(rng, n, 3)
    P = oracle_params(3, n, (0.1,) * 3, PRE, 5 / 3)
    d, _ = oracle.dt(U, P)
    ref, _ = oracle.step(U, P, d)
    big = torch.zeros((5, 17 + 2, 18 + 3, 22 + 6), dtype=torch.float64, device="cuda")
    a = big[:, 1:18, 2:20, 3:25]
    a.copy_(to_dev(U))
    out = torch.zeros((5, 17, 18, 24), dtype=torch.float64, device="cuda")[:, :, :, 1:23]
    ctx = hb.Context(0)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx.hydro_advance_box(hb.box(a, n, (0.1,) * 3, PRE), hb.box(out, n, (0.1,) * 3, PRE),
                              hb.params(3, gamma=5 / 3), d, stream=s)
    s.synchronize()
    got = out.cpu().numpy()
    err = rel_linf(got[:, 4:-4, 4:-4, 4:-4], ref[:, 4:-4, 4:-4, 4:-4])
    assert np.all(err <= 1e-10), err
    ctx.close()


def test_integer_pipe_scaling_is_ieee_exact():
    """The kernels' integer-pipe 2x and x/2 equal IEEE 2.0*x and 0.5*x bit for
    bit, across zeros, subnormals, the normal/subnormal boundary, overflow and
    random bit patterns."""
    rng = np.random.default_rng(99)
    edge = [0.0, -0.0, 5e-324, -5e-324, 1e-323, 1.5e-323, 2.2250738585072014e-308, 2.225073858507201e-308,
            -2.2250738585072014e-308, 4.450147717014403e-308, 1.7976931348623157e308, 8.98846567431158e307,
            -1.7976931348623157e308, np.inf, -np.inf, 1.0, 3.0, 0.1, -7.5]
    pats = rng.integers(0, 2 ** 63 - 1, 200000, dtype=np.int64)
    pats = pats ^ (rng.integers(0, 2, pats.size, dtype=np.int64) << 63)
    x = np.concatenate([np.array(edge), pats.view(np.float64)])
    x = x[~np.isnan(x)]
    for variant in ("default", "exact"):
        t, h = hb.hydro_selftest_scale2(torch.from_numpy(x).cuda(), variant)
        with np.errstate(over="ignore"):
            assert np.array_equal(t.cpu().numpy().view(np.int64), (2.0 * x).view(np.int64))
            assert np.array_equal(h.cpu().numpy().view(np.int64), (0.5 * x).view(np.int64))


def _intpipe_operands(rng):
    """Operand pairs for the integer-pipe product and sum: signed zeros,
    subnormals, the normal/subnormal boundary, the largest values,
    infinities, random bit patterns, products that over- and underflow,
    rounding ties, and sums with every exponent gap including cancellation."""
    edge = np.array([0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, 2.225073858507201e-308,
                     1.7976931348623157e308, -1.7976931348623157e308, np.inf, -np.inf, 1.0, -1.0, 0.5, 3.0,
                     0.1, 1e-300, 1e300, 1.0000000000000002, 0.9999999999999999])
    ex, ey = np.meshgrid(edge, edge)
    n = 400000
    bits = rng.integers(0, 2 ** 63 - 1, (2, n), dtype=np.int64)
    bits ^= rng.integers(0, 2, (2, n), dtype=np.int64) << 63
    rx, ry = bits.view(np.float64)
    # moderate magnitudes with exponent gaps 0..70 and near-cancellation
    m = rng.uniform(1.0, 2.0, n) * 2.0 ** rng.integers(-60, 60, n)
    gap = m * rng.uniform(1.0, 2.0, n) * 2.0 ** -rng.integers(0, 70, n) * rng.choice([-1.0, 1.0], n)
    near = -(m * (1.0 + rng.integers(-8, 8, n) * 2.0 ** -52))
    # products near 1 whose exact significand product ends in a tie or near one
    t1 = 1.0 + rng.integers(0, 2 ** 26, n) * 2.0 ** -26
    t2 = 1.0 + rng.integers(0, 2 ** 27, n) * 2.0 ** -27
    # products across the overflow and underflow thresholds
    big = rng.uniform(1.0, 2.0, n) * 2.0 ** rng.integers(500, 530, n)
    tiny = rng.uniform(1.0, 2.0, n) * 2.0 ** rng.integers(-560, -500, n)
    x = np.concatenate([ex.ravel(), rx, m, m, t1, big, tiny, tiny])
    y = np.concatenate([ey.ravel(), ry, gap, near, t2, big, tiny, big])
    keep = ~(np.isnan(x) | np.isnan(y))
    return x[keep], y[keep]


def test_integer_pipe_products_and_sums_are_ieee_exact():
    """The kernels' integer-pipe x*y and x+y equal the IEEE operations (round
    to nearest even) bit for bit, in both builds; invalid operations give a
    NaN."""
    x, y = _intpipe_operands(np.random.default_rng(1711))
    with np.errstate(over="ignore", under="ignore", invalid="ignore"):
        ref_p, ref_s = x * y, x + y
    for variant in ("default", "exact"):
        p, s = hb.hydro_selftest_intpipe(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), variant)
        for got, ref in ((p.cpu().numpy(), ref_p), (s.cpu().numpy(), ref_s)):
            assert np.array_equal(np.isnan(got), np.isnan(ref))
            ok = ~np.isnan(ref)
            bad = np.flatnonzero(got[ok].view(np.int64) != ref[ok].view(np.int64))
            assert bad.size == 0, (variant, x[ok][bad[:4]], y[ok][bad[:4]], got[ok][bad[:4]], ref[ok][bad[:4]])


def _ulps(a, b):
    """Distance in units in the last place between float64 arrays of one sign."""
    return np.abs(a.view(np.int64) - b.view(np.int64))


def test_reciprocal_quotient_sqrt_error_bounds():
    """The product build's Newton-refined 1/x, y/x and sqrt(x) stay within 2
    ulp of IEEE over magnitudes 1e-300..1e300 (arguments outside the refined
    range, zeros and infinities take the IEEE path); the contraction-free
    build is IEEE exactly."""
    rng = np.random.default_rng(7)
    x = 10.0 ** rng.uniform(-300, 300, 400000)
    x[::7] *= -1.0
    y = rng.standard_normal(x.size) * 10.0 ** rng.uniform(-20, 20, x.size)
    x = np.concatenate([x, [0.0, -0.0, np.inf, 5e-324, 2.2250738585072014e-308, 1.7976931348623157e308]])
    y = np.concatenate([y, [1.0, 1.0, 1.0, 1.0, 1.0, 1.0]])
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        ref = (1.0 / x, y / x, np.sqrt(x))
    for variant, bound in (("exact", 0), ("default", 2)):
        got = hb.hydro_selftest_divsqrt(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), variant)
        for g, w in zip(got, ref):
            g = g.cpu().numpy()
            both_nan = np.isnan(g) & np.isnan(w)
            assert np.array_equal(np.isnan(g), np.isnan(w))
            fin = ~both_nan & np.isfinite(w)
            assert np.array_equal(g[~both_nan & ~np.isfinite(w)], w[~both_nan & ~np.isfinite(w)])
            same_sign = np.signbit(g[fin]) == np.signbit(w[fin])
            assert same_sign.all()
            assert _ulps(g[fin], w[fin]).max() <= bound, (variant, _ulps(g[fin], w[fin]).max())


def test_reciprocal_square_root_error_bound():
    """The product build's refined 1/sqrt(x) (the first solves' sound speed
    and 1/rho come from it) stays within 2 ulp of the correctly rounded value
    over 1e-280..1e280; outside the refined range and in the contraction-free
    build it is IEEE 1.0/sqrt(x)."""
    rng = np.random.default_rng(8)
    x = np.concatenate([10.0 ** rng.uniform(-280, 280, 400000), rng.uniform(0.5, 2.0, 100000),
                        [1.0, 4.0, 0.25, 2.0, 1e-310, 1.7976931348623157e308]])
    want = (1.0 / np.sqrt(x.astype(np.longdouble))).astype(np.float64)
    for variant, bound in (("exact", 1), ("default", 2)):
        got = hb.hydro_selftest_rsqrt(torch.from_numpy(x).cuda(), variant).cpu().numpy()
        assert np.all(np.isfinite(got))
        assert _ulps(got, want).max() <= bound, (variant, _ulps(got, want).max())


def test_host_buffer_step_exact_build_is_the_oracle():
    """The overlapped host-buffer step in the contraction-free build against
    the oracle directly, bit for bit: tall boxes, so that every stage runs in
    many chunks on both compute streams, with every z boundary kind."""
    rng = np.random.default_rng(77)
    ctx = hb.Context(0, "exact")
    for n, bc in (((12, 10, 64), ((O, R), (PER, PER), (O, O))),
                  ((10, 9, 53), ((R, R), (O, O), (PER, PER))),
                  ((9, 11, 40), ((PER, PER), (O, R), (R, O)))):
        U = inputs.random_box(rng, n, 3)
        dx = (0.05, 0.06, 0.04)
        P = oracle_params(3, n, dx, bc, 5 / 3)
        d, _ = oracle.dt(U, P)
        ref, rc = oracle.step(U, P, d)
        assert rc == 0
        hin = torch.from_numpy(U.copy()).pin_memory()
        hout = torch.full_like(hin, float("nan")).pin_memory()
        dn = ctx.hydro_advance_box_host(hb.box(hin, n, dx, bc), hb.box(hout, n, dx, bc), hb.params(3, gamma=5 / 3), d,
                                        want_dt_next=True)
        assert np.array_equal(interior(hout.numpy(), 3), interior(ref, 3)), (n, bc)
        assert dn == oracle.dt(ref, P)[0]
    ctx.close()


def test_host_buffer_step_matches_device_step():
    """hydro_advance_box_host on pageable and pinned host buffers gives the
    device path's result bit for bit: 3-D boxes with derived faces (interior
    planes only cross the host link, in z-chunks that overlap the kernels,
    every stage running over the planes whose inputs have landed, on two
    compute streams; 4 to 100 planes, every z boundary kind), a prefilled
    face (the whole input box crosses) and 2-D; a non-physical input is
    reported.
    It writes none of the output's ghost planes along the slowest axis and
    refuses non-natural layouts."""
    rng = np.random.default_rng(12)
    ctx = hb.Context(0)
    cases = [
        (3, (13, 10, 11), ((hb.BC_PERIODIC,) * 2, (hb.BC_REFLECT, hb.BC_OUTFLOW), (hb.BC_OUTFLOW,) * 2)),
        (3, (12, 9, 10), ((hb.BC_OUTFLOW,) * 2, (hb.BC_PREFILLED, hb.BC_REFLECT), (hb.BC_PERIODIC,) * 2)),
        (2, (14, 11, 1), ((hb.BC_OUTFLOW, hb.BC_REFLECT), (hb.BC_PERIODIC,) * 2, (hb.BC_OUTFLOW,) * 2)),
        # one interior plane per chunk of the overlapped path, and a box of several planes per chunk
        (3, (10, 9, 4), ((hb.BC_REFLECT, hb.BC_OUTFLOW), (hb.BC_OUTFLOW,) * 2, (hb.BC_OUTFLOW,) * 2)),
        (3, (40, 36, 44), ((hb.BC_OUTFLOW,) * 2, (hb.BC_PERIODIC,) * 2, (hb.BC_REFLECT, hb.BC_OUTFLOW))),
        # reflecting z faces with chunks thinner than a ghost layer, and periodic z
        (3, (10, 8, 6), ((hb.BC_OUTFLOW,) * 2, (hb.BC_OUTFLOW,) * 2, (hb.BC_REFLECT,) * 2)),
        (3, (9, 12, 20), ((hb.BC_REFLECT,) * 2, (hb.BC_OUTFLOW,) * 2, (hb.BC_PERIODIC,) * 2)),
        # chunks of 12-13 planes: the z tracing advances by whole tiles between
        # chunks, and the last chunk's final fluxes and update go in pieces
        (3, (24, 20, 100), ((hb.BC_OUTFLOW,) * 2, (hb.BC_REFLECT,) * 2, (hb.BC_PERIODIC,) * 2)),
        (3, (16, 18, 77), ((hb.BC_PERIODIC,) * 2, (hb.BC_OUTFLOW,) * 2, (hb.BC_REFLECT, hb.BC_OUTFLOW))),
    ]
    for dim, n, bc in cases:
        U = inputs.random_box(rng, n, dim)
        dx = (0.05,) * 3
        p = hb.params(dim, gamma=5 / 3)
        P = oracle_params(dim, n[:dim], dx, bc, 5 / 3)
        d, _ = oracle.dt(U, P)
        a = to_dev(U)
        b = torch.empty_like(a)
        dn_dev = ctx.hydro_advance_box(hb.box(a, n, dx, bc), hb.box(b, n, dx, bc), p, d, want_dt_next=True)
        want = b.cpu().numpy()
        for pinned in (False, True):
            hin = torch.from_numpy(U.copy())
            hout = torch.full_like(hin, float("nan"))
            if pinned:
                hin, hout = hin.pin_memory(), hout.pin_memory()
            dn = ctx.hydro_advance_box_host(hb.box(hin, n, dx, bc), hb.box(hout, n, dx, bc), p, d, want_dt_next=True)
            assert dn == dn_dev
            got = hout.numpy()
            assert np.array_equal(interior(got, dim), interior(want, dim))
            # the ghost planes along the slowest axis are not written
            if dim == 3:
                assert np.isnan(got[:, :4]).all() and np.isnan(got[:, -4:]).all()
            else:
                assert np.isnan(got[:, :, :4]).all() and np.isnan(got[:, :, -4:]).all()
    # a non-physical input state is reported by the overlapped path too, and
    # the context is clean again for the next call
    n, dx = (16, 12, 20), (0.05,) * 3
    bc = ((hb.BC_OUTFLOW,) * 2, (hb.BC_REFLECT,) * 2, (hb.BC_OUTFLOW,) * 2)
    U = inputs.random_box(rng, n, 3)
    U[0, 4 + 13, 4 + 5, 4 + 7] = -1.0  # negative density in the interior (plane 13 of 20)
    hin = torch.from_numpy(U.copy()).pin_memory()
    hout = torch.empty((5,) + U.shape[1:], dtype=torch.float64).pin_memory()
    p = hb.params(3, gamma=5 / 3)
    with pytest.raises(hb.HydroError) as e:
        ctx.hydro_advance_box_host(hb.box(hin, n, dx, bc), hb.box(hout, n, dx, bc), p, 1e-3, want_dt_next=True)
    assert e.value.status == hb.HYDRO_EBADSTATE
    U[0, 4 + 13, 4 + 5, 4 + 7] = 1.0
    hin.copy_(torch.from_numpy(U))
    assert ctx.hydro_advance_box_host(hb.box(hin, n, dx, bc), hb.box(hout, n, dx, bc), p, 1e-3, want_dt_next=True) > 0
    n, dx, bc = cases[0][1], (0.05,) * 3, cases[0][2]
    p = hb.params(3, gamma=5 / 3)
    hout = torch.empty((5,) + inputs.grown_shape(n, 3), dtype=torch.float64)
    big = torch.zeros((5, 20, 19, 22), dtype=torch.float64)  # padded rows: not the natural layout
    with pytest.raises(hb.HydroError) as e:
        ctx.hydro_advance_box_host(hb.box(big[:, :, :18, :21], n, dx, bc), hb.box(hout, n, dx, bc), p, 1e-3)
    assert e.value.status == hb.HYDRO_EINVAL
    ctx.close()
