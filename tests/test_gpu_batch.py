"""Batched level step (hydro_advance_batch) against the per-box step and the
oracle.  The batched kernels run the same per-item device code as the
single-box kernels; the results do not depend on the tracing kernel (sweep
segmentation, or warp rows and tiles) the autotuner picks.  With multiply-add contraction on, the compiler may fuse
differently in the batched kernels, so batch and per-box agree to the parity
tolerance (observed: 1 ulp); the contraction-free build is bitwise equal to
the oracle either way."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import blocky_state, rel_linf
from paper_1711_06203_b300 import binding as hb
from paper_1711_06203_b300 import inputs

pytestmark = pytest.mark.gpu

PRE = hb.BC_PREFILLED


def _level(seed, sizes, dim=3):
    rng = np.random.default_rng(seed)
    Us = [inputs.random_box(rng, s, dim) for s in sizes]
    return Us


def _interior(x, dim):
    return x[:, 4:-4, 4:-4, 4:-4] if dim == 3 else x[:, 0, 4:-4, 4:-4]


def _boxes(ts, sizes, dim):
    return [hb.box(t, s, (1.0 / s[0], 1.0 / s[1], 1.0 / s[2] if dim == 3 else 1.0), PRE) for t, s in zip(ts, sizes)]


def _run_batch(ctx, Us, sizes, dim, dts, p, steps=1):
    a = [torch.from_numpy(U).cuda() for U in Us]
    b = [torch.full_like(x, float("nan")) for x in a]
    dt_dev = torch.tensor(dts, dtype=torch.float64, device="cuda")
    dn = torch.zeros(len(Us), dtype=torch.float64, device="cuda")
    for _ in range(steps):
        bad = ctx.hydro_advance_batch(_boxes(a, sizes, dim), _boxes(b, sizes, dim), p, dt_dev, dn, want_bad=True)
        assert bad == -1
        for x, y in zip(a, b):  # carry the ghosts along: they are prefilled data
            inner = y[:, 4:-4, 4:-4, 4:-4].clone() if dim == 3 else y[:, :, 4:-4, 4:-4].clone()
            y.copy_(x)
            if dim == 3:
                y[:, 4:-4, 4:-4, 4:-4] = inner
            else:
                y[:, :, 4:-4, 4:-4] = inner
        a, b = b, a
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in a], dn.cpu().numpy()


def _run_single(ctx, Us, sizes, dim, dts, p):
    outs, nexts = [], []
    for U, s, d in zip(Us, sizes, dts):
        a = torch.from_numpy(U).cuda()
        b = torch.full_like(a, float("nan"))
        box_a, box_b = _boxes([a, b], [s, s], dim)
        nexts.append(ctx.hydro_advance_box(box_a, box_b, p, d, want_dt_next=True))
        outs.append(b.cpu().numpy())
    return outs, np.array(nexts)


SIZES3 = [(16, 24, 16), (32, 16, 24), (24, 24, 24), (16, 16, 32), (48, 16, 16), (24, 32, 16), (16, 16, 16)]


@pytest.mark.parametrize("tune", [True, False])
def test_batch_equals_per_box_and_oracle(tune):
    Us = _level(1711, SIZES3)
    p = hb.params(3, gamma=5 / 3, flatten=True)
    if not tune:
        p.flags |= hb.FLAG_NO_AUTOTUNE
    dts = []
    for U, s in zip(Us, SIZES3):
        P = oracle.params(3, s, dx=(1 / s[0], 1 / s[1], 1 / s[2]), bc=oracle.BC_PREFILLED, gamma=5 / 3)
        dts.append(oracle.dt(U, P)[0] * (0.7 + 0.1 * len(dts) / 7))  # a different dt per box
    ctx = hb.Context(0)
    got, dn = _run_batch(ctx, Us, SIZES3, 3, dts, p)
    single, dn1 = _run_single(ctx, Us, SIZES3, 3, dts, p)
    if tune:
        tuning = ctx.hydro_batch_tuning()
        assert {e for _, e in tuning} >= {16, 24, 32, 48} and {a for a, _ in tuning} == {0, 1, 2}
    ctx.close()
    for g, s1, U, s, d, nx in zip(got, single, Us, SIZES3, dts, dn):
        assert np.all(rel_linf(_interior(g, 3), _interior(s1, 3)) <= 1e-14)
        P = oracle.params(3, s, dx=(1 / s[0], 1 / s[1], 1 / s[2]), bc=oracle.BC_PREFILLED, gamma=5 / 3)
        ref, _ = oracle.step(U, P, d)
        assert np.all(rel_linf(_interior(g, 3), _interior(ref, 3)) <= 1e-10)
        dref, _ = oracle.dt(ref, P)
        assert abs(nx - dref) <= 1e-10 * dref
    assert np.all(np.abs(dn - dn1) <= 1e-14 * dn1)


def test_exact_batch_is_bitwise_equal_to_oracle():
    sizes = SIZES3[:4]
    Us = _level(7, sizes)
    dts = [1e-3, 2e-3, 1.5e-3, 0.5e-3]
    ctx = hb.Context(0, "exact")
    got, _ = _run_batch(ctx, Us, sizes, 3, dts, hb.params(3, gamma=5 / 3))
    ctx.close()
    for g, U, s, d in zip(got, Us, sizes, dts):
        P = oracle.params(3, s, dx=(1 / s[0], 1 / s[1], 1 / s[2]), bc=oracle.BC_PREFILLED, gamma=5 / 3)
        ref, _ = oracle.step(U, P, d)
        assert np.array_equal(_interior(g, 3), _interior(ref, 3))


@pytest.mark.parametrize("mode", ["tiles", "sweeps", "mixed"])
@pytest.mark.parametrize("data", ["random", "blocky"])
def test_exact_batch_with_each_tracing_kernel(mode, data, tmp_path, monkeypatch):
    """The tracing kernel chosen per axis and extent (the sweep with a given
    segment length, or the warp-row / tile kernels), forced through the
    tuning cache file: every choice gives the oracle's result bit for bit,
    in 3-D and 2-D, on random states and on piecewise-constant ones (zones
    at rest, equal neighbours, signed zero velocities: the kernels'
    exact-zero paths)."""
    sizes3 = SIZES3
    sizes2 = [(40, 24, 1), (16, 64, 1), (32, 32, 1)]
    classes = sorted({(a, s[a]) for s in sizes3 for a in range(3)} | {(a, s[a]) for s in sizes2 for a in range(2)})
    pick = {"tiles": lambda a, e: 0, "sweeps": lambda a, e: 2,
            "mixed": lambda a, e: 0 if (a == 0) != (e % 16 == 0) else 3}[mode]
    cache = tmp_path / "tune.txt"
    cache.write_text("".join(f"{a} {e} {pick(a, e)}\n" for a, e in classes))
    monkeypatch.setenv("HYDRO_TUNE_CACHE", str(cache))
    for dim, sizes in ((3, sizes3), (2, sizes2)):
        if data == "random":
            Us = _level(21 + dim, sizes, dim)
        else:
            rng = np.random.default_rng(31 + dim)
            Us = [blocky_state(rng, s[:dim], dim, 5 / 3) for s in sizes]
        dts = [1e-3 * (1 + 0.1 * k) for k in range(len(sizes))]
        ctx = hb.Context(0, "exact")
        got, _ = _run_batch(ctx, Us, sizes, dim, dts, hb.params(dim, gamma=5 / 3))
        tuning = ctx.hydro_batch_tuning()
        ctx.close()
        for a, e in classes:
            if a < dim:
                want = 0 if pick(a, e) == 0 else (e + 2 + pick(a, e) - 1) // pick(a, e)
                assert tuning[a, e] == want
        for g, U, s, d in zip(got, Us, sizes, dts):
            P = oracle.params(dim, s[:dim], dx=(1 / s[0], 1 / s[1], 1 / s[2] if dim == 3 else 1.0),
                              bc=oracle.BC_PREFILLED, gamma=5 / 3)
            ref, _ = oracle.step(U, P, d)
            assert np.array_equal(_interior(g, dim), _interior(ref, dim)), (mode, dim, s)


def test_graph_replay_uses_new_dt_and_ping_pong_plans():
    sizes = SIZES3[:3]
    Us = _level(3, sizes)
    p = hb.params(3, gamma=5 / 3)
    ctx = hb.Context(0)
    # three steps ping-ponging (two plans), dt changed between replays
    a = [torch.from_numpy(U).cuda() for U in Us]
    b = [x.clone() for x in a]
    dt_dev = torch.tensor([1e-3] * 3, dtype=torch.float64, device="cuda")
    refs = [U.copy() for U in Us]
    for k, dt in enumerate((1e-3, 2e-3, 1.5e-3)):
        dt_dev.fill_(dt)
        ctx.hydro_advance_batch(_boxes(a, sizes, 3), _boxes(b, sizes, 3), p, dt_dev)
        a, b = b, a
        for i, s in enumerate(sizes):
            P = oracle.params(3, s, dx=(1 / s[0], 1 / s[1], 1 / s[2]), bc=oracle.BC_PREFILLED, gamma=5 / 3)
            refs[i], _ = oracle.step(refs[i], P, dt)
            # the output ghosts are unspecified: keep the prefilled ghosts of the input
            g = a[i].cpu().numpy()
            g_fixed = refs[i].copy()
            g_fixed[:, 4:-4, 4:-4, 4:-4] = g[:, 4:-4, 4:-4, 4:-4]
            a[i].copy_(torch.from_numpy(g_fixed))
    torch.cuda.synchronize()
    for x, r in zip(a, refs):
        assert np.all(rel_linf(_interior(x.cpu().numpy(), 3), _interior(r, 3)) <= 1e-10)
    ctx.close()


def test_batch_reports_first_bad_box():
    sizes = SIZES3[:5]
    Us = _level(5, sizes)
    Us[3][0, 10, 10, 10] = -2.0
    ctx = hb.Context(0)
    a = [torch.from_numpy(U).cuda() for U in Us]
    b = [torch.empty_like(x) for x in a]
    dt_dev = torch.full((5,), 1e-4, dtype=torch.float64, device="cuda")
    rc, bad = ctx.hydro_advance_batch(_boxes(a, sizes, 3), _boxes(b, sizes, 3), hb.params(3, gamma=5 / 3), dt_dev,
                                      want_bad=True, raise_on_error=False)
    assert rc == hb.HYDRO_EBADSTATE and bad == 3
    ctx.close()


def test_batch_2d():
    sizes = [(40, 24, 1), (16, 64, 1), (32, 32, 1)]
    Us = _level(9, sizes, dim=2)
    p = hb.params(2, gamma=5 / 3)
    dts = [1e-3, 7e-4, 9e-4]
    ctx = hb.Context(0)
    got, _ = _run_batch(ctx, Us, sizes, 2, dts, p)
    ctx.close()
    for g, U, s, d in zip(got, Us, sizes, dts):
        P = oracle.params(2, s[:2], dx=(1 / s[0], 1 / s[1], 1.0), bc=oracle.BC_PREFILLED, gamma=5 / 3)
        ref, _ = oracle.step(U, P, d)
        assert np.all(rel_linf(_interior(g, 2), _interior(ref, 2)) <= 1e-10)


def test_batch_rejects_bad_descriptors():
    ctx = hb.Context(0)
    U = inputs.random_box(np.random.default_rng(0), (16, 16, 16), 3)
    a = torch.from_numpy(U).cuda()
    b = torch.empty_like(a)
    boxes_in, boxes_out = _boxes([a, a], [(16, 16, 16)] * 2, 3), _boxes([b, a], [(16, 16, 16)] * 2, 3)
    dt_dev = torch.full((2,), 1e-4, dtype=torch.float64, device="cuda")
    rc, _ = ctx.hydro_advance_batch(boxes_in, boxes_out, hb.params(3), dt_dev, raise_on_error=False)
    assert rc == hb.HYDRO_EINVAL  # second box writes over its own input
    ctx.close()
