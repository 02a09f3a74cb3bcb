"""Parity at the full sizes of the workloads, in the launch configuration the
benchmark times:
  * Sedov 128^3 for the configuration's 200 steps with the device dt: the
    shock radius follows the self-similar law (exponent 2/5, amplitude from the
    similarity solution), mass and energy are conserved while the blast is
    inside the box, and the octants stay mirror images;
  * Sedov 128^3 (the bench box): after GPU steps, one more step by the GPU
    and by the oracle from the same state, compared over the whole box;
  * the 512-box batched level: one graph-replayed batched step, sampled boxes
    compared with the oracle box by box;
  * the 512^3 stratified atmosphere with gravity (periodic x/y, reflecting z):
    one step, sampled zones compared with the oracle run on small sub-boxes
    whose ghost zones are gathered from the full state through the box's
    boundary maps (the step is local: a zone's update reads 4 zones around it);
  * the unperturbed atmosphere at 128^3, 256^3 and 512^3 for 100 steps: the
    middle half stays at rest (Mach < 1e-3 at 512^3) and the Mach number
    falls with resolution.
"""
import numpy as np
import pytest
import torch

import oracle
import sedov_similarity
from gpu_helpers import rel_linf
from paper_1711_06203_b300 import binding as hb
from paper_1711_06203_b300 import inputs

pytestmark = pytest.mark.gpu

I3 = (slice(None), slice(4, -4), slice(4, -4), slice(4, -4))


def test_sedov_128_full_box_parity():
    n = 128
    U, _ = inputs.sedov(n)
    ctx = hb.Context(0)
    p = hb.params(3, gamma=1.4, cfl=0.5)
    a = torch.from_numpy(U).cuda()
    b = torch.empty_like(a)
    box = lambda t: hb.box(t, (n, n, n), (1.0 / n,) * 3, hb.BC_OUTFLOW)
    dt = ctx.hydro_dt(box(a), p)
    for _ in range(12):
        dt = ctx.hydro_advance_box(box(a), box(b), p, dt, want_dt_next=True)
        a, b = b, a
    state = a.cpu().numpy()
    dn = ctx.hydro_advance_box(box(a), box(b), p, dt, want_dt_next=True)
    got = b.cpu().numpy()
    ctx.close()
    P = oracle.params(3, (n, n, n), gamma=1.4, cfl=0.5)
    ref, rc = oracle.step(state, P, dt)
    assert rc == 0
    assert np.all(rel_linf(got[I3], ref[I3]) <= 1e-10)
    dref, _ = oracle.dt(ref, P)
    assert abs(dn - dref) <= 1e-10 * dref


def test_sedov_128_200_steps_self_similar():
    n, steps = 128, 200
    U, _ = inputs.sedov(n)
    ctx = hb.Context(0)
    p = hb.params(3, gamma=1.4, cfl=0.5)
    a = torch.from_numpy(U).cuda()
    b = torch.empty_like(a)
    box = lambda t: hb.box(t, (n, n, n), (1.0 / n,) * 3, hb.BC_OUTFLOW)
    x = (torch.arange(n, dtype=torch.float64, device="cuda") + 0.5) / n - 0.5
    r = torch.sqrt(x.view(n, 1, 1) ** 2 + x.view(1, n, 1) ** 2 + x.view(1, 1, n) ** 2).ravel()
    nb = n // 2
    idx = torch.clamp((r / 0.5 * nb).long(), max=nb)
    inside = idx < nb
    cnt = torch.bincount(idx[inside], minlength=nb).double()
    rc = (torch.arange(nb, dtype=torch.float64) + 0.5) * (0.5 / nb)
    tot0 = a[:, 4:-4, 4:-4, 4:-4].sum(dim=(1, 2, 3))
    dt = ctx.hydro_dt(box(a), p)
    t, ts, Rpk, Rfr = 0.0, [], [], []
    for s in range(steps):
        d = dt
        dt = ctx.hydro_advance_box(box(a), box(b), p, d, want_dt_next=True)
        a, b = b, a
        t += d
        if s >= steps // 2 and s % 10 == 9:
            rho = a[0, 4:-4, 4:-4, 4:-4].ravel()
            prof = (torch.bincount(idx[inside], weights=rho[inside], minlength=nb) / cnt).cpu().numpy()
            k = int(np.argmax(prof))
            half = 0.5 * (1.0 + prof[k])
            j = k
            while prof[j + 1] > half:
                j += 1
            ts.append(t)
            Rpk.append(float(rc[k]))
            Rfr.append(float(rc[j] + (prof[j] - half) / (prof[j] - prof[j + 1]) * (rc[j + 1] - rc[j])))
    tot1 = a[:, 4:-4, 4:-4, 4:-4].sum(dim=(1, 2, 3))
    rho = a[0, 4:-4, 4:-4, 4:-4].cpu().numpy()
    ctx.close()
    assert Rfr[-1] < 0.45  # the blast is still inside the box
    expo = np.polyfit(np.log(ts), np.log(Rpk), 1)[0]
    assert abs(expo - 0.4) <= 0.02, expo
    ratio = Rfr[-1] / (sedov_similarity.xi0(1.4) * (t * t) ** 0.2)
    assert abs(ratio - 1.0) <= 0.05, ratio
    assert abs((tot1[0] - tot0[0]) / tot0[0]).item() < 1e-13
    assert abs((tot1[4] - tot0[4]) / tot0[4]).item() < 1e-13
    scale = np.abs(rho).max()
    for mir in (rho[::-1], rho[:, ::-1], rho[:, :, ::-1], rho.transpose(1, 0, 2), rho.transpose(2, 1, 0)):
        assert np.abs(rho - mir).max() / scale <= 1e-10


def test_batched_level_512_sampled_boxes():
    sizes, Us = inputs.level_boxes(512, seed=1711)
    dx = (1.0 / 64,) * 3
    p = hb.params(3, gamma=5.0 / 3.0, cfl=0.5)
    ctx = hb.Context(0)
    a = [torch.from_numpy(U).cuda() for U in Us]
    out = [torch.empty_like(x) for x in a]
    bin_ = [hb.box(x, s, dx, hb.BC_PREFILLED) for x, s in zip(a, sizes)]
    bout = [hb.box(x, s, dx, hb.BC_PREFILLED) for x, s in zip(out, sizes)]
    level_dt = min(ctx.hydro_dt(bx, p) for bx in bin_)
    dt_dev = torch.full((512,), level_dt, dtype=torch.float64, device="cuda")
    dt_next = torch.empty_like(dt_dev)
    for _ in range(2):  # plan + tuning, then a graph replay
        ctx.hydro_advance_batch(bin_, bout, p, dt_dev, dt_next)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    for b in sorted(rng.choice(512, 8, replace=False).tolist()) + [int(np.argmax([np.prod(s) for s in sizes]))]:
        s = sizes[b]
        P = oracle.params(3, s, dx=dx, bc=oracle.BC_PREFILLED, gamma=5.0 / 3.0, cfl=0.5)
        ref, rc = oracle.step(Us[b], P, level_dt)
        assert rc == 0
        got = out[b].cpu().numpy()
        assert np.all(rel_linf(got[I3], ref[I3]) <= 1e-10), b
        dref, _ = oracle.dt(ref, P)
        assert abs(dt_next[b].item() - dref) <= 1e-10 * dref
    ctx.close()
    del a, out
    torch.cuda.empty_cache()


def _stratified_device(n, H=0.1, g=1.0, gamma=5.0 / 3.0, perturb=1e-3, seed=1711):
    """The 512^3 atmosphere built on the device (same recipe as inputs.stratified)."""
    gsz = n + 8
    z = ((torch.arange(gsz, dtype=torch.float64, device="cuda") - 4 + 0.5) / n).view(gsz, 1, 1)
    rho = torch.exp(-z / H).expand(gsz, gsz, gsz)
    p = rho * g * H
    if perturb:
        gen = torch.Generator(device="cuda").manual_seed(seed)
        p = p * (1.0 + perturb * torch.randn((gsz, gsz, gsz), generator=gen, dtype=torch.float64, device="cuda"))
    U = torch.zeros((5, gsz, gsz, gsz), dtype=torch.float64, device="cuda")
    U[0] = rho
    U[4] = p / (gamma - 1.0)
    return U


def _subbox(a, n, c, m):
    """Grown sub-box of interior m^3 starting at interior zone c = (x, y, z) of
    the periodic-x/y, reflecting-z device box a, ghosts through the boundary
    maps (reflected z layers get their z-momentum negated); returned on host."""
    idx, flip = [], None
    for ax, c0 in enumerate(c):
        z = np.arange(c0 - 4, c0 + m + 4)
        if ax < 2:  # periodic
            z = np.mod(z, n)
        else:       # reflecting
            flip = (z < 0) | (z >= n)
            z = np.where(z < 0, -1 - z, np.where(z >= n, 2 * n - 1 - z, z))
        idx.append(torch.as_tensor(z + 4, device=a.device))
    S = a.index_select(1, idx[2]).index_select(2, idx[1]).index_select(3, idx[0]).cpu().numpy()
    S[3][flip] *= -1.0
    return np.ascontiguousarray(S)


def test_large_512_box_sampled_zones():
    n = 512
    torch.cuda.empty_cache()
    a = _stratified_device(n)
    b = torch.empty_like(a)
    bc = ((hb.BC_PERIODIC,) * 2, (hb.BC_PERIODIC,) * 2, (hb.BC_REFLECT,) * 2)
    box = lambda t: hb.box(t, (n, n, n), (1.0 / n,) * 3, bc)
    p = hb.params(3, gamma=5.0 / 3.0, cfl=0.5, grav=(0.0, 0.0, -1.0))
    ctx = hb.Context(0)
    dt = ctx.hydro_dt(box(a), p)
    ctx.hydro_advance_box(box(a), box(b), p, dt, want_dt_next=True)
    torch.cuda.synchronize()
    ctx.close()
    m = 4
    rng = np.random.default_rng(3)
    corners = [(0, 0, 0), (n - m, n - m, n - m), (n - m, 5, 0)] + \
              [tuple(int(v) for v in rng.integers(0, n - m, 3)) for _ in range(5)]
    for c in corners:
        S = _subbox(a, n, c, m)
        P = oracle.params(3, (m, m, m), dx=(1.0 / n,) * 3, bc=oracle.BC_PREFILLED, gamma=5.0 / 3.0,
                          grav=(0.0, 0.0, -1.0))
        ref, rc = oracle.step(S, P, dt)
        assert rc == 0
        got = b[:, 4 + c[2]:4 + c[2] + m, 4 + c[1]:4 + c[1] + m, 4 + c[0]:4 + c[0] + m].cpu().numpy()
        assert np.all(rel_linf(got, ref[I3]) <= 1e-10), c
    del a, b
    torch.cuda.empty_cache()


def _hydrostatic_mach(n, steps=100):
    """Max Mach number over the middle half in height after `steps` steps of
    the unperturbed n^3 atmosphere (periodic x/y, reflecting z, g = -1)."""
    torch.cuda.empty_cache()
    a = _stratified_device(n, perturb=0.0)
    b = torch.empty_like(a)
    bc = ((hb.BC_PERIODIC,) * 2, (hb.BC_PERIODIC,) * 2, (hb.BC_REFLECT,) * 2)
    box = lambda t: hb.box(t, (n, n, n), (1.0 / n,) * 3, bc)
    p = hb.params(3, gamma=5.0 / 3.0, cfl=0.5, grav=(0.0, 0.0, -1.0))
    ctx = hb.Context(0)
    dt = ctx.hydro_dt(box(a), p)
    for _ in range(steps):
        dt = ctx.hydro_advance_box(box(a), box(b), p, dt, want_dt_next=True)
        a, b = b, a
    ctx.close()
    mid = a[:, 4 + n // 4:4 + 3 * n // 4, 4:-4, 4:-4]
    rho = mid[0]
    vel = torch.sqrt(mid[1] ** 2 + mid[2] ** 2 + mid[3] ** 2) / rho
    pres = (5.0 / 3.0 - 1.0) * (mid[4] - 0.5 * rho * vel ** 2)
    mach = (vel / torch.sqrt(5.0 / 3.0 * pres / rho)).max().item()
    del a, b, mid, rho, vel, pres
    torch.cuda.empty_cache()
    return mach


def test_unperturbed_atmosphere_stays_hydrostatic_and_converges():
    """100 steps of the unperturbed atmosphere at 128^3, 256^3 and 512^3: away
    from the reflecting walls (whose mirrored ghosts are not in hydrostatic
    balance) the flow stays at rest to a Mach number below 1e-3 at 512^3, and
    the Mach number falls at least twofold with each doubling of resolution."""
    mach = {n: _hydrostatic_mach(n) for n in (128, 256, 512)}
    assert mach[512] < 1e-3, mach
    assert mach[256] <= 0.5 * mach[128] and mach[512] <= 0.5 * mach[256], mach
