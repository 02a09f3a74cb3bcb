"""Two-level subcycled advance on the GPU (hydro_amr_advance) against the
two-level oracle, through the C ABI:

  * a 3-D and a 2-D hierarchy (uneven coarse tiling, fine boxes with a
    concave corner, mixed domain boundary kinds), several coarse steps with
    the device-side dt: bitwise for the contraction-free build, to the parity
    tolerance for the product build;
  * conservation of the composite totals on a periodic domain at the size the
    benchmark times (a property that holds at any size);
  * hierarchies that break the nesting rules are refused.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import rel_linf
from oracle import amr
from paper_1711_06203_b300 import binding as hb
from paper_1711_06203_b300 import inputs

pytestmark = pytest.mark.gpu

O, R, PER = hb.BC_OUTFLOW, hb.BC_REFLECT, hb.BC_PERIODIC


def _interior(U, dim):
    return U[:, 4:-4, 4:-4, 4:-4] if dim == 3 else U[:, 0, 4:-4, 4:-4]


def _tile(Uc, lo, sizes, dim):
    """Per-box grown arrays holding the coarse interior values (ghosts NaN)."""
    out = []
    for c, s in zip(lo, sizes):
        gz = s[2] + 8 if dim == 3 else 1
        B = np.full((5, gz, s[1] + 8, s[0] + 8), np.nan)
        if dim == 3:
            B[:, 4:-4, 4:-4, 4:-4] = Uc[:, 4 + c[2]:4 + c[2] + s[2], 4 + c[1]:4 + c[1] + s[1], 4 + c[0]:4 + c[0] + s[0]]
        else:
            B[:, 0, 4:-4, 4:-4] = Uc[:, 0, 4 + c[1]:4 + c[1] + s[1], 4 + c[0]:4 + c[0] + s[0]]
        out.append(B)
    return out


def _untile(tiles, lo, sizes, dim, domain):
    n = tuple(domain) + (1,) * (3 - len(domain))
    U = np.zeros((5, n[2] if dim == 3 else 1, n[1], n[0]))
    for T, c, s in zip(tiles, lo, sizes):
        if dim == 3:
            U[:, c[2]:c[2] + s[2], c[1]:c[1] + s[1], c[0]:c[0] + s[0]] = T[:, 4:-4, 4:-4, 4:-4]
        else:
            U[:, 0, c[1]:c[1] + s[1], c[0]:c[0] + s[0]] = T[:, 0, 4:-4, 4:-4]
    return U


class Hierarchy:
    """Device-side two-level hierarchy: coarse tiles and fine boxes, each with
    an input and an output tensor swapped after every step."""

    def __init__(self, ctx, dim, domain, bc, Uc, clo, csz, fines, dx, variant_p):
        self.ctx, self.dim, self.domain, self.bc, self.dx, self.p = ctx, dim, domain, bc, dx, variant_p
        self.clo, self.csz = clo, csz
        self.ca = [torch.from_numpy(T).cuda() for T in _tile(Uc, clo, csz, dim)]
        self.cb = [torch.full_like(t, float("nan")) for t in self.ca]
        self.flo = [b.lo for b in fines]
        self.fsz = [b.n for b in fines]
        fa = []
        for b in fines:
            G = np.full_like(b.U, np.nan)
            if dim == 3:
                G[:, 4:-4, 4:-4, 4:-4] = b.U[:, 4:-4, 4:-4, 4:-4]
            else:
                G[:, 0, 4:-4, 4:-4] = b.U[:, 0, 4:-4, 4:-4]
            fa.append(torch.from_numpy(G).cuda())
        self.fa = fa
        self.fb = [torch.full_like(t, float("nan")) for t in fa]
        self.dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.dt_next = torch.zeros(1, dtype=torch.float64, device="cuda")

    def step(self, want_bad=False):
        dxf = tuple(v / 2 for v in self.dx)
        cin = [hb.box(t, s, self.dx) for t, s in zip(self.ca, self.csz)]
        cout = [hb.box(t, s, self.dx) for t, s in zip(self.cb, self.csz)]
        fin = [hb.box(t, s, dxf) for t, s in zip(self.fa, self.fsz)]
        fout = [hb.box(t, s, dxf) for t, s in zip(self.fb, self.fsz)]
        bad = self.ctx.hydro_amr_advance(cin, cout, self.clo, fin, fout, self.flo, self.dim, self.domain, self.bc,
                                         self.p, self.dt, self.dt_next, want_bad=want_bad)
        self.ca, self.cb = self.cb, self.ca
        self.fa, self.fb = self.fb, self.fa
        self.dt.copy_(self.dt_next)
        return bad

    def coarse(self):
        return _untile([t.cpu().numpy() for t in self.ca], self.clo, self.csz, self.dim, self.domain)

    def fine(self, b):
        return _interior(self.fa[b].cpu().numpy(), self.dim)


def _case(dim):
    if dim == 3:
        domain = (24, 24, 24)
        flo, fn = [(12, 12, 12), (24, 12, 12)], [(12, 12, 12), (12, 8, 12)]
        bc = ((PER, PER), (R, R), (O, O))
    else:
        domain = (32, 32)
        flo, fn = [(20, 20, 0), (36, 20, 0), (20, 32, 0)], [(16, 12, 1), (8, 20, 1), (12, 8, 1)]
        bc = ((O, R), (PER, PER), (O, O))
    clo, csz = inputs.level_tiling(domain, sides=(8, 16), seed=3 + dim)
    if dim == 2:
        clo = [(x, y, 0) for x, y, _ in clo]
    return domain, flo, fn, bc, clo, csz


@pytest.mark.parametrize("variant,dim", [("exact", 3), ("default", 3), ("exact", 2), ("default", 2)])
def test_amr_advance_matches_oracle(variant, dim):
    domain, flo, fn, bc, clo, csz = _case(dim)
    Uc, Uf, dx = inputs.amr_two_level(domain, dim, flo, fn, gamma=1.4)
    fines = [amr.FineBox(lo, n, U) for lo, n, U in zip(flo, fn, Uf)]
    ctx = hb.Context(0, variant)
    p = hb.params(dim, gamma=1.4, cfl=0.5)
    H = Hierarchy(ctx, dim, domain, bc, Uc, clo, csz, fines, dx, p)
    dt0 = 0.3 * dx[0] / 4.0
    H.dt.fill_(dt0)
    steps = 3
    C, F, d = Uc, fines, dt0
    gpu_dts, ora_dts = [], []
    for _ in range(steps):
        assert H.step(want_bad=True) == 0
        gpu_dts.append(H.dt.item())
        C, F, d, bad = amr.advance(C, F, d, dim, domain, bc, dx, gamma=1.4, cfl=0.5)
        assert not bad
        ora_dts.append(d)
    gc = H.coarse()
    gf = [H.fine(b) for b in range(len(F))]
    ctx.close()
    wc = _interior(C, dim).reshape(gc.shape)
    if variant == "exact":
        assert gpu_dts == ora_dts
        assert np.array_equal(gc, wc)
        for g, B in zip(gf, F):
            assert np.array_equal(g, _interior(B.U, dim))
    else:
        assert np.allclose(gpu_dts, ora_dts, rtol=1e-12, atol=0)
        assert np.all(rel_linf(gc, wc) <= 1e-10)
        for g, B in zip(gf, F):
            assert np.all(rel_linf(g, _interior(B.U, dim)) <= 1e-10)


def _bench_hierarchy():
    """The benchmarked hierarchy: a 128^3 coarse level in 64^3 boxes with a
    blast at the centre, refined over the central 64^3 coarse zones by eight
    64^3 fine boxes (128^3 fine zones)."""
    domain = (128, 128, 128)
    clo = [(x, y, z) for z in (0, 64) for y in (0, 64) for x in (0, 64)]
    csz = [(64, 64, 64)] * 8
    flo = [(x, y, z) for z in (64, 128) for y in (64, 128) for x in (64, 128)]
    fn = [(64, 64, 64)] * 8
    return domain, clo, csz, flo, fn


def test_amr_conserves_at_bench_size():
    domain, clo, csz, flo, fn = _bench_hierarchy()
    Uc, Uf, dx = inputs.amr_two_level(domain, 3, flo, fn, gamma=1.4, p_amp=20.0, r0=0.08)
    fines = [amr.FineBox(lo, n, U) for lo, n, U in zip(flo, fn, Uf)]
    del Uf
    ctx = hb.Context(0)
    p = hb.params(3, gamma=1.4, cfl=0.5)
    bc = ((PER, PER),) * 3
    H = Hierarchy(ctx, 3, domain, bc, Uc, clo, csz, fines, dx, p)
    del fines

    def totals():
        """(composite totals, coarse totals, normaliser): composite = the
        coarse zones outside the refined region [32, 96)^3 plus the fine
        zones at 1/8 of the coarse volume."""
        c = torch.stack([t[:, 4:-4, 4:-4, 4:-4].sum(dim=(1, 2, 3)) for t in H.ca]).sum(0)
        covered = torch.zeros(5, dtype=torch.float64, device="cuda")
        for t, lo in zip(H.ca, clo):
            sl = [slice(max(32 - lo[a], 0) + 4, min(96 - lo[a], 64) + 4) for a in (2, 1, 0)]
            covered += t[:, sl[0], sl[1], sl[2]].sum(dim=(1, 2, 3))
        f = torch.stack([t[:, 4:-4, 4:-4, 4:-4].sum(dim=(1, 2, 3)) for t in H.fa]).sum(0)
        scale = torch.stack([t[:, 4:-4, 4:-4, 4:-4].abs().sum(dim=(1, 2, 3)) for t in H.ca]).sum(0)
        return (c - covered + f / 8.0).cpu().numpy(), c.cpu().numpy(), scale.cpu().numpy()

    t0, _, scale = totals()
    H.dt.fill_(0.3 * dx[0] / 8.0)
    for _ in range(3):
        assert H.step(want_bad=True) == 0
    t1, c1, _ = totals()
    ctx.close()
    scale = np.where(scale > 0, scale, 1.0)
    assert np.all(np.abs(t1 - t0) / scale <= 1e-13), np.abs(t1 - t0) / scale
    # after the average down the coarse level alone carries the composite totals
    assert np.all(np.abs(c1 - t1) / scale <= 1e-13)


def test_amr_rejects_bad_hierarchies():
    domain, flo, fn, bc, clo, csz = _case(3)
    Uc, Uf, dx = inputs.amr_two_level(domain, 3, flo, fn)
    ctx = hb.Context(0)
    p = hb.params(3, gamma=1.4)
    ca = [torch.from_numpy(T).cuda() for T in _tile(Uc, clo, csz, 3)]
    cb = [torch.empty_like(t) for t in ca]
    cin = [hb.box(t, s, dx) for t, s in zip(ca, csz)]
    cout = [hb.box(t, s, dx) for t, s in zip(cb, csz)]
    dxf = tuple(v / 2 for v in dx)
    dt = torch.full((1,), 1e-3, dtype=torch.float64, device="cuda")
    dn = torch.zeros_like(dt)

    def run(lo, n, fdx=dxf, params=p):
        fa = [torch.zeros((5, s[2] + 8, s[1] + 8, s[0] + 8), dtype=torch.float64, device="cuda") for s in n]
        fb = [torch.zeros_like(t) for t in fa]
        ctx.hydro_amr_advance(cin, cout, clo, [hb.box(t, s, fdx) for t, s in zip(fa, n)],
                              [hb.box(t, s, fdx) for t, s in zip(fb, n)], lo, 3, domain, bc, params, dt, dn)

    for lo, n in [([(13, 12, 12)], [(8, 8, 8)]),                       # odd corner
                  ([(12, 12, 12)], [(9, 8, 8)]),                       # odd size
                  ([(4, 12, 12)], [(8, 8, 8)]),                        # too close to the boundary
                  ([(12, 12, 12), (16, 12, 12)], [(8, 8, 8)] * 2)]:    # overlap
        with pytest.raises(hb.HydroError) as e:
            run(lo, n)
        assert e.value.status == hb.HYDRO_EINVAL
    with pytest.raises(hb.HydroError) as e:   # fine spacing is not half the coarse one
        run([(12, 12, 12)], [(8, 8, 8)], fdx=dx)
    assert e.value.status == hb.HYDRO_EINVAL
    with pytest.raises(hb.HydroError) as e:
        run([(12, 12, 12)], [(8, 8, 8)], params=hb.params(3, gamma=1.4, grav=(0, 0, -1), flux_grav_energy=True))
    assert e.value.status == hb.HYDRO_ENOTIMPL
    # a valid one runs
    run([(12, 12, 12)], [(8, 8, 8)])
    torch.cuda.synchronize()
    ctx.close()
