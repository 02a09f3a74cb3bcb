"""The slab-by-slab step (a context scratch limit smaller than the whole-box
scratch): bitwise the whole-box step, in both builds, for every kind of z
boundary, for slabs of one plane up to most of the box, with the face fluxes
recorded slab by slab equal to the whole-box ones; and within the parity
tolerance of the CPU oracle.  The host-buffer step takes the same path."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import interior, rel_linf, to_dev
from paper_1711_06203_b300 import binding as hb
from paper_1711_06203_b300 import inputs

pytestmark = pytest.mark.gpu

O, R, PER, PRE = hb.BC_OUTFLOW, hb.BC_REFLECT, hb.BC_PERIODIC, hb.BC_PREFILLED


def _plane_bytes(n):
    """Scratch bytes of one grown z-plane (rows padded to even length)."""
    return ((n[0] + 8 + 1) & ~1) * (n[1] + 8) * 123 * 8


def _step(ctx, U, n, dx, bc, p, dt, faces=True):
    a = to_dev(U)
    b = torch.full_like(a, float("nan"))
    ctx.hydro_ctx_record_face_fluxes(faces)
    dn = ctx.hydro_advance_box(hb.box(a, n, dx, bc), hb.box(b, n, dx, bc), p, dt, want_dt_next=True)
    out = {}
    if faces:
        for ax in range(3):
            t = [x for x in range(3) if x != ax]
            for side in (0, 1):
                f = torch.empty((5, n[t[1]], n[t[0]]), dtype=torch.float64, device="cuda")
                ctx.hydro_ctx_face_flux(ax, side, f)
                out[ax, side] = f.cpu().numpy()
    return b.cpu().numpy(), dn, out


BCS = [((O, R), (PER, PER), (R, O)), ((R, R), (O, PRE), (PER, PER)), ((PER, PER), (R, O), (PRE, PRE)),
       ((O, O), (O, O), (O, O))]


@pytest.mark.parametrize("variant", ["exact", "default"])
@pytest.mark.parametrize("bci", range(len(BCS)))
def test_slabs_equal_whole_box(variant, bci):
    rng = np.random.default_rng(100 + bci)
    n = (23, 18, 37)
    bc = BCS[bci]
    U = inputs.random_box(rng, n, 3)
    dx = (1 / 23, 1 / 18, 1 / 37)
    p = hb.params(3, gamma=5 / 3, grav=(0.1, -0.2, 0.3))
    P = oracle.params(3, n, dx=dx, bc=bc, gamma=5 / 3)
    dt = 0.4 * oracle.dt(U, P)[0]
    ctx = hb.Context(0, variant)
    ctx.hydro_ctx_set_scratch_limit(0)
    whole, dn, fw = _step(ctx, U, n, dx, bc, p, dt)
    # slabs of 1, 4, 7, 13 and 33 planes (T + 8 planes fit the limit)
    for T in (1, 4, 7, 13, 33):
        ctx.hydro_ctx_set_scratch_limit((T + 8) * _plane_bytes(n))
        got, dn_s, fs = _step(ctx, U, n, dx, bc, p, dt)
        assert np.array_equal(interior(got, 3), interior(whole, 3)), T
        assert dn_s == dn
        for k in fw:
            assert np.array_equal(fs[k], fw[k]), (T, k)
    ctx.close()


def test_slabs_match_oracle_and_host_path():
    rng = np.random.default_rng(9)
    n = (20, 17, 29)
    bc = ((O, O), (R, R), (PER, PER))
    U = inputs.random_box(rng, n, 3)
    dx = (0.05,) * 3
    P = oracle.params(3, n, dx=dx, bc=bc, gamma=5 / 3)
    d, _ = oracle.dt(U, P)
    ref, rc = oracle.step(U, P, d)
    assert rc == 0
    ctx = hb.Context(0)
    ctx.hydro_ctx_set_scratch_limit(12 * _plane_bytes(n))  # slabs of 4 planes
    got, dn, _ = _step(ctx, U, n, dx, bc, hb.params(3, gamma=5 / 3), d, faces=False)
    assert np.all(rel_linf(interior(got, 3), interior(ref, 3)) <= 1e-10)
    dref, _ = oracle.dt(ref, P)
    assert abs(dn - dref) <= 1e-10 * dref
    # the host-buffer step of a box over the limit takes the slab path too
    hin = torch.from_numpy(U.copy()).pin_memory()
    hout = torch.full_like(hin, float("nan")).pin_memory()
    dn_h = ctx.hydro_advance_box_host(hb.box(hin, n, dx, bc), hb.box(hout, n, dx, bc), hb.params(3, gamma=5 / 3), d,
                                      want_dt_next=True)
    assert dn_h == dn
    assert np.array_equal(interior(hout.numpy(), 3), interior(got, 3))
    ctx.close()
