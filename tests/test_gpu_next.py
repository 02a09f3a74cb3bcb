"""Extensions beyond the base step (the ranked 'next' items of the hot-path
scope): the retry mechanism, Einfeldt wave speeds, flux-based gravity energy."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import rel_linf
from paper_1711_06203_b300 import binding as hb
from paper_1711_06203_b300 import inputs

pytestmark = pytest.mark.gpu

I3 = (slice(None), slice(4, -4), slice(4, -4), slice(4, -4))


def test_retry_halves_dt_until_the_step_is_physical():
    # pressure ratio 1e5: 8x the CFL step produces negative pressure, 4x does not
    n = 32
    U = inputs.two_state(n, 3, 1.4, 1.0, 1000.0, 1.0, 0.01)
    P = oracle.params(3, (n, n, n), gamma=1.4, cfl=0.5)
    d, _ = oracle.dt(U, P)
    ctx = hb.Context(0)
    a = torch.from_numpy(U).cuda()
    b = torch.empty_like(a)
    box = lambda t: hb.box(t, (n, n, n), (1.0 / n,) * 3, hb.BC_OUTFLOW)
    p = hb.params(3, gamma=1.4, cfl=0.5)
    rc, taken, nxt = ctx.hydro_advance_box_retry(box(a), box(b), p, 8 * d, max_retries=0)
    assert rc == hb.HYDRO_EBADSTATE
    rc, taken, nxt = ctx.hydro_advance_box_retry(box(a), box(b), p, 8 * d, max_retries=4)
    assert rc == hb.HYDRO_OK and taken == 4 * d
    ref, rcode = oracle.step(U, P, 4 * d)
    assert rcode == 0
    assert np.all(rel_linf(b.cpu().numpy()[I3], ref[I3]) <= 1e-10)
    dref, _ = oracle.dt(ref, P)
    assert abs(nxt - dref) <= 1e-10 * dref
    ctx.close()


OPTION_CASES = [
    ("einfeldt", dict(einfeldt=True), (0.0, 0.0, 0.0), hb.BC_PERIODIC),
    ("flux_grav", dict(flux_grav_energy=True), (0.3, -0.5, -2.0), hb.BC_REFLECT),
    ("both", dict(einfeldt=True, flux_grav_energy=True), (0.0, 0.0, -1.0), hb.BC_REFLECT),
]


@pytest.mark.parametrize("name,opts,grav,bc", OPTION_CASES)
@pytest.mark.parametrize("variant", ["exact", "default"])
def test_options_match_oracle(name, opts, grav, bc, variant):
    n = (14, 11, 9)
    rng = np.random.default_rng(31)
    U = inputs.random_box(rng, n, 3)
    dx = (1 / 14, 1 / 11, 1 / 9)
    P = oracle.params(3, n, dx=dx, bc=bc, gamma=5 / 3, grav=grav,
                      einfeldt=opts.get("einfeldt", False), flux_grav_energy=opts.get("flux_grav_energy", False))
    d, _ = oracle.dt(U, P)
    ref, rc = oracle.step(U, P, d)
    assert rc == 0
    ctx = hb.Context(0, variant)
    a = torch.from_numpy(U).cuda()
    b = torch.empty_like(a)
    p = hb.params(3, gamma=5 / 3, grav=grav, **opts)
    ctx.hydro_advance_box(hb.box(a, n, dx, bc), hb.box(b, n, dx, bc), p, d, want_dt_next=True)
    got = b.cpu().numpy()
    ctx.close()
    if variant == "exact":
        assert np.array_equal(got[I3], ref[I3])
    else:
        assert np.all(rel_linf(got[I3], ref[I3]) <= 1e-10)
