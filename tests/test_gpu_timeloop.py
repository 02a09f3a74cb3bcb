"""The device-resident time loop, hydro_advance_box_steps: n CFL steps of one
box with the time step handed from step to step in device memory.

  * the 2-D Sod configuration (64^2, outflow, 50 steps): the contraction-free
    build is bitwise the oracle's own 50-step run (same states, same dts,
    same final time), the product build within 1e-10; the density is within
    the configuration's L1 gate of the exact Riemann solution and every row
    is identical;
  * a 3-D random box with mixed boundaries: bitwise the same as stepping it
    with hydro_advance_box in the contraction-free build;
  * an odd number of steps leaves the result in the second box, and
    prefilled faces are refused.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import interior, rel_linf, to_dev
from paper_1711_06203_b300 import binding as hb
from paper_1711_06203_b300 import inputs

pytestmark = pytest.mark.gpu

O, R, PER = hb.BC_OUTFLOW, hb.BC_REFLECT, hb.BC_PERIODIC


def _loop(variant, U, n, dx, bc, p, nsteps, dt0=None):
    ctx = hb.Context(0, variant)
    a = to_dev(U)
    b = torch.full_like(a, float("nan"))
    A, B = hb.box(a, n, dx, bc), hb.box(b, n, dx, bc)
    dt = torch.zeros(2, dtype=torch.float64, device="cuda")
    dt[0] = ctx.hydro_dt(A, p) if dt0 is None else dt0
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.hydro_advance_box_steps(A, B, p, nsteps, dt, t)
    torch.cuda.synchronize()
    assert ctx.hydro_ctx_check() == hb.HYDRO_OK
    res = (b if nsteps % 2 else a).cpu().numpy()
    ctx.close()
    return res, t.item(), dt[nsteps % 2].item()


@pytest.mark.parametrize("variant", ["exact", "default"])
def test_sod_configuration_time_loop(variant):
    n = 64
    U = inputs.sod(n, 2, 0)
    P = oracle.params(2, (n, n), bc=oracle.BC_OUTFLOW, gamma=1.4, cfl=0.5)
    ref, t_ref, dts = oracle.run(U, P, 50)
    got, t, dt_next = _loop(variant, U, (n, n, 1), (1 / n,) * 3, O, hb.params(2, gamma=1.4, cfl=0.5), 50)
    dref, _ = oracle.dt(ref, P)
    if variant == "exact":
        assert np.array_equal(interior(got, 2), interior(ref, 2))
        assert t == t_ref and dt_next == dref
    else:
        assert np.all(rel_linf(interior(got, 2), interior(ref, 2)) <= 1e-10)
        assert abs(t - t_ref) <= 1e-12 * t_ref
    rho = got[0, 0, 4:-4, 4:-4]
    assert np.all(rho == rho[0:1, :])
    x = (np.arange(n) + 0.5) / n
    W = oracle.exact_sample([1, 0, 1], [0.125, 0, 0.1], 1.4, (x - 0.5) / t)
    assert np.mean(np.abs(rho[0] - W[:, 0])) <= 1.5e-2


def test_time_loop_equals_stepping_one_call_at_a_time():
    rng = np.random.default_rng(41)
    n = (19, 14, 11)
    bc = ((O, R), (PER, PER), (R, O))
    U = inputs.random_box(rng, n, 3)
    dx = (0.05, 0.06, 0.07)
    p = hb.params(3, gamma=5 / 3, grav=(0.0, 0.0, -0.5))
    got, t, _ = _loop("exact", U, n, dx, bc, p, 7)
    ctx = hb.Context(0, "exact")
    a = to_dev(U)
    b = torch.empty_like(a)
    dt = ctx.hydro_dt(hb.box(a, n, dx, bc), p)
    t_ref = 0.0
    for _ in range(7):
        t_ref += dt
        dt = ctx.hydro_advance_box(hb.box(a, n, dx, bc), hb.box(b, n, dx, bc), p, dt, want_dt_next=True)
        a, b = b, a
    ref = a.cpu().numpy()
    ctx.close()
    assert np.array_equal(interior(got, 3), interior(ref, 3))
    assert t == t_ref


def test_checkpoint_and_resume_through_host_memory():
    """Checkpoint/resume: the state is the caller's box plus the time step, so
    twenty steps of the device loop equal ten steps, a copy of the state and
    the next dt to host memory and back into fresh buffers (a new context),
    and ten more -- bit for bit."""
    rng = np.random.default_rng(8)
    n, dx, bc = (18, 14, 12), (0.05, 0.06, 0.07), ((O, R), (PER, PER), (R, O))
    U = inputs.random_box(rng, n, 3)
    p = hb.params(3, gamma=5 / 3, grav=(0.0, 0.0, -0.4))
    whole, t_whole, _ = _loop("default", U, n, dx, bc, p, 20)
    half, t_half, dt_next = _loop("default", U, n, dx, bc, p, 10)
    saved = np.array(half, copy=True)  # the checkpoint: the state and the next dt, in host memory
    rest, t_rest, _ = _loop("default", saved, n, dx, bc, p, 10, dt0=dt_next)
    assert np.array_equal(interior(rest, 3), interior(whole, 3))
    assert t_half + t_rest == pytest.approx(t_whole, rel=1e-15)


def test_time_loop_refuses_prefilled_faces():
    n = (8, 8, 8)
    U = inputs.random_box(np.random.default_rng(0), n, 3)
    ctx = hb.Context(0)
    a = to_dev(U)
    b = torch.empty_like(a)
    dt = torch.full((2,), 1e-3, dtype=torch.float64, device="cuda")
    with pytest.raises(hb.HydroError) as e:
        ctx.hydro_advance_box_steps(hb.box(a, n, (0.1,) * 3, hb.BC_PREFILLED), hb.box(b, n, (0.1,) * 3, hb.BC_PREFILLED),
                                    hb.params(3), 3, dt)
    assert e.value.status == hb.HYDRO_EINVAL
    ctx.close()
