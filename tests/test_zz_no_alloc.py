"""The allocation-free step, hydro_advance_box_noalloc.

It exists for callers that cannot allocate device memory while they run:
hosts that have reserved the whole GPU themselves, real-time loops that must
not stall on the synchronisation an allocation may bring, and plug-ins whose
host application owns all allocations.  It runs the same kernels as
hydro_advance_box, with scratch in fixed library storage shared by every call.

Checked here through the C ABI: two calls in a row (different boxes, so the
second call starts from the first call's leftover scratch) agree with
hydro_advance_box and with the CPU oracle to the parity tolerance used
throughout (normwise relative L-infinity <= 1e-10; the two GPU paths are
expected to be identical), the returned CFL step agrees; a box whose scratch
grid fills the fixed storage exactly (32^3) agrees too; a box beyond the
fixed storage is refused with HYDRO_ETOOBIG; a bad state raised by a call
without dt_next_host is reported by the next call that passes one.  This
file runs last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1711_06203_b300 import binding as hb
from paper_1711_06203_b300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _rel_linf(a, b):
    a, b = a.reshape(5, -1), b.reshape(5, -1)
    den = np.abs(b).max(axis=1)
    return np.abs(a - b).max(axis=1) / np.where(den > 0, den, 1.0)


def _interior(t, dim):
    x = t.cpu().numpy()
    return x[:, 4:-4, 4:-4, 4:-4] if dim == 3 else x[:, 0, 4:-4, 4:-4]


def _oracle_interior(U, dim, n, dx, bc, gamma, dt):
    P = oracle.params(dim, n[:dim], dx=dx, bc=bc, gamma=gamma)
    ref, rc = oracle.step(U, P, dt)
    assert rc == 0
    return ref[:, 4:-4, 4:-4, 4:-4] if dim == 3 else ref[:, 0, 4:-4, 4:-4]


def _both_paths(U, dim, n, dx, bc, gamma, dt):
    p = hb.params(dim, gamma=gamma)
    a = torch.from_numpy(U).to("cuda")
    ref_out = torch.full_like(a, float("nan"))
    ctx = hb.Context(0)
    dref = ctx.hydro_advance_box(hb.box(a, n, dx, bc), hb.box(ref_out, n, dx, bc), p, dt, want_dt_next=True)
    ctx.close()
    out = torch.full_like(a, float("nan"))
    rc, dn = hb.hydro_advance_box_noalloc(hb.box(a, n, dx, bc), hb.box(out, n, dx, bc), p, dt, want_dt_next=True)
    torch.cuda.synchronize()
    return rc, _interior(out, dim), _interior(ref_out, dim), dn, dref


def test_noalloc_matches_advance_box_on_two_calls_in_a_row():
    torch.cuda.set_device(0)
    rng = np.random.default_rng(2024)
    # call 1: a ragged 3-D box with caller-filled ghosts (grown 32 x 28 x 24 zones)
    n1 = (24, 20, 16)
    U1 = inputs.random_box(rng, n1, 3)
    rc, got, ref, dn, dref = _both_paths(U1, 3, n1, (1 / 24, 1 / 20, 1 / 16), hb.BC_PREFILLED, 5 / 3, 2e-3)
    assert rc == hb.HYDRO_OK
    assert np.all(_rel_linf(got, ref) <= TOL)
    assert abs(dn - dref) <= TOL * dref
    orc = _oracle_interior(U1, 3, n1, (1 / 24, 1 / 20, 1 / 16), oracle.BC_PREFILLED, 5 / 3, 2e-3)
    assert np.all(_rel_linf(got, orc) <= TOL)
    # call 2, straight after: a different shape and problem (2-D Sod, outflow)
    n2 = (64, 64, 1)
    U2 = inputs.sod(64, 2, 0)
    rc, got, ref, dn, dref = _both_paths(U2, 2, n2, (1 / 64,) * 3, hb.BC_OUTFLOW, 1.4, 4e-3)
    assert rc == hb.HYDRO_OK
    assert np.all(_rel_linf(got, ref) <= TOL)
    assert abs(dn - dref) <= TOL * dref
    orc = _oracle_interior(U2, 2, n2, (1 / 64,) * 3, oracle.BC_OUTFLOW, 1.4, 4e-3)
    assert np.all(_rel_linf(got, orc) <= TOL)


def test_noalloc_box_that_fills_the_storage_exactly():
    """32^3: scratch grid 40 x 40 x 40 = 64,000 zones, the whole storage, so
    the last scratch field ends right where the flag block starts."""
    rng = np.random.default_rng(77)
    n = (32, 32, 32)
    U = inputs.random_box(rng, n, 3)
    dx = (1 / 32,) * 3
    bc = ((hb.BC_PERIODIC,) * 2, (hb.BC_REFLECT, hb.BC_OUTFLOW), (hb.BC_PREFILLED,) * 2)
    rc, got, ref, dn, dref = _both_paths(U, 3, n, dx, bc, 5 / 3, 1e-3)
    assert rc == hb.HYDRO_OK
    assert np.all(_rel_linf(got, ref) <= TOL)
    assert abs(dn - dref) <= TOL * dref
    assert np.all(_rel_linf(got, _oracle_interior(U, 3, n, dx, bc, 5 / 3, 1e-3)) <= TOL)


def test_noalloc_bad_state_is_reported_by_the_next_syncing_call():
    rng = np.random.default_rng(5)
    n = (12, 10, 8)
    dx = (0.1,) * 3
    U = inputs.random_box(rng, n, 3)
    p = hb.params(3, gamma=5 / 3)
    good = torch.from_numpy(U).to("cuda")
    U[0, 4 + 3, 4 + 5, 4 + 6] = -1.0  # negative density in the interior
    bad = torch.from_numpy(U).to("cuda")
    out = torch.empty_like(good)
    box = lambda t: hb.box(t, n, dx, hb.BC_PREFILLED)
    # no dt_next_host: nothing is reported yet
    rc, _ = hb.hydro_advance_box_noalloc(box(bad), box(out), p, 1e-3, want_dt_next=False)
    assert rc == hb.HYDRO_OK
    # the next call that syncs reports it (on a good box), and clears it
    rc, _ = hb.hydro_advance_box_noalloc(box(good), box(out), p, 1e-3, want_dt_next=True)
    assert rc == hb.HYDRO_EBADSTATE
    rc, dn = hb.hydro_advance_box_noalloc(box(good), box(out), p, 1e-3, want_dt_next=True)
    assert rc == hb.HYDRO_OK and dn > 0
    # a bad state in a syncing call is reported by that call
    rc, _ = hb.hydro_advance_box_noalloc(box(bad), box(out), p, 1e-3, want_dt_next=True)
    assert rc == hb.HYDRO_EBADSTATE
    rc, _ = hb.hydro_advance_box_noalloc(box(good), box(out), p, 1e-3, want_dt_next=True)
    assert rc == hb.HYDRO_OK


def test_noalloc_refuses_boxes_beyond_its_storage():
    n = (33, 32, 32)  # scratch grid 42 x 40 x 40 = 67,200 zones > 64,000
    shape = inputs.grown_shape(n, 3)
    a = torch.ones((5,) + shape, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    rc, _ = hb.hydro_advance_box_noalloc(hb.box(a, n, (0.1,) * 3, hb.BC_PREFILLED),
                                         hb.box(b, n, (0.1,) * 3, hb.BC_PREFILLED), hb.params(3), 1e-3,
                                         want_dt_next=True)
    assert rc == hb.HYDRO_ETOOBIG
    assert "fixed storage" in hb.strerror(rc)
