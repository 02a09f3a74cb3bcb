"""Stray writes, caught without a sanitizer: boxes live inside larger buffers
poisoned with a marked NaN, as strided views that leave guard zones before
and after every row, plane and field.  After a step -- whole box, slab by
slab, batched, allocation-free -- the input buffer is bitwise unchanged, the
output buffer outside the box's grown zones still holds the poison, and the
interior is bitwise what contiguous boxes give, with no NaN in it."""
import numpy as np
import pytest
import torch

from gpu_helpers import interior, to_dev
from paper_1711_06203_b300 import binding as hb
from paper_1711_06203_b300 import inputs

pytestmark = pytest.mark.gpu

O, R, PER, PRE = hb.BC_OUTFLOW, hb.BC_REFLECT, hb.BC_PERIODIC, hb.BC_PREFILLED
POISON_BITS = 0x7FF8DEADBEEF0001  # a quiet NaN with a payload, set and compared as bits


def _guarded(shape, U=None):
    """A poisoned buffer holding a box of `shape` (U copied in, if given) as a
    strided view with guard zones on every side."""
    c, gz, gy, gx = shape
    big = torch.full((c, gz + 3, gy + 4, gx + 5), POISON_BITS, dtype=torch.int64, device="cuda").view(torch.float64)
    view = big[:, 1:gz + 1, 2:gy + 2, 3:gx + 3]
    if U is not None:
        view.copy_(torch.from_numpy(U))
    return big, view


def _guard_untouched(big_out, shape):
    c, gz, gy, gx = shape
    mask = torch.ones(big_out.shape, dtype=torch.bool, device=big_out.device)
    mask[:, 1:gz + 1, 2:gy + 2, 3:gx + 3] = False
    return bool((big_out.view(torch.int64)[mask] == POISON_BITS).all())


@pytest.mark.parametrize("mode", ["whole", "slabs"])
def test_single_box_writes_only_its_box(mode):
    rng = np.random.default_rng(3)
    n, dx, bc = (21, 14, 17), (0.05, 0.06, 0.07), ((O, R), (PER, PER), (R, O))
    U = inputs.random_box(rng, n, 3)
    p = hb.params(3, gamma=5 / 3, grav=(0.0, -0.3, 0.1))
    ctx = hb.Context(0)
    if mode == "slabs":
        ctx.hydro_ctx_set_scratch_limit(1)  # one plane per slab
    a, b = to_dev(U), torch.empty_like(to_dev(U))
    dt = ctx.hydro_dt(hb.box(a, n, dx, bc), p)
    ref_dt = ctx.hydro_advance_box(hb.box(a, n, dx, bc), hb.box(b, n, dx, bc), p, dt, want_dt_next=True)
    ref = b.cpu().numpy()
    big_in, vin = _guarded(U.shape, U)
    big_out, vout = _guarded(U.shape)
    before = big_in.view(torch.int64).clone()
    got_dt = ctx.hydro_advance_box(hb.box(vin, n, dx, bc), hb.box(vout, n, dx, bc), p, dt, want_dt_next=True)
    torch.cuda.synchronize()
    ctx.close()
    assert torch.equal(big_in.view(torch.int64), before)
    assert _guard_untouched(big_out, U.shape)
    got = vout.cpu().numpy()
    assert not np.isnan(interior(got, 3)).any()
    assert np.array_equal(interior(got, 3), interior(ref, 3))
    assert got_dt == ref_dt


def test_batched_level_writes_only_its_boxes():
    rng = np.random.default_rng(4)
    sizes = [(16, 24, 16), (24, 16, 32), (32, 32, 16)]
    dx = (1 / 64,) * 3
    p = hb.params(3, gamma=5 / 3)
    Us = [inputs.random_box(rng, s, 3) for s in sizes]
    dt_dev = torch.full((len(sizes),), 1e-4, dtype=torch.float64, device="cuda")
    ctx = hb.Context(0)
    ins = [to_dev(U) for U in Us]
    outs = [torch.empty_like(x) for x in ins]
    ctx.hydro_advance_batch([hb.box(x, s, dx, PRE) for x, s in zip(ins, sizes)],
                            [hb.box(y, s, dx, PRE) for y, s in zip(outs, sizes)], p, dt_dev)
    refs = [y.cpu().numpy() for y in outs]
    guarded_in = [_guarded(U.shape, U) for U in Us]
    guarded_out = [_guarded(U.shape) for U in Us]
    before = [g[0].view(torch.int64).clone() for g in guarded_in]
    ctx.hydro_advance_batch([hb.box(g[1], s, dx, PRE) for g, s in zip(guarded_in, sizes)],
                            [hb.box(g[1], s, dx, PRE) for g, s in zip(guarded_out, sizes)], p, dt_dev)
    torch.cuda.synchronize()
    ctx.close()
    for (big_in, _), b0, (big_out, vout), U, ref in zip(guarded_in, before, guarded_out, Us, refs):
        assert torch.equal(big_in.view(torch.int64), b0)
        assert _guard_untouched(big_out, U.shape)
        got = vout.cpu().numpy()
        assert not np.isnan(interior(got, 3)).any()
        assert np.array_equal(interior(got, 3), interior(ref, 3))


def test_allocation_free_step_writes_only_its_box():
    rng = np.random.default_rng(6)
    n, dx, bc = (20, 16, 12), (0.05,) * 3, ((O, O), (R, R), (PER, PER))
    U = inputs.random_box(rng, n, 3)
    p = hb.params(3, gamma=5 / 3)
    a, b = to_dev(U), torch.empty_like(to_dev(U))
    rc, ref_dt = hb.hydro_advance_box_noalloc(hb.box(a, n, dx, bc), hb.box(b, n, dx, bc), p, 1e-3, want_dt_next=True)
    assert rc == hb.HYDRO_OK
    ref = b.cpu().numpy()
    big_in, vin = _guarded(U.shape, U)
    big_out, vout = _guarded(U.shape)
    before = big_in.view(torch.int64).clone()
    rc, got_dt = hb.hydro_advance_box_noalloc(hb.box(vin, n, dx, bc), hb.box(vout, n, dx, bc), p, 1e-3,
                                              want_dt_next=True)
    assert rc == hb.HYDRO_OK
    torch.cuda.synchronize()
    assert torch.equal(big_in.view(torch.int64), before)
    assert _guard_untouched(big_out, U.shape)
    got = vout.cpu().numpy()
    assert np.array_equal(interior(got, 3), interior(ref, 3))
    assert got_dt == ref_dt
