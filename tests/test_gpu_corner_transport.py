"""The corner-transport corrections of the CUDA step (Sec. 3.2, unsplit PPM) on
the two exact solutions that pin the oracle's transverse terms: a product
profile (bilinear in 2-D, trilinear in 3-D) advected by a uniform oblique
velocity for one CFL step, and a random density moved by exactly one zone
along every axis at unit Courant number.

For each case the contraction-free build is bitwise equal to the oracle, the
product build is within 1e-10 of it (normwise relative L-infinity per field),
and both builds reproduce the exact translated solution to 1e-13.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import gpu_steps, interior, rel_linf
from paper_1711_06203_b300 import binding as hb
from paper_1711_06203_b300 import inputs

pytestmark = pytest.mark.gpu

N = {3: (12, 10, 8), 2: (12, 10, 1)}
VEL = (0.7, 0.4, -0.3)


def _product_case(dim):
    n, dx = N[dim], (1 / 12, 1 / 12, 1 / 12)
    U0 = inputs.product_profile(n, dim, dx, VEL)
    P = oracle.params(dim, n, dx=dx, bc=oracle.BC_PREFILLED, gamma=1.4)
    d, rc = oracle.dt(U0, P)
    assert rc == 0
    return U0, n, dx, P, d, inputs.product_profile(n, dim, dx, VEL, t=d)


def _translation_case(dim, signs):
    n, dx, d = N[dim], (1 / 12, 1 / 10, 1 / 8), 0.05
    U0, want = inputs.translation_box(np.random.default_rng(17), n, dim, dx, d, signs)
    P = oracle.params(dim, n, dx=dx, bc=oracle.BC_PREFILLED, gamma=1.4)
    return U0, n, dx, P, d, want


CASES = [("product", 3, None), ("product", 2, None), ("unit_courant", 3, (1, 1, 1)),
         ("unit_courant", 3, (1, -1, 1)), ("unit_courant", 3, (-1, 1, -1)), ("unit_courant", 2, (-1, 1, 1))]


@pytest.mark.parametrize("kind,dim,signs", CASES)
def test_corner_transport_exact_solutions(kind, dim, signs):
    U0, n, dx, P, d, want = _product_case(dim) if kind == "product" else _translation_case(dim, signs)
    ref, rc = oracle.step(U0, P, d)
    assert rc == 0
    ex, _ = gpu_steps(U0, dim, n, dx, hb.BC_PREFILLED, 1.4, [d], variant="exact")
    assert np.array_equal(interior(ex, dim), interior(ref, dim))
    got, _ = gpu_steps(U0, dim, n, dx, hb.BC_PREFILLED, 1.4, [d])
    assert np.all(rel_linf(interior(got, dim), interior(ref, dim)) <= 1e-10)
    for res in (ex, got):
        assert np.all(rel_linf(interior(res, dim), interior(want, dim)) <= 1e-13)
