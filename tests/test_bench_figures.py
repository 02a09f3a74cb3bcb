"""Host arithmetic behind bench.py's roofline figures (no GPU needed): the
algorithmic bytes of a step and the units each stage processes."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_figures_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("n,bytes_per_update", [(16, 175.0), (64, 96.9), (128, 87.9), (512, 81.9)])
def test_algorithmic_bytes_per_zone_update(n, bytes_per_update):
    # read the 5 FP64 fields of the grown box (4 ghosts a side) once, write the 5 interior fields once;
    # the expected figures are given to one decimal, truncated
    b = _bench()
    got = b.algorithmic_bytes_per_step(n) / n ** 3
    assert bytes_per_update <= got < bytes_per_update + 0.1


def test_stage_units_count_faces_and_sweeps():
    b = _bench()
    n = 96
    u = b.units_per_step(n)
    # counted directly: sweeps over [-1, n] in all three axes, faces [0, n] along d
    sweep = 3 * sum(1 for _ in range(-1, n + 1)) ** 3
    first = sum((n + 1) * (n + 2) * (n + 2) for _ in range(3))
    inter = sum((n + 1) * n * (n + 2) for d in range(3) for t in range(3) if t != d)
    final = sum((n + 1) * n * n for _ in range(3))
    assert u["trace"] == sweep
    assert (u["flux1"], u["flux2"], u["flux3"]) == (first, inter, final)
    # the solve counts the 96^3 captures quote
    assert (u["flux1"], u["flux2"], u["flux3"]) == (2_794_764, 5_475_456, 2_681_856)
    assert u["prim"] == (n + 8) ** 3 and u["update"] == n ** 3


def test_derived_fp64_peak():
    b = _bench()
    assert b.FP64_PEAK_GFLOPS == pytest.approx(148 * 2 * 2 * 2.032)
