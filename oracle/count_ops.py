"""Algorithmic FP64 operation counts per unit of each stage of the step,
tallied by the counting build of the oracle (test infrastructure).

    python -m oracle.count_ops [n] [steps]

advances the Sedov 128^3 workload (or side n) `steps` oracle steps, then
counts one step: prints, per stage, flops (+ - * / sqrt) per unit and the
units per step (grown zone, zone-direction, Riemann solve, interior zone).
"""
import sys

import numpy as np

from . import count_ops_by_stage, dt, params, run
from paper_1711_06203_b300 import inputs


def units(n):
    return {"prim": (n + 8) ** 3, "trace": 3 * (n + 2) ** 3, "flux1": 3 * (n + 1) * (n + 2) ** 2,
            "flux2": 6 * (n + 1) * n * (n + 2), "flux3": 3 * (n + 1) * n * n, "update": n ** 3}


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 128
    steps = int(sys.argv[2]) if len(sys.argv) > 2 else 20
    U, _ = inputs.sedov(n)
    P = params(3, (n, n, n), gamma=1.4, cfl=0.5)
    U, _, _ = run(U, P, steps)
    d, _ = dt(U, P)
    c = count_ops_by_stage(U, P, d)
    u = units(n)
    total = 0
    print(f"Sedov {n}^3 after {steps} steps: algorithmic FP64 operations per unit")
    for k, v in c.items():
        fl = v["add"] + v["mul"] + v["div"] + v["sqrt"]
        total += fl
        print(f"  {k:7s} units/step {u[k]:>10d}  flops/unit {fl / u[k]:8.2f}  (add {v['add'] / u[k]:.2f} "
              f"mul {v['mul'] / u[k]:.2f} div {v['div'] / u[k]:.3f} sqrt {v['sqrt'] / u[k]:.3f}; "
              f"compares {v['cmp'] / u[k]:.2f})")
    print(f"  total flops per zone-update {total / n ** 3:.1f}")


if __name__ == "__main__":
    main()
