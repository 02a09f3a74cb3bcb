"""The overlapped host-buffer step's schedule (hydro_pipe_plan, host only, no
GPU): for every box height, chunk count and low z boundary kind, each stage
covers its range exactly once, reads only what earlier launches formed (the
stencils of the scheme: the z tracing reaches 3 planes up and down, a z-face
needs the two zones beside it, a zone's update its two z-faces), and the
front stages of a chunk never write what the back stages of an earlier
chunk read (the two run side by side on two streams)."""
import pytest

from paper_1711_06203_b300 import binding as hb
from paper_1711_06203_b300 import build as hbuild

NG = 4


@pytest.fixture(scope="module", autouse=True)
def built():
    hbuild.build()  # compiles only when a source is newer than the library


SRC_LOW = {0: lambda nz, m: [0], 1: lambda nz, m: [m - 1], 2: lambda nz, m: [nz - m]}


def _check(nz, C, bc):
    pre, plan = hb.hydro_pipe_plan(nz, C, bc)
    landed = set(range(pre, nz))
    done = {k: set() for k in ("Q", "xy", "tz", "f1z", "f2xz", "f2z", "f3xy", "f3z", "upd")}
    front_writes, back_reads = [], []

    def run(stage, rng, needs, writes=None, reads=None):
        for z in range(*rng):
            assert z not in done[stage], (stage, z, "twice")
            for what, zz in needs(z):
                have = landed if what == "in" else done[what]
                assert zz in have, (stage, z, "needs", what, zz)
            done[stage].add(z)
            if writes is not None:
                writes.add((stage, z))
            if reads is not None:
                reads.update(needs(z))

    for k, c in enumerate(plan):
        lo, hi = c["h2d"]
        assert not (set(range(lo, hi)) & landed)
        landed |= set(range(lo, hi))
        W, R = set(), set()
        run("Q", c["prim"], lambda z: [("in", z)], W)
        if c["ghosts_low"]:
            run("Q", (-NG, 0), lambda z: [("in", s) for s in SRC_LOW[bc](nz, -z)], W)
        if c["ghosts_high"]:
            run("Q", (nz, nz + NG), lambda z: [("in", s) for s in range(nz)], W)
        # front stages
        run("xy", c["xy"], lambda z: [("Q", z)], W)
        run("tz", c["tz"], lambda z: [("Q", z + d) for d in range(-3, 4)], W)
        run("f1z", c["f1z"], lambda f: [("tz", f - 1), ("tz", f)], W)
        front_writes.append(W)
        # back stages; ("xy", z): the x/y first fluxes and conserved traced
        # states of plane z, ("f1z", f): the first z flux of face f and the
        # conserved traced states of the zones beside it
        run("f2xz", c["f2xz"], lambda z: [("xy", z), ("f1z", z), ("f1z", z + 1)], None, R)
        run("f2z", c["f2z"], lambda f: [("f1z", f), ("xy", f - 1), ("xy", f)], None, R)
        run("f3xy", c["f3xy"], lambda z: [("xy", z), ("f2xz", z), ("f2z", z), ("f2z", z + 1)], None, R)
        run("f3z", c["f3z"], lambda f: [("f1z", f), ("xy", f - 1), ("xy", f)], None, R)
        run("upd", c["upd"], lambda z: [("f3xy", z), ("f3z", z), ("f3z", z + 1), ("in", z)], None, R)
        back_reads.append(R)

    assert landed == set(range(nz))
    assert done["Q"] == set(range(-NG, nz + NG))
    for stage, rng in (("xy", (-1, nz + 1)), ("tz", (-1, nz + 1)), ("f1z", (0, nz + 1)), ("f2xz", (0, nz)),
                       ("f2z", (0, nz + 1)), ("f3xy", (0, nz)), ("f3z", (0, nz + 1)), ("upd", (0, nz))):
        assert done[stage] == set(range(*rng)), stage
    for j in range(C):
        for k in range(j + 1, C):
            assert not (front_writes[k] & back_reads[j]), (j, k, sorted(front_writes[k] & back_reads[j])[:4])


@pytest.mark.parametrize("bc", [hb.BC_OUTFLOW, hb.BC_REFLECT, hb.BC_PERIODIC])
def test_schedule_covers_once_in_dependency_order(bc):
    for nz in list(range(4, 50)) + [64, 100, 128, 129, 256]:
        for C in range(1, min(16, nz) + 1):
            _check(nz, C, bc)


def test_schedule_overlaps_and_trails_by_a_few_planes():
    """Sedov 128^3 with 8 chunks: the update starts with the first chunk and
    trails the landed planes by the z stencil plus at most a tile."""
    pre, plan = hb.hydro_pipe_plan(128, 8, hb.BC_OUTFLOW)
    assert pre == 128
    assert plan[0]["upd"][1] > 0
    for c in plan[:-1]:
        assert c["prim"][1] - c["upd"][1] <= 6 + 12


def test_schedule_rejects_bad_arguments():
    for args in ((3, 1, 0), (16, 0, 0), (16, 17, 0), (8, 9, 0), (16, 4, 3), (16, 4, -1)):
        with pytest.raises(hb.HydroError):
            hb.hydro_pipe_plan(*args)
