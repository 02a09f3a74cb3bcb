"""Continuous-batching server: results are the same alone and in a mix of
concurrently running requests, under both scheduling policies (bitwise: the
batched step's arithmetic for a box does not depend on the other boxes or on
which of them step with it), match the CPU oracle, and the request life cycle
(admission, polling, budget refusal, policy changes) behaves."""
import time

import numpy as np
import pytest

import oracle
from gpu_helpers import rel_linf
from paper_1711_06203_b300 import binding as hb
from paper_1711_06203_b300 import inputs

pytestmark = pytest.mark.gpu

I3 = (slice(None), slice(4, -4), slice(4, -4), slice(4, -4))


def _oracle_run(kind, n, steps, gamma, **kw):
    if kind == hb.PROB_SEDOV:
        U, _ = inputs.sedov(n, 3, gamma=gamma, E=kw.get("energy", 1.0), p_amb=kw.get("p_ambient", 1e-5))
    elif kind == hb.PROB_SOD:
        U = inputs.sod(n, 3, 0, gamma)
    else:
        U = inputs.two_state(n, 3, gamma, kw["rho_l"], kw["p_l"], kw["rho_r"], kw["p_r"])
    P = oracle.params(3, (n, n, n), gamma=gamma, cfl=0.5)
    ref, t, _ = oracle.run(U, P, steps)
    return ref, t


REQS = [
    dict(kind=hb.PROB_SOD, n=16, steps=6, gamma=1.4),
    dict(kind=hb.PROB_SEDOV, n=20, steps=5, gamma=1.4),
    dict(kind=hb.PROB_TWO_STATE, n=12, steps=9, gamma=5 / 3, rho_l=2.3, p_l=0.7, rho_r=0.4, p_r=1.9),
    dict(kind=hb.PROB_TWO_STATE, n=24, steps=3, gamma=1.4, rho_l=0.5, p_l=3.0, rho_r=1.5, p_r=0.2),
]


def test_served_results_match_oracle():
    srv = hb.Server(0, max_slots=8)
    ids = [srv.serve_submit(want_state=True, **r) for r in REQS]
    res = [srv.serve_poll(i, timeout_ms=60000) for i in ids]
    srv.close()
    for r, q in zip(res, REQS):
        assert r is not None and r["status"] == hb.HYDRO_OK and r["steps_done"] == q["steps"]
        extra = {k: v for k, v in q.items() if k not in ("kind", "n", "steps", "gamma")}
        ref, t = _oracle_run(q["kind"], q["n"], q["steps"], q["gamma"], **extra)
        assert abs(r["t_final"] - t) <= 1e-10 * t
        assert np.all(rel_linf(r["state"][I3], ref[I3]) <= 1e-10)
        assert r["zone_updates"] == q["steps"] * q["n"] ** 3


@pytest.mark.parametrize("policy", [hb.SERVE_RESPONSE_RATIO, hb.SERVE_ALL])
def test_alone_equals_in_the_mix(policy):
    # each request alone in its own server
    alone = []
    for q in REQS:
        srv = hb.Server(0, max_slots=4)
        rid = srv.serve_submit(want_state=True, **q)
        alone.append(srv.serve_poll(rid, timeout_ms=60000))
        srv.close()
    # in a mix: a long request starts first, the others arrive while it runs
    srv = hb.Server(0, max_slots=8)
    srv.serve_set_policy(policy, 10.0)
    long_id = srv.serve_submit(kind=hb.PROB_SEDOV, n=32, steps=60)
    t0 = time.time()
    while srv.serve_stats()["active"] == 0 and time.time() - t0 < 30:
        time.sleep(0.001)
    ids = []
    for q in REQS:
        ids.append(srv.serve_submit(want_state=True, **q))
        time.sleep(0.002)
    mixed = [srv.serve_poll(i, timeout_ms=60000) for i in ids]
    assert srv.serve_poll(long_id, timeout_ms=60000)["status"] == hb.HYDRO_OK
    stats = srv.serve_stats()
    srv.close()
    for a, m in zip(alone, mixed):
        assert a["status"] == m["status"] == hb.HYDRO_OK
        assert a["t_final"] == m["t_final"]
        assert np.array_equal(a["state"][I3], m["state"][I3])
    assert stats["completed"] == len(REQS) + 1 and stats["admitted"] == len(REQS) + 1
    assert stats["zone_updates"] == 60 * 32 ** 3 + sum(q["steps"] * q["n"] ** 3 for q in REQS)
    assert stats["box_steps"] == 60 + sum(q["steps"] for q in REQS)
    # the requests overlapped the long one: fewer iterations than the sum of all steps
    assert 60 <= stats["iterations"] < 60 + sum(q["steps"] for q in REQS)


def test_response_ratio_quantum_and_policy_changes():
    """With a quantum smaller than one step of any box, every iteration steps
    exactly one request; the policy can change only while the server is idle."""
    srv = hb.Server(0, max_slots=8)
    with pytest.raises(hb.HydroError) as e:
        srv.serve_set_policy(7, 1.0)
    assert e.value.status == hb.HYDRO_EINVAL
    with pytest.raises(hb.HydroError) as e:
        srv.serve_set_policy(hb.SERVE_RESPONSE_RATIO, 0.0)
    assert e.value.status == hb.HYDRO_EINVAL
    srv.serve_set_policy(hb.SERVE_RESPONSE_RATIO, 1e-6)
    long_id = srv.serve_submit(kind=hb.PROB_SEDOV, n=32, steps=200)
    with pytest.raises(hb.HydroError) as e:  # busy
        srv.serve_set_policy(hb.SERVE_ALL)
    assert e.value.status == hb.HYDRO_EAGAIN
    ids = [srv.serve_submit(**q) for q in REQS]
    res = [srv.serve_poll(i, timeout_ms=120000) for i in ids + [long_id]]
    st = srv.serve_stats()
    assert all(r["status"] == hb.HYDRO_OK for r in res)
    assert st["iterations"] == st["box_steps"] == 200 + sum(q["steps"] for q in REQS)
    # the short requests were not held behind the long one: each finished
    # before it
    assert max(r["latency_ms"] for r in res[:-1]) < res[-1]["latency_ms"]
    srv.serve_set_policy(hb.SERVE_ALL)
    srv.close()


def test_poll_and_budget_semantics():
    srv = hb.Server(0, hbm_budget=256 << 20, max_slots=2)
    with pytest.raises(hb.HydroError) as e:
        srv.serve_submit(kind=hb.PROB_SOD, n=96, steps=1)  # 104^3 zones x 109 doubles > 256 MiB
    assert e.value.status == hb.HYDRO_ETOOBIG
    with pytest.raises(hb.HydroError) as e:
        srv.serve_submit(kind=hb.PROB_SOD, n=16, steps=0)
    assert e.value.status == hb.HYDRO_EINVAL
    rid = srv.serve_submit(kind=hb.PROB_SEDOV, n=32, steps=40)
    assert srv.serve_poll(rid, timeout_ms=0) is None  # still running (or queued)
    r = srv.serve_poll(rid, timeout_ms=60000)
    assert r["status"] == hb.HYDRO_OK and r["steps_done"] == 40 and r["latency_ms"] >= r["queue_ms"] >= 0
    with pytest.raises(hb.HydroError) as e:
        srv.serve_poll(rid, timeout_ms=0)  # handle released by the successful poll
    assert e.value.status == hb.HYDRO_EINVAL
    srv.close()


def test_poll_with_a_bounded_wait_times_out():
    """A poll whose wait runs out returns HYDRO_ETIMEDOUT after about that
    wait, leaves the request alive, and a later poll collects it."""
    import ctypes
    srv = hb.Server(0)
    rid = srv.serve_submit(kind=hb.PROB_SEDOV, n=128, steps=100)  # a few hundred ms of GPU work
    res = hb.hydro_result_t()
    t0 = time.perf_counter()
    rc = srv.L.serve_poll(srv.h, ctypes.c_uint64(rid), ctypes.byref(res), 20)
    waited = time.perf_counter() - t0
    assert rc == hb.HYDRO_ETIMEDOUT
    assert 0.015 <= waited < 2.0, waited
    r = srv.serve_poll(rid, timeout_ms=120000)
    assert r["status"] == hb.HYDRO_OK and r["steps_done"] == 100
    srv.close()


def _wait_for(cond, limit_s=60.0):
    t0 = time.perf_counter()
    while not cond():
        assert time.perf_counter() - t0 < limit_s
        time.sleep(0.005)


def test_cancel_queued_running_and_finished_requests():
    """A queued request leaves the queue at once; a running one is retired
    before the scheduler's next iteration with the steps it has done; one
    that finished first keeps its result; the server serves on."""
    srv = hb.Server(0, max_slots=1)
    long_id = srv.serve_submit(kind=hb.PROB_SEDOV, n=128, steps=400)  # about 1.5 s of steps alone
    queued = srv.serve_submit(kind=hb.PROB_SOD, n=32, steps=10)  # waits for the only slot
    srv.serve_cancel(queued)
    r = srv.serve_poll(queued, timeout_ms=60000)
    assert r["status"] == hb.HYDRO_ECANCELED and r["steps_done"] == 0
    _wait_for(lambda: srv.serve_stats()["zone_updates"] > 0)  # the long request is stepping
    srv.serve_cancel(long_id)
    r = srv.serve_poll(long_id, timeout_ms=60000)
    assert r["status"] == hb.HYDRO_ECANCELED and 0 < r["steps_done"] < 400
    rid = srv.serve_submit(kind=hb.PROB_SOD, n=32, steps=10)
    r = srv.serve_poll(rid, timeout_ms=60000)
    assert r["status"] == hb.HYDRO_OK and r["steps_done"] == 10
    rid = srv.serve_submit(kind=hb.PROB_SOD, n=32, steps=5)
    done = srv.serve_stats()["completed"] + 1
    _wait_for(lambda: srv.serve_stats()["completed"] >= done)
    srv.serve_cancel(rid)  # finished first: the result stands
    r = srv.serve_poll(rid, timeout_ms=0)
    assert r["status"] == hb.HYDRO_OK and r["steps_done"] == 5
    with pytest.raises(hb.HydroError) as e:
        srv.serve_cancel(rid)  # collected: unknown handle
    assert e.value.status == hb.HYDRO_EINVAL
    srv.close()


def test_slot_limit_queues_requests():
    srv = hb.Server(0, max_slots=1)
    ids = [srv.serve_submit(kind=hb.PROB_SOD, n=16, steps=4) for _ in range(3)]
    res = [srv.serve_poll(i, timeout_ms=60000) for i in ids]
    st = srv.serve_stats()
    srv.close()
    assert all(r["status"] == hb.HYDRO_OK for r in res)
    # one slot: the requests ran one after another
    assert st["iterations"] == 12
    assert res[2]["queue_ms"] >= res[0]["queue_ms"]
