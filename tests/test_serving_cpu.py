"""Scheduler of the reconstruction server on a simulated device (no GPU):
admission by the device-memory budget, FIFO order, immediate retirement, and
the comparison with one-at-a-time processing."""
import numpy as np
import pytest

from paper_2301_09710_gb300.serving import FakeExecutor, Request, serve, serve_plain


def _req(rid, arrival, nx=8, nz=4, nview=4, niter=3):
    z = np.zeros((nz, nx, nx), np.float32)
    return Request(rid, arrival, nx, nz, nview, niter, z, np.zeros((1, nx, 1), np.float32),
                   np.zeros((1, nx, 1), np.float32), np.zeros((nview, nz, nx), np.float32))


def test_admission_respects_memory_budget_and_completes_everything():
    reqs = [_req(i, 0.001 * i) for i in range(10)]
    per = FakeExecutor.plan_bytes(reqs[0])
    ex = FakeExecutor(iter_cost=0.01)
    st = serve(reqs, ex, mem_budget=3 * per, max_active=8)
    assert [r.rid for r in st.results] == list(range(10))
    assert st.peak_bytes <= 3 * per and st.peak_active == 3
    for r in st.results:
        assert r.admitted >= r.arrival and r.done >= r.admitted + 3 * 0.01 - 1e-9


def test_slots_limit_concurrency():
    reqs = [_req(i, 0.0) for i in range(6)]
    st = serve(reqs, FakeExecutor(), mem_budget=1 << 40, max_active=2)
    assert st.peak_active == 2


def test_fifo_admission_under_pressure():
    reqs = [_req(0, 0.0, niter=10), _req(1, 0.001, nx=16), _req(2, 0.002)]
    per_small = FakeExecutor.plan_bytes(reqs[0])
    ex = FakeExecutor(iter_cost=0.01)
    # budget: the big request (16x16) does not fit beside the first one; the
    # third (small, would fit) must not overtake it
    st = serve(reqs, ex, mem_budget=per_small + FakeExecutor.plan_bytes(reqs[1]) - 1, max_active=4)
    starts = [e for e in ex.log if e[0] == "start"]
    assert [e[1] for e in starts] == [0, 1, 2]


def test_request_beyond_budget_is_refused():
    with pytest.raises(ValueError, match="budget"):
        serve([_req(0, 0.0, nx=64)], FakeExecutor(), mem_budget=10)


def test_concurrency_beats_one_at_a_time_on_the_simulated_device():
    rng = np.random.default_rng(0)
    arr = np.cumsum(rng.exponential(0.005, 30))
    reqs = [_req(i, float(a), niter=int(rng.integers(4, 9))) for i, a in enumerate(arr)]
    served = serve(reqs, FakeExecutor(iter_cost=0.01), mem_budget=1 << 40, max_active=8).summary()
    plain = serve_plain(reqs, FakeExecutor(iter_cost=0.01)).summary()
    assert served["p99_s"] < plain["p99_s"] and served["recon_per_s"] > plain["recon_per_s"]


def test_budget_defaults_to_free_device_memory_less_the_reserve():
    reqs = [_req(i, 0.0) for i in range(8)]
    per = FakeExecutor.plan_bytes(reqs[0])
    ex = FakeExecutor(iter_cost=0.01, device_bytes=4 * per + 1000)
    st = serve(reqs, ex, mem_budget=None, max_active=8, reserve_bytes=1000)
    assert st.budget == 4 * per and st.peak_active == 4 and st.peak_bytes <= 4 * per
    assert len(st.results) == 8


def test_memory_taken_by_another_tenant_holds_admission_back():
    """The budget fits 4 requests, but from t = 0.005 s something else holds
    half the device: admissions after that wait until the live free memory
    allows them, and every request still completes."""
    reqs = [_req(i, 0.001 * i) for i in range(8)]
    per = FakeExecutor.plan_bytes(reqs[0])
    total = 4 * per
    ex = FakeExecutor(iter_cost=0.01, device_bytes=total, other_use=lambda t: 2 * per if t >= 0.005 else 0)
    st = serve(reqs, ex, mem_budget=None, max_active=8, reserve_bytes=0)
    assert len(st.results) == 8
    assert st.held_back > 0
    # while the other tenant holds 2 requests' worth, at most 2 requests are resident
    for t in np.arange(0.006, st.makespan, 0.0005):
        resident = sum(1 for r in st.results if r.admitted <= t < r.done and r.admitted >= 0.005)
        assert resident <= 2


def test_serving_without_a_budget_needs_a_device_that_reports_free_memory():
    with pytest.raises(ValueError, match="mem_budget"):
        serve([_req(0, 0.0)], FakeExecutor(), mem_budget=None)


def test_compact_fallback_admits_what_only_fits_as_a_compact_plan():
    # the second request's full plan fits alone but not beside the first one,
    # its compact plan (a quarter on the simulated device) does
    reqs = [_req(0, 0.0, niter=10), _req(1, 0.001, nx=16), _req(2, 0.002)]
    small, big = FakeExecutor.plan_bytes(reqs[0]), FakeExecutor.plan_bytes(reqs[1])
    budget = big + small // 2
    ex = FakeExecutor(iter_cost=0.01)
    st = serve(reqs, ex, mem_budget=budget, max_active=4, compact_fallback=True)
    starts = {e[1]: (e[2], e[3]) for e in ex.log if e[0] == "start"}
    assert st.compact == 1 and starts[1][1] is True and starts[0][1] is False
    assert starts[1][0] < 0.05, "the compact request waited for the first one to finish"
    assert st.peak_bytes <= budget and [r.rid for r in st.results] == [0, 1, 2]
    # without the fallback the same request waits for the first to finish
    ex2 = FakeExecutor(iter_cost=0.01)
    st2 = serve(reqs, ex2, mem_budget=budget, max_active=4)
    starts2 = {e[1]: e[2] for e in ex2.log if e[0] == "start"}
    assert st2.compact == 0 and starts2[1] >= 10 * 0.01 - 1e-9


def test_compact_fallback_still_refuses_what_no_plan_can_fit():
    reqs = [_req(0, 0.0, nx=16)]
    with pytest.raises(ValueError):
        serve(reqs, FakeExecutor(), mem_budget=FakeExecutor.plan_bytes(reqs[0], compact=True) - 1,
              compact_fallback=True)
    st = serve(reqs, FakeExecutor(), mem_budget=FakeExecutor.plan_bytes(reqs[0], compact=True),
               compact_fallback=True)
    assert st.compact == 1 and len(st.results) == 1
