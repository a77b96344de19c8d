"""Serving (continuous batching of re-solves): results equal the same
request solved alone, warm starts from a session's resident state converge
faster, and admission waits for device memory instead of failing."""
import time

import numpy as np
import pytest

from paper_1903_10041_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_10041_gb300 import build
    build.build()
    from paper_1903_10041_gb300 import capi
    return capi


PAR = W.Params(rho=(1.0, 1.0 / 600, 1.0, 1.0), precision="mixed")


def requests(count, seed):
    out = []
    for t in range(count):
        n, m, q = W.batch_shape(t, seed)
        out.append(W.random_problem(max(20, min(n, 600)), m, q, seed=seed * 1000 + t))
    return out


def wait_all(S, tickets, timeout_s=120.0):
    res, t0 = {}, time.time()
    while len(res) < len(tickets):
        for t in tickets:
            if t not in res:
                r = S.poll(t, wait_ms=5, want_x=True)
                if r is not None:
                    res[t] = r
        assert time.time() - t0 < timeout_s, "served requests did not finish"
    return [res[t] for t in tickets]


def test_served_result_is_the_same_alone_and_in_the_mix(capi, oracle_lib):
    probs = requests(20, seed=5)
    with capi.Server(PAR, tick_iters=40, small_max_elements=4096) as S:
        alone = [wait_all(S, [S.submit(P)])[0] for P in probs[:4]]
        # the same problems again, now submitted together with 16 others at staggered times
        tickets = []
        for t, P in enumerate(probs):
            tickets.append(S.submit(P))
            if t % 5 == 4:
                time.sleep(0.002)
        mix = wait_all(S, tickets)
    for t in range(4):
        assert alone[t]["converged"] and mix[t]["converged"]
        assert alone[t]["iters"] == mix[t]["iters"]
        assert np.array_equal(alone[t]["x"], mix[t]["x"]), t
    for t in (0, 7, 13):
        st_o, _ = oracle_lib.solve(probs[t], PAR.replace(precision="fp64"), threads=16)
        obj_o = oracle_lib.objective(probs[t], st_o["x"])
        assert abs(mix[t]["objective"] - obj_o) <= 1e-6 * max(1.0, abs(obj_o)), t


def test_session_warm_start_after_a_one_step_shift(capi, oracle_lib):
    P0 = W.random_problem(400, 3, 6, seed=77)
    P1 = W.receding_step(P0, step=1)
    with capi.Server(PAR, tick_iters=40) as S:
        r0 = wait_all(S, [S.submit(P0, session=7)])[0]
        r1 = wait_all(S, [S.submit(P1, session=7)])[0]
        cold = wait_all(S, [S.submit(P1)])[0]
    assert r0["converged"] and r1["converged"] and cold["converged"]
    assert r1["warm"] and not cold["warm"]
    assert r1["iters"] < cold["iters"], (r1["iters"], cold["iters"])
    st_o, _ = oracle_lib.solve(P1, PAR.replace(precision="fp64"), threads=16)
    obj_o = oracle_lib.objective(P1, st_o["x"])
    assert abs(r1["objective"] - obj_o) <= 1e-6 * max(1.0, abs(obj_o))


def test_admission_waits_for_device_memory(capi):
    probs = requests(12, seed=9)
    biggest = max(P.m * P.q * ((P.n + 3) // 4 * 4) for P in probs)
    with capi.Server(PAR, tick_iters=20, store_elements=2 * biggest, max_active=64) as S:
        tickets = [S.submit(P) for P in probs]
        seen_queue = S.stats()["queued"] > 0
        res = wait_all(S, tickets)
        st = S.stats()
    assert all(r["converged"] for r in res)
    assert st["finished"] == len(probs)
    assert seen_queue or st["ticks"] > 1


def test_oversized_request_is_rejected(capi):
    P = W.random_problem(100, 5, 2, seed=3)
    with capi.Server(PAR, max_m=4) as S:
        with pytest.raises(capi.AdmmError) as e:
            S.submit(P)
    assert e.value.status == capi.ADMM_EUNSUPPORTED


def test_step_request_slides_the_horizon_on_the_device(capi, oracle_lib):
    """A step request moves the session's resident instance one step on the
    device; the result is the receding-horizon problem's solution."""
    P0 = W.random_problem(400, 3, 6, seed=78)
    P1 = W.receding_step(P0, step=1)
    with capi.Server(PAR, tick_iters=40) as S:
        r0 = wait_all(S, [S.submit(P0, session=9)])[0]
        r1 = wait_all(S, [S.submit_step(9, W.step_data(3, 6, step=1))])[0]
        cold = wait_all(S, [S.submit(P1)])[0]
    assert r0["converged"] and r1["converged"] and cold["converged"]
    assert r1["warm"] and r1["iters"] < cold["iters"], (r1["iters"], cold["iters"])
    st_o, _ = oracle_lib.solve(P1, PAR.replace(precision="fp64"), threads=16)
    obj_o = oracle_lib.objective(P1, st_o["x"])
    assert abs(r1["objective"] - obj_o) <= 1e-6 * max(1.0, abs(obj_o))
    assert abs(cold["objective"] - obj_o) <= 1e-6 * max(1.0, abs(obj_o))


def test_step_requests_with_late_adaptation(capi, oracle_lib):
    """The serving setting for re-solves: adaptation (Sec. IV-A) only from
    iteration 200 on.  A batch and a server give the same bits for the same
    problem, and a warm step re-solve reaches the oracle's optimum."""
    par = PAR.replace(adapt_rho=True, adapt_start=200)
    P0 = W.random_problem(400, 3, 6, seed=79)
    P1 = W.receding_step(P0, step=1)
    with capi.Batch([P0], par) as B:
        B.solve()
        rb = B.wait(want_x=True)[0]
    with capi.Server(par, tick_iters=40) as S:
        r0 = wait_all(S, [S.submit(P0, session=11)])[0]
        r1 = wait_all(S, [S.submit_step(11, W.step_data(3, 6, step=1))])[0]
    assert rb["converged"] and r0["converged"] and r1["converged"] and r1["warm"]
    assert rb["iters"] == r0["iters"] and np.array_equal(rb["x"], r0["x"])
    st_o, _ = oracle_lib.solve(P1, par.replace(precision="fp64"), threads=16)
    obj_o = oracle_lib.objective(P1, st_o["x"])
    assert abs(r1["objective"] - obj_o) <= 1e-6 * max(1.0, abs(obj_o))


def test_step_request_without_a_resident_session_fails_cleanly(capi):
    with capi.Server(PAR) as S:
        t = S.submit_step(123, W.step_data(2, 3, step=1))
        res = None
        for _ in range(200):
            res = S.poll(t, wait_ms=10)
            if res is not None:
                break
    assert res is not None and res["status"] == capi.ADMM_EINVAL


def test_round_robin_ticks_give_the_same_bits(capi):
    """More instances than CTA teams: each tick takes every instance several
    times in round-robin slices, moving its state between SMs.  The results
    equal those of the same requests submitted one at a time."""
    probs = [W.random_problem(40 + (t % 7) * 13, 2 + t % 3, 1 + t % 4, seed=7000 + t) for t in range(700)]
    with capi.Server(PAR, tick_iters=10, small_max_elements=0) as S:
        alone = [wait_all(S, [S.submit(P)])[0] for P in probs[:6]]
        mix = wait_all(S, [S.submit(P) for P in probs], timeout_s=300.0)
        stats = S.stats()
    assert stats["instance_ticks"] / stats["ticks"] > 1.0
    for t in range(6):
        assert alone[t]["converged"] and mix[t]["converged"], t
        assert alone[t]["iters"] == mix[t]["iters"], t
        assert np.array_equal(alone[t]["x"], mix[t]["x"]), t


def test_round_robin_ticks_with_cluster_teams_give_the_same_bits(capi, oracle_lib):
    """Round-robin ticks while cluster teams run the largest requests: each
    cluster instance takes one pass per tick worth the R slices of the CTA
    teams' instances.  Every request gives the bits it gives alone."""
    small = [W.random_problem(40 + (t % 7) * 13, 2 + t % 3, 1 + t % 4, seed=7000 + t) for t in range(700)]
    large = [W.random_problem(600, 3, 4, seed=7900 + t) for t in range(6)]
    cfg = dict(tick_iters=10, small_max_elements=0, cluster_size=2, cluster_min_elements=2000)
    with capi.Server(PAR, **cfg) as S:
        alone = [wait_all(S, [S.submit(P)])[0] for P in large[:2] + small[:2]]
        mix = wait_all(S, [S.submit(P) for P in large + small], timeout_s=300.0)
        stats = S.stats()
    assert stats["instance_ticks"] / stats["ticks"] > 1.0
    for t, u in enumerate((0, 1, 6, 7)):
        assert alone[t]["converged"] and mix[u]["converged"], t
        assert alone[t]["iters"] == mix[u]["iters"], t
        assert np.array_equal(alone[t]["x"], mix[u]["x"]), t
    st_o, _ = oracle_lib.solve(large[0], PAR.replace(precision="fp64"), threads=16)
    obj_o = oracle_lib.objective(large[0], st_o["x"])
    assert abs(mix[0]["objective"] - obj_o) <= 1e-6 * max(1.0, abs(obj_o))


def test_cancel_a_queued_and_a_running_request(capi):
    long_par = PAR.replace(r_tol=0.0, s_tol=0.0, max_iter=5000)  # runs to the iteration cap
    with capi.Server(long_par, max_active=1, tick_iters=5) as S:
        running = S.submit(W.random_problem(4000, 3, 8, seed=91))
        queued = S.submit(W.random_problem(300, 2, 2, seed=92))
        time.sleep(0.2)
        S.cancel(queued)
        rq = S.poll(queued, wait_ms=2000)
        assert rq is not None and rq["status"] == capi.ADMM_ECANCELLED
        S.cancel(running)
        rr = S.poll(running, wait_ms=10000)
        assert rr is not None and rr["status"] == capi.ADMM_ECANCELLED
    with capi.Server(PAR, max_active=1) as S:  # the server keeps serving after cancellations
        t = S.submit(W.random_problem(300, 2, 2, seed=93))
        r = wait_all(S, [t])[0]
        assert r["converged"]
