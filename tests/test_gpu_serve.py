"""Continuous-batching server (imloc_serve_*) through the C ABI.

Checks: results agree with the FP64 oracle; the same query gives the same
pose alone and in a mix of queries that arrive while others run (within
0.05 deg / 5 mm, normally bit-identical since sampling, rounds and reduction
order do not depend on the mix); admission never exceeds the device budget
and a query larger than the budget, a full queue or a full staging ring is
refused; unknown or consumed tickets are reported as such.
"""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2601_04185_gb300 import imloc, synth

from gpu_helpers import pose_close, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def store():
    ms = synth.MapStore(3, 12, width=512, height=384, f=400.0)
    for k in range(12):
        ms.build_view(k)
    t = torch()
    dev_views = []
    for v in ms.views:
        d = dict(v)
        d["depth"] = t.from_numpy(v["depth"]).cuda()
        dev_views.append(d)
    return ms, dev_views


@pytest.fixture(scope="module")
def ctx():
    c = imloc.Context(0, 256 << 20)
    yield c
    c.close()


def make_queries(ms, n, seed, views=(3, 8), per_pair=(1000, 3000)):
    rng = np.random.default_rng(seed)
    return [ms.query(rng, int(rng.integers(*views)), matches_per_pair=int(rng.integers(*per_pair))) for _ in range(n)]


def query_views(dev_views, q):
    return [dev_views[i] for i in q["view_ids"]]


def wait_all(server, tickets, timeout=60.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets) and time.time() - t0 < timeout:
        for tk in tickets:
            if tk in out:
                continue
            st, res, lat = server.poll(tk)
            if st == 0:
                out[tk] = (res, lat)
        time.sleep(0.001)
    assert len(out) == len(tickets), server.stats()
    return out


def opts_for(i, **kw):
    return imloc.default_opts(max_iters=4096, p_miss=1e-4, query_id=i, seed=99, **kw)


def test_served_results_match_the_oracle(store, ctx):
    ms, dev_views = store
    qs = make_queries(ms, 6, 1)
    srv = imloc.Server(ctx, max_slots=8, device_budget_bytes=256 << 20)
    tickets = [srv.submit(query_views(dev_views, q), q["matches"], q["K"], opts_for(i)) for i, q in enumerate(qs)]
    got = wait_all(srv, tickets)
    for i, (q, tk) in enumerate(zip(qs, tickets)):
        res, lat = got[tk]
        assert res["status"] == 0 and lat > 0
        views = [ms.views[j] for j in q["view_ids"]]
        L = oracle.lift(views, q["matches"])
        ref = oracle.ransac_pnp(oracle.Corr(L["x"], L["y"], L["X"], L["w"]), q["K"], max_iters=4096, p_miss=1e-4,
                                query_id=i, seed=99)
        assert pose_close(res["R"], res["t"], ref["R"], ref["t"]), i
        assert res["iterations"] == ref["iterations"] or abs(res["subset_inliers"] - ref["subset_inliers"]) <= 3
    st = srv.stats()
    assert st["completed"] == 6 and st["rejected"] == 0 and st["worker_status"] == 0
    srv.close()


def test_same_result_alone_and_in_the_mix(store, ctx):
    """Query A alone, then A again while a stream of other queries arrives
    before, with and after it (continuous batching)."""
    ms, dev_views = store
    qa = make_queries(ms, 1, 7)[0]
    others = make_queries(ms, 24, 8)
    srv = imloc.Server(ctx, max_slots=6, device_budget_bytes=256 << 20, rounds_per_step=1)
    ta = srv.submit(query_views(dev_views, qa), qa["matches"], qa["K"], opts_for(1000))
    alone = wait_all(srv, [ta])[ta][0]

    tickets = []
    stop = threading.Event()

    def feeder():
        for i, q in enumerate(others):
            tickets.append(srv.submit(query_views(dev_views, q), q["matches"], q["K"], opts_for(i)))
            time.sleep(0.002)

    th = threading.Thread(target=feeder)
    th.start()
    time.sleep(0.01)
    tb = srv.submit(query_views(dev_views, qa), qa["matches"], qa["K"], opts_for(1000))
    th.join()
    got = wait_all(srv, tickets + [tb])
    mixed = got[tb][0]
    assert mixed["status"] == alone["status"] == 0
    assert pose_close(mixed["R"], mixed["t"], alone["R"], alone["t"])
    assert mixed["iterations"] == alone["iterations"]
    st = srv.stats()
    assert st["steps"] > 1 and st["completed"] == 26
    srv.close()


def test_admission_by_device_budget_and_refusals(store, ctx):
    ms, dev_views = store
    qs = make_queries(ms, 10, 11, views=(6, 9), per_pair=(2500, 3000))
    # a budget that holds only a couple of these queries at a time
    srv = imloc.Server(ctx, max_slots=16, device_budget_bytes=8 << 20, max_queue=64)
    tickets = [srv.submit(query_views(dev_views, q), q["matches"], q["K"], opts_for(i)) for i, q in enumerate(qs)]
    assert all(t is not None for t in tickets)
    peak = 0
    t0 = time.time()
    while srv.stats()["completed"] < 10 and time.time() - t0 < 60:
        st = srv.stats()
        assert st["device_bytes_in_use"] <= 8 << 20
        peak = max(peak, st["resident"])
        time.sleep(0.0005)
    got = wait_all(srv, tickets)
    assert all(r[0]["status"] == 0 for r in got.values())
    assert peak < 10  # the budget, not the 16 slots, limited residency
    # a query that can never fit the budget is refused
    big = make_queries(ms, 1, 12, views=(10, 11), per_pair=(17000, 17001))[0]
    assert srv.submit(query_views(dev_views, big), big["matches"], big["K"], opts_for(50)) is None
    assert srv.stats()["rejected"] == 1
    # consumed and unknown tickets
    assert srv.poll(tickets[0])[0] == -6
    assert srv.poll(123456789)[0] == -6
    srv.close()


def test_full_queue_and_full_staging_ring_refuse(store, ctx):
    ms, dev_views = store
    qs = make_queries(ms, 8, 13, views=(4, 5), per_pair=(2000, 2001))
    # tiny queue: submissions beyond it are refused while nothing can be admitted (budget too small for two)
    per_query = len(qs[0]["matches"]["q_u"]) * 20
    srv = imloc.Server(ctx, max_slots=1, device_budget_bytes=6 << 20, max_queue=2, host_staging_bytes=64 << 20)
    res = [srv.submit(query_views(dev_views, q), q["matches"], q["K"], opts_for(i)) for i, q in enumerate(qs)]
    assert any(r is None for r in res)
    ok = [r for r in res if r is not None]
    got = wait_all(srv, ok)
    assert all(v[0]["status"] == 0 for v in got.values())
    srv.close()
    # staging ring smaller than two queries: the second concurrent submission is refused
    srv = imloc.Server(ctx, max_slots=1, device_budget_bytes=6 << 20, host_staging_bytes=per_query + 4096)
    r1 = srv.submit(query_views(dev_views, qs[0]), qs[0]["matches"], qs[0]["K"], opts_for(0))
    r2 = srv.submit(query_views(dev_views, qs[1]), qs[1]["matches"], qs[1]["K"], opts_for(1))
    assert r1 is not None
    wait_all(srv, [r1])
    if r2 is not None:
        wait_all(srv, [r2])
    r3 = srv.submit(query_views(dev_views, qs[2]), qs[2]["matches"], qs[2]["K"], opts_for(2))
    assert r3 is not None  # room again once the ring drained
    wait_all(srv, [r3])
    srv.close()


def test_many_client_threads(store, ctx):
    ms, dev_views = store
    qs = make_queries(ms, 16, 17, views=(3, 5), per_pair=(800, 1500))
    srv = imloc.Server(ctx, max_slots=8, device_budget_bytes=256 << 20)
    tickets = [None] * len(qs)

    def client(k):
        for i in range(k, len(qs), 4):
            q = qs[i]
            tickets[i] = srv.submit(query_views(dev_views, q), q["matches"], q["K"], opts_for(i))

    ths = [threading.Thread(target=client, args=(k,)) for k in range(4)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    got = wait_all(srv, tickets)
    assert all(v[0]["status"] == 0 for v in got.values())
    assert len(set(tickets)) == len(qs)
    srv.close()


def test_device_submitted_matches_give_the_host_submitted_results(store, ctx):
    """imloc_serve_submit_device (matches already in device memory, read in
    place by the lift): the same results as host submission of the same
    queries, mixed in one stream of submissions."""
    ms, dev_views = store
    qs = make_queries(ms, 8, 5)
    t = torch()
    srv = imloc.Server(ctx, max_slots=6, device_budget_bytes=256 << 20)
    keep, tickets_h, tickets_d = [], [], []
    for i, q in enumerate(qs):
        tickets_h.append(srv.submit(query_views(dev_views, q), q["matches"], q["K"], opts_for(i)))
        dm = {k: t.from_numpy(np.ascontiguousarray(q["matches"][k], dtype=np.float32)).cuda()
              for k in ("q_u", "q_v", "db_u", "db_v", "conf")}
        dm.update({k: q["matches"][k] for k in ("seg_off", "seg_view", "seg_dir")})
        p = imloc.Server.prepare_device(query_views(dev_views, q), dm, q["K"], opts_for(i))
        keep.append(p)
        tickets_d.append(srv.submit_prepared(p))
    got = wait_all(srv, tickets_h + tickets_d)
    for i, q in enumerate(qs):
        rh, _ = got[tickets_h[i]]
        rd, _ = got[tickets_d[i]]
        assert rh["status"] == 0 and rd["status"] == 0
        assert pose_close(rh["R"], rh["t"], rd["R"], rd["t"]), i
        assert rh["num_inliers"] == rd["num_inliers"], i
        assert pose_close(rd["R"], rd["t"], q["R_gt"], q["t_gt"], deg=0.5, mm=50), i
    assert srv.stats()["worker_status"] == 0
    srv.close()


def test_slots_reused_while_steps_are_in_flight(store, ctx):
    """Many short queries through two slots: slots are freed and refilled
    while the next step is already on the GPU (the steps are pipelined), and
    a refilled slot must not be retired with the previous query's state.
    Every result equals the same query served alone, the staging ring drains
    (a long second burst is admitted in full), nothing is refused."""
    ms, dev_views = store
    qs = make_queries(ms, 16, 13, views=(3, 5), per_pair=(800, 1500))
    srv = imloc.Server(ctx, max_slots=2, device_budget_bytes=256 << 20, rounds_per_step=1,
                       host_staging_bytes=64 << 20)
    alone = []
    for i, q in enumerate(qs):
        t = srv.submit(query_views(dev_views, q), q["matches"], q["K"], opts_for(i))
        alone.append(wait_all(srv, [t])[t][0])
    for burst in range(3):
        tickets = [srv.submit(query_views(dev_views, q), q["matches"], q["K"], opts_for(i)) for i, q in enumerate(qs)]
        assert all(t is not None for t in tickets)
        got = wait_all(srv, tickets)
        for i, t in enumerate(tickets):
            r = got[t][0]
            assert r["status"] == alone[i]["status"] == 0
            assert pose_close(r["R"], r["t"], alone[i]["R"], alone[i]["t"]), (burst, i)
            assert r["iterations"] == alone[i]["iterations"] and r["num_inliers"] == alone[i]["num_inliers"]
    st = srv.stats()
    assert st["completed"] == 64 and st["rejected"] == 0 and st["resident"] == 0 and st["worker_status"] == 0
    srv.close()
