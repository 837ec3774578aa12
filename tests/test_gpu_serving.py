"""Serving: many analyses interleaved on one GPU give each the same result as
alone; admission respects the analysis count, the chain budget and the memory
budget; requests can be cancelled. All on the GPU through the C ABI."""
import numpy as np
import pytest

import gwinputs as gi
import oracle

pytestmark = pytest.mark.gpu


def _analysis(seed_offset, N=1200, n_live=80, n_det=3, df=None, k=None, snr=None, dl_lo=None):
    w = gi.workload("c1", n_live=n_live, k=k if k else n_live // 2)
    if snr is not None:
        w.snr = snr
    if dl_lo is not None:
        w.lo[gi.P_DL] = dl_lo
    w.N = N
    w.n_det = n_det
    if df is not None:
        w.df = df
    w.seed_noise += seed_offset
    w.seed_injection += seed_offset
    w.seed_sampler += seed_offset
    pb, th = oracle.make_problem(w)
    return dict(kind=pb.kind, lo=pb.lo, hi=pb.hi, data=pb.data(), psd=pb.psd, f0=pb.f0, df=pb.df,
                pos=pb.pos, xarm=pb.xarm, yarm=pb.yarm, n_live=w.n_live, k=w.k,
                steps_per_dim=w.steps_per_dim, seed=w.seed_sampler), pb.dim


@pytest.mark.parametrize("precision", [0, 1])
def test_alone_equals_in_the_mix(gw, precision):
    reqs = [_analysis(i, N=900 + 300 * i, n_live=60 + 20 * i, n_det=2 + (i % 2)) for i in range(3)]
    with gw.Server(precision=precision, slots=2) as srv:
        rid = srv.submit(**reqs[0][0])
        srv.run_until_idle()
        alone = srv.result(rid, reqs[0][1])
        st_alone = srv.poll(rid)
    with gw.Server(precision=precision, slots=2) as srv:
        ids = [srv.submit(**r) for r, _ in reqs]
        max_run = 0
        while True:
            r, p = srv.tick()
            max_run = max(max_run, r)
            if r == 0 and p == 0:
                break
        assert max_run >= 2          # they did share the GPU
        mixed = srv.result(ids[0], reqs[0][1])
        for i in ids:
            assert srv.poll(i)["state"] == gw.NS_REQ_DONE
    assert st_alone["state"] == gw.NS_REQ_DONE
    assert mixed["logZ"] == alone["logZ"] and mixed["dlogZ"] == alone["dlogZ"]
    assert np.array_equal(mixed["u"], alone["u"]) and np.array_equal(mixed["logl"], alone["logl"])


def test_tiled_forms_share_a_server(gw):
    """Mixed analyses whose grids take different mixed forms (32- and 16-bin
    tiles, the per-bin form) interleaved in one server: each result equals the
    analysis alone."""
    reqs = [_analysis(40, N=3000, df=1 / 32), _analysis(41, N=1500, df=1 / 16), _analysis(42)]
    alone = []
    for r, dim in reqs:
        with gw.Server(precision=1, slots=2) as srv:
            rid = srv.submit(**r)
            srv.run_until_idle()
            alone.append(srv.result(rid, dim))
    with gw.Server(precision=1, slots=2) as srv:
        ids = [srv.submit(**r) for r, _ in reqs]
        max_run = 0
        while True:
            n, p = srv.tick()
            max_run = max(max_run, n)
            if n == 0 and p == 0:
                break
        assert max_run == 3
        mixed = [srv.result(i, dim) for i, (_, dim) in zip(ids, reqs)]
    for a, m in zip(alone, mixed):
        assert m["logZ"] == a["logZ"]
        assert np.array_equal(m["logl"], a["logl"])


@pytest.mark.parametrize("precision", [0, 1])
def test_short_and_long_lanes(gw, precision):
    """A long grid (40,000 bins, the server's stream) and two short ones (the
    short lane, iterated again while the long grid's iteration runs) in one
    server: every analysis ends, with the result it has alone and the number of
    iterations it has alone."""
    reqs = [_analysis(60, N=40000, df=1 / 32, n_live=60), _analysis(61, N=1200, n_live=60),
            _analysis(62, N=2000, n_live=80)]
    alone = []
    for r, dim in reqs:
        with gw.Server(precision=precision, slots=2) as srv:
            rid = srv.submit(**r)
            srv.run_until_idle()
            alone.append((srv.result(rid, dim), srv.poll(rid)["iterations"]))
    with gw.Server(precision=precision, slots=2) as srv:
        ids = [srv.submit(**r) for r, _ in reqs]
        ticks = 0
        while True:
            n, p = srv.tick()
            ticks += 1
            if n == 0 and p == 0:
                break
        mixed = [(srv.result(i, dim), srv.poll(i)) for i, (_, dim) in zip(ids, reqs)]
    for (a, it), (m, st) in zip(alone, mixed):
        assert st["state"] == gw.NS_REQ_DONE
        assert st["iterations"] == it
        assert m["logZ"] == a["logZ"] and m["dlogZ"] == a["dlogZ"]
        assert np.array_equal(m["u"], a["u"]) and np.array_equal(m["logl"], a["logl"])
    # the server ran no more ticks than its longest analysis needs iterations
    assert ticks <= max(it for _, it in alone) + 1


def test_server_equals_single_context(gw):
    args, dim = _analysis(7)
    with gw.Server(precision=0, slots=2) as srv:
        rid = srv.submit(**args)
        srv.run_until_idle()
        a = srv.result(rid, dim)
    with gw.Sampler(precision=0, slots=2, **args) as sp:
        sp.run()
        b = sp.result()
    assert a["logZ"] == b["logZ"]
    assert np.array_equal(a["logl"], b["logl"])


def test_admission_by_slots_and_memory(gw):
    reqs = [_analysis(10 + i) for i in range(4)]
    with gw.Server(precision=1, max_active=2) as srv:
        ids = [srv.submit(**r) for r, _ in reqs]
        while True:
            r, p = srv.tick()
            assert r <= 2
            if r == 0 and p == 0:
                break
        assert all(srv.poll(i)["state"] == gw.NS_REQ_DONE for i in ids)
    # a budget that holds one analysis at a time
    fp = None
    with gw.Server(precision=1) as srv:
        fp = srv.poll(srv.submit(**reqs[0][0]))["footprint"]
    with gw.Server(precision=1, mem_budget=int(fp * 1.5)) as srv:
        ids = [srv.submit(**r) for r, _ in reqs[:3]]
        while True:
            r, p = srv.tick()
            assert r <= 1
            if r == 0 and p == 0:
                break
        sts = [srv.poll(i) for i in ids]
        assert all(s["state"] == gw.NS_REQ_DONE for s in sts)
        # served one after another, in arrival order
        assert sts[0]["t_done"] <= sts[1]["t_admit"] <= sts[1]["t_done"] <= sts[2]["t_admit"]
    # a request that can never fit is rejected, the rest still run
    with gw.Server(precision=1, mem_budget=int(fp * 0.5)) as srv:
        rid = srv.submit(**reqs[0][0])
        srv.tick()
        assert srv.poll(rid)["state"] == -4     # NS_ERR_OOM


def test_admission_by_chain_budget(gw):
    reqs = [_analysis(30 + i) for i in range(4)]          # k = 40 chains each
    with gw.Server(precision=1, max_chains=100) as srv:
        ids = [srv.submit(**r) for r, _ in reqs]
        max_run = 0
        while True:
            r, p = srv.tick()
            max_run = max(max_run, r)
            assert r <= 2                                  # 3 x 40 > 100
            if r == 0 and p == 0:
                break
        assert max_run == 2
        assert all(srv.poll(i)["state"] == gw.NS_REQ_DONE for i in ids)
    # an analysis larger than the budget still runs, alone
    with gw.Server(precision=1, max_chains=30) as srv:
        ids = [srv.submit(**r) for r, _ in reqs[:2]]
        while True:
            r, p = srv.tick()
            assert r <= 1
            if r == 0 and p == 0:
                break
        assert all(srv.poll(i)["state"] == gw.NS_REQ_DONE for i in ids)
    with pytest.raises(gw.GWNSError):
        gw.Server(precision=1, max_chains=-1)


def test_cancel(gw):
    reqs = [_analysis(20 + i) for i in range(3)]
    with gw.Server(precision=1, max_active=1) as srv:
        ids = [srv.submit(**r) for r, _ in reqs]
        srv.tick()
        assert srv.poll(ids[0])["state"] == gw.NS_REQ_RUNNING
        srv.cancel(ids[0])            # running
        srv.cancel(ids[1])            # pending
        assert srv.poll(ids[0])["state"] == gw.NS_REQ_CANCELLED
        assert srv.poll(ids[1])["state"] == gw.NS_REQ_CANCELLED
        srv.run_until_idle()
        assert srv.poll(ids[2])["state"] == gw.NS_REQ_DONE
        with pytest.raises(gw.GWNSError):
            srv.cancel(ids[2])


def test_footprint_counts_the_dead_list_growth(gw):
    """An analysis that runs past 64 n dead points doubles its dead list (8
    live points, 4 deleted per iteration, a negative stopping tolerance that is
    never met, and the server's cap of 200 iterations: 800 dead points, the
    list grows at iteration 129). The server adds the growth to the analysis'
    footprint and to the memory in use, so a request that fitted beside the
    analysis' admission footprint waits until the analysis is done."""
    long_req, dim = _analysis(50, n_live=8, k=4)
    long_req = dict(long_req, dlogz_stop=-1.0)
    other, _ = _analysis(51, n_live=8, k=4)
    with gw.Server(precision=1) as probe:
        fa = probe.poll(probe.submit(**long_req))["footprint"]
        fb = probe.poll(probe.submit(**other))["footprint"]
    dead64 = 64 * 8 * (dim + 3) * 8          # the initial dead list: u, log L, log w, n_live
    with gw.Server(precision=1, mem_budget=fa + fb + dead64 // 2, max_iter=200) as srv:
        ra = srv.submit(**long_req)
        for it in range(128):
            srv.tick()
            st = srv.poll(ra)
            assert st["state"] == gw.NS_REQ_RUNNING and st["footprint"] == fa, (it, st)
        srv.tick()                           # iteration 129 needs room for 516 dead points
        st = srv.poll(ra)
        assert st["state"] == gw.NS_REQ_RUNNING and st["footprint"] == fa + dead64
        rb = srv.submit(**other)
        srv.tick()
        assert srv.poll(rb)["state"] == gw.NS_REQ_PENDING
        srv.run_until_idle()
        sa, sb = srv.poll(ra), srv.poll(rb)
        assert sa["state"] == gw.NS_REQ_DONE and sa["iterations"] == 200
        assert sb["state"] == gw.NS_REQ_DONE and sb["t_admit"] >= sa["t_done"]
