"""Serving layer on the GPU: continuous batching, admission by device-memory
budget, CUDA-graph replay, timeouts and cancellation, and per-event results
that are the same alone and in a mix of concurrent requests (bitwise)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_21039_gb300.workloads import DR_MIN, MT, PT_MIN, WORKLOADS  # noqa: E402


@pytest.fixture(scope="module")
def srvmod():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.init()
    from paper_2507_21039_gb300 import serving

    return serving


def pinned_events(orc, name, n, ev0=0):
    w = WORKLOADS[name]
    mom, _, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, ev0, n, w.cut_mask, PT_MIN, DR_MIN)
    t = torch.empty(mom.shape, dtype=torch.float64, pin_memory=True)
    t.copy_(torch.from_numpy(mom))
    return t, mom


def out_like(n):
    return torch.full((n,), -1.0, dtype=torch.float64, pin_memory=True)


@pytest.mark.parametrize("graphs", [True, False])
def test_same_alone_and_in_the_mix(orc, srvmod, graphs):
    import paper_2507_21039_gb300 as me

    srv = srvmod.Server(lanes=3, max_batch=1 << 14, use_graphs=graphs)
    burst = [("gg_ttxgg", 8192, "fp64"), ("gg_ttx", 3000, "mixed"), ("gg_ttxgg", 1234, "mixed"),
             ("ee_mumu", 999, "fp64"), ("gg_ttxg", 4096, "mixed"), ("gg_ttxgg", 2048, "mixed"),
             ("gg_ttx", 517, "fp64"), ("gg_ttxgg", 300, "fp64")]
    # resident handles first (creating one filters its helicities, which waits for the device)
    for name, prec in sorted({(b[0], b[2]) for b in burst}):
        m, _ = pinned_events(orc, name, 64)
        srv.wait(srv.submit(name, m, out_like(64), prec))
    warm = srv.stats()["requests"]
    probe, probe_np = pinned_events(orc, "gg_ttxgg", 777, ev0=5000)
    alone = out_like(777)
    srv.wait(srv.submit("gg_ttxgg", probe, alone, "mixed"))
    # the same request amid a burst of other processes, precisions and sizes (the
    # long FP64 batch first: the others start while it runs)
    others = []
    for i, (name, n, prec) in enumerate(burst):
        m, _ = pinned_events(orc, name, n, ev0=100 * i)
        o = out_like(n)
        others.append((name, prec, m, o, srv.submit(name, m, o, prec)))
    mixed = out_like(777)
    t = srv.submit("gg_ttxgg", probe, mixed, "mixed")
    more = out_like(777)
    t2 = srv.submit("gg_ttxgg", probe, more, "mixed")
    for name, prec, m, o, tk in others:
        srv.wait(tk)
    srv.wait(t)
    srv.wait(t2)
    assert torch.equal(alone, mixed) and torch.equal(alone, more)
    # and equal to the direct ABI call on a handle of the same precision
    h = me.workload_handle("gg_ttxgg", "mixed")
    direct = me.me_sigmakin(h, probe.cuda()).cpu()
    h.close()
    assert torch.equal(direct, alone)
    for name, prec, m, o, tk in others:
        ref = orc.me2(name, m.numpy()[:64], mt=MT, alpha=WORKLOADS[name].alpha)
        rel = np.abs(o.numpy()[:64] / ref - 1)
        assert rel.max() < (1e-12 if prec == "fp64" else 1e-3)
    st = srv.stats()
    assert st["requests"] == warm + 11 and st["failed"] == 0
    if graphs:
        assert st["graph_instantiations"] + st["graph_updates"] >= st["batches"]
    # the burst's batches ran at the same time on the device (timing events
    # around each batch on its lane's stream), not one after another
    assert st["max_lanes_busy"] >= 2 and st["max_device_concurrency"] >= 2, st
    srv.close()


def test_admission_by_device_memory_budget(orc, srvmod):
    npar = 6
    per_event = 8 * (4 * npar + 1)
    budget = per_event * 5000       # room for one 4000-event batch at a time
    srv = srvmod.Server(lanes=4, max_batch=4000, hbm_budget_bytes=budget)
    m, _ = pinned_events(orc, "gg_ttxgg", 4000)
    outs, tks = [], []
    for i in range(6):
        o = out_like(4000)
        outs.append(o)
        tks.append(srv.submit("gg_ttxgg", m, o, "mixed"))
    for t in tks:
        srv.wait(t)
    st = srv.stats()
    assert st["max_bytes_in_flight"] <= budget
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    srv.close()


def test_timeout_cancel_and_bad_requests(orc, srvmod):
    import paper_2507_21039_gb300 as me

    srv = srvmod.Server(lanes=1, max_batch=1 << 16)
    big, _ = pinned_events(orc, "gg_ttxgg", 1 << 16)
    o1, o2, o3 = out_like(1 << 16), out_like(1 << 16), out_like(1 << 16)
    t1 = srv.submit("gg_ttxgg", big, o1, "fp64")        # slow: keeps the only lane busy
    t2 = srv.submit("gg_ttxgg", big, o2, "mixed")
    t3 = srv.submit("gg_ttxg", big[:, :5].contiguous(), o3, "mixed")
    with pytest.raises(me.MEError) as e:
        srv.wait(t2, timeout_ms=0)
    assert e.value.code == me.ME_ETIMEOUT
    srv.cancel(t3)                                        # still queued: dropped
    with pytest.raises(me.MEError):
        srv.wait(t3, timeout_ms=0)                        # ticket released
    assert srv.wait(t1) > 0 and srv.wait(t2) > 0
    assert torch.all(o3 == -1.0)                          # never written
    with pytest.raises(me.MEError) as e:
        srv.submit("no_such_process", big, o1)
    assert e.value.code == me.ME_EINVAL
    too_big = torch.zeros(((1 << 16) + 1, 6, 4), dtype=torch.float64)
    with pytest.raises(me.MEError):
        srv.submit("gg_ttxgg", too_big, out_like((1 << 16) + 1))
    st = srv.stats()
    assert st["cancelled"] == 1
    srv.close()


def test_nonfinite_event_does_not_leak_into_neighbours(orc, srvmod):
    srv = srvmod.Server(lanes=2, max_batch=1 << 12)
    m, _ = pinned_events(orc, "gg_ttxg", 256)
    good = out_like(256)
    srv.wait(srv.submit("gg_ttxg", m, good, "mixed"))
    bad = m.clone().pin_memory()
    bad[17, 4, 2] = float("nan")
    res = out_like(256)
    srv.wait(srv.submit("gg_ttxg", bad, res, "mixed"))
    keep = torch.ones(256, dtype=torch.bool)
    keep[17] = False
    assert torch.equal(res[keep], good[keep])
    assert not torch.isfinite(res[17])
    srv.close()


def test_smaller_request_passes_one_that_does_not_fit(orc, srvmod):
    """Admission without head-of-line blocking: while a large batch holds most
    of the budget, an older large request that does not fit waits and a later
    small one that fits starts (and finishes) first; every result is right."""
    npar = 6
    per_event = 8 * (4 * npar + 1)
    srv = srvmod.Server(lanes=4, max_batch=1 << 14, hbm_budget_bytes=per_event * 12000)
    big, big_np = pinned_events(orc, "gg_ttxgg", 8000)
    small, small_np = pinned_events(orc, "gg_ttx", 500)
    o_a, o_b, o_c = out_like(8000), out_like(8000), out_like(500)
    ta = srv.submit("gg_ttxgg", big, o_a, "fp64")    # holds 8000 events' bytes for a while
    tb = srv.submit("gg_ttxgg", big, o_b, "mixed")   # does not fit beside it: waits
    tc = srv.submit("gg_ttx", small, o_c, "mixed")   # fits: starts before tb
    lat_c = srv.wait(tc)
    lat_b = srv.wait(tb)
    srv.wait(ta)
    st = srv.stats()
    assert st["head_bypasses"] >= 1 and lat_c < lat_b, (st, lat_c, lat_b)
    assert st["max_bytes_in_flight"] <= per_event * 12000
    ref = orc.me2("gg_ttx", small_np[:64], mt=MT, alpha=WORKLOADS["gg_ttx"].alpha)
    assert np.abs(o_c.numpy()[:64] / ref - 1).max() < 1e-3
    ref = orc.me2("gg_ttxgg", big_np[:16], mt=MT, alpha=WORKLOADS["gg_ttxgg"].alpha)
    assert np.abs(o_a.numpy()[:16] / ref - 1).max() < 1e-12
    assert np.abs(o_b.numpy()[:16] / ref - 1).max() < 1e-3
    srv.close()


def test_budget_counts_launch_scratch_and_serves_drell_yan(orc, srvmod):
    """An FP64 gg -> t t~ ggg batch is charged its launch's colour-flow scratch
    (240 KB per resident CTA) beside its momenta and |M|^2; a Drell-Yan request
    is served like the others."""
    from paper_2507_21039_gb300.workloads import ALPHA_S, DY_WORKLOADS

    srv = srvmod.Server(lanes=2, max_batch=1 << 12)
    m, _ = pinned_events(orc, "gg_ttxggg", 64)
    o = out_like(64)
    srv.wait(srv.submit("gg_ttxggg", m, o, "fp64"))
    st = srv.stats()
    assert st["max_bytes_in_flight"] >= 64 * 8 * (4 * 7 + 1) + 240 * 1024, st
    w = DY_WORKLOADS["uux_epemgg"]
    dmom, _, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, 0, 300, w.cut_mask, PT_MIN, DR_MIN)
    d = torch.empty(dmom.shape, dtype=torch.float64, pin_memory=True)
    d.copy_(torch.from_numpy(dmom))
    od = out_like(300)
    srv.wait(srv.submit("uux_epemgg", d, od, "fp64"))
    ref = orc.dy_me2(2, dmom, alpha_s=ALPHA_S)
    assert np.abs(od.numpy() / ref - 1).max() < 1e-12
    srv.close()
