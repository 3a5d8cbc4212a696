"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Inputs are seeded RAMBO points from the oracle's own sampler (never from the
CUDA path).  Tolerances: FP64 within 1e-12 relative per event; FP32 and mixed
with median relative error <= 1e-5 and maximum <= 1e-3 against FP64.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_21039_gb300 as me  # noqa: E402
from paper_2507_21039_gb300.workloads import DR_MIN, MT, PT_MIN, WORKLOADS  # noqa: E402

BUILT = ("ee_mumu", "gg_ttx", "gg_ttxg", "gg_ttxgg", "gg_ttxggg")
FP64_TOL = 1e-12
LOW_MEDIAN, LOW_MAX = 1e-5, 1e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.init()


def oracle_events(orc, name, n, ev0=0):
    w = WORKLOADS[name]
    mom, wt, att = orc.rambo(w.seed, w.sqrt_s, w.masses_final, ev0, n, w.cut_mask, PT_MIN, DR_MIN)
    return mom


def gpu_me2(name, prec, mom, filter_mom=None):
    h = me.workload_handle(name, prec)
    d = torch.from_numpy(np.ascontiguousarray(mom)).cuda()
    if filter_mom is not None:
        me.me_filter_helicities(h, torch.from_numpy(filter_mom).cuda())
    out = me.me_sigmakin(h, d)
    torch.cuda.synchronize()
    res = out.cpu().numpy()
    h.close()
    return res


SIZES = {"ee_mumu": 1001, "gg_ttx": 1001, "gg_ttxg": 1003, "gg_ttxgg": 517, "gg_ttxggg": 67}


@pytest.mark.parametrize("name", BUILT)
def test_fp64_parity(orc, name):
    n = SIZES[name]
    mom = oracle_events(orc, name, n)
    ref = orc.me2(name, mom, mt=MT, alpha=WORKLOADS[name].alpha)
    got = gpu_me2(name, "fp64", mom)
    rel = np.abs(got / ref - 1)
    assert rel.max() < FP64_TOL, (rel.max(), np.argmax(rel))


@pytest.mark.parametrize("prec", ["fp32", "mixed", "mixed64"])
@pytest.mark.parametrize("name", ["gg_ttx", "gg_ttxg", "gg_ttxgg", "gg_ttxggg"])
def test_low_precision_parity(orc, name, prec):
    n = SIZES[name]
    mom = oracle_events(orc, name, n)
    ref = orc.me2(name, mom, mt=MT, alpha=WORKLOADS[name].alpha)
    got = gpu_me2(name, prec, mom)
    rel = np.abs(got / ref - 1)
    assert np.median(rel) <= LOW_MEDIAN and rel.max() <= LOW_MAX, (np.median(rel), rel.max())


@pytest.mark.parametrize("name", BUILT)
def test_per_helicity_parity_and_filter(orc, name):
    w = WORKLOADS[name]
    mom = oracle_events(orc, name, 67 if name != "gg_ttxggg" else 19)
    ref, ref_hel = orc.me2(name, mom, mt=MT, alpha=w.alpha, per_helicity=True)
    h = me.workload_handle(name, "fp64")
    d = torch.from_numpy(mom).cuda()
    ngood = me.me_filter_helicities(h, d)
    good = me.me_good_helicities(h)
    # the filter rule evaluated on the oracle's per-helicity values (same probe events)
    ratio = (ref_hel / ref_hel.sum(1, keepdims=True)).max(0)
    expect = [i for i in range(ref_hel.shape[1]) if ratio[i] > 1e-14]
    assert good == expect and ngood == len(expect)
    me2 = torch.empty(len(mom), dtype=torch.float64, device="cuda")
    hel = torch.empty((len(mom), ngood), dtype=torch.float64, device="cuda")
    me.me_sigmakin_hel(h, d, me2, hel)
    torch.cuda.synchronize()
    got_hel = hel.cpu().numpy()
    iden = orc.iden(name)
    # each helicity's contribution, relative to its event's total
    err = np.abs(got_hel * iden - ref_hel[:, good]) / ref_hel.sum(1, keepdims=True)
    assert err.max() < FP64_TOL, err.max()
    assert np.allclose(got_hel.sum(1), me2.cpu().numpy(), rtol=1e-14, atol=0)
    h.close()


def test_expected_helicity_counts(orc):
    counts = {}
    for name in BUILT:
        mom = oracle_events(orc, name, 64)
        h = me.workload_handle(name, "fp64")
        counts[name] = me.me_filter_helicities(h, torch.from_numpy(mom).cuda())
        h.close()
    assert counts["ee_mumu"] == 4
    assert counts["gg_ttx"] == 12


@pytest.mark.parametrize("name", ["gg_ttx", "gg_ttxg", "gg_ttxgg", "gg_ttxggg"])
def test_gauge_invariance_on_gpu(orc, name):
    """Ward identity: a gluon polarisation replaced by its momentum gives zero.

    In floating point the residual amplitude is rounding of diagrams that each
    scale with the gluon energy E_g (the momentum replaces a unit polarisation),
    so |M_k|^2 / (|M|^2 E_g^2) is bounded by (C u)^2, u the unit roundoff and C
    the cancellation between diagrams; C = 1000 is used.  A wrong vertex or
    sign gives a ratio of order one."""
    mom = oracle_events(orc, name, 33)
    d = torch.from_numpy(mom).cuda()
    for prec, u in (("fp64", 2.0 ** -53), ("fp32", 2.0 ** -24)):
        tol = (1000 * u) ** 2
        h = me.workload_handle(name, prec)
        base = me.me_sigmakin(h, d).cpu().numpy()
        for g in [0, 1] + list(range(4, WORKLOADS[name].npar)):
            me.me_set_option(h, me.ME_OPT_GAUGE_CHECK, g)
            z = me.me_sigmakin(h, d).cpu().numpy()
            ratio = np.abs(z / base) / mom[:, g, 0] ** 2
            assert ratio.max() < tol, (prec, g, ratio.max(), tol)
        me.me_set_option(h, me.ME_OPT_GAUGE_CHECK, -1)
        again = me.me_sigmakin(h, d).cpu().numpy()
        assert np.array_equal(again, base)
        h.close()


def test_edge_cases(orc):
    name = "gg_ttxg"
    mom = oracle_events(orc, name, 40)
    ref = orc.me2(name, mom, mt=MT)
    h = me.workload_handle(name, "fp64")
    d = torch.from_numpy(mom).cuda()
    me.me_filter_helicities(h, d)
    # empty batch is a no-op
    empty = torch.empty((0, 5, 4), dtype=torch.float64, device="cuda")
    out0 = me.me_sigmakin(h, empty)
    assert out0.numel() == 0
    # single event, ragged sizes, offsets: each event independent of its batch
    full = me.me_sigmakin(h, d).cpu().numpy()
    assert np.abs(full / ref - 1).max() < FP64_TOL
    for lo, hi in ((0, 1), (7, 8), (3, 40), (13, 29)):
        part = me.me_sigmakin(h, d[lo:hi].contiguous()).cpu().numpy()
        assert np.array_equal(part, full[lo:hi])
    # host buffers (numpy in, numpy out): staged path, same numbers
    host = me.me_sigmakin(h, np.ascontiguousarray(mom))
    assert np.array_equal(host, full)
    # misaligned momentum pointer (not 16-byte aligned) still works
    buf = torch.zeros(40 * 5 * 4 + 1, dtype=torch.float64, device="cuda")
    mis = buf[1:].view(40, 5, 4)
    mis.copy_(d)
    assert np.array_equal(me.me_sigmakin(h, mis).cpu().numpy(), full)
    h.close()


def test_error_paths(orc):
    name = "gg_ttx"
    mom = oracle_events(orc, name, 8)
    d = torch.from_numpy(mom).cuda()
    h = me.workload_handle(name, "fp64")
    me.me_set_option(h, me.ME_OPT_REQUIRE_FILTER, 1)
    with pytest.raises(me.MEError) as e:
        me.me_sigmakin(h, d)
    assert e.value.code == me.ME_ENOTFILTERED
    me.me_filter_helicities(h, d)
    me.me_set_option(h, me.ME_OPT_CHECK_FINITE, 1)
    bad = d.clone()
    bad[3, 2, 1] = float("nan")
    with pytest.raises(me.MEError) as e:
        me.me_sigmakin(h, bad)
    assert e.value.code == me.ME_ENONFINITE
    ok = me.me_sigmakin(h, d).cpu().numpy()
    assert np.all(np.isfinite(ok))
    with pytest.raises(me.MEError):
        me.me_set_option(h, me.ME_OPT_GAUGE_CHECK, 2)  # not a gluon
    h.close()
    # lazy filtering on the first batch gives the same numbers as explicit filtering
    h1 = me.workload_handle(name, "fp64")
    lazy = me.me_sigmakin(h1, d).cpu().numpy()
    assert np.array_equal(lazy, ok)
    h1.close()


# ---------------------------------------------------------------- sampler
@pytest.mark.parametrize("name", list(WORKLOADS))
def test_rambo_parity(orc, name):
    w = WORKLOADS[name]
    n = 2000
    ev0 = 12345
    masses = [0.0, 0.0] + list(w.masses_final)
    wt = torch.empty(n, dtype=torch.float64, device="cuda")
    got = me.rambo_sample(w.seed, ev0, n, w.sqrt_s, masses, me.cuts_for(name), weights_out=wt, check=True)
    mom, owt, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, ev0, n, w.cut_mask, PT_MIN, DR_MIN)
    g = got.cpu().numpy()
    diff = np.abs(g - mom).max(axis=(1, 2)) / w.sqrt_s
    # same attempt chosen for every event (a different attempt is an O(1) difference);
    # RAMBO's boost amplifies last-ulp differences of log/sin/cos on nearly collinear draws
    assert diff.max() < 1e-9, diff.max()
    assert np.median(diff) < 1e-14
    assert np.allclose(wt.cpu().numpy(), owt, rtol=1e-9, atol=0)


def test_rambo_full_size_sampled(orc):
    """Full-size headline batch (2^20 events): sampled events equal the oracle's."""
    w = WORKLOADS["gg_ttxgg"]
    masses = [0.0, 0.0] + list(w.masses_final)
    got = me.rambo_sample(w.seed, 0, w.nevt, w.sqrt_s, masses, me.cuts_for("gg_ttxgg"), check=True)
    idx = np.unique(np.r_[0, w.nevt - 1, np.random.default_rng(9).integers(0, w.nevt, 64)])
    g = got[torch.from_numpy(idx).cuda()].cpu().numpy()
    for i, e in enumerate(idx):
        mom, _, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, int(e), 1, w.cut_mask, PT_MIN, DR_MIN)
        assert np.abs(g[i] - mom[0]).max() < 1e-9 * w.sqrt_s


@pytest.mark.parametrize("name,prec", [("gg_ttxgg", "mixed"), ("gg_ttxgg", "fp64"), ("gg_ttxgg", "fp32"),
                                       ("gg_ttx", "fp64"), ("gg_ttxg", "fp32"), ("gg_ttxg", "mixed"),
                                       ("gg_ttxggg", "mixed"), ("gg_ttxggg", "fp64")])
def test_full_size_sampled_parity(orc, name, prec):
    """Full-size batch in the benchmark's launch configuration; sampled
    events checked one by one against the oracle."""
    w = WORKLOADS[name]
    mom, _, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, 0, w.nevt, w.cut_mask, PT_MIN, DR_MIN)
    h = me.workload_handle(name, prec)
    d = torch.from_numpy(mom).cuda()
    out = me.me_sigmakin(h, d).cpu().numpy()
    h.close()
    idx = np.unique(np.r_[0, w.nevt - 1, np.random.default_rng(11).integers(0, w.nevt, 96 if name != "gg_ttxggg" else 30)])
    ref = orc.me2(name, mom[idx], mt=MT, alpha=w.alpha)
    rel = np.abs(out[idx] / ref - 1)
    if prec == "fp64":
        assert rel.max() < FP64_TOL
    else:
        assert np.median(rel) <= LOW_MEDIAN and rel.max() <= LOW_MAX
    assert np.all(np.isfinite(out)) and np.all(out > 0)


@pytest.mark.parametrize("name,prec", [("gg_ttx", "fp64"), ("gg_ttxg", "mixed")])
def test_host_buffer_pipeline_matches_device(name, prec):
    """Host buffers of 300000 events (two full pipeline chunks and a ragged
    tail) through rambo_sample and me_sigmakin: bitwise the device-buffer
    results, weights included."""
    w = WORKLOADS[name]
    n = 300000
    masses = [0.0, 0.0] + list(w.masses_final)
    cuts = me.cuts_for(name)
    d_mom = me.rambo_sample(w.seed, 7, n, w.sqrt_s, masses, cuts, check=True)
    d_wt = torch.empty(n, dtype=torch.float64, device="cuda")
    me.rambo_sample(w.seed, 7, n, w.sqrt_s, masses, cuts, momenta_out=d_mom, weights_out=d_wt, check=True)
    h_mom = torch.empty((n, w.npar, 4), dtype=torch.float64, pin_memory=True)
    h_wt = torch.empty(n, dtype=torch.float64, pin_memory=True)
    me.rambo_sample(w.seed, 7, n, w.sqrt_s, masses, cuts, momenta_out=h_mom, weights_out=h_wt, check=True)
    assert torch.equal(h_mom, d_mom.cpu()) and torch.equal(h_wt, d_wt.cpu())
    h = me.workload_handle(name, prec)
    me.me_filter_helicities(h, d_mom[:4096])
    d_me2 = me.me_sigmakin(h, d_mom)
    h_me2 = torch.empty(n, dtype=torch.float64, pin_memory=True)
    me.me_sigmakin(h, h_mom, h_me2)
    assert torch.equal(h_me2, d_me2.cpu())
    pageable = h_mom.numpy().copy()   # pageable host memory takes the same path
    assert np.array_equal(me.me_sigmakin(h, pageable), d_me2.cpu().numpy())
    h.close()


def test_mixed_uses_tensor_core_colour_sum(orc):
    """gg -> t t~ ggg mixed: the 120-flow colour sum runs on BF16 tensor cores
    (hi/lo split, FP32 accumulation).  Its results differ bitwise from the FP32
    scalar colour sum but both agree with the FP64 oracle within the FP32
    tolerances; per-helicity contributions add up to the event total.  At 24
    flows (gg -> t t~ g g) the mixed mode's colour sum is the FP32 scalar one
    (measured faster there), so mixed and FP32 agree bitwise."""
    name = "gg_ttxggg"
    w = WORKLOADS[name]
    mom = oracle_events(orc, name, 64)
    ref = orc.me2(name, mom, mt=MT, alpha=w.alpha)
    d = torch.from_numpy(mom).cuda()
    out = {}
    for prec in ("fp32", "mixed"):
        h = me.workload_handle(name, prec)
        me.me_filter_helicities(h, d)
        ngood = len(me.me_good_helicities(h))
        me2 = torch.empty(len(mom), dtype=torch.float64, device="cuda")
        hel = torch.empty((len(mom), ngood), dtype=torch.float64, device="cuda")
        me.me_sigmakin_hel(h, d, me2, hel)
        plain = me.me_sigmakin(h, d)
        torch.cuda.synchronize()
        assert torch.equal(plain, me2)
        assert np.allclose(hel.sum(1).cpu().numpy(), me2.cpu().numpy(), rtol=1e-6, atol=0)
        out[prec] = me2.cpu().numpy()
        h.close()
    assert not np.array_equal(out["fp32"], out["mixed"])
    for prec in ("fp32", "mixed"):
        rel = np.abs(out[prec] / ref - 1)
        assert np.median(rel) <= LOW_MEDIAN and rel.max() <= LOW_MAX, (prec, np.median(rel), rel.max())
    mom2 = oracle_events(orc, "gg_ttxgg", 300)
    assert np.array_equal(gpu_me2("gg_ttxgg", "fp32", mom2), gpu_me2("gg_ttxgg", "mixed", mom2))
