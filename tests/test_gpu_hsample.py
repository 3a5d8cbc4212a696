"""Helicity sampling (one helicity per event, |M_h|^2 / p_h) against the oracle's
per-helicity |M_h|^2 with the same uniforms and the oracle's own probabilities."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_21039_gb300 as me  # noqa: E402
from paper_2507_21039_gb300.workloads import DR_MIN, MT, PT_MIN, WORKLOADS  # noqa: E402

FILTER_THRESHOLD = 1e-14


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def oracle_sampling(orc, name, mom, uniform=False):
    """kept helicities, per-helicity contributions to |M|^2, probabilities and
    cumulative sums, from the oracle alone (the filter rule, the mean share of
    each kept helicity mixed 0.9 : 0.1 with uniform)"""
    w = WORKLOADS[name]
    mt = 0.0 if name == "ee_mumu" else MT
    tot, hel = orc.me2(name, mom, mt=mt, alpha=w.alpha, per_helicity=True)
    share = hel / hel.sum(1, keepdims=True)
    good = [h for h in range(hel.shape[1]) if share[:, h].max() > FILTER_THRESHOLD]
    contrib = hel * (tot / hel.sum(1))[:, None]
    q = share.mean(0)[good]
    n = len(good)
    p = np.full(n, 1.0 / n) if uniform else 0.9 * q / q.sum() + 0.1 / n
    cdf = np.cumsum(p)
    cdf[-1] = 1.0
    return good, contrib, p, cdf, tot


@pytest.mark.parametrize("name,prec,tol", [("ee_mumu", "fp64", 1e-12), ("gg_ttx", "fp64", 1e-12),
                                           ("gg_ttxg", "fp64", 1e-12), ("gg_ttxgg", "fp64", 1e-12),
                                           ("gg_ttxggg", "fp64", 1e-12), ("gg_ttxg", "mixed", 1e-5),
                                           ("gg_ttxgg", "fp32", 1e-5), ("gg_ttxgg", "mixed", 1e-5),
                                           ("gg_ttxggg", "mixed", 1e-5)])
@pytest.mark.parametrize("uniform", [False, True])
def test_hsample_matches_oracle(orc, name, prec, tol, uniform):
    w = WORKLOADS[name]
    mom, _, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, 0, 256 if name != "gg_ttxggg" else 48, w.cut_mask,
                          PT_MIN, DR_MIN)
    u = np.random.default_rng(17).random(len(mom))
    good, contrib, p, cdf, tot = oracle_sampling(orc, name, mom, uniform)
    d = torch.from_numpy(mom).cuda()
    h = me.workload_handle(name, prec)
    me.me_filter_helicities(h, d)
    me.me_set_option(h, me.ME_OPT_HSAMPLE_UNIFORM, int(uniform))
    assert me.me_good_helicities(h) == good
    assert np.allclose(me.me_hsample_probabilities(h), p, rtol=1e-12, atol=0)
    got, hel = me.me_sigmakin_hsample(h, d, torch.from_numpy(u).cuda())
    got, hel = got.cpu().numpy(), hel.cpu().numpy()
    h.close()
    idx = np.minimum(np.searchsorted(cdf, u, side="right"), len(good) - 1)
    # both sides place u among the cumulative probabilities in FP64; the
    # adaptive ones differ in the last bits, so u that close to a bin edge is skipped
    clear = np.abs(u[:, None] - cdf[None, :]).min(1) > (0.0 if uniform else 1e-12)
    assert clear.sum() > 0.9 * len(u)
    sel = np.array(good)[idx]
    assert np.array_equal(hel[clear], sel[clear])
    exp = contrib[np.arange(len(u)), sel] / p[idx]
    # rounding of one helicity's |M_h|^2 scales with the event's amplitudes,
    # not with that helicity's (possibly suppressed) share: errors are measured
    # against the event's |M|^2, weighted like the estimate (1 / p_h)
    err = np.abs(got - exp)[clear] / (tot / p[idx])[clear]
    assert err.max() <= tol, err.max()


@pytest.mark.parametrize("name", ["gg_ttx", "gg_ttxg"])
def test_hsample_is_unbiased(orc, name):
    """One event, N stratified uniforms u_i = (i + 1/2) / N: the mean of the
    sampled |M_h|^2 / p_h is the helicity sum up to sum_i |M_i|^2 / (p_i N)."""
    w = WORKLOADS[name]
    mom, _, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, 5, 1, w.cut_mask, PT_MIN, DR_MIN)
    n = 8192
    d = torch.from_numpy(np.repeat(mom, n, axis=0)).cuda()
    u = torch.from_numpy((np.arange(n) + 0.5) / n).cuda()
    h = me.workload_handle(name, "fp64")
    me.me_filter_helicities(h, d[:1])
    full = me.me_sigmakin(h, d[:1]).item()
    got, _ = me.me_sigmakin_hsample(h, d, u)
    p = np.array(me.me_hsample_probabilities(h))
    h.close()
    good, contrib, _, _, _ = oracle_sampling(orc, name, mom)
    bound = np.sum(contrib[0, good] / p) / n
    assert abs(got.mean().item() - full) <= bound + 1e-12 * full
