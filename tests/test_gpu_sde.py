"""Single-diagram-enhancement weights (the multi-channel weights of the paper's
event-generation interface, Sec. 3.2) against the oracle's independent diagram
enumeration: weight = sum_h |amp_channel|^2 / sum_h sum_d |amp_d|^2."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_21039_gb300 as me  # noqa: E402
from paper_2507_21039_gb300.gen.plan import build_plan, diagram_lines  # noqa: E402
from paper_2507_21039_gb300.workloads import DR_MIN, MT, PT_MIN, WORKLOADS  # noqa: E402

FILTER_THRESHOLD = 1e-14   # the helicity filter's rule (max over probe events of |M_h|^2 / |M|^2)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def oracle_good_helicities(orc, name, mom):
    mt = 0.0 if name == "ee_mumu" else MT
    _, hel = orc.me2(name, mom, mt=mt, alpha=WORKLOADS[name].alpha, per_helicity=True)
    ratio = (hel / hel.sum(1, keepdims=True)).max(0)
    return [h for h in range(hel.shape[1]) if ratio[h] > FILTER_THRESHOLD]


def channels(P, n):
    """a spread of diagrams, including ones with a four-gluon vertex"""
    full = P.npar - 3
    quartic = [d for d in range(P.ndiagrams) if len(diagram_lines(P, d)) < full]
    pick = sorted(set([0, P.ndiagrams - 1, P.ndiagrams // 2] + quartic[:2] + list(range(1, P.ndiagrams, max(1, P.ndiagrams // n)))))
    return pick[: n + 3]


@pytest.mark.parametrize("name,nevt,prec,tol", [("ee_mumu", 16, "fp64", 1e-12), ("gg_ttx", 16, "fp64", 1e-12),
                                                ("gg_ttxg", 12, "fp64", 1e-12), ("gg_ttxgg", 8, "fp64", 1e-12),
                                                ("gg_ttxggg", 3, "fp64", 1e-12), ("gg_ttxgg", 8, "mixed", 1e-4),
                                                ("gg_ttxggg", 3, "mixed", 1e-4)])
def test_sde_weights_match_oracle(orc, name, nevt, prec, tol):
    w = WORKLOADS[name]
    mom, _, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, 0, nevt, w.cut_mask, PT_MIN, DR_MIN)
    mt = 0.0 if name == "ee_mumu" else MT
    good = oracle_good_helicities(orc, name, mom)
    d = torch.from_numpy(mom).cuda()
    h = me.workload_handle(name, prec)
    me.me_filter_helicities(h, d)
    assert me.me_good_helicities(h) == good          # index work: bit-exact
    P = build_plan(name)
    assert me.me_info(h)["ndiag"] == P.ndiagrams
    ref = [orc.sde(name, p, good, mt) for p in mom]
    index = {key: i for i, key in enumerate(ref[0][1])}
    for c in channels(P, 6):
        key = me.me_diagram_lines(h, c)
        assert key == diagram_lines(P, c)
        _, wgt = me.me_sigmakin_sde(h, d, c)
        got = wgt.cpu().numpy()
        exp = np.array([r[0][index[key]] / r[0].sum() for r in ref])
        assert np.all(np.abs(got - exp) <= tol * np.maximum(exp, 1e-300)), (c, key, got, exp)
    h.close()


@pytest.mark.parametrize("name", ["gg_ttx", "gg_ttxg"])
def test_sde_weights_sum_to_one_and_me2_unchanged(orc, name):
    w = WORKLOADS[name]
    mom, _, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, 100, 64, w.cut_mask, PT_MIN, DR_MIN)
    d = torch.from_numpy(mom).cuda()
    for prec in ("fp64", "fp32"):
        h = me.workload_handle(name, prec)
        base = me.me_sigmakin(h, d)
        total = torch.zeros_like(base)
        for c in range(me.me_info(h)["ndiag"]):
            me2, wgt = me.me_sigmakin_sde(h, d, c)
            assert torch.equal(me2, base)              # the weights ride along; |M|^2 unchanged
            assert bool(((wgt >= 0) & (wgt <= 1)).all())
            total += wgt
        tol = 1e-12 if prec == "fp64" else 1e-5
        assert float((total - 1).abs().max()) < tol
        h.close()


def test_sde_argument_errors(orc):
    w = WORKLOADS["gg_ttx"]
    mom, _, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, 0, 4, w.cut_mask, PT_MIN, DR_MIN)
    d = torch.from_numpy(mom).cuda()
    h = me.workload_handle("gg_ttx", "fp64")
    me.me_filter_helicities(h, d)
    for bad in (-1, 3):
        with pytest.raises(me.MEError):
            me.me_sigmakin_sde(h, d, bad)
    with pytest.raises(me.MEError):
        me.me_sigmakin_sde(h, torch.from_numpy(mom), 0, me2=torch.empty(4, dtype=torch.float64),
                           weight=torch.empty(4, dtype=torch.float64))
    with pytest.raises(me.MEError):
        me.me_diagram_lines(h, 3)
    h.close()
