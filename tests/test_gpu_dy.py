"""GPU parity of the Drell-Yan workload, u u~ -> e+ e- + n g (n = 0..3), the
paper's second standalone process (Sec. 4): photon and Z exchange with the
electroweak parameters of reading R15.

The CUDA path (through the C ABI) is compared with the FP64 CPU oracle
(`orc_dy_me2`: the colour-ordered quark-line recursion with one colourless
insertion, pinned in tests/test_oracle_dy.py) on seeded RAMBO points from the
oracle's own sampler.  Tolerances as for the other processes: FP64 within
1e-12 relative per event; FP32 and mixed median <= 1e-5, maximum <= 1e-3.
Batch sizes are ragged (not a multiple of a CTA's events).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_21039_gb300 as me  # noqa: E402
from paper_2507_21039_gb300.workloads import ALPHA_S, DR_MIN, DY_WORKLOADS, PT_MIN  # noqa: E402

FP64_TOL = 1e-12
LOW_MEDIAN, LOW_MAX = 1e-5, 1e-3
NGLUON = {"uux_epem": 0, "uux_epemg": 1, "uux_epemgg": 2, "uux_epemggg": 3}
SIZES = {"uux_epem": 1001, "uux_epemg": 1003, "uux_epemgg": 517, "uux_epemggg": 131}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.init()


def oracle_events(orc, name, n, ev0=0):
    w = DY_WORKLOADS[name]
    mom, _, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, ev0, n, w.cut_mask, PT_MIN, DR_MIN)
    return mom


def gpu_me2(name, prec, mom):
    h = me.workload_handle(name, prec)
    out = me.me_sigmakin(h, torch.from_numpy(np.ascontiguousarray(mom)).cuda())
    torch.cuda.synchronize()
    res = out.cpu().numpy()
    h.close()
    return res


@pytest.mark.parametrize("name", list(NGLUON))
def test_dy_fp64_parity(orc, name):
    mom = oracle_events(orc, name, SIZES[name])
    ref = orc.dy_me2(NGLUON[name], mom, alpha_s=ALPHA_S)
    got = gpu_me2(name, "fp64", mom)
    assert np.all(ref > 0)
    rel = np.abs(got / ref - 1)
    assert rel.max() < FP64_TOL, (rel.max(), int(np.argmax(rel)))


@pytest.mark.parametrize("prec", ["fp32", "mixed", "mixed64"])
@pytest.mark.parametrize("name", list(NGLUON))
def test_dy_low_precision_parity(orc, name, prec):
    mom = oracle_events(orc, name, SIZES[name])
    ref = orc.dy_me2(NGLUON[name], mom, alpha_s=ALPHA_S)
    rel = np.abs(gpu_me2(name, prec, mom) / ref - 1)
    assert np.median(rel) <= LOW_MEDIAN and rel.max() <= LOW_MAX, (np.median(rel), rel.max())


def test_dy_full_size_sampled(orc):
    """The 2^18-event u u~ -> e+ e- ggg batch in one launch: sampled events
    against the oracle one by one."""
    name = "uux_epemggg"
    w = DY_WORKLOADS[name]
    mom = oracle_events(orc, name, w.nevt)
    got = gpu_me2(name, "mixed", mom)
    idx = np.unique(np.r_[0, w.nevt - 1, np.random.default_rng(3).integers(0, w.nevt, 40)])
    ref = orc.dy_me2(3, mom[idx], alpha_s=ALPHA_S)
    rel = np.abs(got[idx] / ref - 1)
    assert np.median(rel) <= LOW_MEDIAN and rel.max() <= LOW_MAX
    assert np.all(np.isfinite(got)) and np.all(got > 0)


def test_dy_full_size_sampled_gg(orc):
    """The 2^20-event u u~ -> e+ e- gg batch of the benchmark workload in one
    launch (table kernel, FP32): sampled events against the oracle one by one."""
    name = "uux_epemgg"
    w = DY_WORKLOADS[name]
    mom = oracle_events(orc, name, w.nevt)
    got = gpu_me2(name, "fp32", mom)
    idx = np.unique(np.r_[0, w.nevt - 1, np.random.default_rng(4).integers(0, w.nevt, 60)])
    ref = orc.dy_me2(2, mom[idx], alpha_s=ALPHA_S)
    rel = np.abs(got[idx] / ref - 1)
    assert np.median(rel) <= LOW_MEDIAN and rel.max() <= LOW_MAX
    assert np.all(np.isfinite(got)) and np.all(got > 0)


@pytest.mark.parametrize("name", list(NGLUON))
def test_dy_kept_helicities_conserve_helicity(orc, name):
    """The FP64 helicity filter keeps exactly the configurations with opposite
    u, u~ and opposite e+, e- helicity bits (massless fermions: the others vanish
    exactly), 2 x 2 x 2^n of them; the table kernels compute only the table
    variants these read."""
    npar = DY_WORKLOADS[name].npar
    mom = oracle_events(orc, name, 64)
    h = me.workload_handle(name, "fp64")
    me.me_filter_helicities(h, torch.from_numpy(mom).cuda())
    good = me.me_good_helicities(h)
    h.close()
    bit = lambda hh, p: (hh >> (npar - 1 - p)) & 1
    expect = [hh for hh in range(1 << npar) if bit(hh, 0) != bit(hh, 1) and bit(hh, 2) != bit(hh, 3)]
    assert list(good) == expect and len(expect) == 4 << NGLUON[name]


@pytest.mark.parametrize("name", ["uux_epemg", "uux_epemgg", "uux_epemggg"])
def test_dy_gauge_invariance_on_gpu(orc, name):
    """A gluon's polarisation replaced by its momentum: every helicity
    amplitude vanishes, so |M|^2 drops by many orders (FP64)."""
    mom = oracle_events(orc, name, 64)
    d = torch.from_numpy(mom).cuda()
    h = me.workload_handle(name, "fp64")
    ref = me.me_sigmakin(h, d).cpu().numpy()
    npar = DY_WORKLOADS[name].npar
    for g in range(4, npar):
        me.me_set_option(h, me.ME_OPT_GAUGE_CHECK, g)
        got = me.me_sigmakin(h, d).cpu().numpy()
        assert np.all(got < 1e-20 * ref), (g, (got / ref).max())
    me.me_set_option(h, me.ME_OPT_GAUGE_CHECK, -1)
    with pytest.raises(me.MEError):   # the quarks and leptons are not gluons
        me.me_set_option(h, me.ME_OPT_GAUGE_CHECK, 2)
    h.close()


def test_dy_abi_limits():
    """Drell-Yan handles: massless only, default alpha_s, no channel weights."""
    with pytest.raises(me.MEError):
        me.me_init("uux_epemg", [0.0, 0.0, 0.0, 0.0, 1.0], [0.118], "fp64")
    h = me.workload_handle("uux_epemgg", "fp64")
    info = me.me_info(h)
    assert (info["npar"], info["nhel"], info["ncol"], info["ndiag"]) == (6, 64, 2, 8)
    d = torch.zeros((4, 6, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(me.MEError):
        me.me_sigmakin_sde(h, d, 0)
    h.close()
