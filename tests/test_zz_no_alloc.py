"""The helicity filter that allocates no device memory.

Some host programs cannot let a library allocate device memory -- they reserve
the device's memory up front in their own pool, or run loops in which
cudaMalloc / cudaFree (which may synchronise the whole device) are not
acceptable.  me_filter_helicities_noalloc serves them with a fixed scratch array
inside the library.  This file checks, through the C ABI, that it keeps the
same helicities as the ordinary (allocating) filter on two calls in a row, that
the |M|^2 computed afterwards agrees within the FP64 tolerance of the other
tests, that device free memory does not change (also for gg_ttxggg, whose FP64
kernel takes its colour-flow scratch from the same fixed array), and that
oversized or host inputs are refused.  It is collected last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_21039_gb300.workloads import DR_MIN, MT, PT_MIN, WORKLOADS  # noqa: E402

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def me():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2507_21039_gb300 as lib

    torch.cuda.init()
    return lib


# (process, probe events, events checked against the oracle).  gg_ttxggg's FP64
# kernel keeps its colour-flow vectors in global memory: the no-alloc filter
# takes them from the same fixed array, so its probe batch is smaller.
CASES = [("gg_ttx", 2000, 50), ("gg_ttxgg", 2000, 50), ("gg_ttxggg", 1000, 12)]


@pytest.mark.parametrize("name,nprobe,ncheck", CASES, ids=[c[0] for c in CASES])
def test_noalloc_filter_matches_allocating_filter(orc, me, name, nprobe, ncheck):
    w = WORKLOADS[name]
    mom, _, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, 0, nprobe, w.cut_mask, PT_MIN, DR_MIN)
    d = torch.from_numpy(mom).cuda()
    ref = me.workload_handle(name, "fp64")
    n_ref = me.me_filter_helicities(ref, d)
    good_ref = me.me_good_helicities(ref)
    me2_ref = me.me_sigmakin(ref, d).cpu().numpy()
    ref.close()
    oracle_me2 = orc.me2(name, mom[:ncheck], mt=MT, alpha=w.alpha)

    h = me.workload_handle(name, "fp64")
    torch.cuda.synchronize()
    for call in range(2):
        free_before = torch.cuda.mem_get_info()[0]
        n = me.me_filter_helicities_noalloc(h, d)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        assert free_after == free_before, (call, free_before, free_after)
        assert n == n_ref
        assert me.me_good_helicities(h) == good_ref
        got = me.me_sigmakin(h, d).cpu().numpy()
        assert np.abs(got / me2_ref - 1).max() <= FP64_TOL
        assert np.abs(got[:ncheck] / oracle_me2 - 1).max() <= FP64_TOL
    h.close()


def test_noalloc_filter_rejects_what_it_cannot_hold(orc, me):
    w = WORKLOADS["gg_ttxgg"]
    h = me.workload_handle("gg_ttxgg", "fp64")
    big = torch.zeros((20000, w.npar, 4), dtype=torch.float64, device="cuda")   # 20000 x 65 x 8 B > 4 MiB
    with pytest.raises(me.MEError) as e:
        me.me_filter_helicities_noalloc(h, big)
    assert e.value.code == me.ME_ETOOLARGE
    mom, _, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, 0, 16, w.cut_mask, PT_MIN, DR_MIN)
    with pytest.raises(me.MEError) as e:
        me.me_filter_helicities_noalloc(h, np.ascontiguousarray(mom))      # host memory
    assert e.value.code == me.ME_EINVAL
    h.close()
    # gg_ttxggg: 3900 x 129 x 8 B of per-helicity values leave less than one
    # CTA's colour-flow scratch (240 KB) in the 4 MiB array
    w = WORKLOADS["gg_ttxggg"]
    h = me.workload_handle("gg_ttxggg", "fp64")
    big = torch.zeros((3900, w.npar, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(me.MEError) as e:
        me.me_filter_helicities_noalloc(h, big)
    assert e.value.code == me.ME_ETOOLARGE
    h.close()
