"""Multi-rank path on CPU (gloo, world size 2): event-range sharding and the
cross-section reduction give the single-process answer.  The per-rank |M|^2
here is the FP64 oracle on the rank's own RAMBO events, so the test exercises
the host-side sharding logic with real numbers and no GPU."""
import os
import socket

import numpy as np
import pytest

from paper_2507_21039_gb300.shard import event_range


def test_event_ranges_tile_exactly():
    for nevt in (0, 1, 7, 1000, 1 << 20):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                lo, hi = event_range(r, world, nevt, ev0=11)
                assert 11 <= lo <= hi <= 11 + nevt
                seen.extend(range(lo, hi)) if nevt < 5000 else seen.append((lo, hi))
            if nevt < 5000:
                assert seen == list(range(11, 11 + nevt))
            else:
                assert seen[0][0] == 11 and seen[-1][1] == 11 + nevt
                assert all(a[1] == b[0] for a, b in zip(seen, seen[1:]))
    with pytest.raises(ValueError):
        event_range(2, 2, 10)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, nevt, q):
    import torch.distributed as dist

    import oracle
    from paper_2507_21039_gb300.shard import event_range, reduce_estimate
    from paper_2507_21039_gb300.workloads import DR_MIN, MT, PT_MIN, WORKLOADS

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = WORKLOADS["gg_ttxg"]
    lo, hi = event_range(rank, world, nevt)
    mom, wt, _ = oracle.rambo(w.seed, w.sqrt_s, w.masses_final, lo, hi - lo, w.cut_mask, PT_MIN, DR_MIN)
    me2 = oracle.me2("gg_ttxg", mom, mt=MT, alpha=w.alpha, nthreads=1)
    x = wt * me2
    mean, err = reduce_estimate(float(x.sum()), float((x * x).sum()), hi - lo)
    # gather of the |M|^2 slices (the other exchange a caller may want)
    import torch

    sizes = [None] * world
    dist.all_gather_object(sizes, (lo, hi))
    parts = [torch.zeros(b - a, dtype=torch.float64) for a, b in sizes]
    dist.all_gather(parts, torch.from_numpy(me2)) if all(len(p) == len(parts[0]) for p in parts) else None
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mean, err, lo, hi, me2.tolist(), [p.tolist() for p in parts]))


def test_two_rank_gloo_reduction_matches_single_process(orc):
    import torch.multiprocessing as mp

    from paper_2507_21039_gb300.workloads import DR_MIN, MT, PT_MIN, WORKLOADS

    nevt, world = 64, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, nevt, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = WORKLOADS["gg_ttxg"]
    mom, wt, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, 0, nevt, w.cut_mask, PT_MIN, DR_MIN)
    me2 = orc.me2("gg_ttxg", mom, mt=MT, alpha=w.alpha)
    x = wt * me2
    mean = x.mean()
    err = np.sqrt(max((x * x).mean() - mean * mean, 0.0) / nevt)
    for rank, m, e, lo, hi, part, gathered in res:
        assert abs(m / mean - 1) < 1e-12 and abs(e / err - 1) < 1e-9
        assert np.allclose(part, me2[lo:hi], rtol=1e-14, atol=0)
        assert np.allclose(np.concatenate(gathered), me2, rtol=1e-14, atol=0)
