"""Binding of the continuous-batching server (include/me_serve.h) and the
serving load generator used by bench.py.

The server runs in the C++ library; this module marshals arguments and, for
the benchmark, submits a seeded Poisson stream of requests over the process
mix (weights, log-uniform batch sizes 256..65536) and reports p50/p99 latency
beside events/s.
"""
from __future__ import annotations

import ctypes
import json
import math
import time

import numpy as np

from . import ME_OK, PRECISIONS, _check, load

#: symbols declared in include/me_serve.h
SERVE_EXPORTS = ("srv_create", "srv_submit", "srv_wait", "srv_cancel", "srv_stats", "srv_destroy")


class srv_config(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int), ("max_batch", ctypes.c_int64), ("hbm_budget_bytes", ctypes.c_uint64),
                ("use_graphs", ctypes.c_int)]


def _lib():
    lib = load()
    if not getattr(lib, "_srv_ready", False):
        P, i, i64, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
        lib.srv_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(srv_config)]
        lib.srv_submit.argtypes = [P, ctypes.c_char_p, i, P, i64, P, ctypes.POINTER(u64)]
        lib.srv_wait.argtypes = [P, u64, i, ctypes.POINTER(ctypes.c_double)]
        lib.srv_cancel.argtypes = [P, u64]
        lib.srv_stats.argtypes = [P, ctypes.c_char_p, i]
        lib.srv_destroy.argtypes = [P]
        lib.srv_destroy.restype = None
        for n in ("srv_create", "srv_submit", "srv_wait", "srv_cancel", "srv_stats"):
            getattr(lib, n).restype = i
        lib._srv_ready = True
    return lib


class Server:
    def __init__(self, lanes=4, max_batch=1 << 16, hbm_budget_bytes=8 << 30, use_graphs=True):
        self._s = ctypes.c_void_p()
        cfg = srv_config(lanes, max_batch, hbm_budget_bytes, 1 if use_graphs else 0)
        _check(_lib().srv_create(ctypes.byref(self._s), ctypes.byref(cfg)), "srv_create")

    def submit(self, process, momenta, out, precision="mixed") -> int:
        """momenta, out: host torch tensors (pinned preferred) or numpy arrays."""
        from . import _ptr

        t = ctypes.c_uint64()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        _check(_lib().srv_submit(self._s, process.encode(), prec, _ptr(momenta), momenta.shape[0], _ptr(out),
                                 ctypes.byref(t)), "srv_submit")
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        """Returns the request's latency in seconds; raises MEError (ME_ETIMEOUT...)."""
        lat = ctypes.c_double()
        rc = _lib().srv_wait(self._s, ticket, int(timeout_ms), ctypes.byref(lat))
        _check(rc, "srv_wait")
        return lat.value * 1e-6

    def cancel(self, ticket):
        _check(_lib().srv_cancel(self._s, ticket), "srv_cancel")

    def stats(self) -> dict:
        buf = ctypes.create_string_buffer(1024)
        _check(_lib().srv_stats(self._s, buf, 1024), "srv_stats")
        return json.loads(buf.value.decode())

    def close(self):
        if self._s:
            _lib().srv_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------- load
def _mix(processes=None):
    from .workloads import SERVING_MIX

    w = dict(SERVING_MIX["weights"])
    if processes is not None:
        w = {k: v for k, v in w.items() if k in processes}
    tot = sum(w.values())
    return {k: v / tot for k, v in w.items()}


def make_requests(nreq, processes, seed=None, pool=8):
    """Seeded request stream: (process, batch size) for request i, and pinned
    momenta from the device sampler with seed momenta_seed_base + i (a pool of
    `pool` buffers per process is reused cyclically)."""
    import torch

    from . import cuts_for, rambo_sample
    from .workloads import PARTICLES, SERVING_MIX, WORKLOADS

    mix = _mix(processes)
    rng = np.random.default_rng(SERVING_MIX["stream_seed"] if seed is None else seed)
    names = list(mix)
    probs = np.array([mix[n] for n in names])
    lo, hi = math.log(SERVING_MIX["batch_min"]), math.log(SERVING_MIX["batch_max"])
    reqs = []
    for i in range(nreq):
        proc = names[rng.choice(len(names), p=probs)]
        n = int(math.floor(math.exp(rng.uniform(lo, hi))))
        reqs.append((proc, n))
    bufs = {}
    for p in names:
        w = WORKLOADS[p]
        masses = [0.0, 0.0] + list(w.masses_final)
        bufs[p] = []
        for j in range(pool):
            d = rambo_sample(SERVING_MIX["momenta_seed_base"] + j, 0, SERVING_MIX["batch_max"], w.sqrt_s, masses,
                             cuts_for(p))
            h = torch.empty(d.shape, dtype=torch.float64, pin_memory=True)
            h.copy_(d)
            bufs[p].append(h)
    return reqs, bufs


def run_load(server, reqs, bufs, rate_hz, precision="mixed", seed=7):
    """Poisson arrivals at rate_hz; returns latencies (s), events, wall time."""
    import torch

    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=len(reqs)) if rate_hz > 0 else np.zeros(len(reqs))
    outs = [torch.empty(n, dtype=torch.float64, pin_memory=True) for _, n in reqs]
    tickets = []
    t0 = time.perf_counter()
    t_next = t0
    for i, (proc, n) in enumerate(reqs):
        t_next += gaps[i]
        now = time.perf_counter()
        if t_next > now:
            time.sleep(t_next - now)
        mom = bufs[proc][i % len(bufs[proc])][:n]
        tickets.append(server.submit(proc, mom, outs[i], precision))
    lat = [server.wait(t) for t in tickets]
    wall = time.perf_counter() - t0
    return np.array(lat), sum(n for _, n in reqs), wall, outs


def saturation(server, reqs, bufs, precision="mixed"):
    """All requests at once: events/s when the server is never idle."""
    lat, ev, wall, _ = run_load(server, reqs, bufs, 0.0, precision)
    return ev / wall


def bench_point(load=0.7, nreq=300, processes=None, precision="mixed", lanes=4):
    """One serving load point for bench.py: p50/p99 latency at `load` x the
    measured saturation request rate, and the events/s achieved."""
    processes = processes or built_processes()
    reqs, bufs = make_requests(nreq, processes)
    srv = Server(lanes=lanes, max_batch=1 << 17)
    try:
        run_load(srv, reqs[:min(40, nreq)], bufs, 0.0, precision)  # warm-up: handles, graphs
        sat_ev = saturation(srv, reqs, bufs, precision)
        mean_batch = np.mean([n for _, n in reqs])
        rate = load * sat_ev / mean_batch
        lat, ev, wall, _ = run_load(srv, reqs, bufs, rate, precision)
        st = srv.stats()
    finally:
        srv.close()
    return {"load": load, "requests": nreq, "rate_req_per_s": rate, "saturation_events_per_s": sat_ev,
            "events_per_s": ev / wall, "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_batch": float(mean_batch),
            "processes": processes, "precision": precision, "lanes": lanes,
            "batches": st["batches"], "graph_updates": st["graph_updates"]}


def sweep(loads=(0.1, 0.3, 0.5, 0.7, 0.9, 1.1), nreq=2000, processes=None, precision="mixed", lanes=4):
    """Latency against offered load: Poisson arrivals at each `load` x the
    measured saturation request rate, `nreq` requests per point (the same
    seeded request stream at every point)."""
    processes = processes or built_processes()
    reqs, bufs = make_requests(nreq, processes)
    srv = Server(lanes=lanes, max_batch=1 << 17)
    points = []
    try:
        run_load(srv, reqs[:min(40, nreq)], bufs, 0.0, precision)  # warm-up: handles, graphs
        sat_ev = saturation(srv, reqs, bufs, precision)
        mean_batch = float(np.mean([n for _, n in reqs]))
        for load in loads:
            rate = load * sat_ev / mean_batch
            lat, ev, wall, _ = run_load(srv, reqs, bufs, rate, precision)
            points.append({"load": load, "rate_req_per_s": rate, "events_per_s": ev / wall,
                           "p50_ms": float(np.percentile(lat, 50) * 1e3), "p90_ms": float(np.percentile(lat, 90) * 1e3),
                           "p99_ms": float(np.percentile(lat, 99) * 1e3)})
        st = srv.stats()
    finally:
        srv.close()
    return {"requests_per_point": nreq, "saturation_events_per_s": sat_ev, "mean_batch": mean_batch,
            "processes": processes, "precision": precision, "lanes": lanes, "points": points,
            "batches": st["batches"], "graph_updates": st["graph_updates"]}


def built_processes():
    """Processes of the serving mix that this library build contains."""
    from . import load as _load

    lib = _load()
    out = []
    for p in ("ee_mumu", "gg_ttx", "gg_ttxg", "gg_ttxgg", "gg_ttxggg"):
        h = ctypes.c_void_p()
        if lib.me_init(ctypes.byref(h), p.encode(), None, 0, None, 0, 0) == ME_OK:
            lib.me_free(h)
            out.append(p)
    return out


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="serving latency sweep on the current CUDA device")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--loads", default="0.1,0.3,0.5,0.7,0.9,1.1")
    ap.add_argument("--precision", default="mixed")
    args = ap.parse_args()
    print(json.dumps(sweep(tuple(float(x) for x in args.loads.split(",")), args.requests, precision=args.precision)))
