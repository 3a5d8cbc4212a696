"""Seeded synthetic workloads: process, energy, masses, cuts, seed, size.

Pure data shared by the tests, the benchmark and the oracle calls; it holds
none of the method's arithmetic and imports nothing from this package.  The
phase-space points themselves come from the seeded RAMBO sampler (Sec. 4 of
arXiv:2507.21039 uses RAMBO for its standalone benchmark), which each side
implements on its own.
"""
from __future__ import annotations

from dataclasses import dataclass, field

MT = 173.0                 # top-quark mass [GeV]
ALPHA_S = 0.118            # fixed strong coupling, no running
ALPHA_EM = 1.0 / 132.5     # fixed QED coupling, no running
PT_MIN = 20.0              # final-state gluon transverse-momentum cut [GeV]
DR_MIN = 0.4               # pairwise Delta R cut between final-state gluons

#: particle order of each process: initial state first, then final state
PARTICLES = {
    "ee_mumu": ("e-", "e+", "mu-", "mu+"),
    "gg_ttx": ("g", "g", "t", "t~"),
    "gg_ttxg": ("g", "g", "t", "t~", "g"),
    "gg_ttxgg": ("g", "g", "t", "t~", "g", "g"),
    "gg_ttxggg": ("g", "g", "t", "t~", "g", "g", "g"),
    "uux_epem": ("u", "u~", "e+", "e-"),
    "uux_epemg": ("u", "u~", "e+", "e-", "g"),
    "uux_epemgg": ("u", "u~", "e+", "e-", "g", "g"),
    "uux_epemggg": ("u", "u~", "e+", "e-", "g", "g", "g"),
}


@dataclass(frozen=True)
class Workload:
    name: str
    process: str
    sqrt_s: float
    seed: int
    nevt: int
    cuts: bool
    precisions: tuple = ("fp64",)
    notes: str = ""
    masses_final: tuple = field(default=())

    @property
    def npar(self) -> int:
        return len(PARTICLES[self.process])

    @property
    def cut_mask(self):
        """1 for each final-state particle the gluon cuts apply to."""
        fin = PARTICLES[self.process][2:]
        return tuple(1 if (self.cuts and p == "g") else 0 for p in fin)

    @property
    def alpha(self) -> float:
        return ALPHA_EM if self.process == "ee_mumu" else ALPHA_S


def _fin_masses(process):
    return tuple(MT if p in ("t", "t~") else 0.0 for p in PARTICLES[process][2:])


def _w(name, process, sqrt_s, seed, nevt, cuts, precisions, notes=""):
    return Workload(name, process, sqrt_s, seed, nevt, cuts, precisions, notes, _fin_masses(process))


#: the five configurations of the benchmark definition, in order
WORKLOADS = {
    "ee_mumu": _w("ee_mumu", "ee_mumu", 100.0, 1, 16384, False, ("fp64",),
                  "photon only, massless; closed form e^4 (1 + cos^2 theta)"),
    "gg_ttx": _w("gg_ttx", "gg_ttx", 1000.0, 2, 1 << 20, False, ("fp64", "fp32", "mixed"),
                 "closed form (Combridge)"),
    "gg_ttxg": _w("gg_ttxg", "gg_ttxg", 1500.0, 3, 1 << 20, True, ("fp64", "fp32", "mixed")),
    "gg_ttxgg": _w("gg_ttxgg", "gg_ttxgg", 1500.0, 4, 1 << 20, True, ("fp64", "fp32", "mixed"),
                   "headline workload"),
    "gg_ttxggg": _w("gg_ttxggg", "gg_ttxggg", 2000.0, 5, 1 << 18, True, ("fp64", "mixed")),
}

#: the paper's second standalone workload, u u~ -> e+ e- + n g (photon and Z;
#: electroweak parameters fixed as in the library's reading of the paper): a
#: synthetic stand-in at sqrt(s) = 500 GeV with the gluon cuts above
DY_WORKLOADS = {
    "uux_epem": _w("uux_epem", "uux_epem", 500.0, 11, 1 << 20, False, ("fp64", "fp32", "mixed")),
    "uux_epemg": _w("uux_epemg", "uux_epemg", 500.0, 12, 1 << 20, True, ("fp64", "fp32", "mixed")),
    "uux_epemgg": _w("uux_epemgg", "uux_epemgg", 500.0, 13, 1 << 20, True, ("fp64", "fp32", "mixed")),
    "uux_epemggg": _w("uux_epemggg", "uux_epemggg", 500.0, 14, 1 << 18, True, ("fp64", "fp32", "mixed")),
}


def workload(name: str) -> Workload:
    """A benchmark workload or a Drell-Yan workload by name."""
    return WORKLOADS[name] if name in WORKLOADS else DY_WORKLOADS[name]


#: serving mix: process weights, log-uniform batch sizes, per-request seeds
SERVING_MIX = {
    "weights": {"ee_mumu": 0.1, "gg_ttx": 0.3, "gg_ttxg": 0.3, "gg_ttxgg": 0.2, "gg_ttxggg": 0.1},
    "batch_min": 256,
    "batch_max": 65536,
    "momenta_seed_base": 1000,
    "stream_seed": 42,
    "load_points": (0.1, 0.3, 0.5, 0.7, 0.9, 1.1),
    "requests_per_point": 2000,
}
