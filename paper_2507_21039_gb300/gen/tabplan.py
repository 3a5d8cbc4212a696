"""Helicity-recycled evaluation layout for the shared-memory table kernel.

Every off-shell object of the chain (gluon-tree currents, quark-line prefixes
and suffixes, the t tbar pair current) depends only on the helicities of its
own external particles -- its *support*.  Instead of recomputing it for each of
the event's helicity configurations (2^npar), the kernel evaluates each object
once per configuration of its support (2^|support| variants) into a per-event
shared-memory table; the lanes of the event then evaluate only the final
amplitudes (FFV1_0, VVV1_0, VVVV*_0) for their own helicity, reading operands
from the tables.  The Feynman diagrams, vertices and colour coefficients are
exactly those of the plan (Sec. 3.1 of arXiv:2507.21039); only the reuse of
sub-expressions across helicities is new.

Table layout (units of one wavefunction, Wf = 4 complex numbers):
  [0, 2*npar)           external wavefunctions: particle e, helicity bit b at 2e+b
  then, per object X    2^|S_X| consecutive variants; variant index
                        v = sum_j b(p_j) << j over the support particles
                        p_0 > p_1 > ... (b = 1 for helicity +1): the
                        highest-numbered particle -- the lowest helicity bit,
                        which differs between neighbouring lanes -- is the
                        lowest variant bit, so the lanes of one 8-lane
                        shared-memory phase read nearby entries.
Helicity index h: particle i has helicity +1 iff bit (npar-1-i) of h is set.
"""
from __future__ import annotations

from dataclasses import dataclass, field

from .plan import FLOPS, Plan, amputate, build_plan, build_plan_dy, colour_groups

# Drell-Yan lepton-pair objects (both chiralities of the electroweak insertion):
# functions of the e+ (particle 2) and e- (particle 3) states and the event's
# electroweak coefficients, which sit at table entry 2 npar
LEPTON_KINDS = ("ext_lepL", "ext_lepR")
LEPTON_SUPPORT = (3, 2)
# Drell-Yan with massless fermions: helicity conservation along the quark line
# (u, u~ = particles 0, 1) and the lepton pair (2, 3) makes every configuration
# with equal helicity bits in either pair vanish exactly.  Variants of an object
# whose support holds both members of a pair with equal bits are never read by
# a non-vanishing helicity; they are not computed (the kernel returns 0 for
# the vanishing helicities, ProcTab::hel_allowed)
DY_OPPOSITE_PAIRS = ((0, 1), (2, 3))
# flops of one table task: a lepton-pair task forms both chiralities and stores one
TASK_FLOPS = dict(FLOPS, ext_lepR=FLOPS["ext_lepL"])


@dataclass
class Task:
    out: int
    ins: tuple
    lines: tuple   # (la, lb, lo) line indices used by the routine (-1 if unused)


@dataclass
class Round:
    level: int
    kind: str
    tasks: list = field(default_factory=list)


@dataclass
class TabPlan:
    plan: Plan
    support: dict            # op index -> tuple of particles (sorted)
    base: dict               # op index -> table base (Wf units)
    size: int                # table size (Wf units)
    rounds: list             # Round, in dependency order
    nlevels: int
    amp_supports: list       # distinct supports of amplitude operands
    opposite_pairs: tuple = ()  # particle pairs whose helicity bits must differ (else |M_h|^2 = 0)

    def table_flops(self) -> int:
        return sum(TASK_FLOPS[r.kind] * len(r.tasks) for r in self.rounds)

    def amplitude_flops_per_helicity(self, grouped: bool = True) -> int:
        """amplitudes plus their accumulation into J; grouped: amplitudes with
        the same colour vector up to a sign are summed (2 flops per member after
        the first) and the group's terms are added once"""
        P = self.plan
        f = sum(FLOPS[P.ops[a].kind] for a, _ in P.amps)
        if grouped:
            _, _, terms_of, members = colour_groups(P)
            f += sum(2 * (len(m) - 1) for m in members)
        else:
            terms_of = [terms for _, terms in P.amps]
        for terms in terms_of:
            for _, c in terms:
                f += 2 if (abs(c[0]) + abs(c[1]) == 1) else 4
        return f


def _support(P: Plan, i: int, memo: dict):
    if i in memo:
        return memo[i]
    op = P.ops[i]
    if op.kind in LEPTON_KINDS:
        s = LEPTON_SUPPORT
    elif op.kind.startswith("ext_"):
        s = (op.ext,)
    else:
        acc = set()
        for a in op.args:
            acc |= set(_support(P, a, memo))
        s = tuple(sorted(acc, reverse=True))
    memo[i] = s
    return s


def compress(full_bits: dict, support) -> int:
    """variant index of `support` given particle -> bit"""
    return sum(full_bits[p] << j for j, p in enumerate(support))


def _plan_of(process: str) -> Plan:
    from .emit import DY_PROCESSES  # the Drell-Yan process names and their gluon counts

    return build_plan_dy(DY_PROCESSES[process]) if process in DY_PROCESSES else build_plan(process)


def build_tabplan(process: str, amputated: bool = False) -> TabPlan:
    """amputated: every amplitude becomes a contraction of two table objects
    (plan.amputate), the vertex objects joining the table.  Drell-Yan: the
    lepton-pair objects are table objects of support {e+, e-} (level 1), the
    electroweak coefficients table entry 2 npar."""
    P = _plan_of(process)
    memo = {}
    sup = {i: _support(P, i, memo) for i in range(len(P.ops))}
    if amputated:
        P = amputate(P, sup)
        memo = {}
        sup = {i: _support(P, i, memo) for i in range(len(P.ops))}
    external = lambda op: op.kind.startswith("ext_") and op.kind not in LEPTON_KINDS
    dy = any(op.kind in LEPTON_KINDS for op in P.ops)
    base = {}
    for i, op in enumerate(P.ops):
        if external(op):
            base[i] = 2 * op.ext
    ew = 2 * P.npar  # Drell-Yan: the electroweak coefficients' entry
    nxt = 2 * P.npar + (1 if dy else 0)
    level = {}
    for i, op in enumerate(P.ops):
        if external(op):
            level[i] = 0
        else:
            level[i] = 1 + max([level[a] for a in op.args] or [0])
        if op.out != "A" and not external(op):
            base[i] = nxt
            nxt += 1 << len(sup[i])
    pairs = DY_OPPOSITE_PAIRS if dy else ()
    rounds = {}
    for i, op in enumerate(P.ops):
        if op.out == "A" or external(op):
            continue
        key = (level[i], op.kind)
        r = rounds.setdefault(key, Round(level[i], op.kind))
        S = sup[i]
        for v in range(1 << len(S)):
            bits = {p: (v >> j) & 1 for j, p in enumerate(S)}
            if any(a in bits and b in bits and bits[a] == bits[b] for a, b in pairs):
                continue  # read only by vanishing helicities
            if op.kind in LEPTON_KINDS:  # (ubar(e-), v(e+), coefficients), as the straight-line chain passes them
                ins = (2 * 3 + bits[3], 2 * 2 + bits[2], ew)
            else:
                ins = tuple(base[a] + compress(bits, sup[a]) for a in op.args)
            if op.kind == "VVV1P0_1" or op.kind.startswith("VVV1A"):
                ln = (op.mom[0], op.mom[1], op.line)
            else:
                ln = (-1, -1, op.line)
            r.tasks.append(Task(base[i] + v, ins, ln))
    order = sorted(rounds, key=lambda k: (k[0], k[1]))
    amp_sup = sorted({sup[a] for ai, _ in P.amps for a in P.ops[ai].args}, key=lambda s: (len(s), s))
    return TabPlan(P, sup, base, nxt, [rounds[k] for k in order], max(k[0] for k in order) if order else 0, amp_sup,
                   pairs)
