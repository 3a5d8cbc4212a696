"""Staged, descriptor-driven evaluation for the largest process (gg -> t t~ ggg).

The helicity-recycled tables of tabplan.py hold every off-shell object for
every configuration of its support; for 7 external particles that is 12750
wavefunctions per event, far beyond shared memory.  Here the amplitudes are
ordered greedily by colour group (amplitudes whose colour vectors agree up to
a sign are summed before one update of J; each next group needs the fewest new
table entries, its members stay adjacent) and cut into stages.  A stage first computes the objects its amplitudes need that
are not yet in the table (cooperatively, level by level), then every thread
evaluates the stage's amplitudes for its own helicity.  A table object lives
from the stage that computes it to the last stage that reads it; its slots are
then reused (first-fit allocator), so the table only has to hold the peak live
set.  The amplitude phase is a loop over compact descriptors (kind, operands,
line momenta, colour terms) rather than straight-line code, which keeps the
kernel small for 1890 amplitudes per helicity.
"""
from __future__ import annotations

from dataclasses import dataclass, field

from .plan import FLOPS, colour_groups
from .tabplan import build_tabplan, compress

# descriptor codes of the table routines and amplitude kinds (me_kernel_interp.cuh)
ROUTINES = ("VVV1P0_1", "VVVV1P0_1", "VVVV3P0_1", "VVVV4P0_1", "FFV1_2", "FFV1_1", "FFV1P0_3",
            "FFV1A_3", "FFV1A_2", "FFV1A_1", "VVV1A_1", "VVV1A_2", "VVV1A_3", "VVVV1A", "VVVV3A", "VVVV4A")
AMP_KINDS = ("FFV1_0", "VVV1_0", "VVVV1_0", "VVVV3_0", "VVVV4_0", "DOTV", "DOTF")


@dataclass
class Stage:
    rounds: list = field(default_factory=list)     # (kind, [task tuples]) with a barrier between levels
    barriers: list = field(default_factory=list)   # round indices after which a barrier is needed
    amps: list = field(default_factory=list)       # amplitude indices (into plan.amps)
    # split of the amplitudes between the two threads of a helicity (kernels that
    # run two threads per helicity): the first takes amps[:mid], the second
    # amps[mid:]; mid falls on a colour-group boundary, slot_mid = groups before it
    mid: int = 0
    slot_mid: int = 0
    # the stage's table work runs beside the previous stage's amplitudes
    ahead: bool = False


@dataclass
class InterpPlan:
    tab: object
    stages: list
    slot: dict          # object op index -> table base (Wf units)
    table_size: int
    amp_order: list
    supports: list      # distinct supports of amplitude operands
    table_flops: int
    sign: list = field(default_factory=list)    # +-1 of each amplitude in its colour group's sum
    flush: dict = field(default_factory=dict)   # last member of a group -> the group's colour terms
    ahead: bool = False                         # table work one stage ahead of the amplitudes


class _Arena:
    """first-fit allocator over Wf slots (sizes are powers of two)"""

    def __init__(self, base):
        self.free = [(base, 1 << 30)]
        self.peak = base

    def alloc(self, n):
        for i, (s, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (s + n, ln - n)
                self.peak = max(self.peak, s + n)
                return s
        raise RuntimeError("arena exhausted")

    def release(self, s, n):
        self.free.append((s, n))
        self.free.sort()
        merged = []
        for a, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((a, ln))
        self.free = merged


# issue cost of closing a colour group (the BF16 split of G and its operand
# stores), in the units of FLOPS, for balancing the halves of a stage
FLUSH_COST = 24


def _split_amplitudes(ops, amps, stage_amps, flush):
    """Split point of a stage's amplitude list at a colour-group boundary that
    balances the two halves' cost (amplitude flops + group closings); returns
    (mid, groups before mid)."""
    cost = [FLOPS[ops[amps[a][0]].kind] + (FLUSH_COST if a in flush else 0) for a in stage_amps]
    total = sum(cost)
    best, acc, groups = (total, 0, 0), 0, 0
    for i, a in enumerate(stage_amps):
        acc += cost[i]
        if a in flush:
            groups += 1
            key = max(acc, total - acc)
            if key < best[0]:
                best = (key, i + 1, groups)
    return best[1], best[2]


def build_interp(process: str, stage_amps: int = 48, amputated: bool = False, group: bool = True,
                 ahead: bool = False, table_cap: int | None = None) -> InterpPlan:
    """ahead: a stage's table objects may be computed while the previous
    stage's amplitudes are evaluated (one barrier per stage instead of two);
    they then must not reuse the slots that those amplitudes read.  A stage
    runs ahead where its objects fit below table_cap entries that way
    (Stage.ahead); otherwise its table work keeps a phase of its own."""
    T = build_tabplan(process, amputated)
    P = T.plan
    ops = P.ops
    is_obj = lambda i: ops[i].out != "A" and not ops[i].kind.startswith("ext_")
    size = {i: 1 << len(T.support[i]) for i in range(len(ops)) if is_obj(i)}

    def closure(i, acc):
        if i in acc or not is_obj(i):
            return
        for a in ops[i].args:
            closure(a, acc)
        acc.add(i)

    amp_deps = []
    for ai, _ in P.amps:
        s = set()
        for a in ops[ai].args:
            closure(a, s)
        amp_deps.append(s)

    # greedy order over colour groups (amplitudes with the same colour vector up
    # to a sign, summed before the one update of J): next group = fewest new
    # table entries (ties: plan order); members of a group stay adjacent
    group_of, sign_of, group_terms, members = colour_groups(P)
    if not group:  # one amplitude per unit: J updated after every amplitude
        sign_of = [1] * len(P.amps)
        group_terms = [tuple(P.amps[a][1]) for a in range(len(P.amps))]
        members = [[a] for a in range(len(P.amps))]
    unit_deps = [set().union(*(amp_deps[a] for a in m)) for m in members]
    live, order, units, remaining = set(), [], [], set(range(len(members)))
    while remaining:
        best = min(remaining, key=lambda g: (sum(size[o] for o in unit_deps[g] - live), members[g][0]))
        order += members[best]
        units.append(members[best])
        remaining.remove(best)
        live |= unit_deps[best]
    # the last member of each group carries the group's colour terms
    flush = {members[g][-1]: group_terms[g] for g in range(len(members))}

    # stages of at most stage_amps amplitudes, cut between colour groups (a group
    # sum never stays open across a stage, so the amplitudes of a stage can be
    # shared out between threads at any group boundary)
    stages = []
    for u in units:
        assert len(u) <= stage_amps, "a colour group larger than a stage"
        if not stages or len(stages[-1].amps) + len(u) > stage_amps:
            stages.append(Stage())
        stages[-1].amps += u
    for st in stages:
        st.mid, st.slot_mid = _split_amplitudes(ops, P.amps, st.amps, flush)
    first, last = {}, {}
    computed = set()
    for si, st in enumerate(stages):
        need = set()
        for a in st.amps:
            need |= amp_deps[a]
        new = need - computed
        for o in new:
            first[o] = si
        computed |= new
        for o in need:
            last[o] = max(last.get(o, -1), si)
        st.new = new
    # objects read only while computing others in a later stage stay live until then
    for si, st in enumerate(stages):
        for o in st.new:
            for a in ops[o].args:
                if is_obj(a):
                    last[a] = max(last[a], si)

    arena = _Arena(2 * P.npar)
    slot = {}
    pending = []  # objects last read by the previous stage, not yet released
    for si, st in enumerate(stages):
        # allocate this stage's new objects (in dependency order).  Ahead: before
        # the previous stage's dead objects are released, so that none of their
        # slots (read by that stage's amplitudes meanwhile) is reused
        if ahead and si > 0:
            snap = (list(arena.free), arena.peak)
            trial = {o: arena.alloc(size[o]) for o in sorted(st.new)}
            if table_cap is None or arena.peak <= table_cap:
                slot.update(trial)
                st.ahead = True
            else:
                arena.free, arena.peak = snap
        for o in pending:
            arena.release(slot[o], size[o])
        pending = []
        if not st.ahead:
            for o in sorted(st.new):
                slot[o] = arena.alloc(size[o])
        level = {}
        for o in sorted(st.new):  # op indices are topologically ordered
            level[o] = 1 + max([level.get(a, 0) for a in ops[o].args if a in st.new] or [0])
        bykey = {}
        for o in sorted(st.new):
            bykey.setdefault((level[o], ops[o].kind), []).append(o)
        prev = None
        for (lv, kind) in sorted(bykey):
            if prev is not None and lv != prev:
                st.barriers.append(len(st.rounds) - 1)
            prev = lv
            tasks = []
            for o in bykey[(lv, kind)]:
                S = T.support[o]
                op = ops[o]
                for v in range(size[o]):
                    bits = {p: (v >> j) & 1 for j, p in enumerate(S)}
                    ins = []
                    for a in op.args:
                        base = slot[a] if is_obj(a) else 2 * ops[a].ext
                        ins.append(base + compress(bits, T.support[a]))
                    vvv = kind == "VVV1P0_1" or kind.startswith("VVV1A")
                    ln = (op.mom[0], op.mom[1], max(op.line, 0)) if vvv else (0, 0, max(op.line, 0))
                    tasks.append((slot[o] + v, tuple(ins), ln))
            st.rounds.append((kind, tasks))
        # objects last read in this stage are released when the next is placed
        pending = [o for o in slot if last.get(o) == si]
    supports = sorted({T.support[a] for ai, _ in P.amps for a in ops[ai].args}, key=lambda s: (len(s), s))
    tflops = sum(FLOPS[k] * len(t) for st in stages for k, t in st.rounds)
    return InterpPlan(T, stages, slot, arena.peak, order, supports, tflops, sign_of, flush, ahead)
