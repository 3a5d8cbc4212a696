"""Host-side checks that need no GPU: the generator's logic (diagram counts,
exact colour matrices, colour/phase bookkeeping evaluated against the oracle)
and the C-ABI library (builds for sm_103a, loads, exports every declared symbol,
argument validation that happens before any device work)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_2507_21039_gb300.gen import diagrams as D
from paper_2507_21039_gb300.gen.colour import colour_matrix
from paper_2507_21039_gb300.gen.plan import build_plan
from paper_2507_21039_gb300.workloads import MT, WORKLOADS

from plan_eval import evaluate

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# ---------------------------------------------------------------- generator
@pytest.mark.parametrize("k,n,namps", [(2, 3, 3), (3, 16, 18), (4, 123, 159), (5, 1240, 1890)])
def test_diagram_counts(k, n, namps):
    assert D.diagram_count(k) == n
    assert len(D.diagrams(k)) == namps


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_generator_colour_matrix_equals_oracle_brute_force(orc, k):
    num, den = colour_matrix(k)
    C = orc.colour_matrix(k)
    # exact: every numerator recovered from the oracle's floating brute force
    Cn = np.rint(C * den).astype(np.int64)
    assert np.abs(C * den - Cn).max() < 1e-8 * den
    assert np.array_equal(Cn, np.array(num, dtype=np.int64))
    from fractions import Fraction
    g = 0
    for row in num:
        for x in row:
            g = math.gcd(g, x)
    assert math.gcd(g, den) == 1  # lowest terms


@pytest.mark.parametrize("process", ["gg_ttx", "gg_ttxg", "gg_ttxgg", "gg_ttxggg", "ee_mumu"])
def test_generator_plan_reproduces_oracle_partial_amplitudes(orc, process):
    """The generator's diagrams, colour decomposition and phases, evaluated with
    numpy, give the oracle's colour-ordered partial amplitudes."""
    P = build_plan(process)
    w = WORKLOADS[process]
    mom, _, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, 0, 2, w.cut_mask, 20.0, 0.4)
    rng = np.random.default_rng(5)
    for p in mom:
        if process == "ee_mumu":
            me, hel = orc.me2("ee_mumu", p[None], per_helicity=True)
            e4 = (4 * math.pi * w.alpha) ** 2
            for h in range(16):
                J = evaluate(orc, P, p, h, 0.0)
                assert abs(abs(J[0]) ** 2 * e4 - hel[0][h]) <= 1e-13 * hel[0].max()
            continue
        scale = max(np.abs(orc.partial_amps(process, p, h)).max() for h in range(0, 1 << P.npar, 7))
        for h in rng.integers(0, 1 << P.npar, size=3 if process != "gg_ttxggg" else 1):
            J = evaluate(orc, P, p, int(h), MT)
            A = orc.partial_amps(process, p, int(h))
            assert np.abs(J - A).max() < 1e-12 * scale


@pytest.mark.parametrize("process", ["gg_ttx", "gg_ttxg", "gg_ttxgg", "gg_ttxggg"])
def test_amputated_plan_reproduces_oracle_partial_amplitudes(orc, process):
    """Every amplitude rewritten as the contraction of an amputated vertex
    object (no propagator) with the remaining operand gives the oracle's
    colour-ordered partial amplitudes."""
    from paper_2507_21039_gb300.gen.plan import amputate
    from paper_2507_21039_gb300.gen.tabplan import _support

    P = build_plan(process)
    memo = {}
    Q = amputate(P, {i: _support(P, i, memo) for i in range(len(P.ops))})
    assert len(Q.amps) == len(P.amps)
    assert all(Q.ops[a].kind in ("DOTV", "DOTF") for a, _ in Q.amps)
    w = WORKLOADS[process]
    mom, _, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, 4, 1, w.cut_mask, 20.0, 0.4)
    p = mom[0]
    scale = max(np.abs(orc.partial_amps(process, p, h)).max() for h in range(0, 1 << P.npar, 7))
    rng = np.random.default_rng(11)
    for h in rng.integers(0, 1 << P.npar, size=3 if process != "gg_ttxggg" else 1):
        J = evaluate(orc, Q, p, int(h), MT)
        A = orc.partial_amps(process, p, int(h))
        assert np.abs(J - A).max() < 1e-12 * scale


def test_interpreter_descriptor_codes_match_kernel():
    """The generator's routine / amplitude codes are the kernel's enum order."""
    from paper_2507_21039_gb300.gen.interp import AMP_KINDS, ROUTINES

    src = open(os.path.join(ROOT, "paper_2507_21039_gb300", "csrc", "me_kernel_interp.cuh")).read()
    body = lambda name: re.search(r"enum " + name + r" : unsigned char \{(.*?)\};", src, re.S).group(1)
    routines = [x.strip().split("=")[0].strip()[2:] for x in body("IRoutine").split(",") if x.strip()]
    kinds = [x.strip().split("=")[0].strip()[2:] for x in body("IAmpKind").split(",") if x.strip()]
    assert routines == list(ROUTINES)
    assert kinds == list(AMP_KINDS)


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_generator_diagrams_are_the_oracle_diagrams(orc, k):
    """The generator's Feynman diagrams (its amplitudes, grouped by diagram) are
    exactly the oracle's independently enumerated ones, identified by their
    internal lines."""
    from paper_2507_21039_gb300.gen.plan import diagram_lines

    process = {2: "gg_ttx", 3: "gg_ttxg", 4: "gg_ttxgg", 5: "gg_ttxggg"}[k]
    P = build_plan(process)
    gen = set(diagram_lines(P, d) for d in range(P.ndiagrams))
    assert len(gen) == P.ndiagrams == D.diagram_count(k)
    w = WORKLOADS[process]
    mom, _, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, 0, 1, w.cut_mask, 20.0, 0.4)
    _, lines = orc.sde(process, mom[0], [0], MT)
    assert gen == set(lines)


def test_generator_flop_counts_positive():
    for p in ("ee_mumu", "gg_ttx", "gg_ttxg", "gg_ttxgg", "gg_ttxggg"):
        P = build_plan(p)
        assert P.flops_per_helicity() > 0
        assert P.colour_flops_per_helicity() > 0


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_drell_yan_plan_reproduces_oracle_partial_amplitudes(orc, k):
    """The generator's Drell-Yan plans (quark-line diagrams with one photon/Z
    insertion, chiral vertices, colour and phases) give the oracle's
    colour-ordered partial amplitudes of u ubar -> e+ e- + k g."""
    from paper_2507_21039_gb300.gen.plan import build_plan_dy
    from plan_eval import evaluate_dy

    P = build_plan_dy(k)
    assert P.ncol == max(1, math.factorial(k))
    cut = [0, 0] + [1] * k if k else None
    mom, _, _ = orc.rambo(5, 200.0, [0.0] * (2 + k), 0, 2, cut, 20.0, 0.4)
    for p in mom:
        scale = max(np.abs(orc.dy_partial_amps(k, p, h)).max() for h in range(0, 1 << (4 + k), 3))
        for h in range(0, 1 << (4 + k), 5):
            J = evaluate_dy(orc, P, p, h)
            assert np.abs(J - orc.dy_partial_amps(k, p, h)).max() < 1e-12 * scale


@pytest.mark.parametrize("process", ["gg_ttx", "gg_ttxg", "gg_ttxgg", "gg_ttxggg"])
def test_colour_groups_rebuild_every_amplitude_terms(orc, process):
    """Each amplitude's colour terms are its sign times its group's normalised
    terms, the groups are disjoint and cover every amplitude, and J built
    from group sums is J built amplitude by amplitude (random amplitudes)."""
    from paper_2507_21039_gb300.gen.plan import colour_groups

    P = build_plan(process)
    group_of, sign_of, terms_of, members = colour_groups(P)
    assert sorted(a for m in members for a in m) == list(range(len(P.amps)))
    for ai, (_, terms) in enumerate(P.amps):
        g = group_of[ai]
        assert ai in members[g] and sign_of[ai] in (1, -1)
        assert sorted(terms) == sorted((f, (sign_of[ai] * c[0], sign_of[ai] * c[1])) for f, c in terms_of[g])
    for t in terms_of:
        c0 = t[0][1]
        assert c0[1] > 0 or (c0[1] == 0 and c0[0] > 0)
    rng = np.random.default_rng(5)
    x = rng.normal(size=len(P.amps)) + 1j * rng.normal(size=len(P.amps))
    J1 = np.zeros(P.ncol, complex)
    for ai, (_, terms) in enumerate(P.amps):
        for f, c in terms:
            J1[f] += complex(*c) * x[ai]
    J2 = np.zeros(P.ncol, complex)
    for g, m in enumerate(members):
        G = sum(sign_of[a] * x[a] for a in m)
        for f, c in terms_of[g]:
            J2[f] += complex(*c) * G
    assert np.abs(J1 - J2).max() < 1e-12 * np.abs(J1).max()


def test_descriptor_kernel_reads_its_descriptors_from_constant_memory():
    """The default gg -> t t~ ggg schedule keeps its uniform descriptors within
    the 64 KB constant bank (the emitter falls back to global memory, about 20%
    slower, when they do not fit), one set for both precisions."""
    from paper_2507_21039_gb300.gen.emit import INTERP_PROCESSES, emit_interp_struct

    nt, sf, mf, sd, md = INTERP_PROCESSES["gg_ttxggg"]
    assert (sf, mf) == (sd, md)
    src, _ = emit_interp_struct("gg_ttxggg", nt, sf, colour_matrix(5)[0], mf)
    for name in ("c_amps", "c_terms", "c_rounds", "c_stages", "c_stage_term", "c_diag"):
        assert re.search(r"__constant__ \w+( \w+)? " + name + r"\[", src), name
    sizes = {"IAmp": 16, "IRound": 8, "IStage": 16, "unsigned short": 2, "int": 4}
    total = 0
    for ctype, name, n in re.findall(r"__constant__ ([\w ]+?) (c_\w+)\[(\d+)\]", src):
        total += sizes[ctype] * int(n)
    assert total <= 64 * 1024, total


def test_interpreter_descriptors_encode_the_colour_groups():
    """The emitted amplitude descriptors of gg -> t t~ ggg carry, in stage
    order, each amplitude's sign in its colour group (kind bit 7) and, on the
    group's last member only, the group's colour terms (flow, sign of i)."""
    from paper_2507_21039_gb300.gen.emit import INTERP_PROCESSES, emit_interp_struct
    from paper_2507_21039_gb300.gen.interp import AMP_KINDS

    nt, sf, mf, _, _ = INTERP_PROCESSES["gg_ttxggg"]
    src, I = emit_interp_struct("gg_ttxggg", nt, sf, colour_matrix(5)[0], mf)
    amps = re.search(r"c_amps\[\d+\] = \{(.*?)\n\};", src, re.S).group(1)
    rows = [(int(a), int(b)) for a, b in re.findall(r"\}, (\d+), \d+, \d+, (\d+)\}", amps)]
    terms = [int(x) for x in re.findall(r"-?\d+", re.search(r"\bc_terms\[\d+\] = \{(.*?)\};", src, re.S).group(1))]
    order = [ai for st in I.stages for ai in st.amps]
    assert len(rows) == len(order) == len(I.tab.plan.amps)
    P = I.tab.plan
    t = 0
    for (kind, nterm), ai in zip(rows, order):
        assert AMP_KINDS[kind & 0x3F] == P.ops[P.amps[ai][0]].kind
        assert bool(kind & 0x80) == (I.sign[ai] < 0)
        flush = I.flush.get(ai, ())
        assert nterm == len(flush)
        for col, c in flush:
            assert terms[t] == col | (0x8000 if c == (0, -1) else 0)
            t += 1
    assert t == len(terms)


def test_stage_split_between_the_threads_of_a_helicity():
    """The FP32 descriptor kernel runs two threads per helicity; each stage's
    amplitudes are shared out at a colour-group boundary.  Every stage closes
    all its groups (no group sum stays open across a stage), the split point
    lies on a group boundary, the second thread's first update slot counts the
    groups before it and its first colour term their terms, the halves are balanced to within the largest group, and
    the emitted stage descriptors carry the split."""
    from paper_2507_21039_gb300.gen.emit import INTERP_PROCESSES, emit_interp_struct
    from paper_2507_21039_gb300.gen.interp import FLOPS, FLUSH_COST

    nt, sf, mf, _, _ = INTERP_PROCESSES["gg_ttxggg"]
    src, I = emit_interp_struct("gg_ttxggg", nt, sf, colour_matrix(5)[0], mf)
    P = I.tab.plan
    body = re.search(r"c_stages\[\d+\] = \{(.*?)\n\};", src, re.S).group(1)
    rows = [tuple(int(x) for x in r)
            for r in re.findall(r"\{(\d+), (\d+), (\d+), (\d+), (\d+), (\d+), \d+, (\d+)\}", body)]
    assert len(rows) == len(I.stages)
    a0 = 0
    for st, row in zip(I.stages, rows):
        amps = st.amps
        assert 0 < len(amps) <= sf and amps[-1] in I.flush
        assert st.mid == 0 or amps[st.mid - 1] in I.flush
        assert st.slot_mid == sum(1 for a in amps[:st.mid] if a in I.flush)
        # the second thread's first colour term (J updated flow by flow in FP64)
        term_mid = sum(len(I.flush[a]) for a in amps[:st.mid] if a in I.flush)
        assert row[2:] == (a0, a0 + len(amps), a0 + st.mid, st.slot_mid, term_mid)
        cost = [FLOPS[P.ops[P.amps[a][0]].kind] + (FLUSH_COST if a in I.flush else 0) for a in amps]
        ends = [i + 1 for i, a in enumerate(amps) if a in I.flush]
        best = min(max(sum(cost[:m]), sum(cost[m:])) for m in ends)
        assert max(sum(cost[:st.mid]), sum(cost[st.mid:])) == min(best, sum(cost))
        a0 += len(amps)
    assert a0 == len(P.amps)


def test_table_work_ahead_never_overwrites_live_entries():
    """Schedule mode bit 3 (a build option): where a stage's table rounds run beside the previous stage's amplitudes
    (Stage.ahead), every entry written in that phase is disjoint from every
    entry read in it (the amplitudes' operands and the rounds' inputs) and
    from the other writes; the same holds for the table phases of their own.
    The table stays within the cap that keeps two CTAs per SM, and the
    emitted stage descriptors carry the flags."""
    from paper_2507_21039_gb300.gen.emit import INTERP_PROCESSES, _interp_table_cap, emit_interp_struct

    nt, sf, mf, _, _ = INTERP_PROCESSES["gg_ttxggg"]
    src, I = emit_interp_struct("gg_ttxggg", nt, sf, colour_matrix(5)[0], mf | 8)
    P = I.tab.plan
    ops = P.ops
    assert I.table_size <= _interp_table_cap("gg_ttxggg", nt)
    assert sum(st.ahead for st in I.stages) > 0.9 * len(I.stages) and not I.stages[0].ahead
    body = re.search(r"c_stages\[\d+\] = \{(.*?)\n\};", src, re.S).group(1)
    flags = [int(f) for f in re.findall(r"\{\d+, \d+, \d+, \d+, \d+, \d+, (\d+), \d+\}", body)]
    assert flags == [int(st.ahead) for st in I.stages]

    def obj_range(x):
        if ops[x].kind.startswith("ext_"):
            return set(range(2 * ops[x].ext, 2 * ops[x].ext + 2))
        return set(range(I.slot[x], I.slot[x] + (1 << len(I.tab.support[x]))))

    def table_levels(st):  # (reads, writes) of each level, the levels split by CTA barriers
        levels, reads, writes = [], set(), []
        for ri, (_, tl) in enumerate(st.rounds):
            for out, ins, _ in tl:
                reads |= set(ins)
                writes.append(out)
            if ri in st.barriers or ri == len(st.rounds) - 1:
                levels.append((reads, writes))
                reads, writes = set(), []
        return levels

    def amp_reads(st):
        r = set()
        for ai in st.amps:
            for x in ops[P.amps[ai][0]].args:
                r |= obj_range(x)
        return r

    def check(levels, later_reads):
        # writes of a phase are disjoint; a level's reads meet no write of its
        # own or a later level; reads after the phase's last level (amplitudes) no write
        allw = [w for _, ws in levels for w in ws]
        assert len(allw) == len(set(allw))
        for k, (r, _) in enumerate(levels):
            assert not (r & {w for _, ws in levels[k:] for w in ws})
        assert not (later_reads & set(allw))

    for si, st in enumerate(I.stages):
        if not st.ahead:
            check(table_levels(st), set())
        nxt = table_levels(I.stages[si + 1]) if si + 1 < len(I.stages) and I.stages[si + 1].ahead else []
        check(nxt, amp_reads(st))


def test_amplitude_pairs_share_kind_and_half():
    """Descriptor flag AMP_PAIR (0x40): the flagged amplitude and the next one
    are evaluated together, so they have the same kind, lie in the same half
    of the same stage, and the successor of a pair head is not itself a head."""
    from paper_2507_21039_gb300.gen.emit import INTERP_PROCESSES, emit_interp_struct

    nt, sf, mf, _, _ = INTERP_PROCESSES["gg_ttxggg"]
    src, I = emit_interp_struct("gg_ttxggg", nt, sf, colour_matrix(5)[0], mf)
    amps = re.search(r"c_amps\[\d+\] = \{(.*?)\n\};", src, re.S).group(1)
    kinds = [int(k) for k in re.findall(r"\}, (\d+), \d+, \d+, \d+\}", amps)]
    a0, npair = 0, 0
    for st in I.stages:
        n = len(st.amps)
        for i in range(n):
            k = kinds[a0 + i]
            if k & 0x40:
                npair += 1
                assert i + 1 < n and (kinds[a0 + i + 1] & 0x3F) == (k & 0x3F)
                assert (i + 1 < st.mid) or (i >= st.mid)
                assert not kinds[a0 + i + 1] & 0x40
        a0 += n
    assert a0 == len(kinds) and 2 * npair > 0.8 * len(kinds)


def test_fp64_split_into_fp32_parts(tmp_path):
    """me_split.h (the FP32 kernels' per-event split of the FP64 momenta, by
    integer operations) compiled for the host: hi is x truncated to 24
    significant bits, lo the next 24 bits truncated (both exact, checked with
    integer arithmetic on the binary expansion), so |x - hi - lo| < 2^-47 |x|
    wherever the remainder stays in FP32's normal range (|x| >= 2^-73);
    zero keeps its sign, values below FP32's normal range give 0, above it inf,
    NaN stays NaN."""
    import math
    import shutil
    import subprocess

    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "split.cpp"
    src.write_text("""
#include "me_split.h"
#include <cstdio>
int main(int argc, char** argv) {
    FILE* f = fopen(argv[1], "rb"); FILE* o = fopen(argv[2], "wb");
    double x;
    while (fread(&x, sizeof x, 1, f) == 1) { float h, l; me::split_f32(x, h, l); fwrite(&h, 4, 1, o); fwrite(&l, 4, 1, o); }
    fclose(f); fclose(o); return 0;
}
""")
    exe = tmp_path / "split"
    csrc = os.path.join(ROOT, "paper_2507_21039_gb300", "csrc")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", csrc, str(src), "-o", str(exe)], check=True)
    rng = np.random.default_rng(5)
    mags = np.exp(rng.uniform(np.log(1e-30), np.log(1e30), 20000))
    xs = np.concatenate([mags * rng.choice([-1.0, 1.0], len(mags)), rng.normal(0, 500, 5000),
                         [0.0, -0.0, 1.0, -1.0, 2.0 ** -126, 2.0 ** -127, 1e-300, 3e38, 1e39, -1e300,
                          np.inf, -np.inf, np.nan, 1.0 + 2.0 ** -30, 1.0 - 2.0 ** -53]])
    (tmp_path / "in.bin").write_bytes(xs.astype("<f8").tobytes())
    subprocess.run([str(exe), str(tmp_path / "in.bin"), str(tmp_path / "out.bin")], check=True)
    out = np.frombuffer((tmp_path / "out.bin").read_bytes(), dtype="<f4").reshape(-1, 2)
    assert len(out) == len(xs)

    def trunc_bits(v, nbits):  # v > 0: v truncated to nbits significant bits, exactly
        mant, ex = math.frexp(v)  # v = mant * 2^ex, 0.5 <= mant < 1
        q = int(mant * (1 << 53))  # exact: 53-bit integer
        keep = q >> (53 - nbits) << (53 - nbits)
        return math.ldexp(keep, ex - 53)

    for x, (h, l) in zip(xs, out):
        h, l = float(h), float(l)
        if math.isnan(x):
            assert math.isnan(h)
            continue
        if math.isinf(x) or abs(x) >= 2.0 ** 128:
            assert h == math.copysign(math.inf, x) and l == 0.0
            continue
        if abs(x) < 2.0 ** -126:
            assert h == 0.0 and l == 0.0 and math.copysign(1, h) == math.copysign(1, x)
            continue
        a = abs(x)
        th = trunc_bits(a, 24)
        assert abs(h) == th and math.copysign(1, h) == math.copysign(1, x)
        rem = a - th  # exact in FP64 (the low bits of a)
        tl = trunc_bits(rem, 24) if rem >= 2.0 ** -126 else 0.0
        assert abs(l) == tl and (l == 0.0 or math.copysign(1, l) == math.copysign(1, x))
        if a >= 2.0 ** -73:  # the remainder, however small, in FP32's normal range
            assert abs(a - th - tl) < 2.0 ** -47 * a


@pytest.mark.parametrize("process", ["uux_epemgg", "uux_epemggg"])
def test_drell_yan_table_plan_layout(process):
    """Drell-Yan on the helicity-recycled table kernel: the lepton-pair objects
    have support {e+, e-} and read the e- and e+ states of their variant and the
    electroweak coefficients at entry 2 npar, which no object overwrites; every
    task's inputs are externals, that entry or computed variants of objects of
    an earlier level; every index (tasks and amplitude operands) lies inside the
    table; every variant that a non-vanishing helicity (opposite u, u~ and
    opposite e+, e- bits) reads is computed."""
    from paper_2507_21039_gb300.gen.tabplan import LEPTON_KINDS, build_tabplan

    T = build_tabplan(process)
    P = T.plan
    npar, size = P.npar, T.size
    ew = 2 * npar
    level_of = {}
    for r in T.rounds:
        for t in r.tasks:
            assert ew < t.out < size and t.out not in level_of
            level_of[t.out] = r.level
    for r in T.rounds:
        for v, t in enumerate(sorted(r.tasks, key=lambda x: x.out)):
            if r.kind in LEPTON_KINDS:
                assert r.level == 1 and len(t.ins) == 3 and t.ins[2] == ew
                assert t.ins[0] in (6, 7) and t.ins[1] in (4, 5)  # ubar(e-), v(e+) entries 2e + b
            for x in t.ins:
                assert 0 <= x < size
                if x > ew:
                    assert level_of[x] < r.level
    for i, op in enumerate(P.ops):
        if op.kind in LEPTON_KINDS:
            # variant v = b(e-) + 2 b(e+) (support particles in descending order)
            assert T.support[i] == (3, 2)
            lo = T.base[i]
            # only the opposite-helicity variants (v = 1, 2) are computed: equal e+, e-
            # helicities give exactly zero
            tasks = {t.out: t.ins for r in T.rounds if r.kind == op.kind for t in r.tasks}
            assert set(tasks) == {lo + 1, lo + 2}
            for v in (1, 2):
                assert tasks[lo + v] == (6 + (v & 1), 4 + (v >> 1), ew)
    for ai, _ in P.amps:
        for a in P.ops[ai].args:
            assert 0 <= T.base[a] and T.base[a] + (1 << len(T.support[a])) <= size
    from paper_2507_21039_gb300.gen.tabplan import compress

    computed = set(level_of)
    for h in range(1 << npar):
        bits = {p: (h >> (npar - 1 - p)) & 1 for p in range(npar)}
        if bits[0] == bits[1] or bits[2] == bits[3]:
            continue
        for ai, _ in P.amps:
            for a in P.ops[ai].args:
                if T.base[a] > ew:
                    assert T.base[a] + compress(bits, T.support[a]) in computed


def test_stage_sign_matrices_replay_the_flow_updates():
    """The FP32 descriptor kernel accumulates J on the tensor cores: per stage,
    Re J += Im G . B and Im J += Re G . (-B), G the stage's group sums in update
    order (at most 16), B the generator's sign matrix of the stage decoded from
    its BF16 image in the K-major core-matrix operand layout.  For random group
    sums this gives the same J as the flow-by-flow updates J_c += -i G (flag set)
    or +i G, and nothing in the padding flows 120..127."""
    from paper_2507_21039_gb300.gen.emit import emit_interp_struct, umma_k16_offset

    src, I = emit_interp_struct("gg_ttxggg", 128, 16, colour_matrix(5)[0], 0)

    def array(name):
        body = re.search(r"\b" + name + r"\[\d+\] = \{(.*?)\};", src, re.S).group(1)
        return [int(x) for x in re.findall(r"-?\d+", body)]

    terms, words = array("c_terms"), array("c_bmat")
    assert len(words) == 1024 * len(I.stages)
    halves = np.array([(w >> sh) & 0xFFFF for w in words for sh in (0, 16)], dtype=np.uint32)
    values = ((halves << 16).astype(np.uint32)).view(np.float32).astype(float)   # BF16 -> float
    assert set(np.unique(values)) <= {-1.0, 0.0, 1.0}
    rng = np.random.default_rng(9)
    J1 = np.zeros(120, complex)
    Jre, Jim = np.zeros(128), np.zeros(128)
    t = 0
    for si, st in enumerate(I.stages):
        img = values[2048 * si:2048 * (si + 1)]
        B = np.array([[img[umma_k16_offset(n, k) // 2] for k in range(16)] for n in range(128)])
        Gs = np.zeros(16, complex)
        k = 0
        for ai in st.amps:
            if ai not in I.flush:
                continue
            G = complex(*rng.normal(size=2))
            for col, c in I.flush[ai]:
                assert terms[t] == col | (0x8000 if c == (0, -1) else 0)
                J1[col] += (-1j if terms[t] & 0x8000 else 1j) * G
                t += 1
            Gs[k] = G
            k += 1
        assert k <= 16
        Jre += B @ Gs.imag
        Jim += -(B @ Gs.real)
    assert t == len(terms)
    assert np.all(Jre[120:] == 0) and np.all(Jim[120:] == 0)
    assert np.abs(J1 - (Jre[:120] + 1j * Jim[:120])).max() < 1e-12 * np.abs(J1).max()


def test_colour_numerators_as_tensor_core_operand():
    """gg -> t t~ g g's colour numerators as the B operand of the table
    kernel's tcgen05.mma colour sum: the two BF16 K = 16 images decoded through
    the operand layout give N[k][n] for k, n < 24 and zero in the padding."""
    from paper_2507_21039_gb300.gen.emit import emit_process, umma_k16_offset

    src, _ = emit_process("gg_ttxgg")
    body = re.search(r"c_umma_cn\[512\] = \{(.*?)\};", src, re.S).group(1)
    words = [int(x) for x in re.findall(r"\d+", body)]
    halves = np.array([(w >> sh) & 0xFFFF for w in words for sh in (0, 16)], dtype=np.uint32)
    vals = (halves << 16).astype(np.uint32).view(np.float32).astype(float)
    num, _ = colour_matrix(4)
    B = np.zeros((32, 32))
    for ks in range(2):
        for n in range(32):
            for kk in range(16):
                B[n, 16 * ks + kk] = vals[512 * ks + umma_k16_offset(n, kk) // 2]
    ref = np.zeros((32, 32))
    ref[:24, :24] = np.array(num, dtype=float).T
    assert np.array_equal(B, ref)


@pytest.mark.parametrize("process", ["ee_mumu", "gg_ttx", "gg_ttxg", "gg_ttxgg", "gg_ttxggg", "uux_epemg",
                                     "uux_epemgg", "uux_epemggg"])
def test_line_sides_and_gram_denominators(orc, process):
    """The FP32 kernels' per-event setup: each line's momentum written over its
    shorter side (the generator's packed table) equals the line's defining sum
    sum_plus p - sum_minus p, with at most three terms; the FP32 hi + lo split of
    the momenta holds them to 2^-48; and p^2 - m^2 as the FP64 sum of Gram
    entries c_a c_b p_a.p_b over that side equals the square of the FP64
    momentum sum minus m^2 within FP64 rounding of the largest term."""
    from paper_2507_21039_gb300.gen import emit

    from paper_2507_21039_gb300.gen.plan import build_plan_dy
    from paper_2507_21039_gb300.workloads import workload

    dy = process in emit.DY_PROCESSES
    P = build_plan_dy(emit.DY_PROCESSES[process]) if dy else build_plan(process)
    plus, minus, kind = emit._line_tables(P)
    sides, kmax = emit._line_sides(plus, minus, P.npar)
    assert kmax <= 3
    w = workload(process)
    mom, _, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, 0, 64, w.cut_mask, 20.0, 0.4)
    mt = 0.0 if process == "ee_mumu" or dy else MT
    if dy:  # the Drell-Yan quark line: -p_ubar + gluons (+ e+ + e- past the insertion)
        for ln, pm, mm in zip(P.lines, plus, minus):
            if ln.kind == "g":
                continue
            want_p = sum(1 << P.gluon_ext[g] for g in ln.gluons) | (0b1100 if ln.kind == "qe" else 0)
            assert (pm, mm) == (want_p, 0b10)
    hi = mom.astype(np.float32)
    lo = (mom - hi.astype(np.float64)).astype(np.float32)
    assert np.all(np.abs(hi.astype(np.float64) + lo - mom) <= 2.0**-48 * np.abs(mom) + 1e-300)
    mink = np.array([1.0, -1.0, -1.0, -1.0])
    gram = np.einsum("emu,efu,u->emf", mom, mom, mink)
    for pm, mm, kd, word in zip(plus, minus, kind, sides):
        c = np.array([((pm >> i) & 1) - ((mm >> i) & 1) for i in range(P.npar)], dtype=float)
        k = word & 7
        terms = [((word >> (4 * a + 4)) & 7, -1.0 if (word >> (4 * a + 7)) & 1 else 1.0) for a in range(k)]
        q = np.einsum("i,eiu->eu", c, mom)
        q_side = sum(sg * mom[:, i, :] for i, sg in terms)
        scale = mom[:, :, 0].sum(1)[:, None]
        assert np.abs(q_side - q).max() <= 1e-10 * scale.max()
        if kd == 0:
            continue
        m2 = mt * mt if kd == 2 else 0.0
        direct = q[:, 0] ** 2 - (q[:, 1:] ** 2).sum(1) - m2
        via_gram = -m2 + sum((1.0 if a == b else 2.0) * ta[1] * tb[1] * gram[:, ta[0], tb[0]]
                             for a, ta in enumerate(terms) for b, tb in enumerate(terms) if b >= a)
        assert np.all(np.abs(via_gram - direct) <= 1e-9 * scale[:, 0] ** 2)


@pytest.mark.parametrize("process", ["gg_ttxgg", "gg_ttxggg"])
def test_delta_r_guard_band_covers_fp32_error(orc, process):
    """The sampler decides the Delta R cut in FP32 (eta = asinh(pz / pT)) and
    re-decides in FP64 only pairs within 1e-3 of the cut; that band must be far
    wider than the FP32 error of Delta R.  Checked on the oracle's accepted
    momenta against the FP64 formula of the cut definition."""
    w = WORKLOADS[process]
    mom, _, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, 0, 4000, w.cut_mask, 20.0, 0.4)
    glu = [i for i, c in enumerate(w.cut_mask) if c]
    k = mom[:, 2:, :][:, glu, :]
    P = np.sqrt((k[..., 1:] ** 2).sum(-1))
    eta64 = 0.5 * np.log((P + k[..., 3]) / (P - k[..., 3]))
    phi64 = np.arctan2(k[..., 2], k[..., 1])
    k32 = k.astype(np.float32)
    eta32 = np.arcsinh(k32[..., 3] / np.sqrt(k32[..., 1] ** 2 + k32[..., 2] ** 2))
    phi32 = np.arctan2(k32[..., 2], k32[..., 1])
    worst = 0.0
    for i in range(len(glu)):
        for j in range(i + 1, len(glu)):
            d64 = np.remainder(phi64[:, i] - phi64[:, j] + np.pi, 2 * np.pi) - np.pi
            d32 = (phi32[:, i] - phi32[:, j]).astype(np.float32)
            d32 = np.where(d32 > np.pi, d32 - 2 * np.pi, d32)
            d32 = np.where(d32 < -np.pi, d32 + 2 * np.pi, d32)
            dr64 = np.hypot(eta64[:, i] - eta64[:, j], d64)
            dr32 = np.hypot((eta32[:, i] - eta32[:, j]).astype(np.float64), d32.astype(np.float64))
            worst = max(worst, float(np.abs(dr32 - dr64).max()))
            assert np.all(dr64 > 0.4)  # accepted events pass the FP64 cut
    print(process, "largest FP32 error of Delta R", worst)
    assert worst < 1e-4, worst


# ---------------------------------------------------------------- C ABI
def _declared_symbols(header="me.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "switch")))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_21039_gb300 import build as libbuild

    libbuild.build()
    import paper_2507_21039_gb300 as me

    return me.load()


def test_library_exports_every_declared_symbol(lib):
    import paper_2507_21039_gb300 as me

    from paper_2507_21039_gb300 import serving

    headers = sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))
    assert headers == ["me.h", "me_serve.h"]
    declared = _declared_symbols("me.h")
    assert set(declared) == set(me.EXPORTS), declared
    declared_srv = _declared_symbols("me_serve.h")
    assert set(declared_srv) == set(serving.SERVE_EXPORTS), declared_srv
    for name in declared + declared_srv:
        assert hasattr(lib, name), name


def test_library_is_built_for_sm_103a():
    from paper_2507_21039_gb300 import build as libbuild

    assert "arch=compute_103a,code=sm_103a" in " ".join(libbuild.ARCH)
    assert os.path.exists(libbuild.LIB)


def test_abi_validation_without_device(lib):
    import paper_2507_21039_gb300 as me

    assert lib.me_strerror(me.ME_EINVAL).decode() == "invalid argument"
    assert lib.me_version().decode().startswith("libme")
    h = ctypes.c_void_p()
    assert lib.me_init(ctypes.byref(h), b"not_a_process", None, 0, None, 0, 0) == me.ME_EINVAL
    assert lib.me_init(ctypes.byref(h), b"gg_ttx", None, 0, None, 0, 7) == me.ME_EINVAL
    bad = (ctypes.c_double * 4)(0, 0, 173.0, 172.0)   # t and t~ masses differ
    assert lib.me_init(ctypes.byref(h), b"gg_ttx", bad, 4, None, 0, 0) == me.ME_EINVAL
    short = (ctypes.c_double * 3)(0, 0, 173.0)
    assert lib.me_init(ctypes.byref(h), b"gg_ttx", short, 3, None, 0, 0) == me.ME_EINVAL
    neg = (ctypes.c_double * 1)(-0.1)
    assert lib.me_init(ctypes.byref(h), b"gg_ttx", None, 0, neg, 1, 0) == me.ME_EINVAL
    assert lib.me_init(None, b"gg_ttx", None, 0, None, 0, 0) == me.ME_EINVAL
    assert lib.me_sigmakin(None, None, 10, None, None) == me.ME_EINVAL
    assert lib.me_filter_helicities(None, None, 10, None) == me.ME_EINVAL
    assert lib.me_info(None, None, None, None, None, None) == me.ME_EINVAL
    m = (ctypes.c_double * 4)(0, 0, 173.0, 173.0)
    assert lib.rambo_sample(1, 0, 10, 1000.0, m, 2, None, None, None, None, None) == me.ME_EINVAL
    assert lib.rambo_sample(1, 0, -1, 1000.0, m, 4, None, None, None, None, None) == me.ME_EINVAL
    assert lib.rambo_sample(1, 0, 0, 1000.0, m, 4, None, None, None, None, None) == me.ME_OK
    heavy = (ctypes.c_double * 4)(0, 0, 600.0, 600.0)
    out = (ctypes.c_double * 16)()
    assert lib.rambo_sample(1, 0, 1, 1000.0, heavy, 4, None, out, None, None, None) == me.ME_EINVAL
    lib.me_free(None)


@pytest.mark.parametrize("process,stage,amputated", [("gg_ttxgg", 16, False), ("gg_ttxggg", 16, False),
                                                     ("gg_ttxg", 4, True), ("gg_ttxgg", 16, True), ("gg_ttxgg", 60, True),
                                                     ("gg_ttxggg", 16, True)])
def test_staged_schedule_reproduces_oracle(orc, process, stage, amputated):
    """The staged schedules (slot reuse after each object's last reader,
    variant indexing, colour groups; with or without amputated vertex objects,
    and with the groups that share a contraction operand contracted once) give
    the oracle's partial amplitudes."""
    from paper_2507_21039_gb300.gen.interp import build_interp
    from plan_eval import evaluate_staged

    I = build_interp(process, stage, amputated)
    w = WORKLOADS[process]
    mom, _, _ = orc.rambo(w.seed, w.sqrt_s, w.masses_final, 3, 1, w.cut_mask, 20.0, 0.4)
    p = mom[0]
    npar = I.tab.plan.npar
    scale = max(np.abs(orc.partial_amps(process, p, h)).max() for h in range(0, 1 << npar, 9))
    for h in (0b0110101 & ((1 << npar) - 1), (1 << npar) - 1 - 6):
        A = orc.partial_amps(process, p, h)
        for merge in ((False, True) if amputated else (False,)):
            J = evaluate_staged(orc, I, p, h, MT, merge)
            assert np.abs(J - A).max() < 1e-12 * scale
