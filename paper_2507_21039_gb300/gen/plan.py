"""Evaluation plan of the helicity-amplitude chain for one process.

Sec. 3.1 of arXiv:2507.21039: external wavefunctions (vxxxxx, oxxxxx,
ixxxxx) are merged into off-shell currents (VVV1P0_1, FFV1_1, ...) until a
final vertex (FFV1_0, VVV1_0, ...) gives each diagram's amplitude; the
amplitudes enter the colour-flow partial amplitudes J.  Here every off-shell
object is computed once per helicity and shared by all diagrams that contain
it:

* gluon trees  -> vector currents (VVV1P0_1, VVVV{1,3,4}P0_1);
* quark-line prefixes  ubar G1 S1 ... Gj Sj          -> row spinors    (FFV1_2);
* quark-line suffixes  S_j G_{j+1} ... Gm v          -> column spinors (FFV1_1);
* the t tbar pair current  ubar gamma^mu v / q^2     -> vector         (FFV1P0_3).

A diagram (t1 .. tm) with m >= 2 is evaluated as
FFV1_0(prefix(t1..t_{j-1}), J(t_j), suffix(t_{j+1}..tm)) with the split j chosen
greedily to reuse what is already planned; a diagram with a single tree (all
gluons in one tree) is evaluated at the tree's top vertex against the pair
current: VVV1_0 / VVVV*_0.

Lines: every object carries a momentum.  Gluon clusters S (sets of gluons)
carry P_S = sum of outgoing momenta (incoming gluons count with -p) and
1/P_S^2; quark-line propagators carry q = p_t + P_S (S = gluons on the t side)
and 1/(q^2 - m_t^2).  Both are evaluated per event in FP64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

from . import diagrams as D

# real flops per routine as implemented in helas.cuh (one FMA = 2 flops)
FLOPS = {
    "VVV1P0_1": 136,
    "VVVV1P0_1": 86, "VVVV3P0_1": 86, "VVVV4P0_1": 86,
    "FFV1_2": 124, "FFV1_1": 124,
    "FFV1P0_3": 72,
    "FFV1_0": 72,
    "VVV1_0": 90,
    "VVVV1_0": 70, "VVVV3_0": 70, "VVVV4_0": 70,
    # amputated vertices (no propagator) and two-operand contractions, see amputate()
    "FFV1A_3": 64, "FFV1A_2": 64, "FFV1A_1": 64,
    "VVV1A_1": 116, "VVV1A_2": 116, "VVV1A_3": 116,
    "VVVV1A": 78, "VVVV3A": 78, "VVVV4A": 78,
    "DOTV": 30, "DOTF": 30,
    # Drell-Yan insertion (massless quark line): the FFV1 routines with a second
    # 2x2 block and no mass terms; the lepton-pair objects of both chiralities
    # (one call forms both: ext_lepR costs nothing beside ext_lepL in the chain)
    "FFVLR_0": 80, "FFVLR_2": 116, "FFVLR_1": 116, "ext_lepL": 176, "ext_lepR": 0,
}
V4NAMES = ("VVVV1", "VVVV3", "VVVV4")


@dataclass
class Line:
    kind: str          # 'g' gluon cluster, 'q' top propagator
    gluons: frozenset  # gluon positions (indices into the gluon list)


@dataclass
class Op:
    kind: str                  # routine name or ext_v / ext_fo / ext_fi
    args: tuple = ()           # input op indices
    line: int = -1             # output line (momentum / inverse denominator)
    mom: tuple = ()            # line indices whose momenta the vertex needs
    ext: int = -1              # external particle for ext_* ops
    out: str = "V"             # V, Fo (row spinor), Fi (column spinor), A (amplitude)


@dataclass
class Plan:
    process: str
    npar: int
    gluon_ext: tuple           # external index of each gluon position
    gluon_incoming: tuple
    ncol: int
    ops: list = field(default_factory=list)
    lines: list = field(default_factory=list)
    amps: list = field(default_factory=list)   # (op index, ((col, (re, im)), ...))
    ndiagrams: int = 0
    amp_diag: list = field(default_factory=list)   # Feynman diagram of each amplitude
    diag_lines: list = field(default_factory=list)  # internal lines of each diagram (see diagram_lines)

    def flops_per_helicity(self) -> int:
        f = sum(FLOPS.get(o.kind, 0) for o in self.ops)
        # J accumulation: each (amp, colour) term is a complex multiply-add by a
        # Gaussian-integer constant; +-1 / +-i cost one complex add (2 flops)
        for _, terms in self.amps:
            for _, c in terms:
                f += 2 if (abs(c[0]) + abs(c[1]) == 1) else 4
        return f

    def colour_flops_per_helicity(self) -> int:
        n = self.ncol
        # sum_ij C_ij (Re_i Re_j + Im_i Im_j) over the upper triangle, FMA = 2
        return 2 * (2 * (n * (n + 1) // 2) + 2 * n)

    def counts(self) -> dict:
        c = {}
        for o in self.ops:
            c[o.kind] = c.get(o.kind, 0) + 1
        return c


QCD = {"gg_ttx": 2, "gg_ttxg": 3, "gg_ttxgg": 4, "gg_ttxggg": 5}


def build_plan(process: str) -> Plan:
    if process == "ee_mumu":
        return _plan_ee()
    k = QCD[process]
    npar = k + 2
    gluon_ext = tuple([0, 1] + list(range(4, npar)))
    P = Plan(process, npar, gluon_ext, tuple(e < 2 for e in gluon_ext), math.factorial(k))
    line_idx = {}

    def line(kind, gl):
        key = (kind, frozenset(gl))
        if key not in line_idx:
            line_idx[key] = len(P.lines)
            P.lines.append(Line(kind, frozenset(gl)))
        return line_idx[key]

    def add(op):
        P.ops.append(op)
        return len(P.ops) - 1

    # external wavefunctions
    ext_g = [add(Op("ext_v", ext=e, line=line("g", [g]), out="V")) for g, e in enumerate(gluon_ext)]
    ext_fo = add(Op("ext_fo", ext=2, out="Fo", line=line("q", [])))
    ext_fi = add(Op("ext_fi", ext=3, out="Fi"))
    allg = frozenset(range(k))

    cur = {}

    def current(t):
        key = t.key()
        if key in cur:
            return cur[key]
        if t.kind == "leaf":
            cur[key] = ext_g[t.gluon]
            return cur[key]
        ch = [current(c) for c in t.children]
        out_line = line("g", t.leaves)
        if t.kind == "v3":
            mom = tuple(P.ops[c].line for c in ch)
            idx = add(Op("VVV1P0_1", tuple(ch), out_line, mom))
        else:
            idx = add(Op(V4NAMES[t.struct] + "P0_1", tuple(ch), out_line))
        cur[key] = idx
        return idx

    pre = {(): ext_fo}
    suf = {(): ext_fi}

    def prefix(seq):
        key = tuple(t.key() for t in seq)
        if key in pre:
            return pre[key]
        base = prefix(seq[:-1])
        J = current(seq[-1])
        gl = frozenset().union(*(t.leaves for t in seq))
        idx = add(Op("FFV1_2", (base, J), line("q", gl), out="Fo"))
        pre[key] = idx
        return idx

    def suffix(seq):
        key = tuple(t.key() for t in seq)
        if key in suf:
            return suf[key]
        base = suffix(seq[1:])
        J = current(seq[0])
        gl_t_side = allg - frozenset().union(*(t.leaves for t in seq))
        idx = add(Op("FFV1_1", (J, base), line("q", gl_t_side), out="Fi"))
        suf[key] = idx
        return idx

    pair = None

    def new_objects(d, j):
        """objects a split would add: missing prefixes, suffixes, currents"""
        n = 0
        for r in range(1, j):
            if tuple(t.key() for t in d[:r]) not in pre:
                n += 1
        for r in range(j + 1, len(d)):
            if tuple(t.key() for t in d[r:]) not in suf:
                n += 1
        return n

    pidx = D.permutation_index(k)
    terms = D.diagrams(k)
    P.ndiagrams = D.diagram_count(k)
    # diagram ids in order of first appearance; a four-gluon vertex's colour
    # structures are amplitudes of one diagram
    diag_of_term, key_id = [], {}
    for d in terms:
        key = _term_lines(d, gluon_ext)
        if key not in key_id:
            key_id[key] = len(P.diag_lines)
            P.diag_lines.append(key)
        diag_of_term.append(key_id[key])
    # longer diagrams first: their prefixes/suffixes seed the reuse
    order = sorted(range(len(terms)), key=lambda i: (-len(terms[i]), i))
    for di in order:
        d = terms[di]
        ph = D.diagram_phase(d)
        col = D.diagram_colour(d)
        coeffs = []
        for w, c in sorted(col.items()):
            coeffs.append((pidx[w], D.cmul(ph, c)))
        if len(d) == 1:
            t = d[0]
            if pair is None:
                pair = add(Op("FFV1P0_3", (ext_fo, ext_fi), line("g", allg)))
            ch = [current(c) for c in t.children]
            if t.kind == "v3":
                mom = tuple(P.ops[c].line for c in ch)
                a = add(Op("VVV1_0", tuple(ch) + (pair,), -1, mom, out="A"))
            else:
                a = add(Op(V4NAMES[t.struct] + "_0", tuple(ch) + (pair,), -1, out="A"))
        else:
            best = min(range(len(d)), key=lambda j: (new_objects(d, j), abs(2 * j - (len(d) - 1))))
            L = prefix(d[:best])
            Jm = current(d[best])
            R = suffix(d[best + 1:])
            a = add(Op("FFV1_0", (L, Jm, R), -1, out="A"))
        P.amps.append((a, tuple(coeffs)))
        P.amp_diag.append(diag_of_term[di])
    return P


def _term_lines(d, gluon_ext) -> tuple:
    """Internal lines of a diagram (sequence of gluon trees along the quark line
    from the t end): each line as the mask of external particles on its side
    away from the t~ (gluon subtrees: their leaves; quark propagators: the t and
    the gluons attached before them), sorted.  A tree diagram is fixed by this
    set of splits."""
    lines = []

    def tree_lines(t):
        if t.kind == "leaf":
            return
        lines.append(sum(1 << gluon_ext[g] for g in t.leaves))
        for c in t.children:
            tree_lines(c)

    side = 1 << 2
    for j, t in enumerate(d):
        tree_lines(t)
        side |= sum(1 << gluon_ext[g] for g in t.leaves)
        if j < len(d) - 1:
            lines.append(side)
    return tuple(sorted(lines))


def colour_groups(P: Plan):
    """Amplitudes whose colour-flow coefficient vectors are equal up to a sign.

    The colour-flow vector is J_c = sum_a c_{a,c} A_a (Sec. 4.1).  If two
    amplitudes have c_b = -c_a or c_b = c_a, their contribution to J is
    c_a (A_a -+ A_b): the amplitudes are summed first and J is updated once per
    group.  The normalised vector of a group has its lowest-flow coefficient
    equal to +i or, for real coefficients, +1.
    Returns (group of each amplitude, its sign in {+1, -1}, the terms of each
    group, the amplitudes of each group in plan order)."""
    key_of, group_of, sign_of, terms_of, members = {}, [], [], [], []
    for ai, (_, terms) in enumerate(P.amps):
        t = tuple(sorted(terms))
        c0 = t[0][1]
        s = -1 if (c0[1] < 0 or (c0[1] == 0 and c0[0] < 0)) else 1
        key = tuple((f, (s * c[0], s * c[1])) for f, c in t)
        if key not in key_of:
            key_of[key] = len(terms_of)
            terms_of.append(key)
            members.append([])
        g = key_of[key]
        group_of.append(g)
        sign_of.append(s)
        members[g].append(ai)
    return group_of, sign_of, terms_of, members


def diagram_lines(P: Plan, d: int) -> tuple:
    """internal lines of diagram d (masks over the external particles)"""
    return P.diag_lines[d]


def _plan_ee() -> Plan:
    """e-(1) e+(2) -> mu-(3) mu+(4) via one s-channel photon: the e+e- current
    (FFV1P0_3 of vbar(e+) and u(e-)) contracted with the muon line (FFV1_0)."""
    P = Plan("ee_mumu", 4, (), (), 1)
    P.lines = [Line("a", frozenset())]   # photon line: p1 + p2, 1/s
    P.ops = [
        Op("ext_fi", ext=0, out="Fi"),      # u(e-)
        Op("ext_fo", ext=1, out="Fo"),      # vbar(e+)
        Op("ext_fo", ext=2, out="Fo"),      # ubar(mu-)
        Op("ext_fi", ext=3, out="Fi"),      # v(mu+)
        Op("FFV1P0_3", (1, 0), 0),
        Op("FFV1_0", (2, 4, 3), -1, out="A"),
    ]
    # i e gamma at each vertex (charge -1 absorbed in the overall sign), -i/q^2:
    # i * i * (-i) = i
    P.amps = [(5, ((0, (0, 1)),))]
    P.ndiagrams = 1
    P.amp_diag = [0]
    P.diag_lines = [(0b11,)]
    return P


# ---------------------------------------------------------------------------
# amputated form: every amplitude as a two-operand contraction
# ---------------------------------------------------------------------------
# A final vertex is a multilinear form of its operands.  Leaving one operand's
# index open gives an "amputated" vertex object (no propagator) whose
# contraction with that operand is the amplitude:
#   FFV1_0(Fo, V, Fi) = K.V        K^mu = Fo gamma^mu Fi         (FFV1A_3, DOTV)
#                     = R Fi       R    = Fo gamma.V  (row)      (FFV1A_2, DOTF)
#                     = Fo C       C    = gamma.V Fi  (column)   (FFV1A_1, DOTF)
#   VVV1_0(A, B, Q)   = W.Q, W.A, W.B with the open leg Q, A, B  (VVV1A_3/1/2, DOTV)
#   VVVVn_0(A,B,C,Q)  = W.Q        W = VVVVnP0_1(A, B, C) without propagator
# The vertex objects depend on the helicities of their operands only, so the
# table kernel evaluates them once per configuration of that support; per
# helicity only the contraction (30 flops) remains.  Products and sums are the
# same as in the direct vertex, grouped differently.
_SPLITS = {
    # kind -> [(open operand position, vertex kind, vertex operand positions, out)]
    "FFV1_0": [(1, "FFV1A_3", (0, 2), "V"), (2, "FFV1A_2", (0, 1), "Fo"), (0, "FFV1A_1", (1, 2), "Fi")],
    "VVV1_0": [(2, "VVV1A_3", (0, 1), "V"), (0, "VVV1A_1", (1, 2), "V"), (1, "VVV1A_2", (0, 2), "V")],
    "VVVV1_0": [(3, "VVVV1A", (0, 1, 2), "V")],
    "VVVV3_0": [(3, "VVVV3A", (0, 1, 2), "V")],
    "VVVV4_0": [(3, "VVVV4A", (0, 1, 2), "V")],
}


def amputate(P: Plan, support: dict) -> Plan:
    """Rewrite every amplitude of P as a contraction of an amputated vertex
    object with the remaining operand.  `support` maps op index -> tuple of
    external particles.  For each amplitude the split that adds the fewest new
    table variants (2^|support| of a vertex not yet created) is taken; vertex
    objects are shared between amplitudes."""
    Q = Plan(P.process, P.npar, P.gluon_ext, P.gluon_incoming, P.ncol, [], list(P.lines), [], P.ndiagrams,
             list(P.amp_diag), list(P.diag_lines))
    # keep every object of P (the direct amplitude ops go), indices renumbered
    new = {}
    for i, op in enumerate(P.ops):
        if op.out != "A":
            new[i] = len(Q.ops)
            Q.ops.append(Op(op.kind, tuple(new[a] for a in op.args), op.line, op.mom, op.ext, op.out))
    sup_of = {new[i]: support[i] for i in new}
    made = {}
    for ai, terms in P.amps:
        op = P.ops[ai]
        best = None
        for open_pos, vkind, vpos, out in _SPLITS[op.kind]:
            vargs = tuple(new[op.args[i]] for i in vpos)
            key = (vkind, vargs, op.mom)
            sup = set()
            for a in vargs:
                sup |= set(sup_of[a])
            cost = 0 if key in made else (1 << len(sup)) * FLOPS[vkind]
            cand = (cost, len(sup), key, open_pos, out)
            if best is None or cand[:2] < best[:2]:
                best = cand
        _, _, key, open_pos, out = best
        if key not in made:
            vkind, vargs, mom = key
            Q.ops.append(Op(vkind, vargs, -1, mom if vkind.startswith("VVV1A") else (), out=out))
            made[key] = len(Q.ops) - 1
        x = made[key]
        other = new[op.args[open_pos]]
        dk = "DOTF" if out in ("Fo", "Fi") else "DOTV"
        # DOTF takes (row, column)
        args = (x, other) if out == "Fo" else ((other, x) if out == "Fi" else (x, other))
        Q.ops.append(Op(dk, args, -1, out="A"))
        Q.amps.append((len(Q.ops) - 1, terms))
    return Q


def build_plan_dy(k: int) -> Plan:
    """u(0) ubar(1) -> e+(2) e-(3) + k gluons (4..), photon and Z exchange
    (the paper's Drell-Yan workload, Sec. 4).  The quark line runs from the
    ubar row spinor (`ext_fo`, vbar) to the u column spinor (`ext_fi`); the
    lepton pair enters as two vector objects, the left- and right-chirality
    sums over the photon and the Z of (quark coupling) x (lepton current over
    its propagator), `ext_lepL` / `ext_lepR`.  Quark-line objects that contain
    the electroweak insertion use `FFVLR_2` / `FFVLR_1` (the chiral vertex
    slash(L_L) P_L + slash(L_R) P_R and the quark propagator) and the diagram
    split at the insertion uses `FFVLR_0`.  Lines: gluon clusters as in
    `build_plan`; quark lines carry q = -p_ubar + P_S (+ p_e+ + p_e- when the
    insertion is on the ubar side): kind "q" without, "qe" with it.
    Generator-level only for now (evaluated by the host-side tests)."""
    npar = k + 4
    gluon_ext = tuple(range(4, npar))
    P = Plan(f"dy_{k}g", npar, gluon_ext, tuple(False for _ in gluon_ext), max(1, math.factorial(k)))
    line_idx = {}

    def line(kind, gl):
        key = (kind, frozenset(gl))
        if key not in line_idx:
            line_idx[key] = len(P.lines)
            P.lines.append(Line(kind, frozenset(gl)))
        return line_idx[key]

    def add(op):
        P.ops.append(op)
        return len(P.ops) - 1

    ext_g = [add(Op("ext_v", ext=e, line=line("g", [g]), out="V")) for g, e in enumerate(gluon_ext)]
    ext_fo = add(Op("ext_fo", ext=1, out="Fo"))
    ext_fi = add(Op("ext_fi", ext=0, out="Fi"))
    lep = (add(Op("ext_lepL", ext=2, out="V")), add(Op("ext_lepR", ext=2, out="V")))
    allg = frozenset(range(k))
    cur = {}

    def current(t):
        key = t.key()
        if key in cur:
            return cur[key]
        if t.kind == "leaf":
            cur[key] = ext_g[t.gluon]
            return cur[key]
        ch = [current(c) for c in t.children]
        out_line = line("g", t.leaves)
        if t.kind == "v3":
            idx = add(Op("VVV1P0_1", tuple(ch), out_line, tuple(P.ops[c].line for c in ch)))
        else:
            idx = add(Op(V4NAMES[t.struct] + "P0_1", tuple(ch), out_line))
        cur[key] = idx
        return idx

    def seq_key(seq):
        return tuple(t.key() for t in seq)

    def gluons(seq):
        return frozenset().union(*(t.leaves for t in seq)) if seq else frozenset()

    pre, suf = {(): ext_fo}, {(): ext_fi}

    def prefix(seq):
        key = seq_key(seq)
        if key not in pre:
            base, last = prefix(seq[:-1]), seq[-1]
            ln = line("qe" if any(t.kind == "ew" for t in seq) else "q", gluons(seq))
            if last.kind == "ew":
                pre[key] = add(Op("FFVLR_2", (base,) + lep, ln, out="Fo"))
            else:
                pre[key] = add(Op("FFV1_2", (base, current(last)), ln, out="Fo"))
        return pre[key]

    def suffix(seq):
        key = seq_key(seq)
        if key not in suf:
            base, first = suffix(seq[1:]), seq[0]
            # the propagator before the suffix, seen from the ubar side
            ln = line("q" if any(t.kind == "ew" for t in seq) else "qe", allg - gluons(seq))
            if first.kind == "ew":
                suf[key] = add(Op("FFVLR_1", lep + (base,), ln, out="Fi"))
            else:
                suf[key] = add(Op("FFV1_1", (current(first), base), ln, out="Fi"))
        return suf[key]

    def new_objects(d, j):
        n = sum(seq_key(d[:r]) not in pre for r in range(1, j))
        return n + sum(seq_key(d[r:]) not in suf for r in range(j + 1, len(d)))

    pidx = D.permutation_index(k)
    terms = D.dy_diagrams(k)
    P.ndiagrams = len({tuple(D._strip_struct(t) if t.kind != "ew" else "ew" for t in d) for d in terms})
    order = sorted(range(len(terms)), key=lambda i: (-len(terms[i]), i))
    for di in order:
        d = terms[di]
        ph = D.dy_diagram_phase(d)
        coeffs = tuple((pidx[w], D.cmul(ph, c)) for w, c in sorted(D.dy_diagram_colour(d).items()))
        best = min(range(len(d)), key=lambda j: (new_objects(d, j), abs(2 * j - (len(d) - 1))))
        L, R = prefix(d[:best]), suffix(d[best + 1:])
        if d[best].kind == "ew":
            a = add(Op("FFVLR_0", (L,) + lep + (R,), -1, out="A"))
        else:
            a = add(Op("FFV1_0", (L, current(d[best]), R), -1, out="A"))
        P.amps.append((a, coeffs))
        P.amp_diag.append(di)
    return P
