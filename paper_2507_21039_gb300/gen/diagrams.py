"""Feynman diagrams of g g -> t tbar + n g and their colour decomposition.

Sec. 3.1 of arXiv:2507.21039 evaluates each Feynman diagram as a chain of
wavefunction, propagator and vertex routines, then contracts the colour-flow
amplitudes with the colour matrix.  This module enumerates those diagrams for
one quark line (outgoing t, outgoing tbar) and k gluons with the QCD vertices
qqg, ggg and gggg, and expands each diagram's colour factor on the string basis
(T^{a_s1} ... T^{a_sk})_{i_t j_tbar}.

A diagram is an ordered sequence of gluon trees attached along the quark line,
read from the t end to the tbar end; the trees' leaf sets partition the gluons.
A tree is a leaf (an external gluon), a three-gluon node with two children, or
a four-gluon node with three children and one of its three colour structures.
Counting a four-gluon node once per diagram gives 3, 16, 123, 1240 diagrams for
k = 2, 3, 4, 5.

Colour factors follow from f^{abc} T^c = -i [T^a, T^b]:
  three-gluon node (children A, B):      -i [A, B]
  four-gluon structure 0 (f^{abe}f^{cde}): -[[A, B], C]
  four-gluon structure 1 (f^{ace}f^{bde}): -[[A, C], B]
  four-gluon structure 2 (f^{ade}f^{bce}): -[[B, C], A]
with the node's colour contracted into T^d of the line (d the off-shell leg).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass
from functools import lru_cache

# complex coefficients are kept exact as pairs of ints (re, im)


def cmul(a, b):
    return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])


def cadd(a, b):
    return (a[0] + b[0], a[1] + b[1])


ONE = (1, 0)
MINUS_I = (0, -1)


@dataclass(frozen=True)
class Tree:
    """kind: 'leaf' (gluon = index into the gluon list), 'v3', 'v4' (struct 0..2)."""
    kind: str
    children: tuple = ()
    gluon: int = -1
    struct: int = -1

    @property
    def leaves(self) -> frozenset:
        if self.kind == "leaf":
            return frozenset([self.gluon])
        out = frozenset()
        for c in self.children:
            out |= c.leaves
        return out

    @property
    def min_leaf(self) -> int:
        return min(self.leaves)

    def key(self) -> str:
        if self.kind == "leaf":
            return f"g{self.gluon}"
        inner = ",".join(c.key() for c in self.children)
        return f"{self.kind}{self.struct if self.kind == 'v4' else ''}({inner})"

    def n_internal(self) -> int:
        """internal gluon lines (one per non-leaf node, each with a propagator)"""
        if self.kind == "leaf":
            return 0
        return 1 + sum(c.n_internal() for c in self.children)

    def n_v4(self) -> int:
        if self.kind == "leaf":
            return 0
        return (self.kind == "v4") + sum(c.n_v4() for c in self.children)


def _ordered_children(children):
    return tuple(sorted(children, key=lambda t: t.min_leaf))


@lru_cache(maxsize=None)
def trees(leafset: frozenset) -> tuple:
    """All trees (four-gluon nodes expanded into their 3 colour structures)."""
    leaves = sorted(leafset)
    if len(leaves) == 1:
        return (Tree("leaf", gluon=leaves[0]),)
    out = []
    first = leaves[0]
    rest = leaves[1:]
    # unordered 2-partitions {A, B}: A holds the first leaf
    for r in range(0, len(rest)):
        for comb in itertools.combinations(rest, r):
            A = frozenset((first,) + comb)
            B = leafset - A
            if not B:
                continue
            for ta in trees(A):
                for tb in trees(B):
                    out.append(Tree("v3", _ordered_children((ta, tb))))
    # unordered 3-partitions {A, B, C}
    for r in range(0, len(rest)):
        for comb in itertools.combinations(rest, r):
            A = frozenset((first,) + comb)
            R = sorted(leafset - A)
            if len(R) < 2:
                continue
            f2, rest2 = R[0], R[1:]
            for r2 in range(0, len(rest2)):
                for comb2 in itertools.combinations(rest2, r2):
                    B = frozenset((f2,) + comb2)
                    C = frozenset(R) - B
                    if not C:
                        continue
                    for ta in trees(A):
                        for tb in trees(B):
                            for tc in trees(C):
                                ch = _ordered_children((ta, tb, tc))
                                for s in range(3):
                                    out.append(Tree("v4", ch, struct=s))
    return tuple(out)


def ordered_set_partitions(items):
    """All ordered sequences of non-empty disjoint blocks covering items."""
    items = tuple(items)
    if not items:
        yield ()
        return
    n = len(items)
    for r in range(1, n + 1):
        for comb in itertools.combinations(items, r):
            rest = tuple(x for x in items if x not in comb)
            for tail in ordered_set_partitions(rest):
                yield (frozenset(comb),) + tail


def diagrams(k: int):
    """Amplitude terms: each is a tuple of trees (t end first).  Diagrams with
    four-gluon nodes appear once per colour-structure choice."""
    out = []
    for blocks in ordered_set_partitions(range(k)):
        for choice in itertools.product(*(trees(b) for b in blocks)):
            out.append(tuple(choice))
    return out


def diagram_count(k: int) -> int:
    """Feynman diagrams with each four-gluon vertex counted once."""
    seen = set()
    for d in diagrams(k):
        seen.add(tuple(_strip_struct(t) for t in d))
    return len(seen)


def _strip_struct(t: Tree) -> str:
    if t.kind == "leaf":
        return f"g{t.gluon}"
    return t.kind + "(" + ",".join(_strip_struct(c) for c in t.children) + ")"


# ---------------------------------------------------------------- colour
def _comm(A, B):
    """[A, B] for colour expansions {word: coef}"""
    out = {}
    for wa, ca in A.items():
        for wb, cb in B.items():
            c = cmul(ca, cb)
            out[wa + wb] = cadd(out.get(wa + wb, (0, 0)), c)
            out[wb + wa] = cadd(out.get(wb + wa, (0, 0)), (-c[0], -c[1]))
    return {w: c for w, c in out.items() if c != (0, 0)}


def _scale(A, s):
    return {w: cmul(c, s) for w, c in A.items()}


@lru_cache(maxsize=None)
def tree_colour(t: Tree):
    """Colour of a tree contracted with T^c of its root line, as {word: coef}."""
    if t.kind == "leaf":
        return {(t.gluon,): ONE}
    ch = [dict(tree_colour(c)) for c in t.children]
    if t.kind == "v3":
        out = _scale(_comm(ch[0], ch[1]), MINUS_I)
    else:
        A, B, C = ch
        inner = {0: _comm(_comm(A, B), C), 1: _comm(_comm(A, C), B), 2: _comm(_comm(B, C), A)}[t.struct]
        out = _scale(inner, (-1, 0))
    return tuple(sorted(out.items()))


def diagram_colour(d):
    """{permutation tuple: coef} for the product of the trees' colour factors."""
    cur = {(): ONE}
    for t in d:
        tc = dict(tree_colour(t))
        nxt = {}
        for w, c in cur.items():
            for w2, c2 in tc.items():
                key = w + w2
                nxt[key] = cadd(nxt.get(key, (0, 0)), cmul(c, c2))
        cur = {w: c for w, c in nxt.items() if c != (0, 0)}
    return cur


def diagram_phase(d):
    """Constant factor of the Feynman rules other than colour and couplings:
    i per quark-gluon vertex, i per top propagator, -i per gluon propagator,
    -i per four-gluon vertex (the three-gluon vertex carries no i)."""
    m = len(d)
    ph = ONE
    for _ in range(m):
        ph = cmul(ph, (0, 1))  # qqg vertices
    for _ in range(m - 1):
        ph = cmul(ph, (0, 1))  # top propagators
    for t in d:
        for _ in range(t.n_internal()):
            ph = cmul(ph, (0, -1))  # gluon propagators
        for _ in range(t.n_v4()):
            ph = cmul(ph, (0, -1))  # four-gluon vertex -i
    return ph


def permutation_index(k: int):
    """lexicographic permutation order of range(k) -> index"""
    return {p: i for i, p in enumerate(itertools.permutations(range(k)))}


# ---------------------------------------------------------------- Drell-Yan
# u ubar -> e+ e- + n g: the quark line (read from the ubar end) carries the
# gluon trees and one colourless element EW, the photon/Z coupling to the
# lepton pair.  The EW element has no colour and no gluon leaves.
EW = Tree("ew")


def dy_diagrams(k: int):
    """Amplitude terms of u ubar -> e+ e- + k g: every sequence of gluon trees
    along the quark line (as in `diagrams`) with EW inserted at each position."""
    out = []
    seqs = diagrams(k) if k else [()]
    for d in seqs:
        for pos in range(len(d) + 1):
            out.append(d[:pos] + (EW,) + d[pos:])
    return out


def dy_diagram_colour(d):
    """colour of a Drell-Yan term: that of its gluon trees (EW is colourless)"""
    return diagram_colour(tuple(t for t in d if t.kind != "ew"))


def dy_diagram_phase(d):
    """i per quark-line vertex (gluon or EW), i per quark propagator, -i per
    gluon propagator and per four-gluon vertex (the EW element's own factors,
    two vertices and the boson propagator, combine to i and are counted as its
    quark-line vertex)"""
    m = len(d)
    ph = ONE
    for _ in range(2 * m - 1):
        ph = cmul(ph, (0, 1))
    for t in d:
        if t.kind == "ew":
            continue
        for _ in range(t.n_internal() + t.n_v4()):
            ph = cmul(ph, (0, -1))
    return ph
