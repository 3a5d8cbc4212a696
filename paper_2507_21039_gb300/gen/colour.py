"""Exact colour matrix of the string basis (Sec. 4.1 of arXiv:2507.21039:
the colour algebra is an inner product with an integer-coefficient matrix).

C_{s,t} = sum over colours of conj((T^{a_s1}..T^{a_sk})_{ij}) (T^{a_t1}..T^{a_tk})_{ij}
        = sum_a Tr(T^{a_sk} .. T^{a_s1} T^{a_t1} .. T^{a_tk}).
Every adjoint index appears twice in that trace.  Replacing each pair by the
completeness relation sum_a T^a_{ij} T^a_{kl} = 1/2 (d_il d_kj - d_ij d_kl / N)
turns the trace into 2^k products of Kronecker deltas; each product contributes
(1/2)^k (-1/N)^{#second terms} N^{#closed index loops}.  The loops are counted
with a union-find over the 2k index slots of the trace.

C_{s,t} depends only on s^{-1} t (relabelling of summed indices), so one row is
computed and the matrix filled from it.  Output: integer numerators and one
common denominator, C = num / den exactly.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

NC = 3


def _trace_value(word):
    """sum over the labels of Tr(prod_p T^{word[p]}), each label twice."""
    n = len(word)
    pos = {}
    for p, lab in enumerate(word):
        pos.setdefault(lab, []).append(p)
    pairs = list(pos.values())
    total = Fraction(0)
    # generator at position p maps slot p (row index) to slot p+1 (column index)
    for choice in itertools.product((0, 1), repeat=len(pairs)):
        parent = list(range(n))

        def find(x):
            while parent[x] != x:
                parent[x] = parent[parent[x]]
                x = parent[x]
            return x

        def union(a, b):
            ra, rb = find(a), find(b)
            if ra != rb:
                parent[ra] = rb

        coef = Fraction(1, 2 ** len(pairs))
        for (p, q), c in zip(pairs, choice):
            pn, qn = (p + 1) % n, (q + 1) % n
            if c == 0:
                # T_{i_p i_pn} T_{i_q i_qn} -> d(i_p, i_qn) d(i_q, i_pn)
                union(p, qn)
                union(q, pn)
            else:
                # -> -1/N d(i_p, i_pn) d(i_q, i_qn)
                union(p, pn)
                union(q, qn)
                coef *= Fraction(-1, NC)
        loops = len({find(x) for x in range(n)})
        total += coef * NC**loops
    return total


def colour_matrix(k: int):
    """(numerators as list of lists of int, denominator) in lexicographic
    permutation order of the k gluons."""
    perms = list(itertools.permutations(range(k)))
    index = {p: i for i, p in enumerate(perms)}
    row = [_trace_value(tuple(reversed(perms[0])) + p) for p in perms]
    den = 1
    for x in row:
        den = den * x.denominator // math.gcd(den, x.denominator)
    num = [[0] * len(perms) for _ in perms]
    for i, s in enumerate(perms):
        inv = [0] * k
        for a, b in enumerate(s):
            inv[b] = a
        for j, t in enumerate(perms):
            rel = tuple(inv[x] for x in t)
            v = row[index[rel]] * den
            assert v.denominator == 1
            num[i][j] = int(v)
    return num, den
