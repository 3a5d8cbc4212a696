"""Test helper: evaluate a generator plan with numpy, one event and helicity.

Checks the generator's host logic (diagram enumeration, colour coefficients,
phases, reuse of sub-currents) on the CPU.  The routines below restate the
real-coefficient Lorentz structures that the plan names; external
wavefunctions come from the pinned oracle.  This is test code only.
"""
import numpy as np

G = []
_s = [np.eye(2), np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
for _mu in range(4):
    _g = np.zeros((4, 4), dtype=complex)
    _g[:2, 2:] = _s[_mu]
    _g[2:, :2] = _s[_mu] if _mu == 0 else -_s[_mu]
    G.append(_g)
METRIC = np.array([1.0, -1.0, -1.0, -1.0])
AMPUTATED_VERTICES = ("FFV1A_3", "FFV1A_2", "FFV1A_1", "VVV1A_1", "VVV1A_2", "VVV1A_3", "VVVV1A", "VVVV3A", "VVVV4A")


def dot(a, b):
    return np.sum(METRIC * a * b)


def slash(v):
    return G[0] * v[0] - G[1] * v[1] - G[2] * v[2] - G[3] * v[3]


def _vvv_open(kind, a, PA, PB):
    """three-gluon vertex V^{mnr}(k1, k2, k3) A_m B_n Q_r, k1 = -PA, k2 = -PB,
    k3 = PA + PB, with one leg left open (upper index).  kind VVV1A_3: open Q,
    inputs (A, B); VVV1A_1: open A, inputs (B, Q); VVV1A_2: open B, inputs (A, Q)."""
    k1, k2, k3 = -PA, -PB, PA + PB
    d12, d23, d31 = k1 - k2, k2 - k3, k3 - k1
    if kind == "VVV1A_3":
        A, B = a
        return dot(A, B) * d12 + B * dot(d23, A) + A * dot(d31, B)
    if kind == "VVV1A_1":
        B, Q = a
        return B * dot(d12, Q) + dot(B, Q) * d23 + Q * dot(d31, B)
    A, Q = a
    return A * dot(d12, Q) + Q * dot(d23, A) + dot(Q, A) * d31


def _amputated(kind, a, lines, op_mom):
    """amputated vertices (no propagator) and the two-operand contractions"""
    if kind == "FFV1A_3":
        return np.array([a[0] @ G[mu] @ a[1] for mu in range(4)])
    if kind == "FFV1A_2":
        return a[0] @ slash(a[1])
    if kind == "FFV1A_1":
        return slash(a[0]) @ a[1]
    if kind.startswith("VVV1A"):
        return _vvv_open(kind, a, lines[op_mom[0]][0], lines[op_mom[1]][0])
    if kind.startswith("VVVV") and kind.endswith("A"):
        return _v4(kind[:5], a[0], a[1], a[2])
    if kind == "DOTV":
        return dot(a[0], a[1])
    if kind == "DOTF":
        return a[0] @ a[1]
    return None


def evaluate(orc, plan, p, h, mt):
    """Colour-flow amplitudes J (couplings stripped) for event p, helicity h."""
    npar = plan.npar
    lam = [1 if (h >> (npar - 1 - i)) & 1 else -1 for i in range(npar)]
    incoming = [i < 2 for i in range(npar)]
    out_p = np.array([(-p[i] if incoming[i] else p[i]) for i in range(npar)])

    lines = []
    for ln in plan.lines:
        if ln.kind == "a":
            q = p[0] + p[1]
            lines.append((q, 1.0 / dot(q, q)))
        elif ln.kind == "g":
            q = sum(out_p[plan.gluon_ext[g]] for g in ln.gluons)
            lines.append((q, 1.0 / dot(q, q) if len(ln.gluons) > 1 else 0.0))
        else:
            q = p[2] + sum((out_p[plan.gluon_ext[g]] for g in ln.gluons), np.zeros(4))
            lines.append((q, 1.0 / (dot(q, q) - mt * mt)))

    mass = {"ee_mumu": 0.0}.get(plan.process, mt)
    vals = []
    for op in plan.ops:
        a = [vals[i] for i in op.args]
        k = op.kind
        if k == "ext_v":
            e = op.ext
            eps = orc.polvec(p[e], lam[e])
            vals.append(eps if incoming[e] else np.conj(eps))
        elif k == "ext_fo":
            e = op.ext
            if plan.process == "ee_mumu" and e == 1:
                vals.append(orc.bar(orc.spinor_v(p[e], 0.0, lam[e])))
            else:
                vals.append(orc.bar(orc.spinor_u(p[e], mass, lam[e])))
        elif k == "ext_fi":
            e = op.ext
            if plan.process == "ee_mumu" and e == 0:
                vals.append(orc.spinor_u(p[e], 0.0, lam[e]))
            else:
                vals.append(orc.spinor_v(p[e], mass, lam[e]))
        elif k == "VVV1P0_1":
            A, B = a
            PA, PB = lines[op.mom[0]][0], lines[op.mom[1]][0]
            k1, k2, k3 = -PA, -PB, PA + PB
            v = dot(A, B) * (k1 - k2) + B * dot(k2 - k3, A) + A * dot(k3 - k1, B)
            vals.append(lines[op.line][1] * v)
        elif k.startswith("VVVV") and k.endswith("P0_1"):
            A, B, C = a
            v = _v4(k[:5], A, B, C)
            vals.append(lines[op.line][1] * v)
        elif k == "FFV1_2":
            L, V = a
            q, inv = lines[op.line]
            vals.append(inv * (L @ slash(V) @ (slash(q) + mt * np.eye(4))))
        elif k == "FFV1_1":
            V, R = a
            q, inv = lines[op.line]
            vals.append(inv * ((slash(q) + mt * np.eye(4)) @ slash(V) @ R))
        elif k == "FFV1P0_3":
            Fo, Fi = a
            inv = lines[op.line][1]
            vals.append(inv * np.array([Fo @ G[mu] @ Fi for mu in range(4)]))
        elif k == "FFV1_0":
            Fo, V, Fi = a
            vals.append(Fo @ slash(V) @ Fi)
        elif k == "VVV1_0":
            A, B, Q = a
            PA, PB = lines[op.mom[0]][0], lines[op.mom[1]][0]
            k1, k2, k3 = -PA, -PB, PA + PB
            vals.append(dot(A, B) * dot(k1 - k2, Q) + dot(B, Q) * dot(k2 - k3, A) + dot(Q, A) * dot(k3 - k1, B))
        elif k.startswith("VVVV") and k.endswith("_0"):
            A, B, C, Q = a
            vals.append(dot(_v4(k[:5], A, B, C), Q))
        else:
            v = _amputated(k, a, lines, op.mom)
            if v is None:
                raise ValueError(k)
            vals.append(v)
    J = np.zeros(plan.ncol, dtype=complex)
    for ai, terms in plan.amps:
        for col, c in terms:
            J[col] += complex(c[0], c[1]) * vals[ai]
    return J


def _v4(name, A, B, C):
    if name == "VVVV1":
        return dot(A, C) * B - dot(B, C) * A
    if name == "VVVV3":
        return dot(A, B) * C - dot(B, C) * A
    return dot(A, B) * C - dot(A, C) * B


def evaluate_staged(orc, I, p, h, mt, merge=False):
    """Run a staged interpreter schedule (gen/interp.py) in numpy: a slot table
    shared by all helicity variants, filled stage by stage, with slots reused
    after their last reader -- the layout the CUDA kernel executes.  merge:
    colour groups whose members lie in one stage and share a contraction
    operand are contracted once with the signed sum of the other operands, as
    the straight-line table kernel does."""
    from paper_2507_21039_gb300.gen.emit import _group_positions, _shared_operand

    T = I.tab
    P = T.plan
    npar = P.npar
    lam = [1 if (h >> (npar - 1 - i)) & 1 else -1 for i in range(npar)]
    incoming = [i < 2 for i in range(npar)]
    out_p = np.array([(-p[i] if incoming[i] else p[i]) for i in range(npar)])
    lines = []
    for ln in P.lines:
        if ln.kind == "g":
            q = sum(out_p[P.gluon_ext[g]] for g in ln.gluons)
            lines.append((q, 1.0 / dot(q, q) if len(ln.gluons) > 1 else 0.0))
        else:
            q = p[2] + sum((out_p[P.gluon_ext[g]] for g in ln.gluons), np.zeros(4))
            lines.append((q, 1.0 / (dot(q, q) - mt * mt)))
    table = {}
    for e in range(npar):
        for b, l in ((0, -1), (1, 1)):
            if e in (0, 1):
                table[2 * e + b] = orc.polvec(p[e], l)
            elif e == 2:
                table[2 * e + b] = orc.bar(orc.spinor_u(p[e], mt, l))
            elif e == 3:
                table[2 * e + b] = orc.spinor_v(p[e], mt, l)
            else:
                table[2 * e + b] = np.conj(orc.polvec(p[e], l))
    bits = {q: (1 if lam[q] > 0 else 0) for q in range(npar)}

    def var(S):
        return sum(bits[q] << j for j, q in enumerate(S))

    J = np.zeros(P.ncol, dtype=complex)
    gsum = 0.0
    ops = P.ops
    pos = dict(zip(I.amp_order, _group_positions(I.amp_order, I.flush)))
    for st in I.stages:
        for kind, tasks in st.rounds:
            for out, ins, ln in tasks:
                a = [table[i] for i in ins]
                if kind == "VVV1P0_1":
                    PA, PB = lines[ln[0]][0], lines[ln[1]][0]
                    k1, k2, k3 = -PA, -PB, PA + PB
                    v = dot(a[0], a[1]) * (k1 - k2) + a[1] * dot(k2 - k3, a[0]) + a[0] * dot(k3 - k1, a[1])
                    table[out] = lines[ln[2]][1] * v
                elif kind in AMPUTATED_VERTICES:
                    table[out] = _amputated(kind, a, lines, (ln[0], ln[1]))
                elif kind.startswith("VVVV"):
                    table[out] = lines[ln[2]][1] * _v4(kind[:5], a[0], a[1], a[2])
                elif kind == "FFV1_2":
                    q, inv = lines[ln[2]]
                    table[out] = inv * (a[0] @ slash(a[1]) @ (slash(q) + mt * np.eye(4)))
                elif kind == "FFV1_1":
                    q, inv = lines[ln[2]]
                    table[out] = inv * ((slash(q) + mt * np.eye(4)) @ slash(a[0]) @ a[1])
                else:
                    inv = lines[ln[2]][1]
                    table[out] = inv * np.array([a[0] @ G[mu] @ a[1] for mu in range(4)])
        def value(x):
            base = I.slot[x] if (ops[x].out != "A" and not ops[x].kind.startswith("ext_")) else 2 * ops[x].ext
            return table[base + var(T.support[x])]

        amps, k = st.amps, 0
        while k < len(amps):
            ai = amps[k]
            first, last = pos[ai]
            run = [ai]
            if first and not last:
                for b in amps[k + 1:]:
                    if pos[b][0]:
                        break
                    run.append(b)
                    if pos[b][1]:
                        break
            mg = _shared_operand(P, run) if (merge and first and run[-1] in I.flush and len(run) > 1) else None
            if mg:
                kind, y, others = mg
                S = sum(I.sign[a] * value(x) for a, x in zip(run, others))
                gsum = _amputated(kind, [S, value(y)], lines, ())
                for col, c in I.flush[run[-1]]:
                    J[col] += complex(c[0], c[1]) * gsum
                gsum = 0.0
                k += len(run)
                continue
            k += 1
            aop, terms = P.amps[ai]
            op = ops[aop]
            w = [value(x) for x in op.args]
            if op.kind in ("DOTV", "DOTF"):
                x = _amputated(op.kind, w, lines, op.mom)
            elif op.kind == "FFV1_0":
                x = w[0] @ slash(w[1]) @ w[2]
            elif op.kind == "VVV1_0":
                PA, PB = lines[op.mom[0]][0], lines[op.mom[1]][0]
                k1, k2, k3 = -PA, -PB, PA + PB
                x = dot(w[0], w[1]) * dot(k1 - k2, w[2]) + dot(w[1], w[2]) * dot(k2 - k3, w[0]) + \
                    dot(w[2], w[0]) * dot(k3 - k1, w[1])
            else:
                x = dot(_v4(op.kind[:5], w[0], w[1], w[2]), w[3])
            # colour group: signed sum of its amplitudes, added into J with the
            # group's terms by its last member
            gsum += I.sign[ai] * x
            if ai in I.flush:
                for col, c in I.flush[ai]:
                    J[col] += complex(c[0], c[1]) * gsum
                gsum = 0.0
    assert gsum == 0.0
    return J


# Drell-Yan electroweak parameters (the same values the oracle states)
_DY_ALPHA, _DY_MZ, _DY_MW = 1.0 / 132.507, 91.188, 80.419002


def _dy_quark_couplings():
    """(gL, gR) of the u quark to the photon and to the Z"""
    e = np.sqrt(4 * np.pi * _DY_ALPHA)
    cw = _DY_MW / _DY_MZ
    sw = np.sqrt(1 - cw * cw)
    q, t3 = 2 / 3, 0.5
    return (e * q, e * q), (e * (t3 - q * sw * sw) / (sw * cw), -e * q * sw * sw / (sw * cw))


def evaluate_dy(orc, plan, p, h):
    """Colour-flow amplitudes J (gluon couplings stripped) of a Drell-Yan plan
    (gen/plan.py build_plan_dy) for event p, helicity h.  The lepton currents
    over their propagators come from the pinned oracle; the quark-side chiral
    couplings are applied here."""
    npar = plan.npar
    lam = [1 if (h >> (npar - 1 - i)) & 1 else -1 for i in range(npar)]
    qL = p[2] + p[3]
    lines = []
    for ln in plan.lines:
        if ln.kind == "g":
            q = sum(p[plan.gluon_ext[g]] for g in ln.gluons)
            lines.append((q, 1.0 / dot(q, q) if len(ln.gluons) > 1 else 0.0))
        else:
            q = -p[1] + sum((p[plan.gluon_ext[g]] for g in ln.gluons), np.zeros(4)) + (qL if ln.kind == "qe" else 0)
            lines.append((q, 1.0 / dot(q, q)))
    Lv = orc.dy_lepton_currents(p[2], p[3], lam[2], lam[3])
    cq = _dy_quark_couplings()
    LL = cq[0][0] * Lv[0] + cq[1][0] * Lv[1]
    LR = cq[0][1] * Lv[0] + cq[1][1] * Lv[1]
    PL, PR = np.diag([1.0, 1.0, 0.0, 0.0]), np.diag([0.0, 0.0, 1.0, 1.0])

    def mlr(a, b):  # the chiral vertex slash(L_L) P_L + slash(L_R) P_R
        return slash(a) @ PL + slash(b) @ PR

    vals = []
    for op in plan.ops:
        a = [vals[i] for i in op.args]
        k = op.kind
        if k == "ext_v":
            vals.append(np.conj(orc.polvec(p[op.ext], lam[op.ext])))
        elif k == "ext_fo":
            vals.append(orc.bar(orc.spinor_v(p[1], 0.0, lam[1])))
        elif k == "ext_fi":
            vals.append(orc.spinor_u(p[0], 0.0, lam[0]))
        elif k == "ext_lepL":
            vals.append(LL)
        elif k == "ext_lepR":
            vals.append(LR)
        elif k == "VVV1P0_1":
            A, B = a
            PA, PB = lines[op.mom[0]][0], lines[op.mom[1]][0]
            k1, k2, k3 = -PA, -PB, PA + PB
            v = dot(A, B) * (k1 - k2) + B * dot(k2 - k3, A) + A * dot(k3 - k1, B)
            vals.append(lines[op.line][1] * v)
        elif k.startswith("VVVV") and k.endswith("P0_1"):
            vals.append(lines[op.line][1] * _v4(k[:5], *a))
        elif k == "FFV1_2":
            q, inv = lines[op.line]
            vals.append(inv * (a[0] @ slash(a[1]) @ slash(q)))
        elif k == "FFV1_1":
            q, inv = lines[op.line]
            vals.append(inv * (slash(q) @ slash(a[0]) @ a[1]))
        elif k == "FFVLR_2":
            q, inv = lines[op.line]
            vals.append(inv * (a[0] @ mlr(a[1], a[2]) @ slash(q)))
        elif k == "FFVLR_1":
            q, inv = lines[op.line]
            vals.append(inv * (slash(q) @ mlr(a[0], a[1]) @ a[2]))
        elif k == "FFV1_0":
            vals.append(a[0] @ slash(a[1]) @ a[2])
        elif k == "FFVLR_0":
            vals.append(a[0] @ mlr(a[1], a[2]) @ a[3])
        else:
            raise ValueError(k)
    J = np.zeros(plan.ncol, dtype=complex)
    for ai, terms in plan.amps:
        for col, c in terms:
            J[col] += complex(c[0], c[1]) * vals[ai]
    return J
