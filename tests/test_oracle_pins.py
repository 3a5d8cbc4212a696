"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a library
routine (numpy's Philox), closed forms (e+e- -> mu+mu-, gg -> t tbar), textbook
identities (Dirac equation, completeness, SU(3) algebra, Fierz), an independent
brute force (explicit-colour Feynman rules), symmetries (gauge, Lorentz, Bose),
the Parke-Taylor formula for MHV amplitudes, and exact phase-space volumes.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2507_21039_gb300.workloads import ALPHA_EM, ALPHA_S, MT, WORKLOADS

MINK = np.diag([1.0, -1.0, -1.0, -1.0])


def mdot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


def gammas():
    s = [np.eye(2), np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
    out = []
    for mu in range(4):
        g = np.zeros((4, 4), dtype=complex)
        g[:2, 2:] = s[mu]
        g[2:, :2] = s[mu] if mu == 0 else -s[mu]
        out.append(g)
    return out


G = gammas()


def slash(p):
    return G[0] * p[0] - G[1] * p[1] - G[2] * p[2] - G[3] * p[3]


def events(orc, name, n, ev0=0):
    w = WORKLOADS[name]
    mom, wt, att = orc.rambo(w.seed, w.sqrt_s, w.masses_final, ev0, n, w.cut_mask, 20.0, 0.4)
    return mom


def back_to_back(mom, m):
    """Exactly back-to-back 2 -> 2 momenta along the RAMBO directions.  RAMBO's
    conformal boost loses digits when the generated directions are nearly
    collinear (large boost), which leaves the mass shell and momentum balance
    off by up to ~1e-11 relative; the closed forms need consistent inputs."""
    out = mom.copy()
    E = mom[:, 0, 0]
    P = np.sqrt(E * E - m * m)
    n = mom[:, 2, 1:] / np.linalg.norm(mom[:, 2, 1:], axis=1)[:, None]
    out[:, 2, 0] = out[:, 3, 0] = E
    out[:, 2, 1:] = P[:, None] * n
    out[:, 3, 1:] = -P[:, None] * n
    return out


# ---------------------------------------------------------------- RNG
def test_philox_matches_numpy(orc):
    # numpy's Philox (4x64-10) increments its counter before each block
    for key in ([0, 0], [5, 0], [2**63 + 12345, 77]):
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.zeros(4, dtype=np.uint64))
        ref = bg.random_raw(12).reshape(3, 4)
        for blk in range(3):
            got = orc.philox4x64_10([blk + 1, 0, 0, 0], key)
            assert np.array_equal(got, ref[blk])
    bg = np.random.Philox(key=np.array([9, 9], dtype=np.uint64),
                          counter=np.array([2**64 - 1, 3, 0, 1], dtype=np.uint64))
    assert np.array_equal(orc.philox4x64_10([0, 4, 0, 1], [9, 9]), bg.random_raw(4))


def test_u01_open_interval(orc):
    assert orc.u01(0) == 0.5 * 2.0**-53
    assert orc.u01(2**64 - 1) == 1.0 - 0.5 * 2.0**-53
    assert orc.u01(1 << 63) == 0.5 + 0.5 * 2.0**-53


# ---------------------------------------------------------------- spinors, polarisations
@pytest.mark.parametrize("m", [0.0, 173.0])
def test_spinors_dirac_equation_and_completeness(orc, m):
    rng = np.random.default_rng(1)
    dirs = [rng.normal(size=3) for _ in range(6)] + [np.array([0, 0, 1.0]), np.array([0, 0, -1.0])]
    for d in dirs:
        pv = d / np.linalg.norm(d) * rng.uniform(10, 500)
        p = np.array([math.sqrt(m * m + pv @ pv), *pv])
        us = {l: orc.spinor_u(p, m, l) for l in (1, -1)}
        vs = {l: orc.spinor_v(p, m, l) for l in (1, -1)}
        ps = slash(p)
        sig = np.zeros((4, 4), dtype=complex)  # helicity operator Sigma.p/|p|
        pauli = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
        h2 = sum(pv[i] * pauli[i] for i in range(3)) / np.linalg.norm(pv)
        sig[:2, :2] = h2
        sig[2:, 2:] = h2
        scale = p[0]
        for l in (1, -1):
            u, v = us[l], vs[l]
            assert np.allclose(ps @ u, m * u, atol=1e-12 * scale * math.sqrt(scale))
            assert np.allclose(ps @ v, -m * v, atol=1e-12 * scale * math.sqrt(scale))
            assert np.allclose(sig @ u, l * u, atol=1e-12 * math.sqrt(scale))
            # v of helicity l describes the antiparticle: Sigma.p v = -l v
            assert np.allclose(sig @ v, -l * v, atol=1e-12 * math.sqrt(scale))
            assert abs(orc.bar(u) @ u - 2 * m) < 1e-10 * scale
            assert abs(orc.bar(v) @ v + 2 * m) < 1e-10 * scale
        su = sum(np.outer(us[l], orc.bar(us[l])) for l in (1, -1))
        sv = sum(np.outer(vs[l], orc.bar(vs[l])) for l in (1, -1))
        assert np.allclose(su, ps + m * np.eye(4), atol=1e-10 * scale)
        assert np.allclose(sv, ps - m * np.eye(4), atol=1e-10 * scale)
        if m == 0.0:  # chirality: u(+) right-handed, u(-) left-handed
            assert np.allclose(us[1][:2], 0) and np.allclose(us[-1][2:], 0)


def test_polarisation_vectors(orc):
    rng = np.random.default_rng(2)
    dirs = [rng.normal(size=3) for _ in range(6)] + [np.array([0, 0, 1.0]), np.array([0, 0, -1.0])]
    for d in dirs:
        kv = d / np.linalg.norm(d) * 100.0
        k = np.array([100.0, *kv])
        ep, em = orc.polvec(k, 1), orc.polvec(k, -1)
        for e in (ep, em):
            assert abs(mdot(e, k)) < 1e-12
            assert abs(mdot(e, np.conj(e)) + 1) < 1e-14
            assert abs(e[0]) == 0
        assert abs(mdot(ep, np.conj(em))) < 1e-14
        # helicity: i (k_hat x e) = lam e for circular polarisation
        kh = kv / 100.0
        for lam, e in ((1, ep), (-1, em)):
            assert np.allclose(1j * np.cross(kh, e[1:]), lam * e[1:], atol=1e-14)
        # completeness with gauge vector n = (1, -k_hat): sum eps eps* = -g + (k n + n k)/(k.n)
        n = np.array([1.0, *(-kh)])
        S = sum(np.outer(e, np.conj(e)) for e in (ep, em))
        gup = np.diag([1.0, -1, -1, -1])
        R = -gup + (np.outer(k, n) + np.outer(n, k)) / mdot(k, n)
        assert np.allclose(S, R, atol=1e-12)


# ---------------------------------------------------------------- SU(3)
def test_su3_algebra(orc):
    T, f = orc.su3()
    for a in range(8):
        assert np.allclose(T[a], T[a].conj().T)
        assert abs(np.trace(T[a])) < 1e-15
        for b in range(8):
            assert abs(np.trace(T[a] @ T[b]) - 0.5 * (a == b)) < 1e-15
            comm = T[a] @ T[b] - T[b] @ T[a]
            assert np.allclose(comm, 1j * np.einsum("c,cij->ij", f[a, b], T), atol=1e-15)
    assert abs(f[0, 1, 2] - 1.0) < 1e-15 and abs(f[3, 4, 7] - math.sqrt(3) / 2) < 1e-15
    assert np.allclose(f, -np.transpose(f, (1, 0, 2))) and np.allclose(f, np.transpose(f, (1, 2, 0)))
    # Casimirs: f^{acd} f^{bcd} = N delta^{ab};  T^a T^a = C_F = 4/3
    assert np.allclose(np.einsum("acd,bcd->ab", f, f), 3 * np.eye(8))
    assert np.allclose(np.einsum("aij,ajk->ik", T, T), 4 / 3 * np.eye(3))


def _fierz_colour_matrix(k):
    """Exact C_{s,s'} = sum_a Tr(T^{s_k}..T^{s_1} T^{s'_1}..T^{s'_k}) via the Fierz
    reduction Tr(X T^a Y T^a) = 1/2 [Tr X Tr Y - Tr(XY)/N], Tr(1) = N = 3."""
    N = Fraction(3)

    def tr_product(words):
        # words: tuple of traces (tuples of labels); every label appears twice overall
        words = tuple(w for w in words)
        for wi, w in enumerate(words):
            seen = {}
            for pos, lab in enumerate(w):
                if lab in seen:  # both copies in the same trace
                    i, j = seen[lab], pos
                    # Tr(A T B T C) = Tr((C A) T B T): X = C A, Y = B
                    X, Y = w[j + 1:] + w[:i], w[i + 1:j]
                    rest = words[:wi] + words[wi + 1:]
                    return Fraction(1, 2) * (tr_product(rest + (X, Y)) - tr_product(rest + (X + Y,)) / N)
                seen[lab] = pos
        # labels shared between two different traces: merge via Tr(X T^a) Tr(Y T^a) = 1/2[Tr(XY) - Tr X Tr Y / N]
        for wi, w in enumerate(words):
            for pos, lab in enumerate(w):
                for wj in range(wi + 1, len(words)):
                    if lab in words[wj]:
                        v = words[wj]
                        q = v.index(lab)
                        X = w[pos + 1:] + w[:pos]       # Tr(T^a X) cyclic
                        Y = v[q + 1:] + v[:q]
                        rest = tuple(words[t] for t in range(len(words)) if t not in (wi, wj))
                        return Fraction(1, 2) * (tr_product(rest + (X + Y,)) - tr_product(rest + (X, Y)) / N)
        out = Fraction(1)
        for w in words:
            assert len(w) == 0
            out *= N
        return out

    perms = list(itertools.permutations(range(k)))
    C = np.zeros((len(perms), len(perms)), dtype=object)
    for i, s in enumerate(perms):
        for j, t in enumerate(perms):
            C[i, j] = tr_product((tuple(reversed(s)) + tuple(t),))
    return C


@pytest.mark.parametrize("k", [2, 3, 4])
def test_colour_matrix_brute_force(orc, k):
    C = orc.colour_matrix(k)
    n = math.factorial(k)
    assert C.shape == (n, n)
    assert np.allclose(C, C.T, atol=1e-12)
    assert np.allclose(np.diag(C), 3 * (4 / 3) ** k, rtol=1e-13)
    assert np.linalg.eigvalsh(C).min() > -1e-10
    if k == 2:
        assert np.allclose(C, np.array([[16, -2], [-2, 16]]) / 3, atol=1e-13)
    # relabelling invariance: C[s, t] depends on s^-1 t only
    P = orc.perms(k)
    idx = {tuple(p): i for i, p in enumerate(P)}
    for s in range(n):
        inv = np.argsort(P[s])
        for t in range(n):
            rel = tuple(inv[P[t]])
            assert abs(C[s, t] - C[0, idx[rel]]) < 1e-12
    # exact rationals from the independent Fierz reduction, same permutation order
    F = _fierz_colour_matrix(k)
    perms_py = list(itertools.permutations(range(k)))
    assert [tuple(p) for p in P] == perms_py
    Ff = np.array([[float(x) for x in row] for row in F])
    assert np.allclose(C, Ff, atol=1e-12, rtol=0)


@pytest.mark.slow
def test_colour_matrix_k5(orc):
    C = orc.colour_matrix(5)
    assert np.allclose(np.diag(C), 3 * (4 / 3) ** 5, rtol=1e-13)
    assert np.allclose(C, C.T, atol=1e-12)
    F = _fierz_colour_matrix(5)
    assert np.allclose(C, np.array([[float(x) for x in r] for r in F]), atol=1e-11, rtol=0)


# ---------------------------------------------------------------- RAMBO
def test_rambo_kinematics_and_determinism(orc):
    for name in ("ee_mumu", "gg_ttx", "gg_ttxg", "gg_ttxgg", "gg_ttxggg"):
        w = WORKLOADS[name]
        mom = events(orc, name, 256)
        P = mom[:, :2].sum(1) - mom[:, 2:].sum(1)
        assert np.abs(P).max() < 1e-9 * w.sqrt_s
        for j, m in enumerate(w.masses_final):
            p = mom[:, 2 + j]
            m2 = p[:, 0] ** 2 - (p[:, 1:] ** 2).sum(1)
            assert np.allclose(m2, m * m, atol=1e-8 * w.sqrt_s**2)
        assert np.allclose(mom[:, 0], [w.sqrt_s / 2, 0, 0, w.sqrt_s / 2])
        assert np.allclose(mom[:, 1], [w.sqrt_s / 2, 0, 0, -w.sqrt_s / 2])
        # counter-based: event i alone equals event i in a batch
        again = events(orc, name, 5, ev0=100)
        assert np.array_equal(again, mom[100:105])
        # cuts hold
        gl = [2 + j for j, c in enumerate(w.cut_mask) if c]
        for g in gl:
            assert (np.hypot(mom[:, g, 1], mom[:, g, 2]) > 20.0).all()
        for a, b in itertools.combinations(gl, 2):
            def eta(p):
                P = np.linalg.norm(p[:, 1:], axis=1)
                return 0.5 * np.log((P + p[:, 3]) / (P - p[:, 3]))
            dphi = np.angle(np.exp(1j * (np.arctan2(mom[:, a, 2], mom[:, a, 1]) -
                                         np.arctan2(mom[:, b, 2], mom[:, b, 1]))))
            assert (np.hypot(eta(mom[:, a]) - eta(mom[:, b]), dphi) > 0.4).all()


def test_rambo_weights_exact_volumes(orc):
    from scipy import integrate

    # two-body: flat, volume beta / (8 pi)
    s = 1000.0**2
    _, wt, _ = orc.rambo(7, 1000.0, [173.0, 173.0], 0, 64)
    assert np.allclose(wt, math.sqrt(1 - 4 * 173.0**2 / s) / (8 * math.pi), rtol=1e-13)
    _, wt, _ = orc.rambo(7, 100.0, [0.0, 0.0], 0, 8)
    assert np.allclose(wt, 1 / (8 * math.pi), rtol=1e-14)
    # three-body massless: s / (256 pi^3)
    _, wt, _ = orc.rambo(7, 1500.0, [0.0, 0.0, 0.0], 0, 8)
    assert np.allclose(wt, 1500.0**2 / (256 * math.pi**3), rtol=1e-13)
    # three-body (m, m, 0): Monte-Carlo mean of the weights vs Dalitz-plot volume
    rs, m = 1500.0, 173.0
    s = rs * rs
    _, wt, _ = orc.rambo(8, rs, [m, m, 0.0], 0, 200000)

    def m23_range(m12sq):
        m1, m2, m3 = m, m, 0.0
        m12 = math.sqrt(m12sq)
        E2 = (m12sq - m1 * m1 + m2 * m2) / (2 * m12)
        E3 = (s - m12sq - m3 * m3) / (2 * m12)
        p2 = math.sqrt(max(E2 * E2 - m2 * m2, 0))
        p3 = math.sqrt(max(E3 * E3 - m3 * m3, 0))
        return (E2 + E3) ** 2 - (p2 + p3) ** 2, (E2 + E3) ** 2 - (p2 - p3) ** 2

    area, _ = integrate.quad(lambda x: m23_range(x)[1] - m23_range(x)[0], (2 * m) ** 2, s, epsabs=0, epsrel=1e-10)
    vol = (2 * math.pi) ** -5 * math.pi**2 / (4 * s) * area
    err = wt.std() / math.sqrt(wt.size)
    assert abs(wt.mean() - vol) < 5 * err


# ---------------------------------------------------------------- closed forms
def test_ee_mumu_closed_form(orc):
    mom = back_to_back(events(orc, "ee_mumu", 16384), 0.0)
    me, hel = orc.me2("ee_mumu", mom, per_helicity=True)
    cf = np.array([orc.closed_ee(p) for p in mom])
    assert np.max(np.abs(me / cf - 1)) < 1e-13
    # exactly 4 of the 16 helicities contribute
    nz = (hel.max(0) / me.max() > 1e-14)
    assert nz.sum() == 4
    # weighted cos(theta) histogram follows 1 + cos^2(theta) (RAMBO is flat in cos theta)
    c = mom[:, 2, 3] / np.linalg.norm(mom[:, 2, 1:], axis=1)
    assert abs(orc.closed_ee(np.array([[50, 0, 0, 50], [50, 0, 0, -50], [50, 50, 0, 0], [50, -50, 0, 0]])) -
               (4 * math.pi * ALPHA_EM) ** 2) < 1e-16
    h, edges = np.histogram(c, bins=20, range=(-1, 1), weights=me)
    cnt, _ = np.histogram(c, bins=20, range=(-1, 1))
    mid = 0.5 * (edges[1:] + edges[:-1])
    expect = cnt * (4 * math.pi * ALPHA_EM) ** 2 * (1 + mid**2)
    rel = np.abs(h / expect - 1)
    assert rel.max() < 0.01  # bin-centre approximation of a smooth shape


def test_gg_ttx_closed_form(orc):
    mom = back_to_back(events(orc, "gg_ttx", 4096), MT)
    me = orc.me2("gg_ttx", mom)
    cf = np.array([orc.closed_ggtt(p) for p in mom])
    assert np.max(np.abs(me / cf - 1)) < 1e-13
    # worked value at sqrt(s) = 1 TeV, theta = 90 deg, m_t = 173 GeV
    E = 500.0
    pz = math.sqrt(E * E - MT * MT)
    p = np.array([[E, 0, 0, E], [E, 0, 0, -E], [E, pz, 0, 0], [E, -pz, 0, 0]])
    g4 = (4 * math.pi * ALPHA_S) ** 2
    rho = 4 * MT**2 / 1e6
    expect = g4 * (1 / (6 * 0.25) - 3 / 8) * (0.5 + rho - rho**2)
    assert abs(orc.me2("gg_ttx", p[None])[0] / expect - 1) < 1e-13
    assert abs(expect - 0.38824) < 5e-5
    # massless limit: (t^2+u^2)/(6tu) - 3(t^2+u^2)/(8 s^2), times g^4
    mom0 = back_to_back(orc.rambo(11, 1000.0, [0.0, 0.0], 0, 64)[0], 0.0)
    me0 = orc.me2("gg_ttx", mom0, mt=0.0)
    for p, v in zip(mom0, me0):
        s = 2 * mdot(p[0], p[1])
        t = -2 * mdot(p[0], p[2])
        u = -2 * mdot(p[0], p[3])
        ref = g4 * ((t * t + u * u) / (6 * t * u) - 3 * (t * t + u * u) / (8 * s * s))
        assert abs(v / ref - 1) < 1e-12


# ---------------------------------------------------------------- colour decomposition
@pytest.mark.parametrize("name", ["gg_ttx", "gg_ttxg"])
def test_colour_dressed_brute_force_all_helicities(orc, name):
    mom = events(orc, name, 1)
    me, hel = orc.me2(name, mom, per_helicity=True)
    nh = hel.shape[1]
    d = orc.me2_dressed(name, mom[0], list(range(nh)))
    scale = hel[0].max()
    assert np.max(np.abs(d - hel[0])) < 1e-13 * scale


def test_colour_dressed_brute_force_ttgg_some_helicities(orc):
    mom = events(orc, "gg_ttxgg", 1)
    me, hel = orc.me2("gg_ttxgg", mom, per_helicity=True)
    hs = [0b010110, 0b101001, 0b111100]
    d = orc.me2_dressed("gg_ttxgg", mom[0], hs)
    assert np.max(np.abs(d / hel[0][hs] - 1)) < 1e-12


# ---------------------------------------------------------------- symmetries
@pytest.mark.parametrize("name", ["gg_ttx", "gg_ttxg", "gg_ttxgg", "gg_ttxggg"])
def test_gauge_invariance_every_gluon(orc, name):
    mom = events(orc, name, 2)
    npar, k = orc.npar(name), orc.ngluon(name)
    rng = np.random.default_rng(3)
    for p in mom:
        scale = max(np.abs(orc.partial_amps(name, p, h)).max() for h in range(0, 1 << npar, 3))
        for h in rng.integers(0, 1 << npar, size=3):
            for g in range(k):
                Ag = orc.partial_amps(name, p, int(h), gauge_gluon=g)
                assert np.abs(Ag).max() < 1e-10 * scale


def _boost_rotate(mom, rng):
    bvec = rng.normal(size=3)
    bvec *= rng.uniform(0.1, 0.8) / np.linalg.norm(bvec)
    b2 = bvec @ bvec
    g = 1 / math.sqrt(1 - b2)
    L = np.eye(4)
    L[0, 0] = g
    L[0, 1:] = L[1:, 0] = g * bvec
    L[1:, 1:] += (g - 1) * np.outer(bvec, bvec) / b2
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    R = np.eye(4)
    R[1:, 1:] = q
    return mom @ (L @ R).T


@pytest.mark.parametrize("name", ["ee_mumu", "gg_ttx", "gg_ttxg", "gg_ttxgg", "gg_ttxggg"])
def test_lorentz_invariance(orc, name):
    rng = np.random.default_rng(4)
    mom = events(orc, name, 3)
    me = orc.me2(name, mom)
    moved = np.stack([_boost_rotate(p, rng) for p in mom])
    me2 = orc.me2(name, moved)
    assert np.max(np.abs(me2 / me - 1)) < 1e-12


@pytest.mark.parametrize("name", ["gg_ttxg", "gg_ttxgg", "gg_ttxggg"])
def test_bose_symmetry(orc, name):
    mom = events(orc, name, 3)
    me = orc.me2(name, mom)
    npar = orc.npar(name)
    fin_g = list(range(4, npar))
    for perm in list(itertools.permutations(fin_g))[1:3]:
        q = mom.copy()
        q[:, fin_g] = mom[:, list(perm)]
        assert np.max(np.abs(orc.me2(name, q) / me - 1)) < 1e-13
    # swap the two incoming gluons (also flips the z axis: use a rotation by pi about x)
    q = mom[:, [1, 0] + list(range(2, npar))].copy()
    q[:, :, 2] *= -1
    q[:, :, 3] *= -1
    assert np.max(np.abs(orc.me2(name, q) / me - 1)) < 1e-12


# ---------------------------------------------------------------- Parke-Taylor
@pytest.mark.parametrize("name", ["gg_ttx", "gg_ttxg", "gg_ttxgg", "gg_ttxggg"])
def test_parke_taylor_mhv(orc, name):
    """Massless quarks: |A_sigma|^2 = 2^k |<f- j>|^6 |<f+ j>|^2 / prod_cyclic |<ab>|^2
    for one negative-helicity gluon j (all-outgoing helicities) and the conjugate
    form for one positive gluon; helicity-violating and one-minus amplitudes vanish.
    The factor 2^k comes from Tr(T^a T^b) = delta/2 versus the unit-normalised
    generators of the textbook formula."""
    npar, k = orc.npar(name), orc.ngluon(name)
    fin = [0.0] * (npar - 2)
    cand, _, _ = orc.rambo(21, 1000.0, fin, 0, 64)

    def separated(p):  # keep points with every |s_ij| > 1e-3 s (no near-collinear pair)
        q = p.copy()
        q[:2] *= -1
        return min(abs(2 * mdot(q[a], q[b])) for a in range(npar) for b in range(a)) > 1e-3 * 1e6

    mom = [p for p in cand if separated(p)][:2]
    P = orc.perms(k)
    gl_ext = [0, 1] + list(range(4, npar))
    ratios = []
    for p in mom:
        out_p = p.copy()
        out_p[:2] *= -1  # all-outgoing momenta
        s = lambda a, b: abs(2 * mdot(out_p[a], out_p[b]))
        for h in range(1 << npar):
            lam = [1 if (h >> (npar - 1 - i)) & 1 else -1 for i in range(npar)]
            lo = [-l if i < 2 else l for i, l in enumerate(lam)]  # all-outgoing helicities
            A = orc.partial_amps(name, p, h, mt=0.0)
            scale = 1e-3 * np.abs(orc.partial_amps(name, p, 0b1001 << (npar - 4), mt=0.0)).max()
            ft, ftb = lo[2], lo[3]
            gneg = [g for g in gl_ext if lo[g] < 0]
            gpos = [g for g in gl_ext if lo[g] > 0]
            if ft == ftb:
                assert np.abs(A).max() < 1e-12 * max(scale, 1e-300) * 1e3
                continue
            fm, fp = (2, 3) if ft < 0 else (3, 2)
            if len(gneg) == 1:
                j, num = gneg[0], None
            elif len(gpos) == 1:
                j = gpos[0]
                fm, fp = fp, fm  # conjugate formula: positive fermion plays the role of f-
            elif len(gneg) == 0 or len(gpos) == 0:
                assert np.abs(A).max() < 1e-12 * max(scale, 1e-300) * 1e3
                continue
            else:
                continue  # NMHV and beyond: no closed form here
            for si in range(P.shape[0]):
                order = [2] + [gl_ext[g] for g in P[si]] + [3]
                den = 1.0
                for a, b in zip(order, order[1:] + order[:1]):
                    den *= s(a, b)
                pt2 = s(fm, j) ** 3 * s(fp, j) / den
                ratios.append(abs(A[si]) ** 2 / pt2)
    ratios = np.array(ratios)
    assert ratios.size > 0
    assert np.allclose(ratios, 2.0**k, rtol=1e-10)


# ---------------------------------------------------------------- diagrams one by one
@pytest.mark.parametrize("name,count", [("gg_ttx", 3), ("gg_ttxg", 16), ("gg_ttxgg", 123), ("gg_ttxggg", 1240)])
def test_sde_diagram_counts(orc, name, count):
    """The paper's diagram counts for g g -> t t~ + 0..3 g (a four-gluon vertex
    counted once); every diagram is a distinct tree (distinct set of splits)
    with at most npar - 3 internal lines, none containing the t~."""
    p = events(orc, name, 1)[0]
    w2, lines = orc.sde(name, p, [0], MT)
    assert len(w2) == count and len(set(lines)) == count
    npar = WORKLOADS[name].npar
    for key in lines:
        assert 1 <= len(key) <= npar - 3
        assert all(0 < m < (1 << npar) and not (m >> 3) & 1 for m in key)
        assert list(key) == sorted(key)


def test_sde_ee_single_diagram_is_the_matrix_element(orc):
    """e+ e- -> mu+ mu-: one diagram, so its helicity-summed |amp|^2 times the
    couplings and the spin average is |M|^2 (pinned to the closed form)."""
    mom = back_to_back(events(orc, "ee_mumu", 64), 0.0)
    me = orc.me2("ee_mumu", mom)
    for p, v in zip(mom, me):
        w2, lines = orc.sde("ee_mumu", p, list(range(16)), 0.0)
        assert lines == [(0b11,)]
        assert abs((4 * math.pi * ALPHA_EM) ** 2 * w2[0] / 4 / v - 1) < 1e-13


def test_sde_gg_ttx_diagrams_by_traces(orc):
    """g g -> t t~: each diagram's helicity sum recomputed with the trace
    technique (top and antitop spins summed as Tr[(pt + m) G (ptb - m) Gbar],
    no spinors), gluon polarisations summed explicitly."""
    eye = np.eye(4)
    for p in events(orc, "gg_ttx", 8):
        w2, lines = orc.sde("gg_ttx", p, list(range(16)), MT)
        by = dict(zip(lines, w2))
        assert set(by) == {(0b011,), (0b101,), (0b110,)}
        pt, ptb = p[2], p[3]
        Pt, Pb = slash(pt) + MT * eye, slash(ptb) - MT * eye

        def spin_sum(gam):
            gbar = G[0] @ gam.conj().T @ G[0]
            return np.trace(Pt @ gam @ Pb @ gbar).real

        ref = {(0b011,): 0.0, (0b101,): 0.0, (0b110,): 0.0}
        for l0 in (-1, 1):
            for l1 in (-1, 1):
                e0, e1 = orc.polvec(p[0], l0), orc.polvec(p[1], l1)   # incoming gluons: eps
                for first, second, pin, key in ((e0, e1, p[0], (0b101,)), (e1, e0, p[1], (0b110,))):
                    q = pt - pin                                      # t side: t + outgoing(-p_in)
                    gam = slash(first) @ (slash(q) + MT * eye) @ slash(second) / (mdot(q, q) - MT * MT)
                    ref[key] += spin_sum(gam)
                k0, k1 = p[0], p[1]                                   # momenta into the three-gluon vertex
                k3 = -k0 - k1
                J = (np.dot(MINK @ e0, e1) * (k0 - k1) + e1 * np.dot(MINK @ (k1 - k3), e0)
                     + e0 * np.dot(MINK @ (k3 - k0), e1)) / mdot(k0 + k1, k0 + k1)
                ref[(0b011,)] += spin_sum(slash(J))
        for key in ref:
            assert abs(by[key] / ref[key] - 1) < 1e-12, (key, by[key], ref[key])


# ---------------------------------------------------------------- diagrams one by one, any gluon count
def _dirac_rep_gammas():
    """Dirac representation (gamma^0 = diag(1, 1, -1, -1)): traces do not depend
    on the representation, so this pin shares no spinor or matrix convention
    with the oracle (which works in the chiral representation)."""
    pauli = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
    g0 = np.zeros((4, 4), dtype=complex)
    g0[:2, :2], g0[2:, 2:] = np.eye(2), -np.eye(2)
    out = [g0]
    for s in pauli:
        g = np.zeros((4, 4), dtype=complex)
        g[:2, 2:], g[2:, :2] = s, -s
        out.append(g)
    return out


def _linear_polarisations(k3):
    """Two real unit vectors (0, e) transverse to the spatial momentum k3 (Gram-
    Schmidt from fixed reference directions): sum over them of e^mu e^nu is the
    same transverse projector as the sum over the two helicity vectors."""
    n = k3 / np.linalg.norm(k3)
    ref = np.array([0.3, 0.2, 1.0]) if abs(n[2]) < 0.9 else np.array([1.0, 0.4, 0.1])
    e1 = ref - np.dot(ref, n) * n
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    return [np.concatenate(([0.0], e1)), np.concatenate(([0.0], e2))]


def _trees(leaves):
    """Every tree of three- and four-gluon vertices whose external gluons are
    `leaves` (a sorted tuple of external indices): ('leaf', e), ('v3', a, b) or
    ('v4', a, b, c), each split counted once."""
    if len(leaves) == 1:
        return [("leaf", leaves[0])]
    out = []
    first, rest = leaves[0], leaves[1:]
    for r in range(len(rest)):               # {first} + some of the rest | the others
        for extra in itertools.combinations(rest, r):
            a = (first,) + extra
            b = tuple(x for x in rest if x not in extra)
            out += [("v3", ta, tb) for ta in _trees(a) for tb in _trees(b)]
    for r in range(len(rest)):               # three parts, each split counted once
        for extra in itertools.combinations(rest, r):
            a = (first,) + extra
            others = tuple(x for x in rest if x not in extra)
            if len(others) < 2:
                continue
            second, rest2 = others[0], others[1:]
            for r2 in range(len(rest2)):
                for extra2 in itertools.combinations(rest2, r2):
                    b = (second,) + extra2
                    c = tuple(x for x in rest2 if x not in extra2)
                    out += [("v4", ta, tb, tc) for ta in _trees(a) for tb in _trees(b) for tc in _trees(c)]
    return out


def _ordered_partitions(items):
    """Ordered lists of non-empty blocks covering `items` (the trees met along the
    quark line, from the top end)."""
    if not items:
        yield []
        return
    for r in range(1, len(items) + 1):
        for block in itertools.combinations(items, r):
            rest = tuple(x for x in items if x not in block)
            for tail in _ordered_partitions(rest):
                yield [block] + tail


def _leaves_mask(t):
    return 1 << t[1] if t[0] == "leaf" else sum(_leaves_mask(c) for c in t[1:])


def _internal_masks(t):
    return [] if t[0] == "leaf" else [_leaves_mask(t)] + [m for c in t[1:] for m in _internal_masks(c)]


# Feynman-rule tensors with upper indices, contracted with lowered vectors
_V4_STRUCTURES = [np.einsum("ac,bd->abcd", MINK, MINK) - np.einsum("ad,bc->abcd", MINK, MINK),
                  np.einsum("ab,cd->abcd", MINK, MINK) - np.einsum("ad,bc->abcd", MINK, MINK),
                  np.einsum("ab,cd->abcd", MINK, MINK) - np.einsum("ac,bd->abcd", MINK, MINK)]


def _v3_tensor(k1, k2, k3):
    """g^{mn}(k1-k2)^r + g^{nr}(k2-k3)^m + g^{rm}(k3-k1)^n, momenta incoming."""
    return (np.einsum("mn,r->mnr", MINK, k1 - k2) + np.einsum("nr,m->mnr", MINK, k2 - k3)
            + np.einsum("rm,n->mnr", MINK, k3 - k1))


def _tree_currents(t, pol, mom):
    """(currents, outgoing momentum) of tree t: one current per choice of
    four-gluon structure in it, each with its propagator 1/P^2 and no couplings."""
    if t[0] == "leaf":
        return [pol[t[1]].astype(complex)], mom[t[1]]
    subs = [_tree_currents(c, pol, mom) for c in t[1:]]
    P = sum(s[1] for s in subs)
    inv = 1.0 / mdot(P, P)
    lower = lambda j: MINK @ j
    out = []
    if t[0] == "v3":
        V = _v3_tensor(-subs[0][1], -subs[1][1], P)
        for ja in subs[0][0]:
            for jb in subs[1][0]:
                out.append(inv * np.einsum("mnr,m,n->r", V, lower(ja), lower(jb)))
    else:
        for ja in subs[0][0]:
            for jb in subs[1][0]:
                for jc in subs[2][0]:
                    for X in _V4_STRUCTURES:
                        out.append(inv * np.einsum("abcd,a,b,c->d", X, lower(ja), lower(jb), lower(jc)))
    return out, P


def _diagram_weights_by_traces(p, gluons, mt):
    """Per Feynman diagram of g g -> t t~ + gluons: the sum over every helicity of
    |amp_d|^2 (bare vertices, propagators 1/(q^2 - m^2) and 1/P^2), keyed by the
    diagram's internal lines (masks of external particles on the side away from
    the t~).  Top spins are summed as Tr[(pt + m) G (ptb - m) Gbar], gluon
    polarisations over a real transverse basis; a four-gluon vertex gives three
    amplitudes (its Lorentz structures) whose |amp|^2 add."""
    gam = _dirac_rep_gammas()
    sl = lambda v: gam[0] * v[0] - gam[1] * v[1] - gam[2] * v[2] - gam[3] * v[3]
    eye = np.eye(4)
    pt, ptb = p[2], p[3]
    Pt, Pb = sl(pt) + mt * eye, sl(ptb) - mt * eye
    mom = {g: (-p[g] if g < 2 else p[g]) for g in gluons}   # outgoing momenta
    bases = {g: _linear_polarisations(p[g][1:]) for g in gluons}
    diagrams = []
    for blocks in _ordered_partitions(tuple(gluons)):
        for seq in itertools.product(*[_trees(b) for b in blocks]):
            lines, side = [], 1 << 2
            for i, t in enumerate(seq):
                lines += _internal_masks(t)
                side |= _leaves_mask(t)
                if i < len(seq) - 1:
                    lines.append(side)
            diagrams.append((tuple(sorted(lines)), seq))
    out = {key: 0.0 for key, _ in diagrams}
    for choice in itertools.product(*[bases[g] for g in gluons]):
        pol = dict(zip(gluons, choice))
        for key, seq in diagrams:
            cur = [_tree_currents(t, pol, mom) for t in seq]
            for variant in itertools.product(*[c[0] for c in cur]):
                G_ = np.eye(4, dtype=complex)
                q = pt.copy()
                for i, (j, (_, P)) in enumerate(zip(variant, cur)):
                    G_ = G_ @ sl(j)
                    if i < len(seq) - 1:
                        q = q + P
                        G_ = G_ @ (sl(q) + mt * eye) / (mdot(q, q) - mt * mt)
                Gbar = gam[0] @ G_.conj().T @ gam[0]
                out[key] += np.trace(Pt @ G_ @ Pb @ Gbar).real
    return out


@pytest.mark.parametrize("name,nev", [("gg_ttxg", 6), ("gg_ttxgg", 2)])
def test_sde_diagrams_by_traces(orc, name, nev):
    """Every Feynman diagram of g g -> t t~ g (16, one with a four-gluon vertex)
    and g g -> t t~ g g (123, with four-gluon vertices inside larger trees):
    the oracle's per-diagram helicity sum of |amp_d|^2 equals an independent
    evaluation -- diagrams enumerated here from the vertex rules, three- and
    four-gluon vertices as Feynman-rule tensors, top spins summed as traces in
    the Dirac representation, gluon polarisations over a linear basis."""
    npar = WORKLOADS[name].npar
    gluons = [0, 1] + list(range(4, npar))
    for p in events(orc, name, nev):
        w2, lines = orc.sde(name, p, list(range(1 << npar)), MT)
        ref = _diagram_weights_by_traces(p, gluons, MT)
        assert set(ref) == set(lines) and len(ref) == len(lines)
        for key, val in zip(lines, w2):
            assert abs(val / ref[key] - 1) < 1e-10, (key, val, ref[key])


# ---------------------------------------------------------------- normalisation
@pytest.mark.parametrize("name,iden", [("ee_mumu", 4), ("gg_ttx", 256), ("gg_ttxg", 256), ("gg_ttxgg", 512),
                                       ("gg_ttxggg", 1536)])
def test_averaging_and_symmetry_factor(orc, name, iden):
    """Reading R1: |M|^2 is averaged over the incoming spins and colours and
    divided by the number of orderings of identical final-state gluons.  The
    factor is counted here from the states themselves (2 helicities per
    incoming parton, 8 colours per incoming gluon, permutations of the final
    gluons), and |M|^2 equals the sum over all helicities of the unaveraged
    per-helicity values divided by it."""
    w = WORKLOADS[name]
    incoming_states = 2 * 2 * (1 if name == "ee_mumu" else 8 * 8)
    final_gluons = max(w.npar - 4, 0) if name != "ee_mumu" else 0
    counted = incoming_states * math.factorial(final_gluons)
    assert counted == iden
    mom = events(orc, name, 3)
    mt = 0.0 if name == "ee_mumu" else MT
    me, hel = orc.me2(name, mom, mt=mt, alpha=w.alpha, per_helicity=True)
    assert np.allclose(me, hel.sum(1) / iden, rtol=1e-15, atol=0)
