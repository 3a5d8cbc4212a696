"""Pins of the oracle's Drell-Yan process u ubar -> e+ e- + n g (the paper's
second standalone workload, Sec. 4, with photon and Z exchange).

Each test checks the oracle against something other than its own recursion:
the textbook helicity form of q qbar -> gamma/Z -> l+ l- (n = 0), the photon
decoupling identity that writes the photon insertion as the sum of gluon
insertions at every colour position (evaluated by the oracle's separately
pinned gluon recursion), gauge invariance, Lorentz invariance and Bose
symmetry.  CPU only.
"""
import math

import numpy as np
import pytest

# electroweak parameters of the oracle's Drell-Yan process (G_F scheme values)
ALPHA = 1.0 / 132.507
MZ, WZ, MW = 91.188, 2.441404, 80.419002


def mdot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


def events(orc, n, nevt, sqrt_s=200.0, seed=21):
    cut = [0, 0] + [1] * n if n else None
    mom, _, _ = orc.rambo(seed, sqrt_s, [0.0] * (2 + n), 0, nevt, cut, 20.0, 0.4)
    return mom


def chiral_couplings():
    """(gL, gR) of the photon and the Z for the u quark and the electron"""
    e = math.sqrt(4 * math.pi * ALPHA)
    cw = MW / MZ
    sw = math.sqrt(1 - cw * cw)

    def z(t3, q):
        return e * (t3 - q * sw * sw) / (sw * cw), -e * q * sw * sw / (sw * cw)

    return {"u": ((e * 2 / 3, e * 2 / 3), z(0.5, 2 / 3)), "e": ((-e, -e), z(-0.5, -1.0))}


def closed_uu_ee(p):
    """Spin- and colour-averaged |M|^2 of u(p1) ubar(p2) -> e+(p3) e-(p4) through
    a photon and a Z, massless fermions, from the helicity amplitudes: a pair of
    equal chiralities (LL, RR) goes with u^2 = ((p1 - p3)^2)^2, opposite ones with
    t^2 = ((p1 - p4)^2)^2, each |M|^2 = 4 |A_ij|^2 (.)^2 with
    A_ij = g_i^u g_j^e / s (photon) + g_i^u g_j^e / (s - MZ^2 + i MZ WZ) (Z);
    the colour sum gives 3, the average 1/(4 * 9)."""
    c = chiral_couplings()
    s = mdot(p[0] + p[1], p[0] + p[1])
    t = mdot(p[0] - p[3], p[0] - p[3])
    u = mdot(p[0] - p[2], p[0] - p[2])
    dz = s - MZ * MZ + 1j * MZ * WZ
    tot = 0.0
    for i in range(2):          # quark chirality L, R
        for j in range(2):      # lepton chirality L, R
            a = c["u"][0][i] * c["e"][0][j] / s + c["u"][1][i] * c["e"][1][j] / dz
            tot += 4 * abs(a) ** 2 * (u * u if i == j else t * t)
    return 3 * tot / 36


@pytest.mark.parametrize("sqrt_s", [60.0, 91.188, 200.0, 1000.0])
def test_uu_ee_closed_form(orc, sqrt_s):
    """Textbook q qbar -> gamma/Z -> l+ l- at energies below, at and above the
    Z pole (the forward-backward asymmetry fixes the chiral couplings and the
    sign of the photon-Z interference)."""
    mom = events(orc, 0, 64, sqrt_s=sqrt_s)
    got = orc.dy_me2(0, mom)
    exp = np.array([closed_uu_ee(p) for p in mom])
    rel = np.abs(got / exp - 1)
    # nearly collinear events lose a few digits in either evaluation
    assert np.median(rel) < 1e-13 and rel.max() < 1e-10, (np.median(rel), rel.max())


def test_uu_ee_photon_and_z_parts(orc):
    """The photon-only and Z-only pieces are the closed form with the other
    boson's couplings set to zero, and the full result is not their sum
    (interference)."""
    mom = events(orc, 0, 16, sqrt_s=120.0)
    c = chiral_couplings()
    s = np.array([mdot(p[0] + p[1], p[0] + p[1]) for p in mom])
    t = np.array([mdot(p[0] - p[3], p[0] - p[3]) for p in mom])
    u = np.array([mdot(p[0] - p[2], p[0] - p[2]) for p in mom])
    e2 = c["u"][0][0] * c["e"][0][0]     # photon: gL = gR = e Q
    photon = 3 * 4 * (e2 / s) ** 2 * 2 * (u * u + t * t) / 36
    assert np.allclose(orc.dy_me2(0, mom, bosons=1), photon, rtol=1e-12, atol=0)
    full, z_only = orc.dy_me2(0, mom), orc.dy_me2(0, mom, bosons=2)
    assert np.min(np.abs(full - photon - z_only) / full) > 1e-3


def _decoupling_sum(orc, n, p, h):
    """photon insertion as the sum over gluon insertions at every colour
    position, each ordering by the gluon recursion (photon part only)"""
    npar = 4 + n
    lam = [1 if (h >> (npar - 1 - i)) & 1 else -1 for i in range(npar)]
    u = orc.spinor_u(p[0], 0.0, lam[0])
    vb = orc.bar(orc.spinor_v(p[1], 0.0, lam[1]))
    L = orc.dy_lepton_currents(p[2], p[3], lam[2], lam[3], bosons=1)[0]
    e_qu = chiral_couplings()["u"][0][0]
    photon = e_qu * L
    qL = p[2] + p[3]
    glu = [np.conj(orc.polvec(p[4 + g], lam[4 + g])) for g in range(n)]
    out = []
    for order in orc.perms(n) if n else [[]]:
        acc = 0j
        for pos in range(n + 1):
            eps = [glu[g] for g in order]
            mom = [p[4 + g] for g in order]
            eps.insert(pos, photon)
            mom.insert(pos, qL)
            acc += orc.bg_partial(np.array(eps), np.array(mom), vb, -p[1], 0.0, u)
        out.append(acc)
    return np.array(out)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_photon_decoupling_identity(orc, n):
    """The colour-ordered amplitude with a colourless photon on the quark line
    equals the sum of the gluon-recursion amplitudes with the photon current in
    place of a gluon at each of the n+1 colour positions (the gluon
    self-couplings cancel in the sum)."""
    mom = events(orc, n, 2)
    rng = np.random.default_rng(n)
    for p in mom:
        scale = max(np.abs(orc.dy_partial_amps(n, p, h, bosons=1)).max() for h in range(0, 1 << (4 + n), 5))
        for h in rng.integers(0, 1 << (4 + n), size=4):
            got = orc.dy_partial_amps(n, p, int(h), bosons=1)
            exp = _decoupling_sum(orc, n, p, int(h))
            assert np.abs(got - exp).max() < 1e-12 * scale


@pytest.mark.parametrize("n", [1, 2, 3])
def test_dy_gauge_invariance(orc, n):
    """A gluon's polarisation replaced by its momentum: every partial amplitude vanishes."""
    mom = events(orc, n, 2)
    rng = np.random.default_rng(7)
    for p in mom:
        scale = max(np.abs(orc.dy_partial_amps(n, p, h)).max() for h in range(0, 1 << (4 + n), 3))
        for h in rng.integers(0, 1 << (4 + n), size=3):
            for g in range(n):
                assert np.abs(orc.dy_partial_amps(n, p, int(h), gauge_gluon=g)).max() < 1e-11 * scale


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


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_dy_lorentz_invariance(orc, n):
    rng = np.random.default_rng(12)
    mom = events(orc, n, 3)
    me = orc.dy_me2(n, mom)
    moved = np.stack([_boost_rotate(p, rng) for p in mom])
    assert np.max(np.abs(orc.dy_me2(n, moved) / me - 1)) < 1e-11


@pytest.mark.parametrize("n", [2, 3])
def test_dy_bose_symmetry(orc, n):
    mom = events(orc, n, 3)
    me = orc.dy_me2(n, mom)
    q = mom.copy()
    q[:, [4, 5]] = mom[:, [5, 4]]
    assert np.max(np.abs(orc.dy_me2(n, q) / me - 1)) < 1e-12


def test_dy_lepton_current_is_conserved(orc):
    mom = events(orc, 0, 4)
    for p in mom:
        q = p[2] + p[3]
        for le in (-1, 1):
            for lm in (-1, 1):
                L = orc.dy_lepton_currents(p[2], p[3], le, lm)
                for b in range(2):
                    assert abs(mdot(q, L[b])) < 1e-13 * max(1e-300, np.abs(L[b]).max() * abs(q[0]))
