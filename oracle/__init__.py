"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow reference for the batched tree-level |M|^2 of arXiv:2507.21039
(Sec. 3.1 helicity-amplitude chain, Sec. 4.1 colour algebra, Sec. 4 RAMBO
standalone).  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It shares no code with the CUDA
library in ``paper_2507_21039_gb300`` and never imports it.

The arithmetic lives in ``me_oracle.c`` (plain C99, FP64, optional OpenMP over
events); this module only compiles it with gcc and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "me_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

PROCESSES = {"ee_mumu": 0, "gg_ttx": 1, "gg_ttxg": 2, "gg_ttxgg": 3, "gg_ttxggg": 4}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no arch-specific flags; same on x86 and Arm)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            d, i, i64, u64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
            P = ctypes.c_void_p
            lib.orc_philox4x64_10.argtypes = [P, P, P]
            lib.orc_u01.argtypes = [u64]
            lib.orc_u01.restype = d
            lib.orc_rambo.argtypes = [u64, d, P, i, i64, i64, P, d, d, P, P, P]
            lib.orc_rambo.restype = i
            lib.orc_me2.argtypes = [i, P, i64, d, d, P, P, i]
            lib.orc_me2.restype = i
            lib.orc_partial_amps.argtypes = [i, P, d, i, i, P]
            lib.orc_partial_amps.restype = i
            lib.orc_sde.argtypes = [i, P, d, P, i, P, P, P]
            lib.orc_sde.restype = i
            lib.orc_colour_matrix.argtypes = [i, P]
            lib.orc_colour_matrix.restype = i
            lib.orc_me2_dressed.argtypes = [i, P, d, d, P, i, P]
            lib.orc_me2_dressed.restype = i
            lib.orc_closed_ee.argtypes = [P, d]
            lib.orc_closed_ee.restype = d
            lib.orc_closed_ggtt.argtypes = [P, d, d]
            lib.orc_closed_ggtt.restype = d
            lib.orc_spinor_u.argtypes = [P, d, i, P]
            lib.orc_spinor_v.argtypes = [P, d, i, P]
            lib.orc_bar.argtypes = [P, P]
            lib.orc_polvec.argtypes = [P, i, P]
            lib.orc_su3.argtypes = [P, P]
            lib.orc_perms.argtypes = [i, P]
            lib.orc_perms.restype = i
            lib.orc_npar.argtypes = [i]
            lib.orc_npar.restype = i
            lib.orc_ngluon.argtypes = [i]
            lib.orc_ngluon.restype = i
            lib.orc_iden.argtypes = [i]
            lib.orc_iden.restype = d
            lib.orc_max_threads.restype = i
            lib.orc_dy_partial_amps.argtypes = [i, P, i, i, i, P]
            lib.orc_dy_partial_amps.restype = i
            lib.orc_dy_me2.argtypes = [i, P, i64, d, i, P]
            lib.orc_dy_me2.restype = i
            lib.orc_dy_lepton_currents.argtypes = [P, P, i, i, i, P]
            lib.orc_bg_partial.argtypes = [i, P, P, P, P, d, P, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _pid(process) -> int:
    return PROCESSES[process] if isinstance(process, str) else int(process)


def philox4x64_10(counter, key) -> np.ndarray:
    c = np.ascontiguousarray(counter, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    _load().orc_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def u01(x: int) -> float:
    return _load().orc_u01(int(x))


def npar(process) -> int:
    return _load().orc_npar(_pid(process))


def ngluon(process) -> int:
    return _load().orc_ngluon(_pid(process))


def iden(process) -> float:
    return _load().orc_iden(_pid(process))


def rambo(seed, sqrt_s, masses_final, ev0, nevt, cut_mask=None, ptmin=0.0, drmin=0.0):
    """Seeded RAMBO events ev0..ev0+nevt-1 with optional gluon cuts.

    Returns (momenta [nevt, nfin+2, 4], weights [nevt], attempts [nevt]).
    Raises RuntimeError if an event exceeds 1000 attempts or Newton fails."""
    m = np.ascontiguousarray(masses_final, dtype=np.float64)
    nfin = m.size
    mom = np.zeros((nevt, nfin + 2, 4))
    wt = np.zeros(nevt)
    att = np.zeros(nevt, dtype=np.int32)
    cm = None if cut_mask is None else np.ascontiguousarray(cut_mask, dtype=np.int32)
    st = _load().orc_rambo(int(seed), float(sqrt_s), _ptr(m), nfin, int(ev0), int(nevt),
                           None if cm is None else _ptr(cm), float(ptmin), float(drmin),
                           _ptr(mom), _ptr(wt), _ptr(att))
    if st != 0:
        raise RuntimeError(f"oracle rambo failed with status {st}")
    return mom, wt, att


def me2(process, momenta, mt=173.0, alpha=None, per_helicity=False, nthreads=0):
    """Helicity- and colour-summed, averaged |M|^2 per event (FP64)."""
    pid = _pid(process)
    if alpha is None:
        alpha = 1.0 / 132.5 if pid == 0 else 0.118
    p = np.ascontiguousarray(momenta, dtype=np.float64)
    n = p.shape[0]
    out = np.zeros(n)
    nhel = 1 << npar(pid)
    hel = np.zeros((n, nhel)) if per_helicity else None
    st = _load().orc_me2(pid, _ptr(p), n, float(mt), float(alpha), _ptr(out),
                         None if hel is None else _ptr(hel), int(nthreads))
    if st != 0:
        raise RuntimeError("oracle me2 failed")
    return (out, hel) if per_helicity else out


def sde(process, p_event, helicities, mt=173.0):
    """Feynman diagrams one by one (single-diagram enhancement): for one event,
    per diagram the sum over `helicities` of |amp_d|^2 with bare vertex factors
    (no couplings), and each diagram's internal lines as masks over the external
    particles (the side without the tbar), sorted.  Returns (w2, [lines])."""
    pid = _pid(process)
    p = np.ascontiguousarray(p_event, dtype=np.float64)
    hels = np.ascontiguousarray(helicities, dtype=np.int32)
    w2 = np.zeros(1300)
    lines = np.zeros(1300 * 4, dtype=np.int32)
    nl = np.zeros(1300, dtype=np.int32)
    nd = _load().orc_sde(pid, _ptr(p), float(mt), _ptr(hels), len(hels), _ptr(w2), _ptr(lines), _ptr(nl))
    if nd < 0:
        raise RuntimeError("oracle sde failed")
    return w2[:nd].copy(), [tuple(int(x) for x in lines[4 * d:4 * d + nl[d]]) for d in range(nd)]


def partial_amps(process, p_event, helicity, mt=173.0, gauge_gluon=-1) -> np.ndarray:
    """Colour-ordered partial amplitudes (couplings stripped), lexicographic
    permutation order of the gluons."""
    pid = _pid(process)
    p = np.ascontiguousarray(p_event, dtype=np.float64)
    k = ngluon(pid)
    out = np.zeros(int(np.prod(range(1, k + 1))), dtype=np.complex128)
    _load().orc_partial_amps(pid, _ptr(p), float(mt), int(helicity), int(gauge_gluon), _ptr(out))
    return out


def colour_matrix(k: int) -> np.ndarray:
    import math
    n = math.factorial(k)
    C = np.zeros((n, n))
    _load().orc_colour_matrix(int(k), _ptr(C))
    return C


def perms(k: int) -> np.ndarray:
    import math
    out = np.zeros(math.factorial(k) * k, dtype=np.int32)
    n = _load().orc_perms(int(k), _ptr(out))
    return out.reshape(n, k)


def me2_dressed(process, p_event, helicities, mt=173.0, alpha=0.118) -> np.ndarray:
    """Colour-summed |M_h|^2 from the explicit-colour brute force."""
    pid = _pid(process)
    p = np.ascontiguousarray(p_event, dtype=np.float64)
    h = np.ascontiguousarray(helicities, dtype=np.int32)
    out = np.zeros(h.size)
    st = _load().orc_me2_dressed(pid, _ptr(p), float(mt), float(alpha), _ptr(h), h.size, _ptr(out))
    if st != 0:
        raise RuntimeError("oracle me2_dressed failed")
    return out


def closed_ee(p_event, alpha=1.0 / 132.5) -> float:
    p = np.ascontiguousarray(p_event, dtype=np.float64)
    return _load().orc_closed_ee(_ptr(p), float(alpha))


def closed_ggtt(p_event, mt=173.0, alpha_s=0.118) -> float:
    p = np.ascontiguousarray(p_event, dtype=np.float64)
    return _load().orc_closed_ggtt(_ptr(p), float(mt), float(alpha_s))


def spinor_u(p, m, lam) -> np.ndarray:
    pp = np.ascontiguousarray(p, dtype=np.float64)
    out = np.zeros(4, dtype=np.complex128)
    _load().orc_spinor_u(_ptr(pp), float(m), int(lam), _ptr(out))
    return out


def spinor_v(p, m, lam) -> np.ndarray:
    pp = np.ascontiguousarray(p, dtype=np.float64)
    out = np.zeros(4, dtype=np.complex128)
    _load().orc_spinor_v(_ptr(pp), float(m), int(lam), _ptr(out))
    return out


def bar(s) -> np.ndarray:
    ss = np.ascontiguousarray(s, dtype=np.complex128)
    out = np.zeros(4, dtype=np.complex128)
    _load().orc_bar(_ptr(ss), _ptr(out))
    return out


def polvec(k, lam) -> np.ndarray:
    kk = np.ascontiguousarray(k, dtype=np.float64)
    out = np.zeros(4, dtype=np.complex128)
    _load().orc_polvec(_ptr(kk), int(lam), _ptr(out))
    return out


def su3():
    T = np.zeros((8, 3, 3, 2))
    f = np.zeros((8, 8, 8))
    _load().orc_su3(_ptr(T), _ptr(f))
    return T[..., 0] + 1j * T[..., 1], f


def max_threads() -> int:
    return _load().orc_max_threads()


# ---------------------------------------------------------------- Drell-Yan
# u(0) ubar(1) -> e+(2) e-(3) + n gluons (4..), photon and Z exchange; bosons:
# bit 0 photon, bit 1 Z.

def dy_partial_amps(n, p_event, helicity, gauge_gluon=-1, bosons=3) -> np.ndarray:
    """Colour-ordered partial amplitudes of u ubar -> e+ e- + n g (gluon
    couplings stripped, electroweak ones included), lexicographic gluon orders."""
    import math
    p = np.ascontiguousarray(p_event, dtype=np.float64)
    out = np.zeros(math.factorial(n), dtype=np.complex128)
    if _load().orc_dy_partial_amps(int(n), _ptr(p), int(helicity), int(gauge_gluon), int(bosons), _ptr(out)) < 0:
        raise ValueError("oracle dy_partial_amps: n must be 0..4")
    return out


def dy_me2(n, momenta, alpha_s=0.118, bosons=3) -> np.ndarray:
    """Spin- and colour-averaged |M|^2 of u ubar -> e+ e- + n g per event (FP64)."""
    p = np.ascontiguousarray(momenta, dtype=np.float64)
    out = np.zeros(p.shape[0])
    if _load().orc_dy_me2(int(n), _ptr(p), p.shape[0], float(alpha_s), int(bosons), _ptr(out)) != 0:
        raise ValueError("oracle dy_me2: n must be 0..4")
    return out


def dy_lepton_currents(p_ep, p_em, l_ep, l_em, bosons=3) -> np.ndarray:
    """Lepton currents (photon, Z) of the e+ e- pair, each over its propagator."""
    a = np.ascontiguousarray(p_ep, dtype=np.float64)
    b = np.ascontiguousarray(p_em, dtype=np.float64)
    out = np.zeros((2, 4), dtype=np.complex128)
    _load().orc_dy_lepton_currents(_ptr(a), _ptr(b), int(l_ep), int(l_em), int(bosons), _ptr(out))
    return out


def bg_partial(eps, P, ubar, pt, mt, v) -> complex:
    """Colour-ordered quark-line amplitude with k gluon wavefunctions eps[k][4]
    of outgoing momenta P[k][4] (the gluon recursion on its own)."""
    e = np.ascontiguousarray(eps, dtype=np.complex128)
    m = np.ascontiguousarray(P, dtype=np.float64)
    ub = np.ascontiguousarray(ubar, dtype=np.complex128)
    q = np.ascontiguousarray(pt, dtype=np.float64)
    vv = np.ascontiguousarray(v, dtype=np.complex128)
    out = np.zeros(1, dtype=np.complex128)
    _load().orc_bg_partial(e.shape[0], _ptr(e), _ptr(m), _ptr(ub), _ptr(q), float(mt), _ptr(vv), _ptr(out))
    return complex(out[0])
