"""GB300-native batched tree-level |M|^2 (hot path of arXiv:2507.21039).

Thin Python binding over the C ABI of ``_build/libme.so`` (declared in
``include/me.h``): the functions below have the ABI's names and only marshal
arguments -- every step of the computation runs in the library's CUDA
kernels.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays; device
tensors make the calls asynchronous on the given (or current) CUDA stream.
There is no CPU fallback: importing works without a GPU, but every compute
call needs the built library and a CUDA device, and raises otherwise.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("ME_LIBRARY") or os.path.join(_HERE, "_build", "libme.so")

ME_OK = 0
ME_EINVAL = -1
ME_ENOMEM = -2
ME_ECUDA = -3
ME_ENOTFILTERED = -4
ME_ENONFINITE = -5
ME_ETIMEOUT = -6
ME_ESAMPLER = -7
ME_ETOOLARGE = -8

ME_PREC_FP64 = 0
ME_PREC_FP32 = 1
ME_PREC_MIXED = 2
ME_PREC_MIXED64 = 3
ME_OPT_HSAMPLE_UNIFORM = 4
PRECISIONS = {"fp64": ME_PREC_FP64, "fp32": ME_PREC_FP32, "mixed": ME_PREC_MIXED, "mixed64": ME_PREC_MIXED64}

ME_OPT_REQUIRE_FILTER = 1
ME_OPT_CHECK_FINITE = 2
ME_OPT_GAUGE_CHECK = 3

#: symbols declared in include/me.h
EXPORTS = ("me_init", "me_filter_helicities", "me_filter_helicities_noalloc", "me_sigmakin", "me_sigmakin_hel",
           "me_sigmakin_sde", "me_diagram_lines", "me_sigmakin_hsample", "me_hsample_probabilities", "me_info",
           "me_good_helicities", "me_flops_per_event",
           "me_set_option", "me_free", "rambo_sample", "me_strerror", "me_version")

_lock = threading.Lock()
_lib = None


class MEError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class me_cuts(ctypes.Structure):
    _fields_ = [("ptmin", ctypes.c_double), ("drmin", ctypes.c_double), ("final_mask", ctypes.c_uint32)]


def load():
    """Load libme.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        P, i, i64, u64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        lib.me_init.argtypes = [ctypes.POINTER(P), ctypes.c_char_p, P, i, P, i, i]
        lib.me_filter_helicities.argtypes = [P, P, i64, ctypes.POINTER(i)]
        lib.me_filter_helicities_noalloc.argtypes = [P, P, i64, ctypes.POINTER(i)]
        lib.me_sigmakin.argtypes = [P, P, i64, P, P]
        lib.me_sigmakin_hel.argtypes = [P, P, i64, P, P, P]
        lib.me_sigmakin_sde.argtypes = [P, P, i64, i, P, P, P]
        lib.me_diagram_lines.argtypes = [P, i, P, i, ctypes.POINTER(i)]
        lib.me_sigmakin_hsample.argtypes = [P, P, i64, P, P, P, P]
        lib.me_hsample_probabilities.argtypes = [P, P, i, ctypes.POINTER(i)]
        lib.me_info.argtypes = [P, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), P]
        lib.me_good_helicities.argtypes = [P, P, i, ctypes.POINTER(i)]
        lib.me_flops_per_event.argtypes = [P, ctypes.POINTER(d), ctypes.POINTER(d)]
        lib.me_set_option.argtypes = [P, i, i]
        lib.me_free.argtypes = [P]
        lib.me_free.restype = None
        lib.rambo_sample.argtypes = [u64, i64, i64, d, P, i, ctypes.POINTER(me_cuts), P, P,
                                     ctypes.POINTER(i64), P]
        lib.me_strerror.argtypes = [i]
        lib.me_strerror.restype = ctypes.c_char_p
        lib.me_version.restype = ctypes.c_char_p
        for name in ("me_init", "me_filter_helicities", "me_filter_helicities_noalloc", "me_sigmakin", "me_sigmakin_hel",
                     "me_sigmakin_sde", "me_diagram_lines", "me_sigmakin_hsample", "me_hsample_probabilities", "me_info",
           "me_good_helicities", "me_flops_per_event",
                     "me_set_option", "rambo_sample"):
            getattr(lib, name).restype = i
        _lib = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load().me_strerror(int(code)).decode()
    except RuntimeError:
        return f"status {code}"


def _check(code: int, where: str):
    if code != ME_OK:
        raise MEError(code, where)


def _ptr(x):
    """Raw pointer of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    import numpy as np

    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data_as(ctypes.c_void_p)
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream(stream):
    if stream is None:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Handle:
    """Owns one me_handle*.  close() (or garbage collection) frees it."""

    def __init__(self, ptr, process, precision):
        self._ptr = ptr
        self.process = process
        self.precision = precision

    @property
    def ptr(self):
        if self._ptr is None:
            raise RuntimeError("handle is closed")
        return self._ptr

    def close(self):
        if self._ptr is not None and _lib is not None:
            _lib.me_free(self._ptr)
        self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def me_init(process: str, masses=None, couplings=None, precision="mixed") -> Handle:
    lib = load()
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    h = ctypes.c_void_p()
    m = (ctypes.c_double * len(masses))(*masses) if masses is not None else None
    c = (ctypes.c_double * len(couplings))(*couplings) if couplings is not None else None
    rc = lib.me_init(ctypes.byref(h), process.encode(), m, 0 if masses is None else len(masses),
                     c, 0 if couplings is None else len(couplings), prec)
    _check(rc, "me_init")
    return Handle(h, process, prec)


def me_filter_helicities(h: Handle, momenta) -> int:
    n = ctypes.c_int()
    _check(load().me_filter_helicities(h.ptr, _ptr(momenta), momenta.shape[0], ctypes.byref(n)),
           "me_filter_helicities")
    return n.value


def me_filter_helicities_noalloc(h: Handle, momenta) -> int:
    """Helicity filter that allocates no device memory (device momenta only;
    see include/me.h for the size limit and the shared-scratch caveats)."""
    n = ctypes.c_int()
    _check(load().me_filter_helicities_noalloc(h.ptr, _ptr(momenta), momenta.shape[0], ctypes.byref(n)),
           "me_filter_helicities_noalloc")
    return n.value


def me_sigmakin(h: Handle, momenta, me2=None, stream=None):
    """|M|^2 per event.  Allocates me2 like `momenta` (same device) if not given."""
    nevt = momenta.shape[0]
    if me2 is None:
        if hasattr(momenta, "new_empty"):
            me2 = momenta.new_empty((nevt,))
        else:
            import numpy as np

            me2 = np.empty(nevt)
    st = _stream(stream) if (hasattr(momenta, "is_cuda") and momenta.is_cuda) or stream is not None else None
    _check(load().me_sigmakin(h.ptr, _ptr(momenta), nevt, _ptr(me2), st), "me_sigmakin")
    return me2


def me_sigmakin_hel(h: Handle, momenta, me2, hel_out, stream=None):
    _check(load().me_sigmakin_hel(h.ptr, _ptr(momenta), momenta.shape[0], _ptr(me2), _ptr(hel_out),
                                  _stream(stream)), "me_sigmakin_hel")
    return me2, hel_out


def me_sigmakin_sde(h: Handle, momenta, channel, me2=None, weight=None, stream=None):
    """|M|^2 and the single-diagram-enhancement weight of diagram `channel`
    (device tensors); returns (me2, weight)."""
    nevt = momenta.shape[0]
    me2 = momenta.new_empty((nevt,)) if me2 is None else me2
    weight = momenta.new_empty((nevt,)) if weight is None else weight
    _check(load().me_sigmakin_sde(h.ptr, _ptr(momenta), nevt, int(channel), _ptr(me2), _ptr(weight),
                                  _stream(stream)), "me_sigmakin_sde")
    return me2, weight


def me_sigmakin_hsample(h: Handle, momenta, u, me2=None, hel=None, stream=None):
    """helicity sampling: per event one kept helicity drawn with the uniforms u;
    returns (me2 = |M_h|^2 / p_h, hel) (device tensors)"""
    import torch

    nevt = momenta.shape[0]
    me2 = momenta.new_empty((nevt,)) if me2 is None else me2
    hel = torch.empty(nevt, dtype=torch.int32, device=momenta.device) if hel is None else hel
    _check(load().me_sigmakin_hsample(h.ptr, _ptr(momenta), nevt, _ptr(u), _ptr(me2), _ptr(hel), _stream(stream)),
           "me_sigmakin_hsample")
    return me2, hel


def me_hsample_probabilities(h: Handle) -> list:
    n = ctypes.c_int()
    buf = (ctypes.c_double * 128)()
    _check(load().me_hsample_probabilities(h.ptr, buf, 128, ctypes.byref(n)), "me_hsample_probabilities")
    return [buf[i] for i in range(n.value)]


def me_diagram_lines(h: Handle, diagram) -> tuple:
    """internal lines of a Feynman diagram as masks over the external particles"""
    n = ctypes.c_int()
    masks = (ctypes.c_int * 8)()
    _check(load().me_diagram_lines(h.ptr, int(diagram), masks, 8, ctypes.byref(n)), "me_diagram_lines")
    return tuple(masks[i] for i in range(n.value))


def me_info(h: Handle) -> dict:
    npar, nhel, ncol, ndiag = (ctypes.c_int() for _ in range(4))
    words = (ctypes.c_uint64 * 2)()
    _check(load().me_info(h.ptr, ctypes.byref(npar), ctypes.byref(nhel), ctypes.byref(ncol), ctypes.byref(ndiag),
                          words), "me_info")
    return {"npar": npar.value, "nhel": nhel.value, "ncol": ncol.value, "ndiag": ndiag.value,
            "good_mask": int(words[0]) | (int(words[1]) << 64)}


def me_good_helicities(h: Handle) -> list:
    buf = (ctypes.c_int * 128)()
    n = ctypes.c_int()
    _check(load().me_good_helicities(h.ptr, buf, 128, ctypes.byref(n)), "me_good_helicities")
    return [buf[i] for i in range(n.value)]


def me_flops_per_event(h: Handle):
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().me_flops_per_event(h.ptr, ctypes.byref(a), ctypes.byref(b)), "me_flops_per_event")
    return a.value, b.value


def me_set_option(h: Handle, option: int, value: int):
    _check(load().me_set_option(h.ptr, int(option), int(value)), "me_set_option")


def me_free(h: Handle):
    h.close()


def rambo_sample(seed, ev0, nevt, sqrt_s, masses, cuts=None, momenta_out=None, weights_out=None, stream=None,
                 check=False):
    """Seeded RAMBO events ev0..ev0+nevt-1 into momenta_out [nevt, npar, 4]
    (allocated on the current CUDA device if not given).  With check=True the
    call synchronises and raises if any event failed."""
    import torch

    npar = len(masses)
    if momenta_out is None:
        momenta_out = torch.empty((nevt, npar, 4), dtype=torch.float64, device="cuda")
    m = (ctypes.c_double * npar)(*masses)
    cc = None
    if cuts is not None:
        cc = me_cuts(float(cuts[0]), float(cuts[1]), int(cuts[2]))
    nfail = ctypes.c_int64(0)
    st = _stream(stream) if (hasattr(momenta_out, "is_cuda") and momenta_out.is_cuda) or stream is not None else None
    rc = load().rambo_sample(int(seed), int(ev0), int(nevt), float(sqrt_s), m, npar,
                             ctypes.byref(cc) if cc is not None else None, _ptr(momenta_out), _ptr(weights_out),
                             ctypes.byref(nfail) if check else None, st)
    _check(rc, "rambo_sample")
    return momenta_out


def workload_handle(name: str, precision="mixed") -> Handle:
    """Handle for one of the named workloads (see workloads.py)."""
    from .workloads import PARTICLES, MT, workload

    w = workload(name)
    masses = [MT if p in ("t", "t~") else 0.0 for p in PARTICLES[w.process]]
    return me_init(w.process, masses, [w.alpha], precision)


def cuts_for(name: str):
    from .workloads import DR_MIN, PT_MIN, workload

    w = workload(name)
    mask = 0
    for j, c in enumerate(w.cut_mask):
        if c:
            mask |= 1 << j
    return (PT_MIN, DR_MIN, mask) if mask else None
