"""Emit one CUDA translation unit per process from its evaluation plan.

The unit holds: the external-particle and line tables (__constant__), a
straight-line chain routine templated on the amplitude precision (every
wavefunction a named local, so nvcc keeps them in registers), the colour
quadratic form with the integer numerators as immediates, the launchers of
the three precision modes, and a process descriptor for the C ABI.
"""
from __future__ import annotations

import math
import struct

from .colour import colour_matrix
from .plan import FLOPS, Plan, build_plan, build_plan_dy, colour_groups
from .interp import AMP_KINDS, ROUTINES, build_interp
from .tabplan import build_tabplan

EXT_KINDS = {"VIN": 0, "VOUT": 1, "FO_U": 2, "FO_V": 3, "FI_U": 4, "FI_V": 5}
# processes evaluated with the helicity-recycled table kernel (me_kernel_tab.cuh)
# process -> (threads per event, events per CTA in FP32 / mixed, in FP64,
#             schedule mode, amplitudes per stage (0: one resident table),
#             warp fence every n amplitudes in FP32, in FP64)
# schedule mode: bit 0 = amplitudes as contractions of amputated vertex
# objects, bit 1 = no colour groups (J updated after every amplitude), bit 2 =
# no merged contractions (a group's members sharing an operand each contract),
# bit 3 = (descriptor kernel) each stage's table work runs beside the previous
# stage's amplitudes (measured on GB300 over stage sizes, events per CTA and
# fence intervals)
TAB_PROCESSES = {"gg_ttxg": (32, 1, 1, 1, 0, 1, 4), "gg_ttxgg": (64, 2, 2, 5, 60, 7, 4),
                 # Drell-Yan u u~ -> e+ e- + 2, 3 g (16 and 32 kept helicities; resident tables).
                 # Measured FP32 |M|^2 kernel (2^20 / 2^18 events): n = 2 at 16 threads x 8 events,
                 # fence 4: 2.75 ms (4 events 2.76, 16 events with fence 2 3.27, 32 threads 5.05; the
                 # straight-line kernel 3.86); n = 3 at 32 x 2, fence 24: 3.21 ms (fence 4 3.63, 7 3.48,
                 # 12 3.30, 60 3.40; 4 events 3.73; straight-line 5.15)
                 "uux_epemgg": (16, 8, 4, 0, 0, 4, 4), "uux_epemggg": (32, 2, 2, 0, 0, 24, 4)}
# processes evaluated with the staged descriptor kernel (me_kernel_interp.cuh)
# process -> (threads per event, amplitudes per stage and schedule mode (as
#             above) in FP32 / mixed, the same in FP64).  FP32 keeps J in shared
#             memory, so the table peak of its stages must fit beside J; FP64
#             keeps J in a global scratch.  One schedule for both precisions lets
#             them share one descriptor set (in constant memory).
# (mode bit 3, the table work one stage ahead, measured on GB300 for
# gg -> t t~ g g g: mixed 598 ms per 2^18 events against 592 without, FP32 768
# against 773 -- no gain, so it stays off)
INTERP_PROCESSES = {"gg_ttxggg": (128, 16, 0, 16, 0)}


# FP32 straight-line kernels whose chain would otherwise hold more registers
# than leave room for latency hiding: minimum resident CTAs of 128 threads per
# SM (the register cap is 65536 / (128 x n)); build option
# ME_SCALAR_MIN_CTAS="proc=n,..." overrides.  Measured on GB300, |M|^2 kernel
# per 2^20 events: u u~ -> e+ e- g g uncapped 221 registers (2 CTAs) 6.21 ms,
# 3 CTAs 4.70, 4 CTAs 4.11, 5 CTAs 3.95, 6 CTAs (80 registers, 624 bytes
# spilled) 3.92; u u~ -> e+ e- g (146 registers) 1.91 ms uncapped, 2.01 at 4
# CTAs; u u~ -> e+ e- g g g (255 registers) 5.05 ms per 2^18 uncapped, 8.69 at
# 3 CTAs.
SCALAR_MIN_CTAS_F = {"uux_epemgg": 6}


def _scalar_min_ctas(process: str) -> int:
    env = __import__("os").environ.get("ME_SCALAR_MIN_CTAS", "")
    for item in filter(None, env.split(",")):
        name, _, n = item.partition("=")
        if name == process:
            return int(n)
    return SCALAR_MIN_CTAS_F.get(process, 1)


def _apply_kernel_overrides():
    """Build option ME_GEN_KERNEL="proc=interp:NT:STAGE,proc=tab:NT,..." selects
    the kernel family of a process (used to compare kernel designs)."""
    import os

    spec = os.environ.get("ME_GEN_KERNEL", "")
    for item in filter(None, (x.strip() for x in spec.split(","))):
        proc, what = item.split("=")
        parts = what.split(":")
        TAB_PROCESSES.pop(proc, None)
        INTERP_PROCESSES.pop(proc, None)
        if parts[0] == "interp":
            dflt = (0, 16, 0, 16, 1)
            INTERP_PROCESSES[proc] = tuple(int(parts[i + 1]) if len(parts) > i + 1 else dflt[i] for i in range(5))
        elif parts[0] == "tab":
            dflt = (0, 1, 1, 1, 0, 1, 4)
            TAB_PROCESSES[proc] = tuple(int(parts[i + 1]) if len(parts) > i + 1 else dflt[i] for i in range(7))


_apply_kernel_overrides()


# Drell-Yan processes u ubar -> e+ e- + n g (the paper's second standalone
# workload, Sec. 4; photon and Z exchange, reading R15): name -> gluon count
DY_PROCESSES = {"uux_epem": 0, "uux_epemg": 1, "uux_epemgg": 2, "uux_epemggg": 3}


def _ext_table(process: str):
    if process == "ee_mumu":
        # e-(in) u, e+(in) vbar, mu-(out) ubar, mu+(out) v; massless
        return ["FI_U", "FO_V", "FO_U", "FI_V"], [0, 0, 0, 0]
    if process in DY_PROCESSES:
        # u(in) u, ubar(in) vbar, e+(out) v, e-(out) ubar, gluons(out) eps*; massless
        n = DY_PROCESSES[process]
        return ["FI_U", "FO_V", "FI_V", "FO_U"] + ["VOUT"] * n, [0] * (4 + n)
    npar = {"gg_ttx": 4, "gg_ttxg": 5, "gg_ttxgg": 6, "gg_ttxggg": 7}[process]
    kinds = ["VIN", "VIN", "FO_U", "FI_V"] + ["VOUT"] * (npar - 4)
    massive = [0, 0, 1, 1] + [0] * (npar - 4)
    return kinds, massive


def _line_tables(P: Plan):
    plus, minus, kind = [], [], []
    for ln in P.lines:
        pm = mm = 0
        if ln.kind == "a":  # photon: p1 + p2
            pm = 0b11
            kind.append(1)
        elif ln.kind == "g":
            for g in ln.gluons:
                e = P.gluon_ext[g]
                if P.gluon_incoming[g]:
                    mm |= 1 << e
                else:
                    pm |= 1 << e
            kind.append(0 if len(ln.gluons) == 1 else 1)
        elif P.process.startswith("dy_"):  # Drell-Yan quark line ("q", "qe"): -p_ubar + P_S (+ p_e+ + p_e-), massless
            assert ln.kind in ("q", "qe"), ln.kind
            mm |= 1 << 1
            if ln.kind == "qe":
                pm |= 0b1100
            for g in ln.gluons:
                pm |= 1 << P.gluon_ext[g]
            kind.append(1)
        else:  # top propagator: p_t + P_S
            pm |= 1 << 2
            for g in ln.gluons:
                e = P.gluon_ext[g]
                if P.gluon_incoming[g]:
                    mm |= 1 << e
                else:
                    pm |= 1 << e
            kind.append(2)
        plus.append(pm)
        minus.append(mm)
    return plus, minus, kind


def _line_sides(plus, minus, npar):
    """Per line, the shortest signed sum of external momenta equal to its momentum.

    A line's momentum is q = sum_plus p - sum_minus p (physical momenta).  The
    external momenta satisfy sum_i sigma_i p_i = 0 with sigma = -1 for the two
    incoming particles and +1 for the outgoing ones, so q - lam * sum sigma_i p_i
    (lam = +-1) is the same vector written over the other side of the line.  The
    shorter form has at most floor(npar / 2) terms.  Packed per line: bits 0-2
    the number of terms k; term a at bits 4a+4 .. 4a+7 (particle index in bits
    4a+4 .. 4a+6, bit 4a+7 set for a minus sign).  Returns (packed, max k)."""
    sigma = [-1, -1] + [1] * (npar - 2)
    out, kmax = [], 0
    for pm, mm in zip(plus, minus):
        c = [((pm >> i) & 1) - ((mm >> i) & 1) for i in range(npar)]
        best = None
        for lam in (0, 1, -1):
            cc = [ci - lam * si for ci, si in zip(c, sigma)]
            if all(x in (-1, 0, 1) for x in cc):
                n = sum(1 for x in cc if x)
                if best is None or n < best[0]:
                    best = (n, cc)
        n, cc = best
        word = n
        for a, (i, x) in enumerate((i, x) for i, x in enumerate(cc) if x):
            word |= (i | (8 if x < 0 else 0)) << (4 * a + 4)
        out.append(word)
        kmax = max(kmax, n)
    return out, kmax


def umma_k16_offset(row: int, k: int) -> int:
    """Byte offset of element (row, k) in a K = 16 BF16 tensor-core operand,
    K-major core matrices of 8 rows x 16 bytes (me_tmem.cuh: umma_k16_offset)."""
    return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2


def _bf16_bits(x: float) -> int:
    """float -> bfloat16 bits, round to nearest even"""
    f = struct.unpack("<I", struct.pack("<f", float(x)))[0]
    return ((f + 0x7FFF + ((f >> 16) & 1)) >> 16) & 0xFFFF


def _bf16_value(bits: int) -> float:
    return struct.unpack("<f", struct.pack("<I", bits << 16))[0]


def tc_fragments(num):
    """mma.sync m16n8k16 B-operand fragments of the colour numerators: for each
    k-step, n-tile and lane, (b0, b1) packing B[k][n], B[k+1][n] (low, high) at
    k = 16 ks + 2t (+8), n = 8 nt + g (g = lane/4, t = lane%4).  Numerators with
    more than 8 significant bits are split hi + lo, both exact in BF16."""
    n = len(num)
    kp, np_ = (n + 15) // 16 * 16, (n + 7) // 8 * 8
    hi = [[0] * np_ for _ in range(kp)]
    lo = [[0] * np_ for _ in range(kp)]
    split = False
    for k in range(n):
        for j in range(n):
            v = num[k][j]
            hb = _bf16_bits(v)
            rest = v - _bf16_value(hb)
            lb = _bf16_bits(rest)
            assert _bf16_value(hb) + _bf16_value(lb) == v, v
            hi[k][j], lo[k][j] = hb, lb
            split |= rest != 0
    def frags(B):
        out = []
        for ks in range(kp // 16):
            for nt in range(np_ // 8):
                for lane in range(32):
                    g, t = lane >> 2, lane & 3
                    k0, col = 16 * ks + 2 * t, 8 * nt + g
                    b0 = B[k0][col] | (B[k0 + 1][col] << 16)
                    b1 = B[k0 + 8][col] | (B[k0 + 9][col] << 16)
                    out.append((b0, b1))
        return out
    f = frags(hi) + (frags(lo) if split else [])
    return f, split


def _coef_call(col, c, var):
    return f"jacc<{c[0]}, {c[1]}, T>(J[{col}], {var});"


def emit_process(process: str) -> tuple[str, dict]:
    dy = process in DY_PROCESSES
    P = build_plan_dy(DY_PROCESSES[process]) if dy else build_plan(process)
    npar = P.npar
    ncol = P.ncol
    k = len(P.gluon_ext)
    kinds, massive = _ext_table(process)
    plus, minus, lkind = _line_tables(P)
    sides, side_max = _line_sides(plus, minus, npar)
    if process == "ee_mumu":
        num, den = [[1]], 1
        iden, cpow = 4.0, 2
    elif dy:  # quark line with k gluons: the same string basis (delta_ij for k = 0);
        # spin x colour average 4 x 9, k! identical gluons; electroweak couplings fixed
        num, den = colour_matrix(k) if k else ([[3]], 1)
        iden, cpow = 4.0 * 9.0 * math.factorial(k), k
    else:
        num, den = colour_matrix(k)
        iden, cpow = 4.0 * 64.0 * math.factorial(k - 2), k
    j_smem = ncol > 32
    threads = 64 if j_smem else 128
    nlines = len(P.lines)

    diag_of_op = {op: P.amp_diag[n] for n, (op, _) in enumerate(P.amps)}
    body = []
    for i, op in enumerate(P.ops):
        a = [f"w{x}" for x in op.args]
        kd = op.kind
        if kd == "ext_lepL":  # Drell-Yan: both insertion objects from ubar(e-), v(e+) and the coefficients
            iR = next(j for j, o in enumerate(P.ops) if o.kind == "ext_lepR")
            body.append(f"Wf<T> w{i}, w{iR}; LEPLR<T>(ext[6 + ((hel >> {npar - 4}) & 1)], "
                        f"ext[4 + ((hel >> {npar - 3}) & 1)], ext[{2 * npar}], w{i}, w{iR});")
        elif kd == "ext_lepR":
            pass
        elif kd.startswith("ext_"):
            e = op.ext
            body.append(f"const Wf<T>& w{i} = ext[{2 * e} + ((hel >> {npar - 1 - e}) & 1)];")
        elif kd == "VVV1P0_1":
            la, lb = op.mom
            body.append(f"Wf<T> w{i}; VVV1P0_1<T>({a[0]}, ln[{la}].p, {a[1]}, ln[{lb}].p, ln[{op.line}].inv, w{i});")
        elif kd.endswith("P0_1"):
            body.append(f"Wf<T> w{i}; {kd}<T>({a[0]}, {a[1]}, {a[2]}, ln[{op.line}].inv, w{i});")
        elif kd in ("FFV1_2", "FFV1_1"):
            body.append(f"Wf<T> w{i}; {kd}<T>({a[0]}, {a[1]}, ln[{op.line}], mt, w{i});")
        elif kd == "FFVLR_2":
            body.append(f"Wf<T> w{i}; FFVLR_2<T>({a[0]}, {a[1]}, {a[2]}, ln[{op.line}], w{i});")
        elif kd == "FFVLR_1":
            body.append(f"Wf<T> w{i}; FFVLR_1<T>({a[0]}, {a[1]}, {a[2]}, ln[{op.line}], w{i});")
        elif kd == "FFV1P0_3":
            body.append(f"Wf<T> w{i}; FFV1P0_3<T>({a[0]}, {a[1]}, ln[{op.line}].inv, w{i});")
        elif kd == "FFV1_0":
            body.append(f"const cx<T> w{i} = FFV1_0<T>({a[0]}, {a[1]}, {a[2]});")
        elif kd == "VVV1_0":
            la, lb = op.mom
            body.append(f"const cx<T> w{i} = VVV1_0<T>({a[0]}, ln[{la}].p, {a[1]}, ln[{lb}].p, {a[2]});")
        elif kd.endswith("_0"):
            body.append(f"const cx<T> w{i} = {kd}<T>({a[0]}, {a[1]}, {a[2]}, {a[3]});")
        else:
            raise ValueError(kd)
        if op.out == "A":
            terms = dict(P.amps)[i]
            for col, c in terms:
                body.append("  " + _coef_call(col, c, f"w{i}"))
            body.append(f"  ME_SDE(w{i}, {diag_of_op[i]});")

    # colour quadratic form: sum_i Re(conj J_i z_i), z_i = N_ii J_i + sum_{j>i} 2 N_ij J_j
    cbody = []
    for i in range(ncol):
        terms = [(j, num[i][j] * (1 if j == i else 2)) for j in range(i, ncol) if num[i][j] != 0]
        if not terms:
            continue
        j0, c0 = terms[0]
        cbody.append("{")
        cbody.append(f"  const cx<T> a = J[{i}];")
        cbody.append(f"  cx<T> b = J[{j0}];")
        cbody.append(f"  T zr = T({c0}) * b.re, zi = T({c0}) * b.im;")
        for j, c in terms[1:]:
            cbody.append(f"  b = J[{j}]; zr = fma(T({c}), b.re, zr); zi = fma(T({c}), b.im, zi);")
        cbody.append("  s = fma(a.re, zr, fma(a.im, zi, s));")
        cbody.append("}")

    tab_src, TP, IP = ("", None, None)
    if process in TAB_PROCESSES:
        tab_src, TP, tab_flops, tab_amp_flops = emit_tab_struct(process, *TAB_PROCESSES[process], ncol, nlines, cbody)
    elif process in INTERP_PROCESSES:
        nt_i, sa, amp_i, sa_d, amp_d = INTERP_PROCESSES[process]
        tab_src, IP = emit_interp_struct(process, nt_i, sa, num, amp_i)
        if (sa_d, amp_d) != (sa, amp_i):
            tab_src += emit_interp_struct(process, nt_i, sa_d, num, amp_d, "ProcInterpD", "d_")[0]
        else:
            tab_src += "using ProcInterpD = ProcInterp;\n"
        body, cbody = [], []   # the straight-line chain is not used for this process
    kernel_struct = "ProcTab" if TP else ("ProcInterp" if IP else "Proc")
    kernel_struct_d = "ProcInterpD" if IP else kernel_struct
    launch_fn = "launch_tab" if TP else ("launch_interp" if IP else "launch_scalar")
    nhel_all = 1 << npar
    # chain flops per evaluated helicity, and the helicity-independent table
    # flops per event (the table kernels compute every variant of every object
    # once per event, however many helicities are kept)
    table_flops_ev = 0
    if TP:
        flops_hel, table_flops_ev = tab_amp_flops, tab_flops
    elif IP:
        flops_hel = IP.tab.amplitude_flops_per_helicity(not INTERP_PROCESSES[process][2] & 2)
        table_flops_ev = IP.table_flops
    else:
        flops_hel = P.flops_per_helicity()
    tc_members, tc_array = "", ""
    if ncol >= 24:
        fr, nsplit = tc_fragments(num)
        tc_array = (f"__device__ const uint2 c_bfrag[{len(fr)}] = {{\n    "
                    + ",\n    ".join(", ".join("{%du, %du}" % x for x in fr[i:i + 8]) for i in range(0, len(fr), 8))
                    + "\n};\n")
        tc_members = (f"\n    static constexpr bool NSPLIT = {'true' if nsplit else 'false'};"
                      f"\n    __device__ static __forceinline__ const uint2* bfrag() {{ return c_bfrag; }}")
        if ncol <= 32 and not nsplit:
            # colour numerators as the B operand of tcgen05.mma (K-major, N = K = 32,
            # padded with zeros): two K = 16 images, B[n][k] = N[k][n], BF16 exact
            img = [0] * 1024
            for ks in range(2):
                for n_ in range(32):
                    for kk in range(16):
                        k_ = 16 * ks + kk
                        if n_ < ncol and k_ < ncol:
                            img[512 * ks + umma_k16_offset(n_, kk) // 2] = _bf16_bits(num[k_][n_])
            words = [img[i] | (img[i + 1] << 16) for i in range(0, 1024, 2)]
            tc_array += (f"__device__ __align__(16) const unsigned int c_umma_cn[512] = {{\n    "
                         + ",\n    ".join(", ".join("%du" % x for x in words[i:i + 12]) for i in range(0, 512, 12))
                         + "\n};\n")
            tc_members += ("\n    // colour numerators as a tcgen05.mma operand (two K = 16 images of 32 x 16)"
                           "\n    __device__ static __forceinline__ const uint4* umma_cn() "
                           "{ return reinterpret_cast<const uint4*>(c_umma_cn); }")
    ns = f"p_{process}"
    family = 0 if process == "ee_mumu" else (2 if dy else 1)
    # internal-line sets of the diagrams (QCD and e+e-); the Drell-Yan plans carry none
    diag_lines = P.diag_lines if P.diag_lines else [()] * P.ndiagrams
    if IP:  # FP64 chains (FP64, paper-mixed, FP64 channel weights) keep J in global memory
        jscratch_body = ("    return (precision == PREC_FP64 || precision == PREC_MIXED64)\n"
                         "               ? interp_jscratch_per_cta<ProcInterpD, double>()\n"
                         "               : interp_jscratch_per_cta<ProcInterp, float>();")
        jscratch_ctas_body = ("    return (precision == PREC_FP64 || precision == PREC_MIXED64)\n"
                              "               ? interp_resident_ctas<ProcInterpD, double>()\n"
                              "               : interp_resident_ctas<ProcInterp, float>();")
    else:
        jscratch_body = "    (void)precision;\n    return 0;"
        jscratch_ctas_body = "    (void)precision;\n    return 0;"
    cnum_flat = ", ".join(str(x) for row in num for x in row)
    src = f"""// Generated by paper_2507_21039_gb300/gen/emit.py for {process}: do not edit.
// {P.ndiagrams} Feynman diagrams, {len(P.amps)} amplitudes, {len(P.ops)} routine calls,
// {ncol} colour flows, {nlines} lines, {P.flops_per_helicity()} chain flops per helicity.
#include "me_kernel.cuh"
#include "me_colour_tc.cuh"
#include "me_kernel_tab.cuh"
#include "me_kernel_interp.cuh"

namespace me {{
namespace {ns} {{

__constant__ unsigned char c_ext_kind[{npar}] = {{{", ".join(str(EXT_KINDS[x]) for x in kinds)}}};
__constant__ unsigned char c_ext_massive[{npar}] = {{{", ".join(str(x) for x in massive)}}};
__constant__ unsigned short c_line_plus[{max(nlines, 1)}] = {{{", ".join(str(x) for x in plus) or "0"}}};
__constant__ unsigned short c_line_minus[{max(nlines, 1)}] = {{{", ".join(str(x) for x in minus) or "0"}}};
__constant__ unsigned char c_line_kind[{max(nlines, 1)}] = {{{", ".join(str(x) for x in lkind) or "0"}}};
__constant__ unsigned int c_line_side[{max(nlines, 1)}] = {{{", ".join(str(x) for x in sides) or "0"}}};
static const int h_cnum[{ncol * ncol}] = {{{cnum_flat}}};
static const int h_diag_lines[{4 * P.ndiagrams}] = {{{", ".join(str(x) for key in diag_lines for x in (list(key) + [0] * (4 - len(key))))}}};
static const int h_diag_nlines[{P.ndiagrams}] = {{{", ".join(str(len(key)) for key in diag_lines)}}};
{tc_array}
struct Proc {{
    static constexpr int NPAR = {npar}, NCOL = {ncol}, NLINES = {nlines}, THREADS = {threads};
    static constexpr int CDEN = {den};
    // Drell-Yan insertion: its electroweak coefficients follow the 2 NPAR external states
    static constexpr bool EW = {"true" if dy else "false"};
    static constexpr int NEXT = 2 * NPAR + (EW ? 1 : 0);
    // most terms of a line momentum written over its shorter side (line_side)
    static constexpr int SIDE = {max(side_max, 1)};
    static constexpr bool J_SMEM = {"true" if j_smem else "false"};
    // FP32 straight-line kernel: at least this many resident CTAs per SM (register cap)
    static constexpr int MIN_CTAS_F = {_scalar_min_ctas(process)};
    static constexpr bool IS_TAB = false, IS_INTERP = false;{tc_members}
    __device__ static __forceinline__ unsigned ext_kind(int e) {{ return c_ext_kind[e]; }}
    __device__ static __forceinline__ unsigned ext_massive(int e) {{ return c_ext_massive[e]; }}
    __device__ static __forceinline__ unsigned line_plus(int l) {{ return c_line_plus[l]; }}
    __device__ static __forceinline__ unsigned line_minus(int l) {{ return c_line_minus[l]; }}
    __device__ static __forceinline__ unsigned line_kind(int l) {{ return c_line_kind[l]; }}
    __device__ static __forceinline__ unsigned line_side(int l) {{ return c_line_side[l]; }}

    template <class T, bool SDE, class JT>
    __device__ static __forceinline__ void chain(const Wf<T>* __restrict__ ext, int hel, const Ln<T>* __restrict__ ln,
                                                 T mt, JT& J, SdeAcc<T>& sde)
    {{
        (void)sde;
        (void)mt;
{chr(10).join("        " + x for x in body)}
    }}

    template <class T, class JT> __device__ static __forceinline__ T colour(const JT& J)
    {{
        T s = T(0);
{chr(10).join("        " + x for x in cbody)}
        return s;
    }}
}};
{tab_src}
static cudaError_t launch(int precision, const LaunchArgs& a)
{{
    if (a.sde_w) {{  // single-diagram-enhancement weights: FP64 or FP32 chain, scalar colour
        if (precision == PREC_FP64 || precision == PREC_MIXED64)
            return {launch_fn}<{kernel_struct_d}, double{", false" if (IP or TP) else ""}, double, true>(a);
        return {launch_fn}<{kernel_struct}, float{", false" if (IP or TP) else ""}, float, true>(a);
    }}
    switch (precision) {{
    case PREC_FP64: return {launch_fn}<{kernel_struct_d}, double{", false" if IP else ""}>(a);
    case PREC_FP32: return {launch_fn}<{kernel_struct}, float{", false" if IP else ""}>(a);
    case PREC_MIXED: return launch_mixed<{kernel_struct}>(a);
    case PREC_MIXED64: return {launch_fn}<{kernel_struct_d}, double{", false" if (IP or TP) else ""}, float>(a);
    default: return cudaErrorInvalidValue;
    }}
}}

static size_t jscratch_per_cta(int precision)
{{
{jscratch_body}
}}

static int jscratch_ctas(int precision)
{{
{jscratch_ctas_body}
}}

}}  // namespace {ns}

const ProcDesc* procdesc_{process}()
{{
    static const ProcDesc d = {{"{process}", {npar}, {1 << npar}, {ncol}, {P.ndiagrams}, {len(P.amps)}, {k}, {nlines},
                               {threads}, {iden!r}, {den}, {ns}::h_cnum, {flops_hel}LL,
                               {P.colour_flops_per_helicity()}LL, {table_flops_ev}LL, {cpow}, &{ns}::launch, {ns}::h_diag_lines,
                               {ns}::h_diag_nlines, &{ns}::jscratch_per_cta, &{ns}::jscratch_ctas, {family}}};
    return &d;
}}

}}  // namespace me
"""
    meta = {
        "process": process,
        "ndiagrams": P.ndiagrams,
        "namps": len(P.amps),
        "nops": len(P.ops),
        "ncol": ncol,
        "nlines": nlines,
        "flops_per_helicity": flops_hel,
        "table_flops_per_event": table_flops_ev,
        "flops_per_helicity_unrecycled": P.flops_per_helicity(),
        "table_entries": TP.size if TP else 0,
        "colour_flops_per_helicity": P.colour_flops_per_helicity(),
        "counts": P.counts(),
        "cden": den,
    }
    return src, meta


def _support_name(S):
    return "v_" + "_".join(str(p) for p in S)


def _table_call(kind, k="k"):
    if kind == "VVV1P0_1":
        c = f"VVV1P0_1<T>(tab.ld({k}.in0), ln[{k}.la].p, tab.ld({k}.in1), ln[{k}.lb].p, ln[{k}.lo].inv, o);"
    elif kind.startswith("VVVV") and kind.endswith("P0_1"):
        c = f"{kind}<T>(tab.ld({k}.in0), tab.ld({k}.in1), tab.ld({k}.in2), ln[{k}.lo].inv, o);"
    elif kind in ("FFV1_2", "FFV1_1"):
        c = f"{kind}<T>(tab.ld({k}.in0), tab.ld({k}.in1), ln[{k}.lo], mt, o);"
    elif kind == "FFV1P0_3":
        c = f"FFV1P0_3<T>(tab.ld({k}.in0), tab.ld({k}.in1), ln[{k}.lo].inv, o);"
    elif kind in ("FFV1A_3", "FFV1A_2", "FFV1A_1"):
        c = f"{kind}<T>(tab.ld({k}.in0), tab.ld({k}.in1), o);"
    elif kind.startswith("VVV1A_"):
        c = f"VVV1A<{kind[-1]}, T>(tab.ld({k}.in0), tab.ld({k}.in1), ln[{k}.la].p, ln[{k}.lb].p, o);"
    elif kind in ("VVVV1A", "VVVV3A", "VVVV4A"):
        c = f"{kind}<T>(tab.ld({k}.in0), tab.ld({k}.in1), tab.ld({k}.in2), o);"
    elif kind in ("ext_lepL", "ext_lepR"):  # Drell-Yan lepton pair: (ubar(e-), v(e+), coefficients)
        other = "oR" if kind == "ext_lepL" else "oL"
        outs = "o, oR" if kind == "ext_lepL" else "oL, o"
        c = f"Wf<T> {other}; LEPLR<T>(tab.ld({k}.in0), tab.ld({k}.in1), tab.ld({k}.in2), {outs});"
    elif kind in ("FFVLR_2", "FFVLR_1"):
        c = f"{kind}<T>(tab.ld({k}.in0), tab.ld({k}.in1), tab.ld({k}.in2), ln[{k}.lo], o);"
    else:
        raise ValueError(kind)
    return f"Wf<T> o; {c} tab.st({k}.out, o);"


def _amp_call(P, ai, addr):
    """code evaluating amplitude op ai; addr(x) -> table address expression of operand x"""
    op = P.ops[ai]
    args = [f"tab.ld({addr(a)})" for a in op.args]
    if op.kind in ("FFV1_0", "DOTV", "DOTF"):
        return f"{op.kind}<T>({', '.join(args)})"
    if op.kind == "VVV1_0":
        la, lb = op.mom
        return f"VVV1_0<T>({args[0]}, ln[{la}].p, {args[1]}, ln[{lb}].p, {args[2]})"
    return f"{op.kind}<T>({args[0]}, {args[1]}, {args[2]}, {args[3]})"


def _amp_block(P, ai, terms, addr, n_amp, diag):
    out = [f"{{ const cx<T> x = {_amp_call(P, ai, addr)};"]
    for col, c in terms:
        out.append(f"  jacc<{c[0]}, {c[1]}, T>(J[{col}], x);")
    out.append(f"  ME_SDE(x, {diag});")
    out.append("}")
    out.append(f"ME_FENCE(T, {n_amp});")
    return out


def _shared_operand(P, run):
    """For a colour group's members `run` (plan amplitude indices) that are all
    two-operand contractions of one kind (DOTV or DOTF, both bilinear and
    symmetric) sharing one operand: (kind, shared op, [other op of each
    member]); else None."""
    ops = [P.ops[P.amps[a][0]] for a in run]
    if len(run) < 2 or ops[0].kind not in ("DOTV", "DOTF") or any(o.kind != ops[0].kind for o in ops):
        return None
    common = set(ops[0].args).intersection(*(set(o.args) for o in ops[1:]))
    if not common:
        return None
    y = min(common)
    others = [o.args[1] if o.args[0] == y else o.args[0] for o in ops]
    return ops[0].kind, y, others


def _merged_group_block(P, run, addr, n_amp, sign_of, terms, merge):
    """A whole colour group in one block: sum_m s_m K(X_m, Y) = s_1 K(X_1 + sum_m s_1 s_m X_m, Y)
    (K bilinear), one contraction instead of len(run); with single-diagram
    enhancement every member's own amplitude is also formed."""
    kind, y, others = merge
    s1 = sign_of[run[0]]
    out = [f"{{ Wf<T> S = tab.ld({addr(others[0])});"]
    for a, x in zip(run[1:], others[1:]):
        out.append(f"  wf_acc<{s1 * sign_of[a]}>(S, tab.ld({addr(x)}));")
    out.append(f"  const cx<T> G = {kind}<T>(S, tab.ld({addr(y)}));")
    for col, c in terms:
        out.append(f"  jacc<{s1 * c[0]}, {s1 * c[1]}, T>(J[{col}], G);")
    out.append("  if constexpr (SDE) {")
    for a in run:
        out.append(f"    {{ const cx<T> xm = {_amp_call(P, P.amps[a][0], addr)}; ME_SDE(xm, {P.amp_diag[a]}); }}")
    out.append("  }")
    out.append("}")
    for k in range(len(run)):
        out.append(f"ME_FENCE(T, {n_amp + k});")
    return out


def _amp_run_code(P, items, addr, n_amp, sign_of, flush, merging=True):
    """code for consecutive amplitudes `items` [(plan index, first, last)] of one
    stage: whole colour groups that share an operand are merged, the rest go
    amplitude by amplitude.  Returns (code, next amplitude number, amplitude
    flops per helicity saved by the merges)."""
    code, k, saved = [], 0, 0
    while k < len(items):
        pi, first, last = items[k]
        run = [pi]
        if first and not last:
            j = k + 1
            while j < len(items) and not items[j][1]:
                run.append(items[j][0])
                if items[j][2]:
                    break
                j += 1
        merge = _shared_operand(P, run) if (merging and first and run[-1] in flush and len(run) > 1) else None
        if merge:
            code += _merged_group_block(P, run, addr, n_amp, sign_of, flush[run[-1]], merge)
            # per merged member: one contraction and one complex add of the group
            # sum fewer, one wavefunction add (8 flops) more
            saved += (len(run) - 1) * (FLOPS[merge[0]] + 2 - 8)
            n_amp += len(run)
            k += len(run)
            continue
        code += _grouped_amp_block(P, pi, P.amps[pi][0], addr, n_amp, P.amp_diag[pi], sign_of[pi], first, last,
                                   flush.get(pi, ()))
        n_amp += 1
        k += 1
    return code, n_amp, saved


def _group_positions(order, flush):
    """(first, last) flags of each amplitude of `order` within its colour group
    (the members of a group are adjacent in `order`; `flush` holds the last
    member of every group)"""
    return [(k == 0 or order[k - 1] in flush, a in flush) for k, a in enumerate(order)]


def _grouped_amp_block(P, pi, aop, addr, n_amp, diag, sign, first, last, terms):
    """One amplitude of a colour group: the group sum G = sum_m s_m A_m is
    opened by the first member and added into J (the group's normalised
    colour terms) by the last; a group of one adds its own terms directly."""
    if first and last:
        return _amp_block(P, aop, P.amps[pi][1], addr, n_amp, diag)
    out = ["{ cx<T> G;"] if first else []
    out.append(f"{{ const cx<T> x = {_amp_call(P, aop, addr)};")
    if first:
        out.append("  G = x;" if sign > 0 else "  G = cx<T>{-x.re, -x.im};")
    else:
        out.append("  G.re += x.re; G.im += x.im;" if sign > 0 else "  G.re -= x.re; G.im -= x.im;")
    out.append(f"  ME_SDE(x, {diag});")
    out.append("}")
    if last:
        for col, c in terms:
            out.append(f"jacc<{c[0]}, {c[1]}, T>(J[{col}], G);")
        out.append("}")
    out.append(f"ME_FENCE(T, {n_amp});")
    return out


def _variant_code(npar, supports):
    bits = [f"const int b{p} = (h >> {npar - 1 - p}) & 1;" for p in range(npar)]
    sups = []
    for S in sorted(supports, key=lambda x: (len(x), x)):
        expr = " | ".join(f"(b{p} << {j})" if j else f"b{p}" for j, p in enumerate(S))
        sups.append(f"const int {_support_name(S)} = {expr};")
    return bits + sups


def _allowed_expr(TP):
    """C expression of the helicity index h: every pair of TP.opposite_pairs has
    different helicity bits (particle p's bit is bit npar - 1 - p of h)"""
    n = TP.plan.npar
    terms = [f"(((h >> {n - 1 - a}) ^ (h >> {n - 1 - b})) & 1)" for a, b in TP.opposite_pairs]
    return " && ".join(terms) if terms else "true"


def emit_tab_struct(process: str, nt: int, epc_f: int, epc_d: int, amputated: int, stage: int,
                    fence_f: int, fence_d: int, ncol: int, nlines: int, colour_body: list):
    """ProcTab: task table, table rounds and per-helicity amplitudes.

    stage == 0: one resident table (every object, all levels), then the
    amplitudes of each helicity (`tables` + `amps`).  stage > 0: the staged
    schedule of gen/interp.py as straight-line code (`staged`): per stage, the
    table rounds of the objects that become live, then the stage's amplitudes,
    slots reused after each object's last reader; one helicity per thread."""
    saved = 0
    tasks = []
    # rounds of one level run without barriers between them; each round's
    # tasks start at the warp after the one where the previous round's ended,
    # so that small rounds do not all land on the first warp
    rot = [0]

    def round_code(kind, tl, level_note):
        start = len(tasks)
        for out, ins, ln in tl:
            ins = list(ins) + [0] * (3 - len(ins))
            tasks.append((out, ins[0], ins[1], ins[2], *(max(x, 0) for x in ln)))
        off = rot[0]
        rot[0] = (off + -(-len(tl) // 32) * 32) % nt
        first = "tid" if off == 0 else f"(tid + {nt - off}) % NT"
        return (f"for (int t = {first}; t < {len(tl)}; t += NT) {{ const TabTask k = ld_task(c_tasks + {start} + t); "
                f"{_table_call(kind)} }}  // {level_note}{kind}")

    if stage == 0:
        TP = build_tabplan(process, bool(amputated & 1))
        P = TP.plan
        npar = P.npar
        size, table_flops = TP.size, TP.table_flops()
        rounds_code, prev = [], None
        for r in TP.rounds:
            if prev is not None and r.level != prev:
                rounds_code.append("__syncthreads();")
            prev = r.level
            rounds_code.append(round_code(r.kind, [(t.out, t.ins, t.lines) for t in r.tasks], f"level {r.level}: "))
        addr = lambda a: f"{TP.base[a]} + {_support_name(TP.support[a])}"
        group_of, sign_of, group_terms, members = colour_groups(P)
        if amputated & 2:  # no colour groups
            members = [[a] for a in range(len(P.amps))]
        order = [a for m in members for a in m]
        flush = {m[-1]: group_terms[group_of[m[-1]]] for m in members}
        items = [(pi, f, l) for pi, (f, l) in zip(order, _group_positions(order, flush))]
        acode, _, saved = _amp_run_code(P, items, addr, 0, sign_of, flush, not amputated & 4)
        used = {TP.support[a] for ai, _ in P.amps for a in P.ops[ai].args}
        body = f"""
    static constexpr bool STAGED = false;
    template <class T>
    __device__ static __forceinline__ void tables(const TabRef<T, TAB>& tab, const Ln<T>* __restrict__ ln, T mt, int tid)
    {{
        (void)mt;
{NL.join("        " + x for x in rounds_code)}
    }}

    template <class T, bool SDE, class JT>
    __device__ static __forceinline__ void amps(const TabRef<T, TAB>& tab, int h, const Ln<T>* __restrict__ ln, JT& J,
                                                SdeAcc<T>& sde)
    {{
        (void)sde;
{NL.join("        " + x for x in _variant_code(npar, used))}
{NL.join("        " + x for x in acode)}
    }}"""
    else:
        I = build_interp(process, stage, bool(amputated & 1), not amputated & 2)
        TP = I.tab
        P = TP.plan
        npar = P.npar
        if nt < (1 << npar):
            raise ValueError("the staged table kernel takes every helicity in one pass: NT >= 2^npar")
        size, table_flops = I.table_size, I.table_flops
        ops = P.ops
        is_obj = lambda x: ops[x].out != "A" and not ops[x].kind.startswith("ext_")
        addr = lambda a: f"{I.slot[a] if is_obj(a) else 2 * ops[a].ext} + {_support_name(TP.support[a])}"
        code, n_amp = [], 0
        pos = dict(zip(I.amp_order, _group_positions(I.amp_order, I.flush)))
        for si, st in enumerate(I.stages):
            code.append(f"// stage {si}: {sum(len(t) for _, t in st.rounds)} table tasks, {len(st.amps)} amplitudes")
            for ri, (kind, tl) in enumerate(st.rounds):
                code.append(round_code(kind, tl, ""))
                if ri in st.barriers:
                    code.append("__syncthreads();")
            code.append("__syncthreads();")
            run_code, n_amp, sv = _amp_run_code(P, [(ai, *pos[ai]) for ai in st.amps], addr, n_amp, I.sign,
                                                I.flush, not amputated & 4)
            saved += sv
            code += run_code
            code.append("__syncthreads();  // the stage's dead slots are reused by the next one")
        used = {TP.support[a] for ai, _ in P.amps for a in ops[ai].args}
        body = f"""
    static constexpr bool STAGED = true;
    // every stage in order; all threads of the CTA call it (CTA barriers inside)
    template <class T, bool SDE, class JT>
    __device__ static __forceinline__ void staged(const TabRef<T, TAB>& tab, const Ln<T>* __restrict__ ln, T mt, int tid,
                                                  int h, JT& J, SdeAcc<T>& sde)
    {{
        (void)mt;
        (void)sde;
{NL.join("        " + x for x in _variant_code(npar, used))}
{NL.join("        " + x for x in code)}
    }}"""

    amp_flops = TP.amplitude_flops_per_helicity(not amputated & 2) - saved
    task_init = ",\n    ".join("{%d, %d, %d, %d, %d, %d, %d, 0, 0}" % t for t in tasks)
    desc = (f"{'staged (' + str(stage) + ' amplitudes per stage)' if stage else 'resident'}"
            f"{', amputated vertex objects' if amputated & 1 else ''}{'' if amputated & 2 else ', colour groups'}")
    src = f"""
__device__ const TabTask c_tasks[{max(len(tasks), 1)}] = {{
    {task_init if tasks else "{0, 0, 0, 0, 0, 0, 0, 0, 0}"}
}};

// helicity-recycled evaluation, {desc}: {size} table entries, {len(tasks)} table tasks,
// {table_flops} table flops per event, {amp_flops} amplitude flops per helicity
struct ProcTab : Proc {{
    static constexpr int NT = {nt}, TAB = {(size + 7) // 8 * 8};
    // events per CTA (own shared-memory region each; CTA barriers keep their
    // warps at the same point of the code), in FP32 / mixed and in FP64
    static constexpr int EPC_F = {epc_f}, EPC_D = {epc_d};
    // register budget: FP32 <= 128 per thread (occupancy bound by shared memory
    // anyway), FP64 <= 255 (its tables are twice as large)
    static constexpr int MIN_CTAS_F = {max(1, 65536 // (nt * epc_f * 128))}, MIN_CTAS_D = {max(1, 65536 // (nt * epc_d * 255))};
    static constexpr bool IS_TAB = true, IS_INTERP = false;
    static constexpr long long TABLE_FLOPS = {table_flops}LL, AMP_FLOPS = {amp_flops}LL;
    // warp fence every n amplitudes (FP32, FP64)
    static constexpr int FENCE_F = {fence_f}, FENCE_D = {fence_d};
    // helicities that can be non-zero; the others are exactly 0 and the table
    // variants only they would read are not computed
    __device__ static __forceinline__ bool hel_allowed(int h) {{ (void)h; return {_allowed_expr(TP)}; }}
{body}
}};
"""
    return src, TP, table_flops, amp_flops


NL = "\n"


# uniform descriptors of the staged descriptor kernel in constant memory (build
# option ME_INTERP_CONST=0 keeps them in global memory)
CONST_DESCRIPTORS = __import__("os").environ.get("ME_INTERP_CONST", "1") != "0"
# accumulator slots per thread for the colour windows of the staged descriptor


# shared memory of the FP32 descriptor kernel with J in tensor memory, two CTAs
# per SM (me_kernel_interp.cuh InterpLayout): 228 KB per SM, per CTA 1 KB
# reserved and up to 1.5 KB of static arrays; after the table the six A
# operands (4352 bytes each, 1 KB-aligned start) and B (4096 bytes)
SMEM_PER_SM, SMEM_CTA_RESERVED, INTERP_STATIC_SMEM = 233472, 1024, 1536
INTERP_OPERAND_BYTES = 6 * 4352 + 4096


def _interp_table_cap(process: str, nt: int) -> int:
    """most table entries (FP32 wavefunctions, 32 bytes) that keep two CTAs of
    the descriptor kernel resident per SM"""
    P = build_plan(process)
    npar, nl = P.npar, len(P.lines)
    from .interp import build_interp as _bi  # supports of the default schedule bound NSUP
    nsup = len(_bi(process, INTERP_PROCESSES.get(process, (0, 16))[1]).supports)
    a16 = lambda x: (x + 15) // 16 * 16
    table_off = a16(a16(npar * 4 * 8 * 2 + npar * (npar + 1) // 2 * 8 + nl * 20) + nsup * nt)
    dyn = SMEM_PER_SM // 2 - SMEM_CTA_RESERVED - INTERP_STATIC_SMEM
    jsm_max = (dyn - INTERP_OPERAND_BYTES) // 1024 * 1024
    return (jsm_max - table_off) // 32 // 8 * 8


def _pair_heads(kinds, mid):
    """positions i of a stage's amplitude list whose amplitude is evaluated
    together with amplitude i + 1 (descriptor flag AMP_PAIR): greedily, where
    both have the same kind and lie on the same side of the split at `mid`"""
    heads, i = set(), 0
    while i + 1 < len(kinds):
        if kinds[i] == kinds[i + 1] and (i + 1 < mid or i >= mid):
            heads.add(i)
            i += 2
        else:
            i += 1
    return heads


def emit_interp_struct(process: str, nt: int, stage_amps: int, num, mode: int = 0,
                       name: str = "ProcInterp", prefix: str = ""):
    """ProcInterp: staged table tasks, amplitude descriptors, colour terms
    (arrays named with `prefix`, struct `name`)."""
    amputated = bool(mode & 1)
    I = build_interp(process, stage_amps, amputated, not mode & 2, bool(mode & 8),
                     _interp_table_cap(process, nt) if mode & 8 else None)
    T = I.tab
    P = T.plan
    npar = P.npar
    ops = P.ops
    tasks, rounds, stages, amps, terms, stage_term, diags = [], [], [], [], [], [], []
    # per stage, the colour-group updates as a tensor-core operand (J accumulated
    # by tcgen05.mma in FP32 kernels): B[n][k] = sigma of flow n in the stage's
    # k-th group update, where that update adds -i G (sigma = +1) or +i G
    # (sigma = -1) to J_n; Re J += Im G . B and Im J += Re G . (-B).  BF16
    # +-1 / 0 in the K-major core-matrix layout of a 128 x 16 operand
    # (me_tmem.cuh: umma_k16_offset), one 4096-byte image per stage.
    bmat, maxflush = [], 0
    for st in I.stages:
        r0 = len(rounds)
        for ri, (kind, tl) in enumerate(st.rounds):
            rounds.append((len(tasks), len(tl), ROUTINES.index(kind), 1 if ri in st.barriers else 0))
            for out, ins, ln in tl:
                ins = list(ins) + [0] * (3 - len(ins))
                tasks.append((out, ins[0], ins[1], ins[2], ln[0], ln[1], ln[2]))
        a0 = len(amps)
        stage_term.append(len(terms))
        sup_index = {S: i for i, S in enumerate(I.supports)}
        heads = _pair_heads([ops[P.amps[ai][0]].kind for ai in st.amps], st.mid)
        for pos, ai in enumerate(st.amps):
            aop, coefs = P.amps[ai]
            op = ops[aop]
            bases, sups = [], []
            for x in op.args:
                base = I.slot[x] if (ops[x].out != "A" and not ops[x].kind.startswith("ext_")) else 2 * ops[x].ext
                bases.append(base)
                sups.append(sup_index[T.support[x]])
            while len(bases) < 4:
                bases.append(0)
                sups.append(0)
            la, lb = (op.mom if op.kind == "VVV1_0" else (0, 0))
            diags.append(P.amp_diag[ai])
            # colour group: the amplitude enters the group sum with its sign
            # (kind bit 7 = minus); the group's last member carries the terms
            gterms = I.flush.get(ai, ())
            assert len(op.args) <= 4 and len(gterms) < 256 and all(c in ((0, 1), (0, -1)) for _, c in coefs + gterms)
            kind = AMP_KINDS.index(op.kind) | (0x80 if I.sign[ai] < 0 else 0) | (0x40 if pos in heads else 0)
            amps.append((bases, sups, kind, la, lb, len(gterms)))
            for col, c in gterms:
                terms.append(col | (0x8000 if c == (0, -1) else 0))
        img = [0] * 2048   # BF16 halves of one stage's 128 x 16 operand
        flushes = [ai for ai in st.amps if ai in I.flush]
        maxflush = max(maxflush, len(flushes))
        for k, ai in enumerate(flushes[:16]):
            for col, c in I.flush[ai]:
                assert col < 128
                img[umma_k16_offset(col, k) // 2] = 0x3F80 if c == (0, -1) else 0xBF80
        bmat += [img[i] | (img[i + 1] << 16) for i in range(0, 2048, 2)]
        term_mid = sum(len(I.flush[ai]) for ai in st.amps[:st.mid] if ai in I.flush)
        stages.append((r0, len(rounds), a0, len(amps), a0 + st.mid, st.slot_mid, int(st.ahead), term_mid))
    masks = []
    for S in I.supports:
        m = 0
        for p in S:
            m |= 1 << (npar - 1 - p)
        masks.append(m)
    n = len(num)
    cnum2 = [num[i][j] * (1 if i == j else 2) if j >= i else 0 for i in range(n) for j in range(n)]

    # the descriptors every thread of a CTA reads at the same index (rounds,
    # stages, amplitudes, colour terms, diagrams) go to constant memory when they
    # fit its 64 KB (uniform reads through the constant cache), for the first
    # struct of the unit only; per-thread data (table tasks) stays in global memory
    uniform = ("c_rounds", "c_stages", "c_amps", "c_terms", "c_stage_term", "c_diag")
    cbytes = 8 * len(rounds) + 16 * len(stages) + 16 * len(amps) + 2 * len(terms) + 4 * len(stage_term) + 2 * len(diags)
    use_const = CONST_DESCRIPTORS and not prefix and cbytes <= 60 * 1024

    def arr(aname, ctype, rows, fmt, per_line=6):
        body = ",\n    ".join(", ".join(fmt(x) for x in rows[i:i + per_line]) for i in range(0, len(rows), per_line))
        space = "__constant__" if use_const and aname in uniform else "__device__ const"
        return f"{space} {ctype} {prefix}{aname}[{max(len(rows), 1)}] = {{\n    {body if rows else '0'}\n}};\n"

    def rd(aname, index):  # read of a descriptor array
        return f"{prefix}{aname}[{index}]" if use_const and aname in uniform else f"__ldg({prefix}{aname} + {index})"

    src = ""
    src += arr("c_itasks", "TabTask", tasks, lambda t: "{%d, %d, %d, %d, %d, %d, %d, 0, 0}" % t, 4)
    src += arr("c_rounds", "IRound", rounds, lambda r: "{%du, %d, %d, %d}" % r, 8)
    src += arr("c_stages", "IStage", stages, lambda r: "{%d, %d, %d, %d, %d, %d, %d, %d}" % r, 4)
    src += arr("c_amps", "IAmp", amps, lambda a: "{{%d, %d, %d, %d}, {%d, %d, %d, %d}, %d, %d, %d, %d}" % (
        *a[0], *a[1], a[2], a[3], a[4], a[5]), 3)
    src += arr("c_terms", "unsigned short", terms, lambda x: "%d" % x, 16)
    src += arr("c_stage_term", "int", stage_term, lambda x: "%d" % x, 16)
    src += (f"__device__ __align__(128) const unsigned int {prefix}c_bmat[{len(bmat)}] = {{\n    "
            + ",\n    ".join(", ".join("%du" % x for x in bmat[i:i + 12]) for i in range(0, len(bmat), 12)) + "\n};\n")
    src += arr("c_supmask", "unsigned short", masks, lambda x: "%d" % x, 16)
    src += arr("c_cnum2", "short", cnum2, lambda x: "%d" % x, 24)
    src += arr("c_diag", "unsigned short", diags, lambda x: "%d" % x, 16)
    src += f"""
// staged evaluation{' with amputated vertex objects' if amputated else ''}: {len(I.stages)} stages of <= {stage_amps} amplitudes, table peak {I.table_size} entries,
// {len(tasks)} table tasks ({I.table_flops} flops per event), {len(terms)} colour terms
struct {name} : Proc {{
    static constexpr int NT = {nt}, TAB = {(I.table_size + 7) // 8 * 8}, NSUP = {len(I.supports)}, NSTAGE = {len(I.stages)};
    static constexpr bool IS_TAB = false, IS_INTERP = true;
    // table objects of stage s + 1 computed beside the amplitudes of stage s
    // (slots reused two stages after their last reader)
    static constexpr bool TABLE_AHEAD = {"true" if I.ahead else "false"};
    static constexpr long long TABLE_FLOPS = {I.table_flops}LL, AMP_FLOPS = {T.amplitude_flops_per_helicity(not mode & 2)}LL;
    __device__ static __forceinline__ const TabTask* tasks() {{ return {prefix}c_itasks; }}
    __device__ static __forceinline__ IRound round(int r) {{ return {prefix}c_rounds[r]; }}
    __device__ static __forceinline__ IStage stage(int s) {{ return {prefix}c_stages[s]; }}
    __device__ static __forceinline__ IAmp amp(int a) {{ return {prefix}c_amps[a]; }}
    __device__ static __forceinline__ unsigned short term(int t) {{ return {rd("c_terms", "t")}; }}
    __device__ static __forceinline__ int stage_term_begin(int s) {{ return {prefix}c_stage_term[s]; }}
    // colour-group updates per stage as tensor-core operands (4096 bytes each);
    // most group updates in one stage (the tensor-core path takes at most 16)
    static constexpr int MAXFLUSH = {maxflush};
    __device__ static __forceinline__ const uint4* bmat(int s) {{ return reinterpret_cast<const uint4*>({prefix}c_bmat) + 256 * s; }}
    __device__ static __forceinline__ unsigned support_mask(int s) {{ return {prefix}c_supmask[s]; }}
    __device__ static __forceinline__ int cnum2(int i, int j) {{ return __ldg({prefix}c_cnum2 + i * NCOL + j); }}
    __device__ static __forceinline__ int diag(int a) {{ return {rd("c_diag", "a")}; }}
}};
"""
    return src, I


PROCESSES = ("ee_mumu", "gg_ttx", "gg_ttxg", "gg_ttxgg", "gg_ttxggg") + tuple(DY_PROCESSES)


def emit_registry(processes=PROCESSES) -> str:
    decls = "\n".join(f"const ProcDesc* procdesc_{p}();" for p in processes)
    checks = "\n".join(
        f'    if (std::strcmp(name, "{p}") == 0) return procdesc_{p}();' for p in processes)
    return f"""// Generated by paper_2507_21039_gb300/gen/emit.py: process registry.
#include <cstring>
#include "me_proc.h"

namespace me {{
{decls}

const ProcDesc* find_process(const char* name)
{{
    if (!name) return nullptr;
{checks}
    return nullptr;
}}
}}  // namespace me
"""
