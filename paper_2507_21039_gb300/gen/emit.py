"""Emit one CUDA translation unit per process from its evaluation plan.

The unit holds: the external-particle and line tables (__constant__), a
straight-line chain routine templated on the amplitude precision (every
wavefunction a named local, so nvcc keeps them in registers), the colour
quadratic form with the integer numerators as immediates, the launchers of
the three precision modes, and a process descriptor for the C ABI.
"""
from __future__ import annotations

import math

from .colour import colour_matrix
from .plan import Plan, build_plan

EXT_KINDS = {"VIN": 0, "VOUT": 1, "FO_U": 2, "FO_V": 3, "FI_U": 4, "FI_V": 5}
CHUNK_ROUTINES = ()


def _ext_table(process: str):
    if process == "ee_mumu":
        # e-(in) u, e+(in) vbar, mu-(out) ubar, mu+(out) v; massless
        return ["FI_U", "FO_V", "FO_U", "FI_V"], [0, 0, 0, 0]
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


def _coef_call(col, c, var):
    return f"jacc<{c[0]}, {c[1]}, T>(J[{col}], {var});"


def emit_process(process: str) -> tuple[str, dict]:
    P = build_plan(process)
    npar = P.npar
    ncol = P.ncol
    k = len(P.gluon_ext)
    kinds, massive = _ext_table(process)
    plus, minus, lkind = _line_tables(P)
    if process == "ee_mumu":
        num, den = [[1]], 1
        iden, cpow = 4.0, 2
    else:
        num, den = colour_matrix(k)
        iden, cpow = 4.0 * 64.0 * math.factorial(k - 2), k
    j_smem = ncol > 32
    threads = 64 if j_smem else 128
    nlines = len(P.lines)

    body = []
    for i, op in enumerate(P.ops):
        a = [f"w{x}" for x in op.args]
        kd = op.kind
        if kd.startswith("ext_"):
            e = op.ext
            body.append(f"const Wf<T>& w{i} = ext[{2 * e} + ((hel >> {npar - 1 - e}) & 1)];")
        elif kd == "VVV1P0_1":
            la, lb = op.mom
            body.append(f"Wf<T> w{i}; VVV1P0_1<T>({a[0]}, ln[{la}].p, {a[1]}, ln[{lb}].p, ln[{op.line}].inv, w{i});")
        elif kd.endswith("P0_1"):
            body.append(f"Wf<T> w{i}; {kd}<T>({a[0]}, {a[1]}, {a[2]}, ln[{op.line}].inv, w{i});")
        elif kd in ("FFV1_2", "FFV1_1"):
            body.append(f"Wf<T> w{i}; {kd}<T>({a[0]}, {a[1]}, ln[{op.line}], mt, w{i});")
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

    ns = f"p_{process}"
    cnum_flat = ", ".join(str(x) for row in num for x in row)
    src = f"""// Generated by paper_2507_21039_gb300/gen/emit.py for {process}: do not edit.
// {P.ndiagrams} Feynman diagrams, {len(P.amps)} amplitudes, {len(P.ops)} routine calls,
// {ncol} colour flows, {nlines} lines, {P.flops_per_helicity()} chain flops per helicity.
#include "me_kernel.cuh"
#include "me_colour_tc.cuh"

namespace me {{
namespace {ns} {{

__constant__ unsigned char c_ext_kind[{npar}] = {{{", ".join(str(EXT_KINDS[x]) for x in kinds)}}};
__constant__ unsigned char c_ext_massive[{npar}] = {{{", ".join(str(x) for x in massive)}}};
__constant__ unsigned short c_line_plus[{nlines}] = {{{", ".join(str(x) for x in plus)}}};
__constant__ unsigned short c_line_minus[{nlines}] = {{{", ".join(str(x) for x in minus)}}};
__constant__ unsigned char c_line_kind[{nlines}] = {{{", ".join(str(x) for x in lkind)}}};
static const int h_cnum[{ncol * ncol}] = {{{cnum_flat}}};

struct Proc {{
    static constexpr int NPAR = {npar}, NCOL = {ncol}, NLINES = {nlines}, THREADS = {threads};
    static constexpr int CDEN = {den};
    static constexpr bool J_SMEM = {"true" if j_smem else "false"};
    __device__ static __forceinline__ unsigned ext_kind(int e) {{ return c_ext_kind[e]; }}
    __device__ static __forceinline__ unsigned ext_massive(int e) {{ return c_ext_massive[e]; }}
    __device__ static __forceinline__ unsigned line_plus(int l) {{ return c_line_plus[l]; }}
    __device__ static __forceinline__ unsigned line_minus(int l) {{ return c_line_minus[l]; }}
    __device__ static __forceinline__ unsigned line_kind(int l) {{ return c_line_kind[l]; }}

    template <class T, class JT>
    __device__ static __forceinline__ void chain(const Wf<T>* __restrict__ ext, int hel, const Ln<T>* __restrict__ ln,
                                                 T mt, JT& J)
    {{
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

static cudaError_t launch(int precision, const LaunchArgs& a)
{{
    switch (precision) {{
    case PREC_FP64: return launch_scalar<Proc, double>(a);
    case PREC_FP32: return launch_scalar<Proc, float>(a);
    case PREC_MIXED: return launch_mixed<Proc>(a);
    default: return cudaErrorInvalidValue;
    }}
}}

}}  // namespace {ns}

const ProcDesc* procdesc_{process}()
{{
    static const ProcDesc d = {{"{process}", {npar}, {1 << npar}, {ncol}, {P.ndiagrams}, {len(P.amps)}, {k}, {nlines},
                               {threads}, {iden!r}, {den}, {ns}::h_cnum, {P.flops_per_helicity()}LL,
                               {P.colour_flops_per_helicity()}LL, {cpow}, &{ns}::launch}};
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
        "flops_per_helicity": P.flops_per_helicity(),
        "colour_flops_per_helicity": P.colour_flops_per_helicity(),
        "counts": P.counts(),
        "cden": den,
    }
    return src, meta


PROCESSES = ("ee_mumu", "gg_ttx", "gg_ttxg", "gg_ttxgg", "gg_ttxggg")


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
