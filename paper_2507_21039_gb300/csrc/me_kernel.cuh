// Batched |M|^2 kernel template (arXiv:2507.21039 Sec. 3.1: per event, the
// helicity-amplitude chain for every good helicity, the colour sum J^+ C J and
// the helicity sum).
//
// Work layout (GB300-first, not the paper's event-per-thread layout):
//   * a CTA owns E = THREADS / S consecutive events; S lanes (a power of two,
//     <= 32) share one event and split its good helicities between them, so the
//     helicity sum is a warp-shuffle reduction inside an S-lane segment;
//   * the CTA loads its events' momenta ([nevt][npar][4] FP64, contiguous) with
//     16-byte coalesced loads into shared memory;
//   * everything that does not depend on the helicity -- the external
//     wavefunctions for both helicities of every particle, every line's
//     momentum and propagator denominator p^2 - m^2 -- is computed once per
//     event in FP64 by the CTA's threads and kept in shared memory (rounded to
//     the amplitude precision T); FP64 work per (event, helicity) is zero;
//   * each lane runs the generated straight-line chain with its wavefunctions
//     and the colour-flow vector J in registers (or J in shared memory for the
//     120-flow basis), then the colour quadratic form, accumulating |M_h|^2 in
//     FP64.
#pragma once
#include <type_traits>

#include "helas.cuh"
#include "me_proc.h"
#include "me_split.h"

namespace me {

enum ExtKind : unsigned char { VIN = 0, VOUT = 1, FO_U = 2, FO_V = 3, FI_U = 4, FI_V = 5 };
enum LineKind : unsigned char { L_EXT = 0, L_MASSLESS = 1, L_MASSIVE = 2 };

// shared-memory bytes for E events of process P at precision T (+ J storage)
// Straight-line kernel, per CTA of E events: FP64 momenta, external states
// (and the Drell-Yan coefficients), lines; for T = float also the momenta split
// into FP32 hi + lo and the FP64 Gram matrix of the FP32 setup (see below)
template <class P, class T> __host__ __device__ constexpr size_t scalar_line_offset(int E)
{
    return (size_t)E * P::NPAR * 4 * sizeof(double) + (size_t)E * P::NEXT * sizeof(Wf<T>);
}
template <class P, class T> __host__ __device__ constexpr size_t scalar_pf_offset(int E)
{
    return (scalar_line_offset<P, T>(E) + (size_t)E * P::NLINES * sizeof(Ln<T>) + 15) / 16 * 16;
}
template <class P, class T> __host__ __device__ constexpr size_t scalar_gram_offset(int E)
{
    return scalar_pf_offset<P, T>(E) + (std::is_same<T, float>::value ? (size_t)E * P::NPAR * 4 * sizeof(float2) : 0);
}
template <class P, class T> __host__ __device__ constexpr size_t setup_bytes(int E)
{
    return (scalar_gram_offset<P, T>(E) +
            (std::is_same<T, float>::value ? (size_t)E * (P::NPAR * (P::NPAR + 1) / 2) * sizeof(double) : 0) + 15) /
           16 * 16;
}

// Single-diagram enhancement (the multi-channel weight of the paper's event
// generation): per thread, |x|^2 of every amplitude x into den and of the
// chosen diagram's amplitudes into num, summed over the thread's helicities.
// The generated amplitude code calls ME_SDE after each amplitude; it compiles
// to nothing unless the kernel's SDE flag is set.
template <class T> struct SdeAcc {
    T num, den;
    int chan;
};
#define ME_SDE(x, d)                                            \
    do {                                                        \
        if constexpr (SDE) {                                    \
            const auto sde_w2 = fma((x).re, (x).re, (x).im * (x).im); \
            sde.den += sde_w2;                                  \
            if ((d) == sde.chan) sde.num += sde_w2;             \
        }                                                       \
    } while (0)

// Strided shared-memory accumulator for a per-thread J (column-major over the CTA)
template <class T, int STRIDE> struct JSmem {
    cx<T>* base;
    __device__ __forceinline__ cx<T>& operator[](int c) const { return base[c * STRIDE]; }
};

// External wavefunction of particle e with helicity bit b from its momentum pe
// and mass m, both in the amplitude precision T
template <class P, class T>
__device__ __forceinline__ Wf<T> ext_wavefunction_at(const T (&pe)[4], int e, int b, T m, int gauge_ext)
{
    const int lam = b ? 1 : -1;
    Wf<T> o;
    if (e == gauge_ext) {  // diagnostic: gluon polarisation replaced by its momentum
        for (int mu = 0; mu < 4; ++mu) o.c[mu] = {pe[mu], T(0)};
        return o;
    }
    switch (P::ext_kind(e)) {
    case VIN: vxxxxx<T>(pe, lam, -1, o.c); break;
    case VOUT: vxxxxx<T>(pe, lam, +1, o.c); break;
    case FO_U: oxxxxx<T>(pe, m, lam, +1, o.c); break;
    case FO_V: oxxxxx<T>(pe, m, lam, -1, o.c); break;
    case FI_U: ixxxxx<T>(pe, m, lam, +1, o.c); break;
    default: ixxxxx<T>(pe, m, lam, -1, o.c); break;
    }
    return o;
}

// External wavefunction `item` = 2 e + b (particle e, helicity bit b), computed
// in the amplitude precision T from the FP64 momenta
template <class P, class T>
__device__ __forceinline__ Wf<T> ext_wavefunction(const double* __restrict__ p, int item, double mt, int gauge_ext)
{
    const int e = item >> 1;
    T pe[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) pe[mu] = (T)p[4 * e + mu];
    return ext_wavefunction_at<P, T>(pe, e, item & 1, P::ext_massive(e) ? (T)mt : T(0), gauge_ext);
}

// Line l: momentum (signed sum of external momenta, FP64) and 1/(p^2 - m^2)
template <class P, class T> __device__ __forceinline__ Ln<T> line_data(const double* __restrict__ p, int l, double mt)
{
    const unsigned plus = P::line_plus(l), minus = P::line_minus(l);
    double q[4] = {0.0, 0.0, 0.0, 0.0};
    for (int e = 0; e < P::NPAR; ++e) {
        const double s = ((plus >> e) & 1) ? 1.0 : (((minus >> e) & 1) ? -1.0 : 0.0);
        if (s != 0.0)
            for (int mu = 0; mu < 4; ++mu) q[mu] += s * p[4 * e + mu];
    }
    const unsigned kind = P::line_kind(l);
    Ln<T> o;
    o.inv = T(0);
    if (kind != L_EXT) {
        // the denominator p^2 - m^2 in FP64: its cancellation near collinear
        // and soft limits is what FP32 cannot resolve; once formed, rounding it
        // to T keeps T's relative precision, so the reciprocal is taken in T
        const double m2 = kind == L_MASSIVE ? mt * mt : 0.0;
        const double d = q[0] * q[0] - q[1] * q[1] - q[2] * q[2] - q[3] * q[3] - m2;
        o.inv = T(1) / (T)d;
    }
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) o.p[mu] = (T)q[mu];
    return o;
}

// ---------------------------------------------------------------------------
// FP32 kernels: per-event FP64 work only where cancellation needs it.
//
// GB300 runs FP64 at 1/64 of the FP32 rate.  In the FP32 and mixed kernels the
// per-event setup therefore keeps FP64 for the propagator denominators p^2 - m^2
// alone, and forms them from few FP64 instructions:
//   * every momentum component is split once into FP32 hi + lo (p = hi + lo to
//     2^-47 relative: by conversions in the table kernels, by integer operations
//     on the bit pattern in the straight-line kernels, see split_or_gram).  hi
//     feeds the external wavefunctions; each line momentum is a
//     compensated FP32 sum of the hi and lo parts (the rounding of every hi
//     addition is recovered exactly and added back), i.e. the FP32 rounding of
//     its FP64 value up to the last bit;
//   * the Gram matrix p_i.p_j (i <= j) is formed once per event in FP64, and a
//     line's p^2 - m^2 is the FP64 sum of c_a c_b p_a.p_b over the particles of
//     the line's shorter side (at most three for up to seven particles: six
//     FP64 fused multiply-adds), which is the same quantity as the square of the
//     FP64 momentum sum, rounded differently.
// ---------------------------------------------------------------------------
template <int NPAR> struct Gram {
    static constexpr int N = NPAR * (NPAR + 1) / 2;
    // entry of p_i.p_j for i <= j (rows of the upper triangle)
    __host__ __device__ static constexpr int idx(int i, int j) { return i * NPAR - i * (i - 1) / 2 + (j - i); }
};

// setup item `it` of the first phase: it < 4 NPAR splits momentum component it
// into pf[it] = {hi, lo}; otherwise the Gram entry it - 4 NPAR (row order).
// INT_SPLIT: by integer operations on the bit pattern (me_split.h: no FP64-pipe
// work, about twenty integer instructions), for kernels bound by the FP64 pipe;
// otherwise by conversions (hi the FP32 rounding of p, lo that of the
// remainder: three conversions and one FP64 add, fewer issue slots), for the
// issue-bound table kernels (measured: the integer split cost gg -> t t~ g g
// 2.6%, and gained e+ e- -> mu+ mu- 22%, u u~ -> e+ e- g 12%)
template <int NPAR, bool INT_SPLIT = false>
__device__ __forceinline__ void split_or_gram(const double* __restrict__ p, int it, float2* __restrict__ pf,
                                              double* __restrict__ gram)
{
    if (it < 4 * NPAR) {
        const double x = p[it];
        float hi, lo;
        if constexpr (INT_SPLIT) {
            split_f32(x, hi, lo);
        } else {
            hi = __double2float_rn(x);
            lo = __double2float_rn(x - (double)hi);
        }
        pf[it] = make_float2(hi, lo);
    } else {
        int k = it - 4 * NPAR, i = 0;
        while (k >= NPAR - i) {
            k -= NPAR - i;
            ++i;
        }
        const double* a = p + 4 * i;
        const double* b = p + 4 * (i + k);
        gram[it - 4 * NPAR] = fma(-a[3], b[3], fma(-a[2], b[2], fma(-a[1], b[1], a[0] * b[0])));
    }
}

// Line l in FP32 from the split momenta and the FP64 Gram matrix (m2 = mt^2)
template <class P>
__device__ __forceinline__ Ln<float> line_data_split(const float2* __restrict__ pf, const double* __restrict__ gram,
                                                     int l, double m2)
{
    constexpr int S = P::SIDE;
    const unsigned sd = P::line_side(l);
    const int k = (int)(sd & 7u);
    int id[S];
    float sf[S];
#pragma unroll
    for (int a = 0; a < S; ++a) {  // terms past k: particle 0 with coefficient 0
        const unsigned t = sd >> (4 * a + 4);
        id[a] = a < k ? (int)(t & 7u) : 0;
        sf[a] = a < k ? ((t & 8u) ? -1.0f : 1.0f) : 0.0f;
    }
    Ln<float> o;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        float s = 0.0f, c = 0.0f;
#pragma unroll
        for (int a = 0; a < S; ++a) {
            const float2 v = pf[4 * id[a] + mu];
            const float x = sf[a] * v.x;          // exact (a sign or zero)
            const float t = s + x;                // two-sum: s + x = t + err exactly
            const float z = t - s;
            c += ((s - (t - z)) + (x - z)) + sf[a] * v.y;
            s = t;
        }
        o.p[mu] = s + c;
    }
    o.inv = 0.0f;
    const unsigned kind = P::line_kind(l);
    if (kind != L_EXT) {
        double d = kind == L_MASSIVE ? -m2 : 0.0;
#pragma unroll
        for (int a = 0; a < S; ++a)
#pragma unroll
            for (int b = a; b < S; ++b) {
                const bool neg = ((sd >> (4 * a + 4)) ^ (sd >> (4 * b + 4))) & 8u;
                const double cab = b < k ? (a == b ? 1.0 : (neg ? -2.0 : 2.0)) : 0.0;
                const int i = min(id[a], id[b]), j = max(id[a], id[b]);
                d = fma(cab, gram[Gram<P::NPAR>::idx(i, j)], d);
            }
        o.inv = 1.0f / __double2float_rn(d);
    }
    return o;
}

// External wavefunction `item` = 2 e + b in FP32 from the split momenta
template <class P>
__device__ __forceinline__ Wf<float> ext_wavefunction_split(const float2* __restrict__ pf, int item, float mt,
                                                            int gauge_ext)
{
    const int e = item >> 1;
    float pe[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) pe[mu] = pf[4 * e + mu].x;
    return ext_wavefunction_at<P, float>(pe, e, item & 1, P::ext_massive(e) ? mt : 0.0f, gauge_ext);
}

// Item of the first setup phase taken by thread tid of an NT-thread event group
// in a single pass: splits on the first warp, Gram entries on the second, so
// that neither warp diverges between the two; -1 = none.  Groups of one warp
// loop over all items instead (split_items_one_pass false).
template <int NPAR, int NT> __host__ __device__ constexpr bool split_items_one_pass()
{
    return NT >= 64 && 4 * NPAR <= 32 && Gram<NPAR>::N <= NT - 32;
}
template <int NPAR> __device__ __forceinline__ int split_item_of(int tid)
{
    if (tid < 32) return tid < 4 * NPAR ? tid : -1;
    return tid - 32 < Gram<NPAR>::N ? 4 * NPAR + tid - 32 : -1;
}

// Compensated FP32 sum (s + c): the helicity sum of the FP32 kernels, formed
// without FP64 until the per-event total
struct FSum {
    float s, c;
};
__device__ __forceinline__ FSum fsum_add(FSum a, FSum b)
{
    const float t = a.s + b.s;
    const float z = t - a.s;
    return {t, a.c + b.c + ((a.s - (t - z)) + (b.s - z))};
}
// over aligned groups of W lanes (W a power of two <= 32; 32: the whole warp)
template <int W = 32> __device__ __forceinline__ FSum fsum_warp(FSum v)
{
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) {
        const FSum o{__shfl_xor_sync(0xffffffffu, v.s, off), __shfl_xor_sync(0xffffffffu, v.c, off)};
        v = fsum_add(v, o);
    }
    return v;
}

// Drell-Yan electroweak parameters (reading R15: G_F-scheme values, fixed
// widths; couplings -i gamma^mu (gL P_L + gR P_R), photon gL = gR = e Q, Z
// gL = e (T3 - Q sw^2) / (sw cw), gR = -e Q sw^2 / (sw cw))
constexpr double kDyAlpha = 1.0 / 132.507, kDyMZ = 91.188, kDyWZ = 2.441404, kDyMW = 80.419002;

// The four electroweak coefficients of the Drell-Yan insertion for the event's
// lepton pair (particles 2 = e+, 3 = e-), in FP64 and rounded to T:
//   c[0] = sum_V gL^u gL^e / D_V,  c[1] = sum_V gL^u gR^e / D_V,
//   c[2] = sum_V gR^u gL^e / D_V,  c[3] = sum_V gR^u gR^e / D_V,
// D_photon = s, D_Z = s - M_Z^2 + i M_Z Gamma_Z, s = (p_e+ + p_e-)^2
template <class T> __device__ __forceinline__ Wf<T> ew_coefficients(const double* __restrict__ p)
{
    double q[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) q[mu] = p[8 + mu] + p[12 + mu];
    const double s = q[0] * q[0] - q[1] * q[1] - q[2] * q[2] - q[3] * q[3];
    const double e = sqrt(4.0 * M_PI * kDyAlpha);
    const double cw = kDyMW / kDyMZ, sw = sqrt(1.0 - cw * cw), swcw = sw * cw;
    // couplings [boson][L/R]: u quark (Q = 2/3, T3 = 1/2) and electron (Q = -1, T3 = -1/2)
    const double gu[2][2] = {{e * 2.0 / 3.0, e * 2.0 / 3.0},
                             {e * (0.5 - 2.0 / 3.0 * sw * sw) / swcw, -e * 2.0 / 3.0 * sw * sw / swcw}};
    const double ge[2][2] = {{-e, -e}, {e * (-0.5 + sw * sw) / swcw, e * sw * sw / swcw}};
    // 1 / D_V: photon 1/s; Z 1/(a + i b) = (a - i b) / (a^2 + b^2)
    const double za = s - kDyMZ * kDyMZ, zb = kDyMZ * kDyWZ, zn = 1.0 / (za * za + zb * zb);
    const double inv_re[2] = {1.0 / s, za * zn}, inv_im[2] = {0.0, -zb * zn};
    Wf<T> c;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const int cu = x >> 1, ce = x & 1;  // quark chirality (L, R), lepton chirality (L, R)
        double re = 0.0, im = 0.0;
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const double g = gu[v][cu] * ge[v][ce];
            re += g * inv_re[v];
            im += g * inv_im[v];
        }
        c.c[x] = {(T)re, (T)im};
    }
    return c;
}

// Setup item of the straight-line kernel: external wavefunctions (2 NPAR),
// then, for a process with the Drell-Yan insertion, its electroweak
// coefficients (one table entry), then the lines
template <class P, class T>
__device__ __forceinline__ void event_setup(const double* __restrict__ p, int item, double mt, int gauge_ext,
                                            Wf<T>* __restrict__ ext, Ln<T>* __restrict__ ln)
{
    if (item < 2 * P::NPAR) ext[item] = ext_wavefunction<P, T>(p, item, mt, gauge_ext);
    else if (item < P::NEXT) ext[item] = ew_coefficients<T>(p);
    else ln[item - P::NEXT] = line_data<P, T>(p, item - P::NEXT, mt);
}

// Colour form J^+ N J in precision C of a colour-flow vector J held in
// precision T: with C != T the amplitudes are cast to C first (the paper's
// mixed mode evaluates them in FP64 and the colour algebra in FP32).
template <class P, class T, class C, class JT> __device__ __forceinline__ T colour_as(const JT& J)
{
    if constexpr (std::is_same<C, T>::value) {
        return P::template colour<T>(J);
    } else {
        cx<C> Jc[P::NCOL];
#pragma unroll
        for (int c = 0; c < P::NCOL; ++c) {
            const cx<T> j = J[c];
            Jc[c] = {(C)j.re, (C)j.im};
        }
        return (T)P::template colour<C>(Jc);
    }
}

// Scalar colour contraction and helicity sum.  T: chain precision, C: colour.
template <class P, class T, class C = T, bool SDE = false>
// (a minimum of 0 CTAs per SM leaves the register allocation unconstrained: an
// explicit 1 made ptxas give gg -> t t~ 125 registers instead of 96)
__global__ void __launch_bounds__(P::THREADS, (std::is_same<T, float>::value && P::MIN_CTAS_F > 1) ? P::MIN_CTAS_F : 0)
    me_kernel_scalar(LaunchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NPAR = P::NPAR, NL = P::NLINES, TH = P::THREADS;
    const int S = a.slots;
    const int E = TH / S;
    const long long e0 = (long long)blockIdx.x * E;
    const int ne = (int)min((long long)E, a.nevt - e0);

    double* smom = reinterpret_cast<double*>(smem);
    Wf<T>* sext = reinterpret_cast<Wf<T>*>(smom + E * NPAR * 4);
    Ln<T>* sln = reinterpret_cast<Ln<T>*>(smem + scalar_line_offset<P, T>(E));
    constexpr bool F32 = std::is_same<T, float>::value;
    constexpr int NG = NPAR * (NPAR + 1) / 2;
    float2* spf = reinterpret_cast<float2*>(smem + scalar_pf_offset<P, T>(E));
    double* sgram = reinterpret_cast<double*>(smem + scalar_gram_offset<P, T>(E));

    // (a1) coalesced load of this CTA's momenta
    const double* g = a.mom + e0 * NPAR * 4;
    if ((reinterpret_cast<uintptr_t>(g) & 15) == 0) {
        const double2* g2 = reinterpret_cast<const double2*>(g);
        double2* s2 = reinterpret_cast<double2*>(smom);
        for (int i = threadIdx.x; i < ne * NPAR * 2; i += TH) s2[i] = __ldg(g2 + i);
    } else {
        for (int i = threadIdx.x; i < ne * NPAR * 4; i += TH) smom[i] = __ldg(g + i);
    }
    __syncthreads();

    // (a2, a3 denominators) helicity-independent per-event data: FP64 in FP64
    // kernels; in FP32 kernels from the split momenta, with FP64 only for the Gram
    // matrix and the line denominators (the FP32 setup of the table kernels)
    constexpr int PER = P::NEXT + NL;
    if constexpr (F32) {
        // without lines there is no denominator to protect: the first phase then
        // only takes each momentum component's leading 24 bits (the hi part of the
        // split), once per event rather than once per external state that reads it
        constexpr int NA = NL > 0 ? 4 * NPAR + NG : 4 * NPAR;
        for (int it = threadIdx.x; it < ne * NA; it += TH) {
            if constexpr (NL > 0) {
                const int ev = it / NA, j = it - ev * NA;
                split_or_gram<NPAR, true>(smom + ev * NPAR * 4, j, spf + ev * NPAR * 4, sgram + ev * NG);
            } else {
                float hi, lo;
                split_f32(smom[it], hi, lo);
                spf[it] = make_float2(hi, 0.0f);
            }
        }
        __syncthreads();
        const double m2 = a.mt * a.mt;
        const float mtf = (float)a.mt;
        for (int it = threadIdx.x; it < ne * PER; it += TH) {
            const int ev = it / PER, j = it - ev * PER;
            if (j < 2 * NPAR) sext[ev * P::NEXT + j] = ext_wavefunction_split<P>(spf + ev * NPAR * 4, j, mtf, a.gauge_ext);
            else if (j < P::NEXT) sext[ev * P::NEXT + j] = ew_coefficients<T>(smom + ev * NPAR * 4);
            else sln[ev * NL + j - P::NEXT] = line_data_split<P>(spf + ev * NPAR * 4, sgram + ev * NG, j - P::NEXT, m2);
        }
    } else {
        for (int it = threadIdx.x; it < ne * PER; it += TH) {
            const int ev = it / PER, j = it - ev * PER;
            event_setup<P, T>(smom + ev * NPAR * 4, j, a.mt, a.gauge_ext, sext + ev * P::NEXT, sln + ev * NL);
        }
    }
    __syncthreads();

    // (a3-a6) chain, colour sum, helicity accumulation
    const int ev = threadIdx.x / S, slot = threadIdx.x - ev * S;
    double acc = 0.0, snum = 0.0, sden = 0.0;
    FSum facc{0.0f, 0.0f};  // FP32 kernels: compensated helicity sum, one conversion per event
    if (ev < ne) {
        const Wf<T>* ext = sext + ev * P::NEXT;
        const Ln<T>* ln = sln + ev * NL;
        for (int i = slot; i < a.nlist; i += S) {
            // helicity sampling: one helicity per event (external states of
            // both helicities are in shared memory, so lanes with different
            // helicities run the same instructions)
            const int hel = a.hel_ev ? a.hel_ev[e0 + ev] : a.hel_list[i];
            SdeAcc<T> sde{T(0), T(0), a.sde_channel};
            T v;
            if constexpr (P::J_SMEM) {
                cx<T>* jb = reinterpret_cast<cx<T>*>(smem + setup_bytes<P, T>(E)) + threadIdx.x;
                JSmem<T, TH> J{jb};
                for (int c = 0; c < P::NCOL; ++c) J[c] = {T(0), T(0)};
                P::template chain<T, SDE>(ext, hel, ln, (T)a.mt, J, sde);
                v = colour_as<P, T, C>(J);
            } else {
                cx<T> J[P::NCOL];
#pragma unroll
                for (int c = 0; c < P::NCOL; ++c) J[c] = {T(0), T(0)};
                P::template chain<T, SDE>(ext, hel, ln, (T)a.mt, J, sde);
                v = colour_as<P, T, C>(J);
            }
            if constexpr (F32) facc = fsum_add(facc, FSum{(float)v, 0.0f});
            else acc += (double)v;
            if constexpr (SDE) {
                snum += (double)sde.num;
                sden += (double)sde.den;
            }
            if (a.hel_out) a.hel_out[(e0 + ev) * a.nlist + i] = (double)v * a.norm;
        }
    }
    // (a6) helicity sum: reduce over the S lanes of each event
    for (int off = S >> 1; off > 0; off >>= 1) {
        if constexpr (F32) {
            const FSum o{__shfl_xor_sync(0xffffffffu, facc.s, off), __shfl_xor_sync(0xffffffffu, facc.c, off)};
            facc = fsum_add(facc, o);
        } else {
            acc += __shfl_xor_sync(0xffffffffu, acc, off);
        }
        if constexpr (SDE) {
            snum += __shfl_xor_sync(0xffffffffu, snum, off);
            sden += __shfl_xor_sync(0xffffffffu, sden, off);
        }
    }
    // (a7) normalisation g^{2k} / (IDEN * colour denominator)
    if (ev < ne && slot == 0) {
        if constexpr (F32) acc = (double)facc.s + (double)facc.c;
        a.me2[e0 + ev] = acc * a.norm * (a.w_ev ? a.w_ev[e0 + ev] : 1.0);
        if constexpr (SDE) a.sde_w[e0 + ev] = sden > 0.0 ? snum / sden : 0.0;
    }
}

template <class P, class T> size_t scalar_smem_bytes(int E)
{
    size_t b = setup_bytes<P, T>(E);
    if constexpr (P::J_SMEM) b += (size_t)P::THREADS * P::NCOL * sizeof(cx<T>);
    return b;
}

// Raise a kernel's dynamic shared-memory limit to `bytes` once (monotone).
// A failed request leaves no stale error behind for later launches.
template <class K> cudaError_t ensure_smem(K kernel, size_t bytes, size_t& granted)
{
    if (bytes <= 48 * 1024 || bytes <= granted) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;
    }
    granted = bytes;
    return cudaSuccess;
}

template <class P, class T, class C = T, bool SDE = false> cudaError_t launch_scalar(const LaunchArgs& a)
{
    const int E = P::THREADS / a.slots;
    const long long grid = (a.nevt + E - 1) / E;
    const size_t smem = scalar_smem_bytes<P, T>(E);
    static size_t granted = 0;  // per instantiation; idempotent if raced
    cudaError_t e = ensure_smem(me_kernel_scalar<P, T, C, SDE>, smem, granted);
    if (e != cudaSuccess) return e;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
    me_kernel_scalar<P, T, C, SDE><<<(unsigned)grid, P::THREADS, smem, a.stream>>>(a);
    return cudaGetLastError();
}

}  // namespace me
