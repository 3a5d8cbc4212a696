// Device wavefunction and vertex routines of the helicity-amplitude chain
// (arXiv:2507.21039 Sec. 3.1: vxxxxx / ixxxxx / oxxxxx external states,
// VVV1P0_1-type off-shell currents, FFV1_0-type amplitudes).
//
// Conventions: metric (+,-,-,-); chiral Dirac matrices
// gamma^mu = [[0, s^mu], [sb^mu, 0]], s = (1, sigma), sb = (1, -sigma), upper two
// spinor components left-handed.  Vector wavefunctions are stored with upper
// index; every contraction is the Minkowski bilinear product.  Vertex routines
// implement real-coefficient Lorentz structures only: the factors i of the
// Feynman rules, the couplings and the colour coefficients are folded by the
// generator into the constant with which each amplitude enters the colour-flow
// vector J.  T is the amplitude precision (float or double).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace me {

template <class T> struct cx { T re, im; };
template <class T> struct Wf { cx<T> c[4]; };          // spinor or vector wavefunction
template <class T> struct Ln { T p[4]; T inv; };       // line momentum and 1/(p^2 - m^2)

template <class T> __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <class T> __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <class T> __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class T> __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return {s * a.re, s * a.im}; }
// a*b + c
template <class T> __device__ __forceinline__ cx<T> cfma(cx<T> a, cx<T> b, cx<T> c)
{
    return {fma(a.re, b.re, fma(-a.im, b.im, c.re)), fma(a.re, b.im, fma(a.im, b.re, c.im))};
}
// s*a + c, s real
template <class T> __device__ __forceinline__ cx<T> rfma(T s, cx<T> a, cx<T> c)
{
    return {fma(s, a.re, c.re), fma(s, a.im, c.im)};
}

// Minkowski bilinear product of complex four-vectors
template <class T> __device__ __forceinline__ cx<T> mdot(const Wf<T>& a, const Wf<T>& b)
{
    cx<T> s = a.c[0] * b.c[0];
    s = cfma({-a.c[1].re, -a.c[1].im}, b.c[1], s);
    s = cfma({-a.c[2].re, -a.c[2].im}, b.c[2], s);
    s = cfma({-a.c[3].re, -a.c[3].im}, b.c[3], s);
    return s;
}
// real four-vector k with complex four-vector a
template <class T> __device__ __forceinline__ cx<T> rdot(const T* k, const Wf<T>& a)
{
    cx<T> s = k[0] * a.c[0];
    s = rfma(-k[1], a.c[1], s);
    s = rfma(-k[2], a.c[2], s);
    s = rfma(-k[3], a.c[3], s);
    return s;
}

// 2x2 blocks of V_mu s^mu  (s00 s01; s10 s11); V_mu sb^mu = (s11 -s01; -s10 s00)
template <class T> struct Blk { cx<T> s00, s01, s10, s11; };
template <class T> __device__ __forceinline__ Blk<T> sblk(const Wf<T>& V)
{
    Blk<T> b;
    b.s00 = V.c[0] - V.c[3];
    b.s11 = V.c[0] + V.c[3];
    b.s01 = {-(V.c[1].re + V.c[2].im), V.c[2].re - V.c[1].im};   // -V1 + i V2
    b.s10 = {V.c[2].im - V.c[1].re, -(V.c[1].im + V.c[2].re)};   // -V1 - i V2
    return b;
}

// ---------------------------------------------------------------------------
// amplitudes
// ---------------------------------------------------------------------------
// FFV1_0: Fo gamma^mu V_mu Fi
template <class T> __device__ __forceinline__ cx<T> FFV1_0(const Wf<T>& Fo, const Wf<T>& V, const Wf<T>& Fi)
{
    Blk<T> b = sblk(V);
    // (o0,o1) s (i2,i3) + (o2,o3) sb (i0,i1)
    cx<T> t0 = cfma(b.s01, Fi.c[3], b.s00 * Fi.c[2]);
    cx<T> t1 = cfma(b.s11, Fi.c[3], b.s10 * Fi.c[2]);
    cx<T> t2 = b.s11 * Fi.c[0] - b.s01 * Fi.c[1];
    cx<T> t3 = b.s00 * Fi.c[1] - b.s10 * Fi.c[0];
    cx<T> a = Fo.c[0] * t0;
    a = cfma(Fo.c[1], t1, a);
    a = cfma(Fo.c[2], t2, a);
    a = cfma(Fo.c[3], t3, a);
    return a;
}

// VVV1_0: V^{mnr}(k1,k2,k3) A_m B_n Q_r with k1 = -PA, k2 = -PB, k3 = PA + PB
template <class T>
__device__ __forceinline__ cx<T> VVV1_0(const Wf<T>& A, const T* PA, const Wf<T>& B, const T* PB, const Wf<T>& Q)
{
    T d12[4], d23[4], d31[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        d12[m] = PB[m] - PA[m];
        d23[m] = -fma(T(2), PB[m], PA[m]);
        d31[m] = fma(T(2), PA[m], PB[m]);
    }
    cx<T> ab = mdot(A, B), bq = mdot(B, Q), qa = mdot(Q, A);
    return ab * rdot(d12, Q) + bq * rdot(d23, A) + qa * rdot(d31, B);
}

// four-gluon structures contracted with the fourth leg Q
//   VVVV1: (A.C)(B.Q) - (B.C)(A.Q)   [f^{abe} f^{cde}]
//   VVVV3: (A.B)(C.Q) - (B.C)(A.Q)   [f^{ace} f^{bde}]
//   VVVV4: (A.B)(C.Q) - (A.C)(B.Q)   [f^{ade} f^{bce}]
template <class T> __device__ __forceinline__ cx<T> VVVV1_0(const Wf<T>& A, const Wf<T>& B, const Wf<T>& C, const Wf<T>& Q)
{
    return mdot(A, C) * mdot(B, Q) - mdot(B, C) * mdot(A, Q);
}
template <class T> __device__ __forceinline__ cx<T> VVVV3_0(const Wf<T>& A, const Wf<T>& B, const Wf<T>& C, const Wf<T>& Q)
{
    return mdot(A, B) * mdot(C, Q) - mdot(B, C) * mdot(A, Q);
}
template <class T> __device__ __forceinline__ cx<T> VVVV4_0(const Wf<T>& A, const Wf<T>& B, const Wf<T>& C, const Wf<T>& Q)
{
    return mdot(A, B) * mdot(C, Q) - mdot(A, C) * mdot(B, Q);
}

// ---------------------------------------------------------------------------
// off-shell currents (propagator 1/(q^2 - m^2) applied through ln.inv)
// ---------------------------------------------------------------------------
// VVV1P0_1: inv * [ (A.B)(k1-k2) + B ((k2-k3).A) + A ((k3-k1).B) ]
template <class T>
__device__ __forceinline__ void VVV1P0_1(const Wf<T>& A, const T* PA, const Wf<T>& B, const T* PB, T inv, Wf<T>& out)
{
    T d12[4], d23[4], d31[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        d12[m] = PB[m] - PA[m];
        d23[m] = -fma(T(2), PB[m], PA[m]);
        d31[m] = fma(T(2), PA[m], PB[m]);
    }
    cx<T> ab = inv * mdot(A, B), a = inv * rdot(d23, A), b = inv * rdot(d31, B);
#pragma unroll
    for (int m = 0; m < 4; ++m) out.c[m] = cfma(B.c[m], a, cfma(A.c[m], b, d12[m] * ab));
}

// four-gluon currents: inv * [structure with open fourth index]
template <class T>
__device__ __forceinline__ void VVVV1P0_1(const Wf<T>& A, const Wf<T>& B, const Wf<T>& C, T inv, Wf<T>& out)
{
    cx<T> x = inv * mdot(A, C), y = inv * mdot(B, C);
#pragma unroll
    for (int m = 0; m < 4; ++m) out.c[m] = x * B.c[m] - y * A.c[m];
}
template <class T>
__device__ __forceinline__ void VVVV3P0_1(const Wf<T>& A, const Wf<T>& B, const Wf<T>& C, T inv, Wf<T>& out)
{
    cx<T> x = inv * mdot(A, B), y = inv * mdot(B, C);
#pragma unroll
    for (int m = 0; m < 4; ++m) out.c[m] = x * C.c[m] - y * A.c[m];
}
template <class T>
__device__ __forceinline__ void VVVV4P0_1(const Wf<T>& A, const Wf<T>& B, const Wf<T>& C, T inv, Wf<T>& out)
{
    cx<T> x = inv * mdot(A, B), y = inv * mdot(A, C);
#pragma unroll
    for (int m = 0; m < 4; ++m) out.c[m] = x * C.c[m] - y * B.c[m];
}

// FFV1P0_3: inv * Fo gamma^mu Fi   (vector current of a fermion pair)
template <class T> __device__ __forceinline__ void FFV1P0_3(const Wf<T>& Fo, const Wf<T>& Fi, T inv, Wf<T>& out)
{
    const cx<T>*o = Fo.c, *i = Fi.c;
    cx<T> a = o[0] * i[2], b = o[1] * i[3], c = o[2] * i[0], d = o[3] * i[1];
    cx<T> e = o[0] * i[3], f = o[1] * i[2], g = o[2] * i[1], h = o[3] * i[0];
    cx<T> j0 = a + b + c + d;
    cx<T> j1 = e + f - g - h;
    cx<T> s2 = f + g - e - h;                  // J2 = i * s2
    cx<T> j3 = a - b - c + d;
    out.c[0] = inv * j0;
    out.c[1] = inv * j1;
    out.c[2] = {-inv * s2.im, inv * s2.re};
    out.c[3] = inv * j3;
}

// FFV1_2: Fo' = inv * Fo gamma.V (qslash + m)   (row spinor, outgoing-fermion side)
template <class T>
__device__ __forceinline__ void FFV1_2(const Wf<T>& Fo, const Wf<T>& V, const Ln<T>& q, T m, Wf<T>& out)
{
    Blk<T> b = sblk(V);
    // X = Fo gamma.V: X_L = (o2,o3) sb, X_R = (o0,o1) s ;  sb = (s11 -s01; -s10 s00)
    cx<T> xl0 = Fo.c[2] * b.s11 - Fo.c[3] * b.s10;
    cx<T> xl1 = Fo.c[3] * b.s00 - Fo.c[2] * b.s01;
    cx<T> xr0 = cfma(Fo.c[1], b.s10, Fo.c[0] * b.s00);
    cx<T> xr1 = cfma(Fo.c[1], b.s11, Fo.c[0] * b.s01);
    // Y_L = X_R (q.sb) + m X_L ; Y_R = X_L (q.s) + m X_R
    // q.s = (q0-q3, -q1+i q2; -q1-i q2, q0+q3), q.sb = (q0+q3, q1-i q2; q1+i q2, q0-q3)
    const T q0 = q.p[0], q1 = q.p[1], q2 = q.p[2], q3 = q.p[3], inv = q.inv;
    cx<T> qs01 = {-q1, q2}, qs10 = {-q1, -q2};
    cx<T> yl0 = rfma(q0 + q3, xr0, rfma(m, xl0, xr1 * cx<T>{q1, q2}));
    cx<T> yl1 = rfma(q0 - q3, xr1, rfma(m, xl1, xr0 * cx<T>{q1, -q2}));
    cx<T> yr0 = rfma(q0 - q3, xl0, rfma(m, xr0, xl1 * qs10));
    cx<T> yr1 = rfma(q0 + q3, xl1, rfma(m, xr1, xl0 * qs01));
    out.c[0] = inv * yl0;
    out.c[1] = inv * yl1;
    out.c[2] = inv * yr0;
    out.c[3] = inv * yr1;
}

// FFV1_1: Fi' = inv * (qslash + m) gamma.V Fi   (column spinor, incoming side)
template <class T>
__device__ __forceinline__ void FFV1_1(const Wf<T>& V, const Wf<T>& Fi, const Ln<T>& q, T m, Wf<T>& out)
{
    Blk<T> b = sblk(V);
    // X = gamma.V Fi: X_L = s (i2,i3), X_R = sb (i0,i1)
    cx<T> xl0 = cfma(b.s01, Fi.c[3], b.s00 * Fi.c[2]);
    cx<T> xl1 = cfma(b.s11, Fi.c[3], b.s10 * Fi.c[2]);
    cx<T> xr0 = b.s11 * Fi.c[0] - b.s01 * Fi.c[1];
    cx<T> xr1 = b.s00 * Fi.c[1] - b.s10 * Fi.c[0];
    // Y_L = (q.s) X_R + m X_L ; Y_R = (q.sb) X_L + m X_R
    const T q0 = q.p[0], q1 = q.p[1], q2 = q.p[2], q3 = q.p[3], inv = q.inv;
    cx<T> yl0 = rfma(q0 - q3, xr0, rfma(m, xl0, cx<T>{-q1, q2} * xr1));
    cx<T> yl1 = rfma(q0 + q3, xr1, rfma(m, xl1, cx<T>{-q1, -q2} * xr0));
    cx<T> yr0 = rfma(q0 + q3, xl0, rfma(m, xr0, cx<T>{q1, -q2} * xl1));
    cx<T> yr1 = rfma(q0 - q3, xl1, rfma(m, xr1, cx<T>{q1, q2} * xl0));
    out.c[0] = inv * yl0;
    out.c[1] = inv * yl1;
    out.c[2] = inv * yr0;
    out.c[3] = inv * yr1;
}

// ---------------------------------------------------------------------------
// Chiral vertices of the Drell-Yan quark line (the colourless photon/Z
// insertion; reading R15).  Upper spinor components are left-handed, so in
// gamma.V = [[0, V.s], [V.sb, 0]] the V.s block meets right-handed and the
// V.sb block left-handed components.  The insertion slash(LL) P_L + slash(LR)
// P_R = [[0, LR.s], [LL.sb, 0]]: the FFV1 routines with the s block taken from
// LR and the sb block from LL.
// ---------------------------------------------------------------------------
// FFVLR_0: Fo (slash(LL) P_L + slash(LR) P_R) Fi
template <class T>
__device__ __forceinline__ cx<T> FFVLR_0(const Wf<T>& Fo, const Wf<T>& LL, const Wf<T>& LR, const Wf<T>& Fi)
{
    const Blk<T> r = sblk(LR), l = sblk(LL);
    cx<T> t0 = cfma(r.s01, Fi.c[3], r.s00 * Fi.c[2]);
    cx<T> t1 = cfma(r.s11, Fi.c[3], r.s10 * Fi.c[2]);
    cx<T> t2 = l.s11 * Fi.c[0] - l.s01 * Fi.c[1];
    cx<T> t3 = l.s00 * Fi.c[1] - l.s10 * Fi.c[0];
    cx<T> a = Fo.c[0] * t0;
    a = cfma(Fo.c[1], t1, a);
    a = cfma(Fo.c[2], t2, a);
    a = cfma(Fo.c[3], t3, a);
    return a;
}

// FFVLR_2: Fo' = inv * Fo (slash(LL) P_L + slash(LR) P_R) qslash   (massless quark)
template <class T>
__device__ __forceinline__ void FFVLR_2(const Wf<T>& Fo, const Wf<T>& LL, const Wf<T>& LR, const Ln<T>& q, Wf<T>& out)
{
    const Blk<T> r = sblk(LR), l = sblk(LL);
    // X_L = (o2,o3) LL.sb, X_R = (o0,o1) LR.s
    cx<T> xl0 = Fo.c[2] * l.s11 - Fo.c[3] * l.s10;
    cx<T> xl1 = Fo.c[3] * l.s00 - Fo.c[2] * l.s01;
    cx<T> xr0 = cfma(Fo.c[1], r.s10, Fo.c[0] * r.s00);
    cx<T> xr1 = cfma(Fo.c[1], r.s11, Fo.c[0] * r.s01);
    // Y_L = X_R (q.sb), Y_R = X_L (q.s)
    const T q0 = q.p[0], q1 = q.p[1], q2 = q.p[2], q3 = q.p[3], inv = q.inv;
    cx<T> yl0 = rfma(q0 + q3, xr0, xr1 * cx<T>{q1, q2});
    cx<T> yl1 = rfma(q0 - q3, xr1, xr0 * cx<T>{q1, -q2});
    cx<T> yr0 = rfma(q0 - q3, xl0, xl1 * cx<T>{-q1, -q2});
    cx<T> yr1 = rfma(q0 + q3, xl1, xl0 * cx<T>{-q1, q2});
    out.c[0] = inv * yl0;
    out.c[1] = inv * yl1;
    out.c[2] = inv * yr0;
    out.c[3] = inv * yr1;
}

// FFVLR_1: Fi' = inv * qslash (slash(LL) P_L + slash(LR) P_R) Fi   (massless quark)
template <class T>
__device__ __forceinline__ void FFVLR_1(const Wf<T>& LL, const Wf<T>& LR, const Wf<T>& Fi, const Ln<T>& q, Wf<T>& out)
{
    const Blk<T> r = sblk(LR), l = sblk(LL);
    // X upper = LR.s (i2,i3), lower = LL.sb (i0,i1)
    cx<T> xl0 = cfma(r.s01, Fi.c[3], r.s00 * Fi.c[2]);
    cx<T> xl1 = cfma(r.s11, Fi.c[3], r.s10 * Fi.c[2]);
    cx<T> xr0 = l.s11 * Fi.c[0] - l.s01 * Fi.c[1];
    cx<T> xr1 = l.s00 * Fi.c[1] - l.s10 * Fi.c[0];
    const T q0 = q.p[0], q1 = q.p[1], q2 = q.p[2], q3 = q.p[3], inv = q.inv;
    cx<T> yl0 = rfma(q0 - q3, xr0, cx<T>{-q1, q2} * xr1);
    cx<T> yl1 = rfma(q0 + q3, xr1, cx<T>{-q1, -q2} * xr0);
    cx<T> yr0 = rfma(q0 + q3, xl0, cx<T>{q1, -q2} * xl1);
    cx<T> yr1 = rfma(q0 - q3, xl1, cx<T>{q1, q2} * xl0);
    out.c[0] = inv * yl0;
    out.c[1] = inv * yl1;
    out.c[2] = inv * yr0;
    out.c[3] = inv * yr1;
}

// Lepton-pair objects of the insertion: with S = Fo gamma P_R Fi and
// Sb = Fo gamma P_L Fi (Fo = ubar(e-), Fi = v(e+), upper index),
//   LL = c.c[0] Sb + c.c[1] S,   LR = c.c[2] Sb + c.c[3] S,
// c the event's electroweak coefficients (sums over photon and Z of quark
// coupling x lepton coupling / propagator denominator; see ew_coefficients).
template <class T>
__device__ __forceinline__ void LEPLR(const Wf<T>& Fo, const Wf<T>& Fi, const Wf<T>& c, Wf<T>& LL, Wf<T>& LR)
{
    const cx<T>*o = Fo.c, *i = Fi.c;
    const cx<T> a = o[0] * i[2], b = o[1] * i[3], e = o[0] * i[3], f = o[1] * i[2];   // right-handed
    const cx<T> cc = o[2] * i[0], d = o[3] * i[1], g = o[2] * i[1], h = o[3] * i[0]; // left-handed
    const cx<T> fe = f - e, gh = g - h;
    Wf<T> S, Sb;
    S.c[0] = a + b;
    S.c[1] = e + f;
    S.c[2] = {-fe.im, fe.re};    // i (f - e)
    S.c[3] = a - b;
    Sb.c[0] = cc + d;
    Sb.c[1] = {-(g.re + h.re), -(g.im + h.im)};
    Sb.c[2] = {-gh.im, gh.re};   // i (g - h)
    Sb.c[3] = d - cc;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        LL.c[m] = cfma(c.c[0], Sb.c[m], c.c[1] * S.c[m]);
        LR.c[m] = cfma(c.c[2], Sb.c[m], c.c[3] * S.c[m]);
    }
}

// ---------------------------------------------------------------------------
// amputated vertices (no propagator) and two-operand contractions.  A final
// vertex with one operand's index left open; contracting it with that operand
// gives the amplitude of the direct vertex routine (same products, grouped
// differently), e.g. FFV1_0(Fo, V, Fi) = DOTV(FFV1A_3(Fo, Fi), V)
// = DOTF(FFV1A_2(Fo, V), Fi) = DOTF(Fo, FFV1A_1(V, Fi)).
// ---------------------------------------------------------------------------
// spinor contraction (row) . (column), no metric
template <class T> __device__ __forceinline__ cx<T> sdot(const Wf<T>& a, const Wf<T>& b)
{
    cx<T> s = a.c[0] * b.c[0];
    s = cfma(a.c[1], b.c[1], s);
    s = cfma(a.c[2], b.c[2], s);
    s = cfma(a.c[3], b.c[3], s);
    return s;
}
// a += S b (S = +1 or -1), componentwise: the contractions are bilinear, so a
// colour group's members sharing one operand are contracted once with the
// signed sum of their other operands
template <int S, class T> __device__ __forceinline__ void wf_acc(Wf<T>& a, const Wf<T>& b)
{
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if constexpr (S > 0) { a.c[i].re += b.c[i].re; a.c[i].im += b.c[i].im; }
        else { a.c[i].re -= b.c[i].re; a.c[i].im -= b.c[i].im; }
    }
}
template <class T> __device__ __forceinline__ cx<T> DOTV(const Wf<T>& a, const Wf<T>& b) { return mdot(a, b); }
template <class T> __device__ __forceinline__ cx<T> DOTF(const Wf<T>& a, const Wf<T>& b) { return sdot(a, b); }

// K^mu = Fo gamma^mu Fi
template <class T> __device__ __forceinline__ void FFV1A_3(const Wf<T>& Fo, const Wf<T>& Fi, Wf<T>& out)
{
    const cx<T>*o = Fo.c, *i = Fi.c;
    cx<T> a = o[0] * i[2], b = o[1] * i[3], c = o[2] * i[0], d = o[3] * i[1];
    cx<T> e = o[0] * i[3], f = o[1] * i[2], g = o[2] * i[1], h = o[3] * i[0];
    const cx<T> s2 = f + g - e - h;            // K2 = i * s2
    out.c[0] = a + b + c + d;
    out.c[1] = e + f - g - h;
    out.c[2] = {-s2.im, s2.re};
    out.c[3] = a - b - c + d;
}
// row spinor Fo gamma.V
template <class T> __device__ __forceinline__ void FFV1A_2(const Wf<T>& Fo, const Wf<T>& V, Wf<T>& out)
{
    Blk<T> b = sblk(V);
    out.c[0] = Fo.c[2] * b.s11 - Fo.c[3] * b.s10;
    out.c[1] = Fo.c[3] * b.s00 - Fo.c[2] * b.s01;
    out.c[2] = cfma(Fo.c[1], b.s10, Fo.c[0] * b.s00);
    out.c[3] = cfma(Fo.c[1], b.s11, Fo.c[0] * b.s01);
}
// column spinor gamma.V Fi
template <class T> __device__ __forceinline__ void FFV1A_1(const Wf<T>& V, const Wf<T>& Fi, Wf<T>& out)
{
    Blk<T> b = sblk(V);
    out.c[0] = cfma(b.s01, Fi.c[3], b.s00 * Fi.c[2]);
    out.c[1] = cfma(b.s11, Fi.c[3], b.s10 * Fi.c[2]);
    out.c[2] = b.s11 * Fi.c[0] - b.s01 * Fi.c[1];
    out.c[3] = b.s00 * Fi.c[1] - b.s10 * Fi.c[0];
}
// three-gluon vertex V^{mnr}(k1, k2, k3) A_m B_n Q_r (k1 = -PA, k2 = -PB,
// k3 = PA + PB) with one leg open: OPEN = 3 (Q; inputs A, B), 1 (A; inputs B,
// Q), 2 (B; inputs A, Q).  PA, PB are the momenta of legs A and B.
template <int OPEN, class T>
__device__ __forceinline__ void VVV1A(const Wf<T>& X, const Wf<T>& Y, const T* PA, const T* PB, Wf<T>& out)
{
    T d12[4], d23[4], d31[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        d12[m] = PB[m] - PA[m];
        d23[m] = -fma(T(2), PB[m], PA[m]);
        d31[m] = fma(T(2), PA[m], PB[m]);
    }
    if constexpr (OPEN == 3) {         // X = A, Y = B: (A.B) d12 + B (d23.A) + A (d31.B)
        const cx<T> ab = mdot(X, Y), a = rdot(d23, X), b = rdot(d31, Y);
#pragma unroll
        for (int m = 0; m < 4; ++m) out.c[m] = cfma(Y.c[m], a, cfma(X.c[m], b, d12[m] * ab));
    } else if constexpr (OPEN == 1) {  // X = B, Y = Q: B (d12.Q) + (B.Q) d23 + Q (d31.B)
        const cx<T> bq = mdot(X, Y), q = rdot(d12, Y), b = rdot(d31, X);
#pragma unroll
        for (int m = 0; m < 4; ++m) out.c[m] = cfma(X.c[m], q, cfma(Y.c[m], b, d23[m] * bq));
    } else {                           // X = A, Y = Q: A (d12.Q) + Q (d23.A) + (Q.A) d31
        const cx<T> qa = mdot(Y, X), q = rdot(d12, Y), a = rdot(d23, X);
#pragma unroll
        for (int m = 0; m < 4; ++m) out.c[m] = cfma(X.c[m], q, cfma(Y.c[m], a, d31[m] * qa));
    }
}
// four-gluon structures with the fourth leg open (VVVVnP0_1 without propagator)
template <class T> __device__ __forceinline__ void VVVV1A(const Wf<T>& A, const Wf<T>& B, const Wf<T>& C, Wf<T>& out)
{
    const cx<T> x = mdot(A, C), y = mdot(B, C);
#pragma unroll
    for (int m = 0; m < 4; ++m) out.c[m] = x * B.c[m] - y * A.c[m];
}
template <class T> __device__ __forceinline__ void VVVV3A(const Wf<T>& A, const Wf<T>& B, const Wf<T>& C, Wf<T>& out)
{
    const cx<T> x = mdot(A, B), y = mdot(B, C);
#pragma unroll
    for (int m = 0; m < 4; ++m) out.c[m] = x * C.c[m] - y * A.c[m];
}
template <class T> __device__ __forceinline__ void VVVV4A(const Wf<T>& A, const Wf<T>& B, const Wf<T>& C, Wf<T>& out)
{
    const cx<T> x = mdot(A, B), y = mdot(A, C);
#pragma unroll
    for (int m = 0; m < 4; ++m) out.c[m] = x * C.c[m] - y * B.c[m];
}

// J_c += (R + i I) a for a Gaussian-integer colour/phase coefficient
template <int R, int I, class T, class C> __device__ __forceinline__ void jacc(C& j, cx<T> a)
{
    cx<T> t = j;
    if constexpr (R == 1) { t.re += a.re; t.im += a.im; }
    else if constexpr (R == -1) { t.re -= a.re; t.im -= a.im; }
    else if constexpr (R != 0) { t.re = fma(T(R), a.re, t.re); t.im = fma(T(R), a.im, t.im); }
    if constexpr (I == 1) { t.re -= a.im; t.im += a.re; }
    else if constexpr (I == -1) { t.re += a.im; t.im -= a.re; }
    else if constexpr (I != 0) { t.re = fma(T(-I), a.im, t.re); t.im = fma(T(I), a.re, t.im); }
    j = t;
}

// ---------------------------------------------------------------------------
// external wavefunctions (evaluated per event in FP64, then rounded to T)
// ---------------------------------------------------------------------------
// In FP64 mode these run in FP64; in FP32 / mixed mode in FP32 from the
// rounded momenta (their relative error, ~1e-7, is that of the FP32 chain).
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }

// two-spinors chi_lam(p): chi_+ = (P+pz, px+i py)/n, chi_- = (-px+i py, P+pz)/n,
// n = sqrt(2P(P+pz)); p along -z: chi_+ = (0,1), chi_- = (-1,0); at rest along +z.
template <class C> __device__ __forceinline__ void chi2(const C* p, int lam, cx<C>* out)
{
    const C px = p[1], py = p[2], pz = p[3];
    const C pt2 = px * px + py * py;
    const C P = sqrt(pt2 + pz * pz);
    if (P == C(0)) {
        out[0] = {lam > 0 ? C(1) : C(0), C(0)};
        out[1] = {lam > 0 ? C(0) : C(1), C(0)};
        return;
    }
    const C ppz = pz >= C(0) ? P + pz : pt2 / (P - pz);
    if (ppz == C(0)) {
        out[0] = {lam > 0 ? C(0) : C(-1), C(0)};
        out[1] = {lam > 0 ? C(1) : C(0), C(0)};
        return;
    }
    const C rn = rsq(C(2) * P * ppz);
    if (lam > 0) {
        out[0] = {ppz * rn, C(0)};
        out[1] = {px * rn, py * rn};
    } else {
        out[0] = {-px * rn, py * rn};
        out[1] = {ppz * rn, C(0)};
    }
}

// omega_+ = sqrt(E + |p|), omega_- = m / sqrt(E + |p|)
template <class C> __device__ __forceinline__ void omegas(const C* p, C m, C& wp, C& wm)
{
    const C P = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
    wp = sqrt(p[0] + P);
    wm = m == C(0) ? C(0) : m / wp;
}

// ixxxxx: flowing-in spinor; nsf = +1 -> u(p, lam) (incoming fermion),
// nsf = -1 -> v(p, lam) (outgoing antifermion)
template <class C> __device__ __forceinline__ void ixxxxx(const C* p, C m, int lam, int nsf, cx<C>* w)
{
    C wp, wm;
    omegas(p, m, wp, wm);
    cx<C> c[2];
    const C wl = lam > 0 ? wp : wm, wml = lam > 0 ? wm : wp;
    if (nsf > 0) {
        chi2(p, lam, c);
        w[0] = wml * c[0]; w[1] = wml * c[1];
        w[2] = wl * c[0];  w[3] = wl * c[1];
    } else {
        chi2(p, -lam, c);
        const C sl = lam > 0 ? C(1) : C(-1);
        w[0] = (-sl * wl) * c[0]; w[1] = (-sl * wl) * c[1];
        w[2] = (sl * wml) * c[0]; w[3] = (sl * wml) * c[1];
    }
}

// oxxxxx: flowing-out (barred) spinor; nsf = +1 -> ubar(p, lam) (outgoing
// fermion), nsf = -1 -> vbar(p, lam) (incoming antifermion).  psibar = psi^+ gamma^0.
template <class C> __device__ __forceinline__ void oxxxxx(const C* p, C m, int lam, int nsf, cx<C>* w)
{
    cx<C> s[4];
    ixxxxx(p, m, lam, nsf, s);
    w[0] = {s[2].re, -s[2].im};
    w[1] = {s[3].re, -s[3].im};
    w[2] = {s[0].re, -s[0].im};
    w[3] = {s[1].re, -s[1].im};
}

// vxxxxx: massless vector boson polarisation eps(k, lam) = (-lam e1 - i e2)/sqrt2,
// e1 = (0, ct cf, ct sf, -st), e2 = (0, -sf, cf, 0); nsv = -1 incoming (eps),
// nsv = +1 outgoing (conj eps)
template <class C> __device__ __forceinline__ void vxxxxx(const C* k, int lam, int nsv, cx<C>* w)
{
    const C kx = k[1], ky = k[2], kz = k[3];
    const C pt = sqrt(kx * kx + ky * ky);
    const C P = sqrt(pt * pt + kz * kz);
    const C ct = kz / P, st = pt / P;
    const C cf = pt > C(0) ? kx / pt : C(1), sf = pt > C(0) ? ky / pt : C(0);
    const C r2 = C(0.70710678118654752440);
    const C sl = lam > 0 ? C(1) : C(-1);
    const C im_sign = nsv < 0 ? C(1) : C(-1);   // conj for outgoing
    w[0] = {C(0), C(0)};
    w[1] = {-sl * ct * cf * r2, im_sign * sf * r2};
    w[2] = {-sl * ct * sf * r2, -im_sign * cf * r2};
    w[3] = {sl * st * r2, C(0)};
}

}  // namespace me
