/*
 * FP64 CPU ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct reference for the batched tree-level squared
 * matrix element |M|^2 (summed over helicities and colours) computed by the
 * standalone amplitude code of arXiv:2507.21039 (Sec. 3.1 "Parallel scattering
 * amplitudes", Sec. 4 "Standalone application").  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load this library;
 * the product library never links, loads or calls it, and the two share no
 * source.
 *
 * Algorithm (independent of the GPU's Feynman-diagram chain):
 *   - colour-ordered partial amplitudes A_sigma of one quark line plus k gluons
 *     from the Berends-Giele off-shell recursion (Berends & Giele 1988), with
 *     colour-ordered vertices derived from the QCD Feynman rules below;
 *   - the colour matrix C_{sigma sigma'} = sum_colours conj(S_sigma) S_sigma'
 *     of the string basis S_sigma = (T^{a_sigma1} ... T^{a_sigmak})_{ij}, by
 *     brute-force summation over all adjoint and fundamental indices with
 *     explicit Gell-Mann matrices (Sec. 4.1: colour algebra is the inner product
 *     of colour-ordered amplitudes with an integer colour matrix);
 *   - |M|^2 = (1/IDEN) sum_h g^{2k} A_h^dagger C A_h, with no helicity filter
 *     (Sec. 3.1 sums all non-vanishing spin configurations; summing all of them
 *     is the same number and catches a wrong GPU helicity mask).
 * Drell-Yan u ubar -> e+ e- + n g (the paper's second standalone workload,
 * Sec. 4) uses the same quark-line recursion with one colourless photon/Z
 * insertion (section at the end of this file).
 * Extra pins live here too: a colour-dressed brute force (explicit colour
 * indices, full f^{abc} vertices, no colour decomposition), the closed forms for
 * e+e- -> mu+mu- (photon only) and gg -> t tbar (Combridge 1979), and
 * RAMBO (Kleiss, Stirling, Ellis 1986) with a Philox4x64-10 counter RNG
 * (Salmon et al., SC'11).
 *
 * Conventions (stated once, implemented separately by the GPU side):
 *   metric (+,-,-,-); chiral Dirac matrices gamma^mu = [[0, s^mu],[sb^mu, 0]],
 *   s^mu = (1, sigma), sb^mu = (1, -sigma); upper two components left-handed.
 *   Two-spinors chi_+(p) = (|p|+pz, px+i py)/sqrt(2|p|(|p|+pz)),
 *               chi_-(p) = (-px+i py, |p|+pz)/sqrt(2|p|(|p|+pz)),
 *   with chi_+ = (0,1), chi_- = (-1,0) for p along -z and p along +z at rest.
 *   u(p,l) = (w_{-l} chi_l ; w_l chi_l),  v(p,l) = (-l w_l chi_{-l} ; l w_{-l} chi_{-l}),
 *   w_{+-} = sqrt(E +- |p|).  eps(k,l) = (-l e1 - i e2)/sqrt(2) with
 *   e1 = (0, cos t cos f, cos t sin f, -sin t), e2 = (0, -sin f, cos f, 0)
 *   (f = 0 when k has no transverse part).  Incoming gluon: eps; outgoing:
 *   conj(eps).  Outgoing quark: ubar; outgoing antiquark: v; incoming e-: u;
 *   incoming e+: vbar.
 *   Feynman rules (D = d - i g A^a T^a, Tr T^a T^b = delta/2):
 *     qqg  i g gamma^mu T^a;   ggg  g f^{abc} [g^{mn}(k1-k2)^r + g^{nr}(k2-k3)^m + g^{rm}(k3-k1)^n]
 *     gggg -i g^2 [f^{abe}f^{cde}(g^{mr}g^{ns}-g^{ms}g^{nr}) + f^{ace}f^{bde}(g^{mn}g^{rs}-g^{ms}g^{nr})
 *                  + f^{ade}f^{bce}(g^{mn}g^{rs}-g^{mr}g^{ns})]   (all momenta incoming)
 *     gluon propagator -i g_{mn}/q^2 (Feynman gauge); quark propagator
 *     i(qslash + m)/(q^2 - m^2), width zero.
 *   Colour decomposition M = g^k sum_sigma (T^{a_s1}..T^{a_sk})_{i_t j_tbar} A_sigma
 *   with the string read from the outgoing quark t to the outgoing antiquark.
 *   Colour-ordered rules that follow (f^{abc}T^c = -i[T^a,T^b]):
 *     quark vertex i gamma^mu; three-gluon vertex -i V^{mnr}(k1,k2,k3) for legs
 *     1,2 in colour order; four-gluon vertex i(2 g^{mr}g^{ns} - g^{mn}g^{rs} - g^{ms}g^{nr})
 *     for legs 1,2,3 in colour order and leg 4 the off-shell one.
 *   Helicity index h in [0, 2^npar): particle i has helicity +1 if bit
 *   (npar-1-i) of h is set, else -1 (physical helicities of the particles).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cx;

#define MAXG 5            /* max gluons (gg -> t tbar ggg) */
#define MAXPAR 7
#define MAXPERM 120       /* 5! */

/* ------------------------------------------------------------------ */
/* Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw,  */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11).              */
/* ------------------------------------------------------------------ */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL;
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73BULL;

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * c0;
        unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 53 random bits mapped to the open interval (0,1): ((x >> 11) + 1/2) 2^-53. */
double orc_u01(uint64_t x) { return ((double)(x >> 11) + 0.5) * 0x1p-53; }

/* ------------------------------------------------------------------ */
/* Minkowski algebra and Dirac matrices                                */
/* ------------------------------------------------------------------ */
static double mdot(const double a[4], const double b[4])
{
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}
static cx cdot(const cx a[4], const cx b[4]) /* bilinear, no conjugation */
{
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}
static cx rcdot(const double a[4], const cx b[4])
{
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

static cx GAM[4][4][4]; /* GAM[mu][row][col] */
static int gam_ready = 0;

static void init_gamma(void)
{
    if (gam_ready) return;
    const cx sig[4][2][2] = {
        {{1, 0}, {0, 1}},
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    memset(GAM, 0, sizeof GAM);
    for (int mu = 0; mu < 4; ++mu)
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                GAM[mu][a][2 + b] = sig[mu][a][b];                       /* s^mu  */
                GAM[mu][2 + a][b] = (mu == 0 ? 1.0 : -1.0) * sig[mu][a][b]; /* sb^mu */
            }
    gam_ready = 1;
}

/* slash(J) = gamma^mu J_mu (J given with upper index) */
static void slash_c(const cx J[4], cx S[4][4])
{
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c)
            S[r][c] = GAM[0][r][c] * J[0] - GAM[1][r][c] * J[1] - GAM[2][r][c] * J[2] - GAM[3][r][c] * J[3];
}
static void slash_r(const double q[4], cx S[4][4])
{
    cx J[4] = {q[0], q[1], q[2], q[3]};
    slash_c(J, S);
}
static void row_times(const cx x[4], cx M[4][4], cx out[4])
{
    for (int c = 0; c < 4; ++c) {
        cx s = 0;
        for (int r = 0; r < 4; ++r) s += x[r] * M[r][c];
        out[c] = s;
    }
}
static void mat_times_col(cx M[4][4], const cx x[4], cx out[4])
{
    for (int r = 0; r < 4; ++r) {
        cx s = 0;
        for (int c = 0; c < 4; ++c) s += M[r][c] * x[c];
        out[r] = s;
    }
}

/* ------------------------------------------------------------------ */
/* External states (Sec. 3.1: vxxxxx / ixxxxx / oxxxxx compute these)  */
/* ------------------------------------------------------------------ */
static void chi(const double p[4], int lam, cx out[2])
{
    double px = p[1], py = p[2], pz = p[3];
    double P = sqrt(px * px + py * py + pz * pz);
    if (P == 0.0) { /* at rest: quantise along +z */
        if (lam > 0) { out[0] = 1; out[1] = 0; }
        else { out[0] = 0; out[1] = 1; }
        return;
    }
    double ppz = (pz >= 0) ? P + pz : (px * px + py * py) / (P - pz);
    if (ppz == 0.0) { /* along -z */
        if (lam > 0) { out[0] = 0; out[1] = 1; }
        else { out[0] = -1; out[1] = 0; }
        return;
    }
    double n = sqrt(2.0 * P * ppz);
    if (lam > 0) { out[0] = ppz / n; out[1] = (px + I * py) / n; }
    else { out[0] = (-px + I * py) / n; out[1] = ppz / n; }
}

static void omegas(const double p[4], double m, double *wp, double *wm)
{
    double P = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
    double E = p[0];
    *wp = sqrt(E + P);
    *wm = (m == 0.0) ? 0.0 : sqrt(m * m / (E + P));
}

void orc_spinor_u(const double p[4], double m, int lam, cx u[4])
{
    cx c[2];
    double wp, wm;
    chi(p, lam, c);
    omegas(p, m, &wp, &wm);
    double wl = lam > 0 ? wp : wm, wml = lam > 0 ? wm : wp; /* w_l, w_{-l} */
    u[0] = wml * c[0]; u[1] = wml * c[1];
    u[2] = wl * c[0];  u[3] = wl * c[1];
}

void orc_spinor_v(const double p[4], double m, int lam, cx v[4])
{
    cx c[2];
    double wp, wm;
    chi(p, -lam, c);
    omegas(p, m, &wp, &wm);
    double wl = lam > 0 ? wp : wm, wml = lam > 0 ? wm : wp;
    v[0] = -lam * wl * c[0]; v[1] = -lam * wl * c[1];
    v[2] = lam * wml * c[0]; v[3] = lam * wml * c[1];
}

/* Dirac adjoint psibar = psi^dagger gamma^0, returned as a row spinor */
void orc_bar(const cx s[4], cx sb[4])
{
    sb[0] = conj(s[2]); sb[1] = conj(s[3]); sb[2] = conj(s[0]); sb[3] = conj(s[1]);
}

void orc_polvec(const double k[4], int lam, cx eps[4])
{
    double kx = k[1], ky = k[2], kz = k[3];
    double pt = sqrt(kx * kx + ky * ky);
    double P = sqrt(kx * kx + ky * ky + kz * kz);
    double ct = kz / P, st = pt / P;
    double cf = (pt > 0) ? kx / pt : 1.0, sf = (pt > 0) ? ky / pt : 0.0;
    double e1[4] = {0, ct * cf, ct * sf, -st};
    double e2[4] = {0, -sf, cf, 0};
    for (int mu = 0; mu < 4; ++mu) eps[mu] = (-lam * e1[mu] - I * e2[mu]) / sqrt(2.0);
}

/* ------------------------------------------------------------------ */
/* RAMBO phase space (Sec. 4; Kleiss, Stirling, Ellis 1986)           */
/* ------------------------------------------------------------------ */
/* counter layout: (event index, attempt, final-state particle, 0); key (seed, 0) */
static void rambo_uniforms(uint64_t seed, int64_t ev, int attempt, int j, double r[4])
{
    uint64_t ctr[4] = {(uint64_t)ev, (uint64_t)attempt, (uint64_t)j, 0};
    uint64_t key[2] = {seed, 0};
    uint64_t o[4];
    orc_philox4x64_10(ctr, key, o);
    for (int i = 0; i < 4; ++i) r[i] = orc_u01(o[i]);
}

static double factorial(int n) { double f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; }

/* One RAMBO point for nfin final-state particles.  Returns 0, or -1 when the
 * Newton solve for the massive rescaling does not converge.  mom[j][4] are the
 * final-state momenta, *wt the phase-space weight (2 pi)^{4-3n} normalisation. */
static int rambo_point(uint64_t seed, int64_t ev, int attempt, double sqrt_s, const double *m, int n,
                       double mom[][4], double *wt)
{
    double q[MAXPAR][4], Q[4] = {0, 0, 0, 0};
    for (int j = 0; j < n; ++j) {
        double r[4];
        rambo_uniforms(seed, ev, attempt, j, r);
        double c = 2.0 * r[0] - 1.0, s = sqrt(1.0 - c * c), f = 2.0 * M_PI * r[1];
        double q0 = -log(r[2] * r[3]);
        q[j][0] = q0; q[j][1] = q0 * s * cos(f); q[j][2] = q0 * s * sin(f); q[j][3] = q0 * c;
        for (int mu = 0; mu < 4; ++mu) Q[mu] += q[j][mu];
    }
    double M = sqrt(mdot(Q, Q));
    double b[3] = {-Q[1] / M, -Q[2] / M, -Q[3] / M};
    double x = sqrt_s / M, gam = Q[0] / M, a = 1.0 / (1.0 + gam);
    for (int j = 0; j < n; ++j) {
        double bq = b[0] * q[j][1] + b[1] * q[j][2] + b[2] * q[j][3];
        mom[j][0] = x * (gam * q[j][0] + bq);
        for (int i = 0; i < 3; ++i) mom[j][i + 1] = x * (q[j][i + 1] + b[i] * q[j][0] + a * bq * b[i]);
    }
    double w = pow(M_PI / 2.0, n - 1) * pow(sqrt_s * sqrt_s, n - 2) / (factorial(n - 1) * factorial(n - 2));
    w *= pow(2.0 * M_PI, 4 - 3 * n);
    double msum = 0;
    int massive = 0;
    for (int j = 0; j < n; ++j) { msum += m[j]; if (m[j] > 0) massive = 1; }
    if (massive) {
        /* solve sum_j sqrt(m_j^2 + xi^2 |p_j|^2) = sqrt_s by Newton's method */
        double P2[MAXPAR];
        for (int j = 0; j < n; ++j) P2[j] = mom[j][0] * mom[j][0]; /* massless: |p|^2 = E^2 */
        double xi = sqrt(1.0 - (msum / sqrt_s) * (msum / sqrt_s));
        int ok = 0;
        for (int it = 0; it < 50; ++it) {
            double f = -sqrt_s, fp = 0;
            for (int j = 0; j < n; ++j) {
                double e = sqrt(m[j] * m[j] + xi * xi * P2[j]);
                f += e; fp += xi * P2[j] / e;
            }
            if (fabs(f) <= 1e-14 * sqrt_s) { ok = 1; break; }
            xi -= f / fp;
        }
        if (!ok) return -1;
        double wt2 = 1, wt3 = 0;
        for (int j = 0; j < n; ++j) {
            double k0 = sqrt(m[j] * m[j] + xi * xi * P2[j]);
            for (int i = 1; i < 4; ++i) mom[j][i] *= xi;
            mom[j][0] = k0;
            double kk = xi * sqrt(P2[j]);
            wt2 *= kk / k0;
            wt3 += kk * kk / k0;
        }
        w *= pow(xi, 2 * n - 3) * wt2 * sqrt_s / wt3;
    }
    *wt = w;
    return 0;
}

static double pseudorapidity(const double p[4])
{
    double P = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
    return 0.5 * log((P + p[3]) / (P - p[3]));
}

/* gluon cuts: pT > ptmin for each flagged particle, Delta R > drmin for each flagged pair */
static int pass_cuts(double mom[][4], int n, const int *is_cut, double ptmin, double drmin)
{
    for (int i = 0; i < n; ++i) {
        if (!is_cut[i]) continue;
        double pt = sqrt(mom[i][1] * mom[i][1] + mom[i][2] * mom[i][2]);
        if (!(pt > ptmin)) return 0;
    }
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            if (!is_cut[i] || !is_cut[j]) continue;
            double de = pseudorapidity(mom[i]) - pseudorapidity(mom[j]);
            double dphi = atan2(mom[i][2], mom[i][1]) - atan2(mom[j][2], mom[j][1]);
            while (dphi > M_PI) dphi -= 2 * M_PI;
            while (dphi < -M_PI) dphi += 2 * M_PI;
            if (!(sqrt(de * de + dphi * dphi) > drmin)) return 0;
        }
    return 1;
}

/* Events ev0 .. ev0+nevt-1: momenta [nevt][nfin+2][4] with the two incoming
 * partons along +z and -z (E = sqrt_s/2), weights [nevt], attempts [nevt].
 * Returns 0, -2 if an event needs more than 1000 attempts, -3 on a Newton failure. */
int orc_rambo(uint64_t seed, double sqrt_s, const double *mfin, int nfin, int64_t ev0, int64_t nevt,
              const int *is_cut, double ptmin, double drmin, double *mom_out, double *wt_out, int *att_out)
{
    int status = 0;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nevt; ++e) {
        double mom[MAXPAR][4], wt = 0;
        int att, done = 0;
        for (att = 0; att < 1000; ++att) {
            if (rambo_point(seed, ev0 + e, att, sqrt_s, mfin, nfin, mom, &wt) != 0) {
#pragma omp atomic write
                status = -3;
                break;
            }
            if (!is_cut || pass_cuts(mom, nfin, is_cut, ptmin, drmin)) { done = 1; break; }
        }
        if (!done && status == 0) {
#pragma omp atomic write
            status = -2;
        }
        double *o = mom_out + (size_t)e * (nfin + 2) * 4;
        o[0] = sqrt_s / 2; o[1] = 0; o[2] = 0; o[3] = sqrt_s / 2;
        o[4] = sqrt_s / 2; o[5] = 0; o[6] = 0; o[7] = -sqrt_s / 2;
        for (int j = 0; j < nfin; ++j)
            for (int mu = 0; mu < 4; ++mu) o[8 + 4 * j + mu] = mom[j][mu];
        if (wt_out) wt_out[e] = wt;
        if (att_out) att_out[e] = att;
    }
    return status;
}

/* ------------------------------------------------------------------ */
/* Processes                                                           */
/* ------------------------------------------------------------------ */
/* 0 ee_mumu: e-(in) e+(in) mu-(out) mu+(out)
 * 1..4 gg_ttx + k-2 gluons: g(in) g(in) t(out) tbar(out) g(out)... */
int orc_npar(int proc) { return proc == 0 ? 4 : proc + 3; }
int orc_ngluon(int proc) { return proc == 0 ? 0 : proc + 1; }
double orc_iden(int proc)
{
    /* spin average 2*2, colour average 8*8 for gg, identical final gluons n! */
    if (proc == 0) return 4.0;
    return 4.0 * 64.0 * factorial(proc - 1);
}

static int gluon_pos(int proc, int i) /* external index of the i-th gluon */
{
    (void)proc;
    return i < 2 ? i : i + 2;
}

/* lexicographic permutations of {0..k-1}; perm[idx][pos] */
static int next_perm(int *a, int k)
{
    int i = k - 2;
    while (i >= 0 && a[i] >= a[i + 1]) --i;
    if (i < 0) return 0;
    int j = k - 1;
    while (a[j] <= a[i]) --j;
    int t = a[i]; a[i] = a[j]; a[j] = t;
    for (int l = i + 1, r = k - 1; l < r; ++l, --r) { t = a[l]; a[l] = a[r]; a[r] = t; }
    return 1;
}
int orc_perms(int k, int *out)
{
    int a[MAXG], n = 0;
    for (int i = 0; i < k; ++i) a[i] = i;
    do { for (int i = 0; i < k; ++i) out[n * k + i] = a[i]; ++n; } while (next_perm(a, k));
    return n;
}

/* ------------------------------------------------------------------ */
/* SU(3): Gell-Mann generators T^a = lambda^a / 2, structure constants */
/* ------------------------------------------------------------------ */
static cx TG[8][3][3];
static double FABC[8][8][8];
static int su3_ready = 0;

static void init_su3(void)
{
    if (su3_ready) return;
    memset(TG, 0, sizeof TG);
    double s3 = 1.0 / sqrt(3.0);
    TG[0][0][1] = TG[0][1][0] = 0.5;
    TG[1][0][1] = -0.5 * I; TG[1][1][0] = 0.5 * I;
    TG[2][0][0] = 0.5; TG[2][1][1] = -0.5;
    TG[3][0][2] = TG[3][2][0] = 0.5;
    TG[4][0][2] = -0.5 * I; TG[4][2][0] = 0.5 * I;
    TG[5][1][2] = TG[5][2][1] = 0.5;
    TG[6][1][2] = -0.5 * I; TG[6][2][1] = 0.5 * I;
    TG[7][0][0] = TG[7][1][1] = 0.5 * s3; TG[7][2][2] = -s3;
    /* f^{abc} = -2 i Tr([T^a, T^b] T^c) */
    for (int a = 0; a < 8; ++a)
        for (int b = 0; b < 8; ++b)
            for (int c = 0; c < 8; ++c) {
                cx tr = 0;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        for (int l = 0; l < 3; ++l)
                            tr += (TG[a][i][j] * TG[b][j][l] - TG[b][i][j] * TG[a][j][l]) * TG[c][l][i];
                FABC[a][b][c] = creal(-2.0 * I * tr);
            }
    su3_ready = 1;
}

void orc_su3(double *T_re_im /*[8][3][3][2]*/, double *f /*[8][8][8]*/)
{
    init_su3();
    for (int a = 0; a < 8; ++a)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                T_re_im[((a * 3 + i) * 3 + j) * 2] = creal(TG[a][i][j]);
                T_re_im[((a * 3 + i) * 3 + j) * 2 + 1] = cimag(TG[a][i][j]);
            }
    memcpy(f, FABC, sizeof FABC);
}

/* Colour matrix of the string basis for k gluons, by brute force over all
 * adjoint indices a_1..a_k in 1..8 and fundamental end indices i, j. */
int orc_colour_matrix(int k, double *C /*[k!][k!]*/)
{
    init_su3();
    int perms[MAXPERM * MAXG];
    int np = orc_perms(k, perms);
    long ncfg = 1;
    for (int i = 0; i < k; ++i) ncfg *= 8;
    memset(C, 0, sizeof(double) * np * np);
#pragma omp parallel
    {
        double *Cl = calloc((size_t)np * np, sizeof(double));
        cx (*S)[3][3] = malloc(sizeof(cx) * 9 * np);
#pragma omp for schedule(static)
        for (long cfg = 0; cfg < ncfg; ++cfg) {
            int a[MAXG];
            long r = cfg;
            for (int i = 0; i < k; ++i) { a[i] = (int)(r % 8); r /= 8; }
            for (int s = 0; s < np; ++s) {
                cx M[3][3];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) M[i][j] = TG[a[perms[s * k]]][i][j];
                for (int l = 1; l < k; ++l) {
                    cx N[3][3];
                    const cx (*T)[3] = TG[a[perms[s * k + l]]];
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j)
                            N[i][j] = M[i][0] * T[0][j] + M[i][1] * T[1][j] + M[i][2] * T[2][j];
                    memcpy(M, N, sizeof M);
                }
                memcpy(S[s], M, sizeof M);
            }
            for (int s = 0; s < np; ++s)
                for (int t = 0; t < np; ++t) {
                    cx acc = 0;
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j) acc += conj(S[s][i][j]) * S[t][i][j];
                    Cl[s * np + t] += creal(acc);
                }
        }
#pragma omp critical
        for (int i = 0; i < np * np; ++i) C[i] += Cl[i];
        free(Cl);
        free(S);
    }
    return np;
}

static double *colour_cache[MAXG + 1];

static const double *colour_matrix_cached(int k)
{
    if (!colour_cache[k]) {
        int np = (int)factorial(k);
        double *C = malloc(sizeof(double) * np * np);
        orc_colour_matrix(k, C);
        colour_cache[k] = C;
    }
    return colour_cache[k];
}

/* ------------------------------------------------------------------ */
/* Vertices shared by the colour-ordered and colour-dressed recursions */
/* ------------------------------------------------------------------ */
/* V^{mnr}(k1,k2,k3) J1_m J2_n with k3 = -k1-k2 (all incoming), open index r up */
static void v3(const cx J1[4], const double k1[4], const cx J2[4], const double k2[4], cx out[4])
{
    double k3[4], d12[4], d23[4], d31[4];
    for (int mu = 0; mu < 4; ++mu) {
        k3[mu] = -k1[mu] - k2[mu];
        d12[mu] = k1[mu] - k2[mu];
        d23[mu] = k2[mu] - k3[mu];
        d31[mu] = k3[mu] - k1[mu];
    }
    cx j12 = cdot(J1, J2), a = rcdot(d23, J1), b = rcdot(d31, J2);
    for (int mu = 0; mu < 4; ++mu) out[mu] = j12 * d12[mu] + J2[mu] * a + J1[mu] * b;
}

/* ------------------------------------------------------------------ */
/* Colour-ordered Berends-Giele recursion: one quark line + k gluons    */
/* ------------------------------------------------------------------ */
/* eps[i], P[i]: wavefunction and OUTGOING momentum of the gluon at colour
 * position i (already permuted).  ubar: outgoing-quark row spinor with momentum
 * pt; v: outgoing-antiquark column spinor.  Returns the partial amplitude with
 * couplings stripped (M = g^k sum S_sigma A_sigma). */
/* Off-shell gluon currents J[i][j] of every contiguous colour-ordered range
 * i..j of the k gluons (Berends-Giele), with their summed momenta PS[i][j]. */
static void gluon_currents(int k, cx eps[][4], double P[][4], cx J[MAXG][MAXG][4], double PS[MAXG][MAXG][4])
{
    for (int len = 1; len <= k; ++len)
        for (int i = 0; i + len - 1 < k; ++i) {
            int j = i + len - 1;
            if (len == 1) {
                memcpy(J[i][i], eps[i], sizeof(cx) * 4);
                memcpy(PS[i][i], P[i], sizeof(double) * 4);
                continue;
            }
            for (int mu = 0; mu < 4; ++mu) PS[i][j][mu] = PS[i][i][mu] + PS[i + 1][j][mu];
            cx tmp[4] = {0, 0, 0, 0};
            for (int m = i; m < j; ++m) { /* three-gluon vertex, colour-ordered: -i V */
                double kL[4], kR[4];
                for (int mu = 0; mu < 4; ++mu) { kL[mu] = -PS[i][m][mu]; kR[mu] = -PS[m + 1][j][mu]; }
                cx o[4];
                v3(J[i][m], kL, J[m + 1][j], kR, o);
                for (int mu = 0; mu < 4; ++mu) tmp[mu] += -I * o[mu];
            }
            for (int m = i; m < j; ++m) /* four-gluon vertex, colour-ordered */
                for (int n = m + 1; n < j; ++n) {
                    const cx *A = J[i][m], *B = J[m + 1][n], *Cc = J[n + 1][j];
                    cx ac = cdot(A, Cc), ab = cdot(A, B), bc = cdot(B, Cc);
                    for (int mu = 0; mu < 4; ++mu)
                        tmp[mu] += I * (2.0 * ac * B[mu] - ab * Cc[mu] - bc * A[mu]);
                }
            double p2 = mdot(PS[i][j], PS[i][j]);
            for (int mu = 0; mu < 4; ++mu) J[i][j][mu] = (-I / p2) * tmp[mu];
        }
}

static cx bg_partial(int k, cx eps[][4], double P[][4], const cx ubar[4], const double pt[4], double mt,
                     const cx v[4])
{
    cx J[MAXG][MAXG][4];
    double PS[MAXG][MAXG][4];
    gluon_currents(k, eps, P, J, PS);
    /* quark line from the outgoing quark */
    cx U[MAXG + 1][4];
    memcpy(U[0], ubar, sizeof(cx) * 4);
    cx amp = 0;
    for (int j = 1; j <= k; ++j) {
        cx X[4] = {0, 0, 0, 0};
        for (int m = 0; m < j; ++m) {
            cx S[4][4], t[4];
            slash_c(J[m][j - 1], S);
            row_times(U[m], S, t);
            for (int c = 0; c < 4; ++c) X[c] += I * t[c];
        }
        if (j < k) {
            double q[4];
            for (int mu = 0; mu < 4; ++mu) q[mu] = pt[mu] + PS[0][j - 1][mu];
            cx S[4][4], t[4];
            slash_r(q, S);
            for (int r = 0; r < 4; ++r) S[r][r] += mt;
            row_times(X, S, t);
            double den = mdot(q, q) - mt * mt;
            for (int c = 0; c < 4; ++c) U[j][c] = I * t[c] / den;
        } else {
            for (int c = 0; c < 4; ++c) amp += X[c] * v[c];
        }
    }
    return amp;
}

/* external wavefunctions of the QCD processes for helicity index h */
static void qcd_externals(int proc, const double *p, double mt, int h, int gauge_gluon, cx eps[][4],
                          double P[][4], cx ubar[4], cx v[4])
{
    int npar = orc_npar(proc), k = orc_ngluon(proc);
    for (int g = 0; g < k; ++g) {
        int e = gluon_pos(proc, g);
        int lam = ((h >> (npar - 1 - e)) & 1) ? 1 : -1;
        const double *pe = p + 4 * e;
        int incoming = e < 2;
        if (g == gauge_gluon) {
            for (int mu = 0; mu < 4; ++mu) eps[g][mu] = pe[mu];
        } else {
            orc_polvec(pe, lam, eps[g]);
            if (!incoming)
                for (int mu = 0; mu < 4; ++mu) eps[g][mu] = conj(eps[g][mu]);
        }
        for (int mu = 0; mu < 4; ++mu) P[g][mu] = incoming ? -pe[mu] : pe[mu];
    }
    int lt = ((h >> (npar - 1 - 2)) & 1) ? 1 : -1;
    int ltb = ((h >> (npar - 1 - 3)) & 1) ? 1 : -1;
    cx u[4];
    orc_spinor_u(p + 8, mt, lt, u);
    orc_bar(u, ubar);
    orc_spinor_v(p + 12, mt, ltb, v);
}

/* all k! colour-ordered partial amplitudes for one event and helicity */
int orc_partial_amps(int proc, const double *p, double mt, int h, int gauge_gluon, cx *A_out)
{
    init_gamma();
    int k = orc_ngluon(proc);
    if (k < 2) return -1;
    cx eps[MAXG][4], ubar[4], v[4];
    double P[MAXG][4];
    qcd_externals(proc, p, mt, h, gauge_gluon, eps, P, ubar, v);
    int perms[MAXPERM * MAXG];
    int np = orc_perms(k, perms);
    for (int s = 0; s < np; ++s) {
        cx e2[MAXG][4];
        double P2[MAXG][4];
        for (int i = 0; i < k; ++i) {
            memcpy(e2[i], eps[perms[s * k + i]], sizeof(cx) * 4);
            memcpy(P2[i], P[perms[s * k + i]], sizeof(double) * 4);
        }
        A_out[s] = bg_partial(k, e2, P2, ubar, p + 8, mt, v);
    }
    return np;
}

/* ------------------------------------------------------------------ */
/* e+ e- -> mu+ mu- via one s-channel photon                           */
/* ------------------------------------------------------------------ */
static double ee_hel(const double *p, int h)
{
    int l[4];
    for (int i = 0; i < 4; ++i) l[i] = ((h >> (3 - i)) & 1) ? 1 : -1;
    cx u1[4], v2[4], v2b[4], u3[4], u3b[4], v4[4];
    orc_spinor_u(p + 0, 0.0, l[0], u1);
    orc_spinor_v(p + 4, 0.0, l[1], v2);
    orc_bar(v2, v2b);
    orc_spinor_u(p + 8, 0.0, l[2], u3);
    orc_bar(u3, u3b);
    orc_spinor_v(p + 12, 0.0, l[3], v4);
    cx je[4], jm[4];
    for (int mu = 0; mu < 4; ++mu) {
        cx t[4];
        row_times(v2b, GAM[mu], t);
        je[mu] = t[0] * u1[0] + t[1] * u1[1] + t[2] * u1[2] + t[3] * u1[3];
        row_times(u3b, GAM[mu], t);
        jm[mu] = t[0] * v4[0] + t[1] * v4[1] + t[2] * v4[2] + t[3] * v4[3];
    }
    double s = mdot((double[4]){p[0] + p[4], p[1] + p[5], p[2] + p[6], p[3] + p[7]},
                    (double[4]){p[0] + p[4], p[1] + p[5], p[2] + p[6], p[3] + p[7]});
    cx amp = cdot(je, jm) / s; /* couplings e^2 applied by the caller */
    return creal(amp * conj(amp));
}

/* ------------------------------------------------------------------ */
/* |M|^2 per event (colour-ordered recursion + brute-force colour)      */
/* ------------------------------------------------------------------ */
static double me2_event(int proc, const double *p, double mt, double alpha, double *hel_out)
{
    int npar = orc_npar(proc), nhel = 1 << npar;
    double tot = 0;
    if (proc == 0) {
        double e2 = 4.0 * M_PI * alpha;
        for (int h = 0; h < nhel; ++h) {
            double v = e2 * e2 * ee_hel(p, h);
            if (hel_out) hel_out[h] = v;
            tot += v;
        }
        return tot / orc_iden(proc);
    }
    int k = orc_ngluon(proc), np = (int)factorial(k);
    const double *C = colour_matrix_cached(k);
    double gk = pow(4.0 * M_PI * alpha, k); /* g^{2k} */
    cx A[MAXPERM];
    for (int h = 0; h < nhel; ++h) {
        orc_partial_amps(proc, p, mt, h, -1, A);
        double s = 0;
        for (int a = 0; a < np; ++a) {
            cx row = 0;
            for (int b = 0; b < np; ++b) row += C[a * np + b] * A[b];
            s += creal(conj(A[a]) * row);
        }
        double v = gk * s;
        if (hel_out) hel_out[h] = v;
        tot += v;
    }
    return tot / orc_iden(proc);
}

int orc_me2(int proc, const double *mom, int64_t nevt, double mt, double alpha, double *me2_out,
            double *hel_out, int nthreads)
{
    if (proc < 0 || proc > 4) return -1;
    init_gamma();
    init_su3();
    if (proc > 0) colour_matrix_cached(orc_ngluon(proc));
    int npar = orc_npar(proc), nhel = 1 << npar;
    /* nthreads > 0 limits this call only; the process-wide default stays */
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
    for (int64_t e = 0; e < nevt; ++e)
        me2_out[e] = me2_event(proc, mom + (size_t)e * npar * 4, mt, alpha, hel_out ? hel_out + (size_t)e * nhel : NULL);
    return 0;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Colour-dressed brute force: explicit colour indices, full Feynman   */
/* rules (f^{abc}, T^a), unordered subset recursion, no decomposition. */
/* ------------------------------------------------------------------ */
static double F4A[8][8][8][8], F4B[8][8][8][8], F4C[8][8][8][8];
static int f4_ready = 0;

static void init_f4(void)
{
    if (f4_ready) return;
    init_su3();
    for (int a = 0; a < 8; ++a)
        for (int b = 0; b < 8; ++b)
            for (int c = 0; c < 8; ++c)
                for (int d = 0; d < 8; ++d) {
                    double x = 0, y = 0, z = 0;
                    for (int e = 0; e < 8; ++e) {
                        x += FABC[a][b][e] * FABC[c][d][e];
                        y += FABC[a][c][e] * FABC[b][d][e];
                        z += FABC[a][d][e] * FABC[b][c][e];
                    }
                    F4A[a][b][c][d] = x; F4B[a][b][c][d] = y; F4C[a][b][c][d] = z;
                }
    f4_ready = 1;
}

/* one colour configuration: gluon colours ag[k], quark colour it, antiquark jt */
static cx dressed_amp(int k, cx eps[][4], double P[][4], const int *ag, int it, int jt, const cx ubar[4],
                      const double pt[4], double mt, const cx v[4])
{
    int nsub = 1 << k;
    static __thread cx Jd[1 << MAXG][8][4];
    static __thread double PSd[1 << MAXG][4];
    for (int S = 1; S < nsub; ++S) {
        int pc = __builtin_popcount(S);
        memset(PSd[S], 0, sizeof PSd[S]);
        for (int g = 0; g < k; ++g)
            if (S >> g & 1)
                for (int mu = 0; mu < 4; ++mu) PSd[S][mu] += P[g][mu];
        memset(Jd[S], 0, sizeof Jd[S]);
        if (pc == 1) {
            int g = __builtin_ctz(S);
            memcpy(Jd[S][ag[g]], eps[g], sizeof(cx) * 4);
            continue;
        }
        cx tmp[8][4];
        memset(tmp, 0, sizeof tmp);
        int low = S & -S;
        /* unordered pairs {A, B}: A holds the lowest gluon of S */
        for (int A = (S - 1) & S; A > 0; A = (A - 1) & S) {
            if (!(A & low)) continue;
            int B = S ^ A;
            if (!B) continue;
            double kA[4], kB[4];
            for (int mu = 0; mu < 4; ++mu) { kA[mu] = -PSd[A][mu]; kB[mu] = -PSd[B][mu]; }
            for (int a = 0; a < 8; ++a)
                for (int b = 0; b < 8; ++b) {
                    cx o[4];
                    v3(Jd[A][a], kA, Jd[B][b], kB, o);
                    for (int c = 0; c < 8; ++c) {
                        double f = FABC[a][b][c];
                        if (f == 0) continue;
                        for (int mu = 0; mu < 4; ++mu) tmp[c][mu] += f * o[mu];
                    }
                }
        }
        /* unordered triples {A, B, C}: A holds the lowest gluon, B the lowest of the rest */
        for (int A = S; A > 0; A = (A - 1) & S) {
            if (!(A & low) || A == S) continue;
            int R = S ^ A, lowR = R & -R;
            for (int B = R; B > 0; B = (B - 1) & R) {
                if (!(B & lowR) || B == R) continue;
                int Cm = R ^ B;
                for (int a = 0; a < 8; ++a)
                    for (int b = 0; b < 8; ++b)
                        for (int c = 0; c < 8; ++c) {
                            const cx *J1 = Jd[A][a], *J2 = Jd[B][b], *J3 = Jd[Cm][c];
                            cx j13 = cdot(J1, J3), j23 = cdot(J2, J3), j12 = cdot(J1, J2);
                            cx X1[4], X2[4], X3[4];
                            for (int mu = 0; mu < 4; ++mu) {
                                X1[mu] = j13 * J2[mu] - j23 * J1[mu];
                                X2[mu] = j12 * J3[mu] - j23 * J1[mu];
                                X3[mu] = j12 * J3[mu] - j13 * J2[mu];
                            }
                            for (int d = 0; d < 8; ++d) {
                                double fa = F4A[a][b][c][d], fb = F4B[a][b][c][d], fc = F4C[a][b][c][d];
                                if (fa == 0 && fb == 0 && fc == 0) continue;
                                for (int mu = 0; mu < 4; ++mu)
                                    tmp[d][mu] += -I * (fa * X1[mu] + fb * X2[mu] + fc * X3[mu]);
                            }
                        }
            }
        }
        double p2 = mdot(PSd[S], PSd[S]);
        for (int c = 0; c < 8; ++c)
            for (int mu = 0; mu < 4; ++mu) Jd[S][c][mu] = (-I / p2) * tmp[c][mu];
    }
    /* quark line: U[S][colour][spinor], S = gluons already attached */
    static __thread cx U[1 << MAXG][3][4];
    memset(U, 0, sizeof(cx) * nsub * 12);
    memcpy(U[0][it], ubar, sizeof(cx) * 4);
    cx amp = 0;
    for (int S = 1; S < nsub; ++S) {
        cx X[3][4];
        memset(X, 0, sizeof X);
        for (int A = S; A > 0; A = (A - 1) & S) { /* A = last attached cluster */
            int Rm = S ^ A;
            for (int a = 0; a < 8; ++a) {
                cx Sl[4][4];
                slash_c(Jd[A][a], Sl);
                for (int c = 0; c < 3; ++c) {
                    cx t[4];
                    row_times(U[Rm][c], Sl, t);
                    for (int c2 = 0; c2 < 3; ++c2) {
                        cx tc = TG[a][c][c2];
                        if (tc == 0) continue;
                        for (int s = 0; s < 4; ++s) X[c2][s] += I * tc * t[s];
                    }
                }
            }
        }
        if (S != nsub - 1) {
            double q[4];
            for (int mu = 0; mu < 4; ++mu) q[mu] = pt[mu] + PSd[S][mu];
            cx Sq[4][4];
            slash_r(q, Sq);
            for (int r = 0; r < 4; ++r) Sq[r][r] += mt;
            double den = mdot(q, q) - mt * mt;
            for (int c = 0; c < 3; ++c) {
                cx t[4];
                row_times(X[c], Sq, t);
                for (int s = 0; s < 4; ++s) U[S][c][s] = I * t[s] / den;
            }
        } else {
            for (int s = 0; s < 4; ++s) amp += X[jt][s] * v[s];
        }
    }
    return amp;
}

/* colour-summed |M_h|^2 (couplings included, no averaging) for the listed helicities */
int orc_me2_dressed(int proc, const double *p, double mt, double alpha, const int *hels, int nh,
                    double *out)
{
    if (proc < 1 || proc > 4) return -1;
    init_gamma();
    init_f4();
    int k = orc_ngluon(proc);
    long ncol = 9;
    for (int i = 0; i < k; ++i) ncol *= 8;
    double gk = pow(4.0 * M_PI * alpha, k);
    for (int ih = 0; ih < nh; ++ih) {
        cx eps[MAXG][4], ubar[4], v[4];
        double P[MAXG][4];
        qcd_externals(proc, p, mt, hels[ih], -1, eps, P, ubar, v);
        double sum = 0;
#pragma omp parallel for reduction(+ : sum) schedule(dynamic, 16)
        for (long cfg = 0; cfg < ncol; ++cfg) {
            long r = cfg;
            int it = (int)(r % 3); r /= 3;
            int jt = (int)(r % 3); r /= 3;
            int ag[MAXG];
            for (int i = 0; i < k; ++i) { ag[i] = (int)(r % 8); r /= 8; }
            cx a = dressed_amp(k, eps, P, ag, it, jt, ubar, p + 8, mt, v);
            sum += creal(a * conj(a));
        }
        out[ih] = gk * sum;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Closed forms                                                        */
/* ------------------------------------------------------------------ */
/* e+e- -> mu+mu- (massless, photon only), spin averaged: e^4 (1 + cos^2 theta) */
double orc_closed_ee(const double *p, double alpha)
{
    double e2 = 4.0 * M_PI * alpha;
    double P1 = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
    double P3 = sqrt(p[9] * p[9] + p[10] * p[10] + p[11] * p[11]);
    double c = (p[1] * p[9] + p[2] * p[10] + p[3] * p[11]) / (P1 * P3);
    return e2 * e2 * (1.0 + c * c);
}

/* gg -> Q Qbar, spin/colour averaged (Combridge 1979):
 * g^4 [1/(6 t1 t2) - 3/8] [t1^2 + t2^2 + rho - rho^2/(4 t1 t2)],
 * t1 = (m^2 - t)/s, t2 = (m^2 - u)/s, rho = 4 m^2 / s. */
double orc_closed_ggtt(const double *p, double mt, double alpha_s)
{
    double P[4], T[4], Uu[4];
    for (int mu = 0; mu < 4; ++mu) {
        P[mu] = p[mu] + p[4 + mu];
        T[mu] = p[mu] - p[8 + mu];
        Uu[mu] = p[mu] - p[12 + mu];
    }
    double s = mdot(P, P), t = mdot(T, T), u = mdot(Uu, Uu), m2 = mt * mt;
    double t1 = (m2 - t) / s, t2 = (m2 - u) / s, rho = 4 * m2 / s;
    double g2 = 4.0 * M_PI * alpha_s;
    return g2 * g2 * (1.0 / (6 * t1 * t2) - 3.0 / 8.0) * (t1 * t1 + t2 * t2 + rho - rho * rho / (4 * t1 * t2));
}

/* ------------------------------------------------------------------ */
/* Feynman diagrams one by one: single-diagram-enhancement weights     */
/* ------------------------------------------------------------------ */
/* The paper's multi-channel integration weights a phase-space channel by
 * |amp_d|^2 / sum_d' |amp_d'|^2, amp_d the amplitude of one Feynman diagram,
 * summed over helicities (its single-diagram enhancement).  Here every tree
 * diagram of g g -> t tbar + n g is enumerated directly (independently of the
 * colour-ordered recursion above) and evaluated with the bare vertex factors:
 * no couplings and no factors of i, so amp_d is fixed up to a phase.
 *
 *   gluon tree: a leaf (external gluon), a three-gluon vertex with two
 *     children, or a four-gluon vertex with three children; children are
 *     unordered.  A four-gluon vertex has three Lorentz structures (one per
 *     colour structure), (A.C)B-(B.C)A, (A.B)C-(B.C)A, (A.B)C-(A.C)B, each a
 *     separate amplitude of the same diagram; |amp_d|^2 sums them.
 *   current of a tree with leaf set S (outgoing momentum P_S): the vertex
 *     contracted with the children's currents, times 1/P_S^2.
 *   diagram: an ordered sequence of trees along the quark line, read from the
 *     outgoing t (ubar) to the outgoing tbar (v), leaf sets partitioning the
 *     gluons; amp = ubar [J1.gamma] S(q1) [J2.gamma] ... [Jm.gamma] v with
 *     S(q) = (qslash + m) / (q^2 - m^2), q_j = p_t + sum_{i<=j} P_i.
 *     (m = 1: the single tree meets the t tbar pair directly.)
 * A diagram is identified by its internal lines: each line is the set of
 * external particles on one side of it (the side without the tbar), and a
 * tree diagram is fixed by this set of splits.  Counting a four-gluon vertex
 * once gives 3, 16, 123, 1240 diagrams for 2..5 gluons. */

#define SDE_MAXTREE 1024   /* distinct gluon trees over all subsets of 5 gluons */
#define SDE_MAXVAR 9       /* four-gluon structure variants of one tree (<= 2 vertices) */
#define SDE_MAXDIAG 1300
#define SDE_MAXLINES 4

typedef struct {
    int mask;        /* leaf set (bits over gluon positions) */
    int kind;        /* 0 leaf, 3 three-gluon, 4 four-gluon */
    int child[3];
    int nvar;        /* structure variants */
    int leaf;        /* gluon position of a leaf */
} sde_tree;

typedef struct {
    int m;                  /* trees along the quark line */
    int tree[MAXG];
    int nlines;
    int lines[SDE_MAXLINES]; /* internal-line masks over external particles, sorted */
} sde_diag;

static sde_tree sde_trees[SDE_MAXTREE];
static int sde_ntree;
static int sde_first[1 << MAXG], sde_count[1 << MAXG]; /* trees of each leaf set (contiguous) */
static sde_diag sde_diags[MAXG + 1][SDE_MAXDIAG];
static int sde_ndiag[MAXG + 1];
static int sde_k = -1; /* gluon count the tables above were built for */

static int lowbit(int x) { return x & -x; }

/* all trees with leaf set S, appended contiguously (children first) */
static void sde_build_trees(int k)
{
    sde_ntree = 0;
    for (int S = 1; S < (1 << k); ++S) {
        /* subsets in increasing order: every proper subset is done before S */
        sde_first[S] = sde_ntree;
        if ((S & (S - 1)) == 0) {
            sde_tree t = {S, 0, {-1, -1, -1}, 1, __builtin_ctz(S)};
            sde_trees[sde_ntree++] = t;
        } else {
            int lo = lowbit(S);
            /* three-gluon vertex: {A, B}, A holds the lowest leaf */
            for (int A = (S - 1) & S; A > 0; A = (A - 1) & S) {
                if (!(A & lo)) continue;
                int B = S & ~A;
                for (int a = 0; a < sde_count[A]; ++a)
                    for (int b = 0; b < sde_count[B]; ++b) {
                        int ta = sde_first[A] + a, tb = sde_first[B] + b;
                        sde_tree t = {S, 3, {ta, tb, -1}, sde_trees[ta].nvar * sde_trees[tb].nvar, -1};
                        sde_trees[sde_ntree++] = t;
                    }
            }
            /* four-gluon vertex: {A, B, C}, A holds the lowest leaf of S, B the
             * lowest leaf of S \ A */
            for (int A = (S - 1) & S; A > 0; A = (A - 1) & S) {
                if (!(A & lo)) continue;
                int R = S & ~A, lo2 = lowbit(R);
                for (int B = (R - 1) & R; B > 0; B = (B - 1) & R) {
                    if (!(B & lo2)) continue;
                    int C = R & ~B;
                    for (int a = 0; a < sde_count[A]; ++a)
                        for (int b = 0; b < sde_count[B]; ++b)
                            for (int c = 0; c < sde_count[C]; ++c) {
                                int ta = sde_first[A] + a, tb = sde_first[B] + b, tc = sde_first[C] + c;
                                sde_tree t = {S, 4, {ta, tb, tc},
                                              3 * sde_trees[ta].nvar * sde_trees[tb].nvar * sde_trees[tc].nvar, -1};
                                sde_trees[sde_ntree++] = t;
                            }
                }
            }
        }
        sde_count[S] = sde_ntree - sde_first[S];
    }
}

static int sde_ext_mask(int proc, int gmask)
{
    int m = 0;
    for (int g = 0; gmask; ++g, gmask >>= 1)
        if (gmask & 1) m |= 1 << gluon_pos(proc, g);
    return m;
}

static void sde_tree_lines(int proc, int t, int *lines, int *n)
{
    const sde_tree *T = &sde_trees[t];
    if (T->kind == 0) return;
    lines[(*n)++] = sde_ext_mask(proc, T->mask);
    for (int c = 0; c < (T->kind == 3 ? 2 : 3); ++c) sde_tree_lines(proc, T->child[c], lines, n);
}

static int cmp_int(const void *a, const void *b) { return *(const int *)a - *(const int *)b; }

static void sde_add_diagram(int proc, int k, const int *seq, int m)
{
    sde_diag *D = &sde_diags[k][sde_ndiag[k]++];
    D->m = m;
    int n = 0, side = 1 << 2; /* the t side of a quark propagator: t and the gluons before it */
    for (int i = 0; i < m; ++i) {
        D->tree[i] = seq[i];
        sde_tree_lines(proc, seq[i], D->lines, &n);
        side |= sde_ext_mask(proc, sde_trees[seq[i]].mask);
        if (i < m - 1) D->lines[n++] = side;
    }
    D->nlines = n;
    qsort(D->lines, n, sizeof(int), cmp_int);
}

static void sde_sequences(int proc, int k, int remaining, int *seq, int m)
{
    if (!remaining) {
        sde_add_diagram(proc, k, seq, m);
        return;
    }
    for (int A = remaining; A > 0; A = (A - 1) & remaining)
        for (int a = 0; a < sde_count[A]; ++a) {
            seq[m] = sde_first[A] + a;
            sde_sequences(proc, k, remaining & ~A, seq, m + 1);
        }
}

static void sde_init(int proc) /* not thread-safe: the tables are rebuilt when k changes */
{
    int k = orc_ngluon(proc);
    if (sde_k == k) return;
    sde_build_trees(k);
    sde_ndiag[k] = 0;
    int seq[MAXG];
    sde_sequences(proc, k, (1 << k) - 1, seq, 0);
    sde_k = k;
}

/* current variants of tree t for the externals eps / P */
static void sde_current(int t, cx eps[][4], double P[][4], cx cur[][SDE_MAXVAR][4], double PS[][4])
{
    const sde_tree *T = &sde_trees[t];
    if (T->kind == 0) {
        memcpy(cur[t][0], eps[T->leaf], sizeof(cx) * 4);
        memcpy(PS[t], P[T->leaf], sizeof(double) * 4);
        return;
    }
    int nc = T->kind == 3 ? 2 : 3;
    for (int mu = 0; mu < 4; ++mu) {
        PS[t][mu] = 0;
        for (int c = 0; c < nc; ++c) PS[t][mu] += PS[T->child[c]][mu];
    }
    double inv = 1.0 / mdot(PS[t], PS[t]);
    int v = 0;
    if (T->kind == 3) {
        const int a = T->child[0], b = T->child[1];
        double ka[4], kb[4];
        for (int mu = 0; mu < 4; ++mu) { ka[mu] = -PS[a][mu]; kb[mu] = -PS[b][mu]; }
        for (int va = 0; va < sde_trees[a].nvar; ++va)
            for (int vb = 0; vb < sde_trees[b].nvar; ++vb, ++v) {
                cx o[4];
                v3(cur[a][va], ka, cur[b][vb], kb, o);
                for (int mu = 0; mu < 4; ++mu) cur[t][v][mu] = inv * o[mu];
            }
    } else {
        const int a = T->child[0], b = T->child[1], c = T->child[2];
        for (int va = 0; va < sde_trees[a].nvar; ++va)
            for (int vb = 0; vb < sde_trees[b].nvar; ++vb)
                for (int vc = 0; vc < sde_trees[c].nvar; ++vc) {
                    const cx *A = cur[a][va], *B = cur[b][vb], *C = cur[c][vc];
                    cx ab = cdot(A, B), ac = cdot(A, C), bc = cdot(B, C);
                    for (int mu = 0; mu < 4; ++mu) {
                        cur[t][v][mu] = inv * (ac * B[mu] - bc * A[mu]);
                        cur[t][v + 1][mu] = inv * (ab * C[mu] - bc * A[mu]);
                        cur[t][v + 2][mu] = inv * (ab * C[mu] - ac * B[mu]);
                    }
                    v += 3;
                }
    }
}

/* sum over the variants of diagram D of |amp|^2 (one helicity) */
static double sde_diagram_w2(const sde_diag *D, cx cur[][SDE_MAXVAR][4], double PS[][4], const cx ubar[4],
                             const double pt[4], double mt, const cx v[4])
{
    int nv = 1;
    for (int i = 0; i < D->m; ++i) nv *= sde_trees[D->tree[i]].nvar;
    double w2 = 0;
    for (int var = 0; var < nv; ++var) {
        int rem = var;
        cx U[4];
        memcpy(U, ubar, sizeof(cx) * 4);
        double q[4] = {pt[0], pt[1], pt[2], pt[3]};
        for (int i = 0; i < D->m; ++i) {
            const int t = D->tree[i], nvt = sde_trees[t].nvar;
            cx S[4][4], X[4];
            slash_c(cur[t][rem % nvt], S);
            rem /= nvt;
            row_times(U, S, X);
            if (i < D->m - 1) {
                for (int mu = 0; mu < 4; ++mu) q[mu] += PS[t][mu];
                cx Q[4][4];
                slash_r(q, Q);
                for (int r = 0; r < 4; ++r) Q[r][r] += mt;
                row_times(X, Q, U);
                const double den = mdot(q, q) - mt * mt;
                for (int c = 0; c < 4; ++c) U[c] /= den;
            } else {
                cx a = X[0] * v[0] + X[1] * v[1] + X[2] * v[2] + X[3] * v[3];
                w2 += creal(a * conj(a));
            }
        }
    }
    return w2;
}

/* Per-diagram sum over the given helicities of |amp_d|^2 for one event.
 * Returns the number of diagrams; lines_out[d * 4 + i] (i < nlines_out[d])
 * are diagram d's internal-line masks over the external particles (sorted). */
int orc_sde(int proc, const double *p, double mt, const int *hels, int nh, double *w2_out, int *lines_out,
            int *nlines_out)
{
    init_gamma();
    if (proc == 0) { /* one diagram: the s-channel photon, line {e-, e+} */
        double s = 0;
        for (int i = 0; i < nh; ++i) s += ee_hel(p, hels[i]);
        w2_out[0] = s;
        lines_out[0] = 0x3;
        nlines_out[0] = 1;
        return 1;
    }
    if (proc < 1 || proc > 4) return -1;
    sde_init(proc);
    const int k = orc_ngluon(proc), nd = sde_ndiag[k];
    static __thread cx cur[SDE_MAXTREE][SDE_MAXVAR][4];
    static __thread double PS[SDE_MAXTREE][4];
    for (int d = 0; d < nd; ++d) {
        w2_out[d] = 0;
        nlines_out[d] = sde_diags[k][d].nlines;
        for (int i = 0; i < SDE_MAXLINES; ++i) lines_out[d * 4 + i] = i < sde_diags[k][d].nlines ? sde_diags[k][d].lines[i] : 0;
    }
    for (int ih = 0; ih < nh; ++ih) {
        cx eps[MAXG][4], ubar[4], v[4];
        double P[MAXG][4];
        qcd_externals(proc, p, mt, hels[ih], -1, eps, P, ubar, v);
        for (int t = 0; t < sde_ntree; ++t) sde_current(t, eps, P, cur, PS);
        for (int d = 0; d < nd; ++d) w2_out[d] += sde_diagram_w2(&sde_diags[k][d], cur, PS, ubar, p + 8, mt, v);
    }
    return nd;
}

/* ------------------------------------------------------------------ */
/* Drell-Yan u ubar -> e+ e- + n g through a photon and a Z             */
/* ------------------------------------------------------------------ */
/* Particles: 0 u (incoming), 1 ubar (incoming), 2 e+, 3 e-, 4.. gluons
 * (outgoing).  Electroweak parameters fixed (G_F scheme values): alpha =
 * 1/132.507, M_Z = 91.188, Gamma_Z = 2.441404, M_W = 80.419002, sin^2 theta_W
 * = 1 - M_W^2/M_Z^2.  Vertices -i gamma^mu (gL P_L + gR P_R) with
 * P_L = diag(1,1,0,0) (left-handed upper components): photon gL = gR = e Q;
 * Z gL = e (T3 - Q sw^2)/(sw cw), gR = -e Q sw^2/(sw cw).  Propagators
 * -i g_{mn}/s (photon) and -i g_{mn}/(s - M_Z^2 + i M_Z Gamma_Z) (Z; its
 * k_m k_n term vanishes on the conserved massless lepton current).  The
 * boson and the lepton pair enter the quark line as one colourless insertion
 * i gamma^mu (gL^u P_L + gR^u P_R) L_mu (the three factors -i combine to i),
 * L^mu = sum_V ubar(e-) gamma^mu (gL^e P_L + gR^e P_R) v(e+) / D_V.
 * Colour: M = g^n sum_sigma (T^{a_s1}..T^{a_sn})_{i j} A_sigma, the string
 * read along the quark line from the ubar end, n = 0 giving delta_ij. */
static const double DY_ALPHA = 1.0 / 132.507, DY_MZ = 91.188, DY_WZ = 2.441404, DY_MW = 80.419002;

static void dy_couplings(int boson, double t3, double q, double *gl, double *gr)
{
    const double e = sqrt(4.0 * M_PI * DY_ALPHA);
    const double cw = DY_MW / DY_MZ, sw = sqrt(1.0 - cw * cw);
    if (boson == 0) {
        *gl = *gr = e * q;
    } else {
        *gl = e * (t3 - q * sw * sw) / (sw * cw);
        *gr = -e * q * sw * sw / (sw * cw);
    }
}

/* lepton currents L_V^mu (upper index) of the photon (V = 0) and the Z (V = 1),
 * each divided by its propagator denominator; bosons: bit 0 photon, bit 1 Z
 * (a boson left out gets a zero current) */
void orc_dy_lepton_currents(const double *p_ep, const double *p_em, int l_ep, int l_em, int bosons, cx L[2][4])
{
    init_gamma();
    cx v[4], u[4], ub[4];
    orc_spinor_v(p_ep, 0.0, l_ep, v);
    orc_spinor_u(p_em, 0.0, l_em, u);
    orc_bar(u, ub);
    double q[4];
    for (int mu = 0; mu < 4; ++mu) q[mu] = p_ep[mu] + p_em[mu];
    const double s = mdot(q, q);
    for (int b = 0; b < 2; ++b) {
        for (int mu = 0; mu < 4; ++mu) L[b][mu] = 0;
        if (!((bosons >> b) & 1)) continue;
        double gl, gr;
        dy_couplings(b, -0.5, -1.0, &gl, &gr);
        const cx den = b == 0 ? (cx)s : s - DY_MZ * DY_MZ + I * DY_MZ * DY_WZ;
        const cx vc[4] = {gl * v[0], gl * v[1], gr * v[2], gr * v[3]}; /* (gL P_L + gR P_R) v */
        for (int mu = 0; mu < 4; ++mu) {
            cx t[4];
            row_times(ub, GAM[mu], t);
            L[b][mu] = (t[0] * vc[0] + t[1] * vc[1] + t[2] * vc[2] + t[3] * vc[3]) / den;
        }
    }
}

/* colour-ordered partial amplitude of u ubar -> e+ e- + n g for the gluons
 * in colour order eps[0..n-1] (outgoing momenta P): the quark line runs from
 * the ubar row spinor vb (fermion flow outgoing with momentum -p_ubar) to the
 * u column spinor u; the colourless insertion of the lepton currents L
 * (momentum qL) is placed at every position along the line */
static cx dy_partial(int n, cx eps[][4], double P[][4], const cx vb[4], const double p_ubar[4], const cx u[4],
                     cx L[2][4], const double qL[4])
{
    cx J[MAXG][MAXG][4];
    double PS[MAXG][MAXG][4];
    if (n > 0) gluon_currents(n, eps, P, J, PS);
    /* insertion matrix without its factor i: sum_V gamma^mu L_V,mu (gL^u P_L + gR^u P_R) */
    cx M[4][4];
    memset(M, 0, sizeof M);
    for (int b = 0; b < 2; ++b) {
        double gl, gr;
        dy_couplings(b, 0.5, 2.0 / 3.0, &gl, &gr);
        cx S[4][4];
        slash_c(L[b], S);
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) M[r][c] += S[r][c] * (c < 2 ? gl : gr);
    }
    /* U0[j]: gluons 0..j-1 attached, no insertion; U1[j]: gluons 0..j-1 and
     * the insertion attached; both carry their propagator */
    cx U0[MAXG + 1][4], U1[MAXG + 1][4];
    memcpy(U0[0], vb, sizeof(cx) * 4);
    cx amp = 0;
    for (int j = 0; j <= n; ++j) {
        double q0[4];
        for (int mu = 0; mu < 4; ++mu) q0[mu] = -p_ubar[mu] + (j > 0 ? PS[0][j - 1][mu] : 0.0);
        if (j > 0) { /* the gluon range m..j-1 attached last, no insertion yet */
            cx X[4] = {0, 0, 0, 0};
            for (int m = 0; m < j; ++m) {
                cx S[4][4], t[4];
                slash_c(J[m][j - 1], S);
                row_times(U0[m], S, t);
                for (int c = 0; c < 4; ++c) X[c] += I * t[c];
            }
            cx S[4][4], t[4];
            slash_r(q0, S);
            row_times(X, S, t);
            const double d0 = mdot(q0, q0);
            for (int c = 0; c < 4; ++c) U0[j][c] = I * t[c] / d0;
        }
        /* the insertion attached last (after gluons 0..j-1), or a gluon range
         * m..j-1 attached after it */
        cx Y[4], t[4];
        row_times(U0[j], M, t);
        for (int c = 0; c < 4; ++c) Y[c] = I * t[c];
        for (int m = 0; m < j; ++m) {
            cx S[4][4];
            slash_c(J[m][j - 1], S);
            row_times(U1[m], S, t);
            for (int c = 0; c < 4; ++c) Y[c] += I * t[c];
        }
        if (j == n) {
            for (int c = 0; c < 4; ++c) amp += Y[c] * u[c];
        } else {
            double q1[4];
            for (int mu = 0; mu < 4; ++mu) q1[mu] = q0[mu] + qL[mu];
            cx S[4][4];
            slash_r(q1, S);
            row_times(Y, S, t);
            const double d1 = mdot(q1, q1);
            for (int c = 0; c < 4; ++c) U1[j][c] = I * t[c] / d1;
        }
    }
    return amp;
}

/* external states of u ubar -> e+ e- + n g for helicity index h (bit
 * (npar-1-i) set: particle i has helicity +1); gauge_gluon >= 0 replaces that
 * gluon's polarisation by its momentum */
static void dy_externals(int n, const double *p, int h, int gauge_gluon, int bosons, cx eps[][4], double P[][4],
                         cx vb[4], cx u[4], cx L[2][4], double qL[4])
{
    const int npar = 4 + n;
    int l[4 + MAXG];
    for (int i = 0; i < npar; ++i) l[i] = ((h >> (npar - 1 - i)) & 1) ? 1 : -1;
    orc_spinor_u(p + 0, 0.0, l[0], u);
    cx v[4];
    orc_spinor_v(p + 4, 0.0, l[1], v);
    orc_bar(v, vb);
    orc_dy_lepton_currents(p + 8, p + 12, l[2], l[3], bosons, L);
    for (int mu = 0; mu < 4; ++mu) qL[mu] = p[8 + mu] + p[12 + mu];
    for (int g = 0; g < n; ++g) {
        const double *pe = p + 4 * (4 + g);
        if (g == gauge_gluon) {
            for (int mu = 0; mu < 4; ++mu) eps[g][mu] = pe[mu];
        } else {
            orc_polvec(pe, l[4 + g], eps[g]);
            for (int mu = 0; mu < 4; ++mu) eps[g][mu] = conj(eps[g][mu]);
        }
        for (int mu = 0; mu < 4; ++mu) P[g][mu] = pe[mu];
    }
}

/* all n! partial amplitudes (gluon orders lexicographic) of one event and helicity */
int orc_dy_partial_amps(int n, const double *p, int h, int gauge_gluon, int bosons, cx *A_out)
{
    if (n < 0 || n > 4) return -1;
    init_gamma();
    cx eps[MAXG][4], vb[4], u[4], L[2][4];
    double P[MAXG][4], qL[4];
    dy_externals(n, p, h, gauge_gluon, bosons, eps, P, vb, u, L, qL);
    if (n == 0) {
        A_out[0] = dy_partial(0, eps, P, vb, p + 4, u, L, qL);
        return 1;
    }
    int perms[MAXPERM * MAXG];
    const int np = orc_perms(n, perms);
    for (int s = 0; s < np; ++s) {
        cx e2[MAXG][4];
        double P2[MAXG][4];
        for (int i = 0; i < n; ++i) {
            memcpy(e2[i], eps[perms[s * n + i]], sizeof(cx) * 4);
            memcpy(P2[i], P[perms[s * n + i]], sizeof(double) * 4);
        }
        A_out[s] = dy_partial(n, e2, P2, vb, p + 4, u, L, qL);
    }
    return np;
}

/* the colour-ordered Berends-Giele amplitude of one quark line and k gluons
 * with given external wavefunctions (exposed for the identities that relate
 * the Drell-Yan recursion to the gluon recursion) */
void orc_bg_partial(int k, const cx *eps /*[k][4]*/, const double *P /*[k][4]*/, const cx ubar[4], const double pt[4],
                    double mt, const cx v[4], cx *out)
{
    init_gamma();
    cx e2[MAXG][4];
    double P2[MAXG][4];
    for (int i = 0; i < k; ++i) {
        memcpy(e2[i], eps + 4 * i, sizeof(cx) * 4);
        memcpy(P2[i], P + 4 * i, sizeof(double) * 4);
    }
    *out = bg_partial(k, e2, P2, ubar, pt, mt, v);
}

/* |M|^2 of u ubar -> e+ e- + n g per event: sum over all 2^(4+n) helicities
 * and colours, averaged over the initial spins (4) and colours (9), divided
 * by n! for the identical gluons; alpha_s for the gluon couplings */
int orc_dy_me2(int n, const double *mom, int64_t nevt, double alpha_s, int bosons, double *me2_out)
{
    if (n < 0 || n > 4) return -1;
    init_gamma();
    init_su3();
    const double *C = n > 0 ? colour_matrix_cached(n) : NULL;
    const int npar = 4 + n, nhel = 1 << npar, np = (int)factorial(n);
    const double gs2n = pow(4.0 * M_PI * alpha_s, n);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t e = 0; e < nevt; ++e) {
        const double *p = mom + (size_t)e * npar * 4;
        double tot = 0;
        cx A[MAXPERM];
        for (int h = 0; h < nhel; ++h) {
            orc_dy_partial_amps(n, p, h, -1, bosons, A);
            double s = 0;
            if (n == 0) {
                s = 3.0 * creal(A[0] * conj(A[0])); /* sum_ij |delta_ij|^2 = 3 */
            } else {
                for (int a = 0; a < np; ++a) {
                    cx row = 0;
                    for (int b = 0; b < np; ++b) row += C[a * np + b] * A[b];
                    s += creal(conj(A[a]) * row);
                }
            }
            tot += gs2n * s;
        }
        me2_out[e] = tot / (4.0 * 9.0 * factorial(n));
    }
    return 0;
}
