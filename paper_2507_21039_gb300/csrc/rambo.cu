// Seeded flat phase-space sampler on the device (arXiv:2507.21039 Sec. 4: the
// standalone application draws RAMBO points; RAMBO is Kleiss, Stirling, Ellis
// 1986).  One thread per event; the event depends only on (seed, index), so any
// range can be regenerated and sharded without communication.
//
// Random numbers: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), key
// (seed, 0), counter (event, attempt, final-particle index, 0); one block
// yields the four uniforms of one final-state particle, u = ((x >> 11) + 1/2) 2^-53.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "me.h"
#include "me_pool.h"

namespace {

constexpr int kMaxFinal = 6;
constexpr int kMaxAttempts = 1000;
#ifndef ME_PIPE_CHUNK_LOG2
#define ME_PIPE_CHUNK_LOG2 17  // build option: log2 of the events per host-output pipeline chunk
#endif
constexpr int64_t kPipeChunk = int64_t(1) << ME_PIPE_CHUNK_LOG2;

struct U4 { uint64_t x[4]; };

__device__ __forceinline__ U4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                                            uint64_t k1)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return {{c0, c1, c2, c3}};
}

__device__ __forceinline__ double u01(uint64_t x) { return ((double)(x >> 11) + 0.5) * 0x1p-53; }

struct Params {
    uint64_t seed;
    long long ev0, nevt;
    double sqrt_s;
    double m[kMaxFinal];
    int nfin;
    bool massive;
    double msum;
    double w0;  // massless weight (pi/2)^{n-1} s^{n-2} / ((n-1)!(n-2)!) (2 pi)^{4-3n}
    double ptmin, drmin;
    uint32_t cutmask;
    int chunk;  // events per warp (a multiple of 32)
    double* mom;
    double* wt;
    unsigned long long* nfail;
};

// generation cuts on the final particles selected by cutmask: pT > ptmin for
// each, Delta R = sqrt(Delta eta^2 + Delta phi^2) > drmin for each pair.  The
// pseudorapidity and azimuth of each particle are computed once.
// Delta R = sqrt(Delta eta^2 + Delta phi^2) of two momenta in FP64, Delta phi
// wrapped to [-pi, pi]
__device__ double delta_r(const double* ki, const double* kj)
{
    const double Pi = sqrt(ki[1] * ki[1] + ki[2] * ki[2] + ki[3] * ki[3]);
    const double Pj = sqrt(kj[1] * kj[1] + kj[2] * kj[2] + kj[3] * kj[3]);
    const double de = 0.5 * log((Pi + ki[3]) / (Pi - ki[3])) - 0.5 * log((Pj + kj[3]) / (Pj - kj[3]));
    double dphi = atan2(ki[2], ki[1]) - atan2(kj[2], kj[1]);
    while (dphi > M_PI) dphi -= 2.0 * M_PI;
    while (dphi < -M_PI) dphi += 2.0 * M_PI;
    return sqrt(de * de + dphi * dphi);
}

__device__ bool passes(const double (*k)[4], int n, const Params& a)
{
    if (!a.cutmask) return true;
    for (int i = 0; i < n; ++i) {
        if (!((a.cutmask >> i) & 1)) continue;
        if (!(sqrt(k[i][1] * k[i][1] + k[i][2] * k[i][2]) > a.ptmin)) return false;
    }
    if (__popc(a.cutmask) < 2) return true;  // no pairs
    // Delta R of each pair in FP32 (eta = asinh(pz / pT), well conditioned);
    // a pair within a guard band of the cut, far wider than the FP32 error of
    // Delta R, is decided in FP64 exactly as the definition states it
    constexpr float kBand = 1e-3f;
    float etf[kMaxFinal], phf[kMaxFinal];
    for (int i = 0; i < n; ++i) {
        if (!((a.cutmask >> i) & 1)) continue;
        const float px = (float)k[i][1], py = (float)k[i][2], pz = (float)k[i][3];
        etf[i] = asinhf(pz / sqrtf(px * px + py * py));
        phf[i] = atan2f(py, px);
    }
    const float drf = (float)a.drmin;
    const float lo2 = drf > kBand ? (drf - kBand) * (drf - kBand) : -1.0f, hi2 = (drf + kBand) * (drf + kBand);
    for (int i = 0; i < n; ++i) {
        if (!((a.cutmask >> i) & 1)) continue;
        for (int j = i + 1; j < n; ++j) {
            if (!((a.cutmask >> j) & 1)) continue;
            const float de = etf[i] - etf[j];
            float dphi = phf[i] - phf[j];
            if (dphi > (float)M_PI) dphi -= 2.0f * (float)M_PI;
            if (dphi < -(float)M_PI) dphi += 2.0f * (float)M_PI;
            const float dr2 = de * de + dphi * dphi;
            if (dr2 > hi2) continue;
            if (dr2 < lo2) return false;
            if (!(delta_r(k[i], k[j]) > a.drmin)) return false;  // near the cut (or not finite): FP64
        }
    }
    return true;
}

// one RAMBO point; returns false when the Newton solve does not converge
__device__ bool rambo_point(const Params& a, long long ev, int attempt, double (*k)[4], double& w)
{
    const int n = a.nfin;
    double q[kMaxFinal][4];
    double Q0 = 0, Q1 = 0, Q2 = 0, Q3 = 0;
    for (int j = 0; j < n; ++j) {
        const U4 r = philox4x64_10((uint64_t)ev, (uint64_t)attempt, (uint64_t)j, 0, a.seed, 0);
        const double c = 2.0 * u01(r.x[0]) - 1.0;
        const double s = sqrt(1.0 - c * c);
        const double f = 2.0 * M_PI * u01(r.x[1]);
        const double q0 = -log(u01(r.x[2]) * u01(r.x[3]));
        double sf, cf;
        sincos(f, &sf, &cf);
        q[j][0] = q0;
        q[j][1] = q0 * s * cf;
        q[j][2] = q0 * s * sf;
        q[j][3] = q0 * c;
        Q0 += q[j][0];
        Q1 += q[j][1];
        Q2 += q[j][2];
        Q3 += q[j][3];
    }
    const double M = sqrt(Q0 * Q0 - Q1 * Q1 - Q2 * Q2 - Q3 * Q3);
    const double b1 = -Q1 / M, b2 = -Q2 / M, b3 = -Q3 / M;
    const double x = a.sqrt_s / M, gam = Q0 / M, aa = 1.0 / (1.0 + gam);
    for (int j = 0; j < n; ++j) {
        const double bq = b1 * q[j][1] + b2 * q[j][2] + b3 * q[j][3];
        k[j][0] = x * (gam * q[j][0] + bq);
        k[j][1] = x * (q[j][1] + b1 * q[j][0] + aa * bq * b1);
        k[j][2] = x * (q[j][2] + b2 * q[j][0] + aa * bq * b2);
        k[j][3] = x * (q[j][3] + b3 * q[j][0] + aa * bq * b3);
    }
    w = a.w0;
    if (!a.massive) return true;
    double P2[kMaxFinal];
    for (int j = 0; j < n; ++j) P2[j] = k[j][0] * k[j][0];
    const double r = a.msum / a.sqrt_s;
    // Newton for xi: first in FP32 (fast square roots and divisions) to about
    // FP32 resolution, then in FP64 to the FP64 tolerance (one or two steps
    // from there, as the convergence is quadratic)
    float xf = sqrtf(1.0f - (float)(r * r));
    const float sf = (float)a.sqrt_s;
    for (int it = 0; it < 12; ++it) {
        float f = -sf, fp = 0.0f;
        for (int j = 0; j < n; ++j) {
            const float p2 = (float)P2[j], m = (float)a.m[j];
            const float e = sqrtf(fmaf(xf * xf, p2, m * m));
            f += e;
            fp += xf * p2 / e;
        }
        if (fabsf(f) <= 4e-7f * sf) break;
        xf -= f / fp;
    }
    double xi = (xf > 0.0f && xf <= 1.0f) ? (double)xf : sqrt(1.0 - r * r);
    bool ok = false;
    double e[kMaxFinal];  // energies at the converged xi (the loop stops before updating it)
    for (int it = 0; it < 50; ++it) {
        double f = -a.sqrt_s, fp = 0.0;
        for (int j = 0; j < n; ++j) {
            e[j] = sqrt(a.m[j] * a.m[j] + xi * xi * P2[j]);
            f += e[j];
            fp += xi * P2[j] / e[j];
        }
        if (fabs(f) <= 1e-14 * a.sqrt_s) {
            ok = true;
            break;
        }
        xi -= f / fp;
    }
    if (!ok) return false;
    // weight factors; the energies of the converged solve are reused, |k_j| is xi
    // times the massless energy, and xi^(2n-3) is a product (FP64 square roots,
    // divisions and pow cost dozens of FP64-pipe instructions each on GB300)
    double wt2 = 1.0, wt3 = 0.0, xin = 1.0;
    for (int j = 0; j < n; ++j) {
        const double k0 = e[j];
        const double kk = xi * k[j][0];
        k[j][1] *= xi;
        k[j][2] *= xi;
        k[j][3] *= xi;
        k[j][0] = k0;
        wt2 *= kk / k0;
        wt3 += kk * kk / k0;
    }
    for (int j = 0; j < 2 * n - 3; ++j) xin *= xi;
    w *= xin * wt2 * a.sqrt_s / wt3;
    return true;
}

// Each warp generates a contiguous chunk of a.chunk events.  A lane that has
// finished its event (accepted, Newton failure, or out of attempts) takes the
// warp's next unstarted event, so lanes do not idle while a neighbour retries a
// rejected attempt (with one event per lane for the whole kernel, a warp runs as
// many attempts as its unluckiest lane).  Every attempt's random numbers depend
// only on (event, attempt), so which lane runs it does not change the result.
// Chunks of 256 events pay off when pair cuts reject often; without them one
// event per lane (chunk 32) keeps more warps in flight.
constexpr int kChunkCut = 256, kChunkPlain = 32;

__device__ void rambo_store(const Params& a, long long i, const double (*k)[4], double w, bool ok)
{
    const int npar = a.nfin + 2;
    double* o = a.mom + i * npar * 4;
    const double h = 0.5 * a.sqrt_s;
    o[0] = h; o[1] = 0.0; o[2] = 0.0; o[3] = h;
    o[4] = h; o[5] = 0.0; o[6] = 0.0; o[7] = -h;
    for (int j = 0; j < a.nfin; ++j)
        for (int mu = 0; mu < 4; ++mu) o[8 + 4 * j + mu] = k[j][mu];
    if (!ok) {
        w = -1.0;
        if (a.nfail) atomicAdd(a.nfail, 1ULL);
    }
    if (a.wt) a.wt[i] = w;
}

__global__ void rambo_kernel(Params a)
{
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long c0 = warp * a.chunk;
    if (c0 >= a.nevt) return;  // the whole warp leaves together
    const long long c1 = c0 + a.chunk < a.nevt ? c0 + a.chunk : a.nevt;
    long long i = c0 + lane;   // this lane's event (index into the batch)
    long long next = c0 + 32;  // the warp's next unstarted event (the same in every lane)
    int att = 0;
    for (;;) {
        const bool active = i < c1;
        if (!__any_sync(0xffffffffu, active)) break;
        bool finished = false;
        if (active) {
            double k[kMaxFinal][4];
            double w = 0.0;
            const bool newton_ok = rambo_point(a, a.ev0 + i, att, k, w);
            const bool done = newton_ok && passes(k, a.nfin, a);
            if (done || !newton_ok || att + 1 >= kMaxAttempts) {
                rambo_store(a, i, k, w, done);
                finished = true;
            } else {
                ++att;
            }
        }
        const unsigned fin = __ballot_sync(0xffffffffu, finished);
        if (finished) {
            i = next + __popc(fin & ((1u << lane) - 1u));
            att = 0;
        }
        next += __popc(fin);
    }
}

unsigned rambo_blocks(int64_t n, int chunk, int threads)
{
    const int64_t warps = (n + chunk - 1) / chunk;
    return (unsigned)((warps * 32 + threads - 1) / threads);
}

bool is_dev(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int rambo_sample(uint64_t seed, int64_t ev0, int64_t nevt, double sqrt_s, const double* masses, int npar,
                            const me_cuts* cuts, double* momenta_out, double* weights_out, int64_t* nfail_out,
                            void* cuda_stream)
{
    if (nevt < 0 || ev0 < 0 || npar < 3 || npar > kMaxFinal + 2 || !masses) return ME_EINVAL;
    if (nevt == 0) return ME_OK;
    if (!momenta_out || !(sqrt_s > 0.0) || masses[0] != 0.0 || masses[1] != 0.0) return ME_EINVAL;
    Params a{};
    a.seed = seed;
    a.ev0 = ev0;
    a.nevt = nevt;
    a.sqrt_s = sqrt_s;
    a.nfin = npar - 2;
    double msum = 0.0;
    for (int j = 0; j < a.nfin; ++j) {
        const double m = masses[2 + j];
        if (!(m >= 0.0)) return ME_EINVAL;
        a.m[j] = m;
        msum += m;
        if (m > 0.0) a.massive = true;
    }
    if (!(msum < sqrt_s)) return ME_EINVAL;
    a.msum = msum;
    const int n = a.nfin;
    double fact1 = 1.0, fact2 = 1.0;
    for (int i = 2; i <= n - 1; ++i) fact1 *= i;
    for (int i = 2; i <= n - 2; ++i) fact2 *= i;
    a.w0 = std::pow(M_PI / 2.0, n - 1) * std::pow(sqrt_s * sqrt_s, n - 2) / (fact1 * fact2) *
           std::pow(2.0 * M_PI, 4 - 3 * n);
    if (cuts) {
        a.ptmin = cuts->ptmin;
        a.drmin = cuts->drmin;
        a.cutmask = cuts->final_mask & ((1u << n) - 1u);
    }
    a.chunk = __builtin_popcount(a.cutmask) >= 2 ? kChunkCut : kChunkPlain;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const bool dev_m = is_dev(momenta_out);
    const bool dev_w = !weights_out || is_dev(weights_out);
    const size_t mbytes = sizeof(double) * 4 * npar * (size_t)nevt;
    double *d_m = nullptr, *d_w = nullptr;
    unsigned long long* d_fail = nullptr;
    int rc = ME_OK;
    if (!dev_m && me::staging_alloc(&d_m, mbytes, st) != cudaSuccess) return ME_ENOMEM;
    if (weights_out && !dev_w && me::staging_alloc(&d_w, sizeof(double) * nevt, st) != cudaSuccess) rc = ME_ENOMEM;
    const bool want_fail = nfail_out != nullptr || !dev_m || !dev_w;
    if (rc == ME_OK && want_fail) {
        if (me::staging_alloc(&d_fail, sizeof(unsigned long long), st) != cudaSuccess) rc = ME_ENOMEM;
        else if (cudaMemsetAsync(d_fail, 0, sizeof(unsigned long long), st) != cudaSuccess) rc = ME_ECUDA;
    }
    a.mom = dev_m ? momenta_out : d_m;
    a.wt = weights_out ? (dev_w ? weights_out : d_w) : nullptr;
    a.nfail = d_fail;
    const int th = 128;
    if (rc == ME_OK && !dev_m && nevt >= 2 * kPipeChunk) {
        // host output: chunks on two streams, so that the copy of one chunk
        // overlaps the sampling of the next; ordered after the caller's stream
        // and joined back into it
        cudaStream_t s2[2] = {nullptr, nullptr};
        cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
        bool ok = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess &&
                  cudaEventRecord(fork, st) == cudaSuccess;
        for (int i = 0; i < 2 && ok; ++i)
            ok = cudaStreamCreateWithFlags(&s2[i], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming) == cudaSuccess &&
                 cudaStreamWaitEvent(s2[i], fork, 0) == cudaSuccess;
        const int64_t chunk = std::max(kPipeChunk, (nevt + 7) / 8);
        const size_t per = sizeof(double) * 4 * npar;
        for (int64_t c0 = 0, k = 0; c0 < nevt && ok; c0 += chunk, ++k) {
            const int64_t n = std::min(chunk, nevt - c0);
            Params b = a;
            b.ev0 = a.ev0 + c0;
            b.nevt = n;
            b.mom = a.mom + c0 * 4 * npar;
            b.wt = a.wt ? a.wt + c0 : nullptr;
            rambo_kernel<<<rambo_blocks(n, a.chunk, th), th, 0, s2[k & 1]>>>(b);
            ok = cudaGetLastError() == cudaSuccess &&
                 cudaMemcpyAsync(reinterpret_cast<char*>(momenta_out) + c0 * per, b.mom, per * n, cudaMemcpyDeviceToHost,
                                 s2[k & 1]) == cudaSuccess;
            if (ok && d_w)
                ok = cudaMemcpyAsync(weights_out + c0, b.wt, sizeof(double) * n, cudaMemcpyDeviceToHost, s2[k & 1]) ==
                     cudaSuccess;
        }
        for (int i = 0; i < 2; ++i) {
            if (!s2[i]) continue;
            if (!join[i] || cudaEventRecord(join[i], s2[i]) != cudaSuccess || cudaStreamWaitEvent(st, join[i], 0) != cudaSuccess) {
                cudaStreamSynchronize(s2[i]);
                ok = false;
            }
        }
        for (int i = 0; i < 2; ++i) {
            if (s2[i]) cudaStreamDestroy(s2[i]);
            if (join[i]) cudaEventDestroy(join[i]);
        }
        if (fork) cudaEventDestroy(fork);
        if (!ok) {
            cudaGetLastError();
            rc = ME_ECUDA;
        }
    } else if (rc == ME_OK) {
        rambo_kernel<<<rambo_blocks(nevt, a.chunk, th), th, 0, st>>>(a);
        if (cudaGetLastError() != cudaSuccess) rc = ME_ECUDA;
        if (rc == ME_OK && !dev_m && cudaMemcpyAsync(momenta_out, d_m, mbytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            rc = ME_ECUDA;
        if (rc == ME_OK && d_w &&
            cudaMemcpyAsync(weights_out, d_w, sizeof(double) * nevt, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            rc = ME_ECUDA;
    }
    unsigned long long nfail = 0;
    if (rc == ME_OK && d_fail && cudaMemcpyAsync(&nfail, d_fail, sizeof(nfail), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = ME_ECUDA;
    if (d_m) cudaFreeAsync(d_m, st);
    if (d_w) cudaFreeAsync(d_w, st);
    if (d_fail) cudaFreeAsync(d_fail, st);
    if (want_fail && cudaStreamSynchronize(st) != cudaSuccess && rc == ME_OK) rc = ME_ECUDA;
    if (rc == ME_OK && nfail_out) *nfail_out = (int64_t)nfail;
    if (rc == ME_OK && nfail > 0) rc = ME_ESAMPLER;
    return rc;
}
