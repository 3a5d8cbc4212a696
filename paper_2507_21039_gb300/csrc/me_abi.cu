// C ABI of libme (declared in include/me.h): handles, pointer-kind detection,
// host staging, helicity filtering (arXiv:2507.21039 Sec. 3.1 "non-vanishing
// helicities"), dispatch to the generated per-process kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "me.h"
#include "me_pool.h"
#include "me_proc.h"

using me::LaunchArgs;
using me::ProcDesc;

struct me_handle {
    const ProcDesc* proc;
    int precision;
    int device;
    double mt;
    double alpha;
    double norm;          // (4 pi alpha)^power / (iden * cden)
    int nhel;
    int ngood;
    short good[128];      // host copy of the kept helicities
    short* d_hel;         // device copy
    // helicity sampling over the kept helicities: probabilities (adaptive:
    // the filter probe's mean share of each helicity mixed with a uniform
    // floor; or uniform), their cumulative sums and inverses (host), and the
    // cumulative sums and inverses on the device (d_hs[0..127], d_hs[128..255])
    double hs_mean[128];
    double hs_p[128], hs_cdf[128], hs_invp[128];
    double* d_hs;
    int hs_uniform;
    int filtered;
    int require_filter;
    int check_finite;
    int gauge_ext;
    // host-buffer pipeline: two streams (created on first use) and the events
    // that order them after / before the caller's stream
    std::mutex pipe_mutex;
    cudaStream_t pipe[2];
    cudaEvent_t fork, join[2];
    bool pipe_ready;
};

namespace {

constexpr int kMaxProbe = 16384;
constexpr double kFilterThreshold = 1e-14;

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int slots_for(int nlist)
{
    int s = 1;
    while (s < nlist && s < 32) s <<= 1;
    return s;
}

// per helicity, over the probe events: the maximum of |M_h|^2 / |M|^2 into
// ratio[h] (the filter decision) and its mean into ratio[nhel + h] (the
// helicity-sampling probabilities)
__global__ void filter_reduce(const double* __restrict__ hel_out, const double* __restrict__ me2, int nprobe,
                              int nhel, double* __restrict__ ratio)
{
    const int h = blockIdx.x;
    double m = 0.0, sum = 0.0;
    int cnt = 0;
    for (int e = threadIdx.x; e < nprobe; e += blockDim.x) {
        const double tot = me2[e];
        if (tot > 0.0 && isfinite(tot)) {
            const double r = hel_out[(long long)e * nhel + h] / tot;
            m = fmax(m, r);
            sum += r;
            ++cnt;
        }
    }
    __shared__ double red[256], reds[256];
    __shared__ int redc[256];
    red[threadIdx.x] = m;
    reds[threadIdx.x] = sum;
    redc[threadIdx.x] = cnt;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
            reds[threadIdx.x] += reds[threadIdx.x + s];
            redc[threadIdx.x] += redc[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ratio[h] = red[0];
        ratio[nhel + h] = redc[0] > 0 ? reds[0] / redc[0] : 0.0;
    }
}

__global__ void count_nonfinite(const double* __restrict__ p, long long n, unsigned long long* bad)
{
    unsigned long long local = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!isfinite(p[i])) ++local;
    if (local) atomicAdd(bad, local);
}

// helicity sampling: the kept helicity whose cumulative-probability bin holds
// u (the smallest i with u < cdf[i]; the last bin takes the rest) and 1 / p
__global__ void hsample_select(const double* __restrict__ u, long long n, const double* __restrict__ hs, int ngood,
                               const short* __restrict__ list, short* __restrict__ hel_ev, double* __restrict__ w_ev,
                               int* __restrict__ hel_out)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double x = u[e];
    int i = 0;
    while (i < ngood - 1 && !(x < hs[i])) ++i;
    hel_ev[e] = list[i];
    w_ev[e] = hs[128 + i];
    if (hel_out) hel_out[e] = list[i];
}

int launch_me(me_handle* h, int precision, const double* d_mom, int64_t nevt, double* d_me2, double* d_hel_out,
              const short* d_list, int nlist, cudaStream_t st, double* d_sde_w = nullptr, int sde_channel = 0,
              const short* d_hel_ev = nullptr, const double* d_w_ev = nullptr, void* d_jscratch = nullptr,
              size_t jscratch_bytes = 0)
{
    LaunchArgs a{};
    a.mom = d_mom;
    a.nevt = nevt;
    a.me2 = d_me2;
    a.hel_out = d_hel_out;
    a.hel_list = d_list;
    a.nlist = nlist;
    a.slots = slots_for(nlist);
    a.norm = h->norm;
    a.mt = h->mt;
    a.gauge_ext = h->gauge_ext;
    a.stream = st;
    a.sde_w = d_sde_w;
    a.sde_channel = sde_channel;
    a.hel_ev = d_hel_ev;
    a.w_ev = d_w_ev;
    if (d_hel_ev) a.slots = 1;
    a.jscratch = d_jscratch;
    a.jscratch_bytes = jscratch_bytes;
    cudaError_t e = h->proc->launch(precision, a);
    return e == cudaSuccess ? ME_OK : ME_ECUDA;
}

// Helicity-sampling probabilities over the kept helicities: adaptive,
// p_i = 0.9 q_i / sum q + 0.1 / ngood with q_i the mean share of helicity i in
// the filter probe (every kept helicity keeps probability >= 0.1 / ngood, so
// the estimator stays unbiased with bounded weights); or uniform, 1 / ngood.
// Cumulative sums are formed left to right in FP64; the last one is 1.
int set_hsample(me_handle* h)
{
    const int n = h->ngood;
    double q = 0.0;
    for (int i = 0; i < n; ++i) q += h->hs_mean[h->good[i]];
    double c = 0.0;
    for (int i = 0; i < n; ++i) {
        const double p = (h->hs_uniform || !(q > 0.0)) ? 1.0 / n : 0.9 * h->hs_mean[h->good[i]] / q + 0.1 / n;
        h->hs_p[i] = p;
        h->hs_invp[i] = 1.0 / p;
        c += p;
        h->hs_cdf[i] = i == n - 1 ? 1.0 : c;
    }
    double dev[256] = {};
    memcpy(dev, h->hs_cdf, sizeof(double) * n);
    memcpy(dev + 128, h->hs_invp, sizeof(double) * n);
    return cudaMemcpy(h->d_hs, dev, sizeof dev, cudaMemcpyHostToDevice) == cudaSuccess ? ME_OK : ME_ECUDA;
}

int set_good(me_handle* h, const short* list, int n)
{
    memcpy(h->good, list, sizeof(short) * n);
    h->ngood = n;
    if (cudaMemcpy(h->d_hel, h->good, sizeof(short) * n, cudaMemcpyHostToDevice) != cudaSuccess) return ME_ECUDA;
    return set_hsample(h);
}

// FP64 per-helicity evaluation of the probe events and the filter decision
int filter_device(me_handle* h, const double* d_mom, int64_t nevt)
{
    const int nprobe = (int)(nevt < kMaxProbe ? nevt : kMaxProbe);
    const int nhel = h->nhel;
    short all[128];
    for (int i = 0; i < nhel; ++i) all[i] = (short)i;
    double *d_hel_out = nullptr, *d_me2 = nullptr, *d_ratio = nullptr;
    short* d_all = nullptr;
    int rc = ME_OK;
    if (cudaMalloc(&d_hel_out, sizeof(double) * (size_t)nprobe * nhel) != cudaSuccess ||
        cudaMalloc(&d_me2, sizeof(double) * nprobe) != cudaSuccess ||
        cudaMalloc(&d_ratio, sizeof(double) * 2 * nhel) != cudaSuccess ||
        cudaMalloc(&d_all, sizeof(short) * nhel) != cudaSuccess) {
        rc = ME_ENOMEM;
    }
    double ratio[256];
    if (rc == ME_OK && cudaMemcpy(d_all, all, sizeof(short) * nhel, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = ME_ECUDA;
    if (rc == ME_OK) rc = launch_me(h, me::PREC_FP64, d_mom, nprobe, d_me2, d_hel_out, d_all, nhel, 0);
    if (rc == ME_OK) {
        filter_reduce<<<nhel, 256>>>(d_hel_out, d_me2, nprobe, nhel, d_ratio);
        if (cudaGetLastError() != cudaSuccess) rc = ME_ECUDA;
    }
    if (rc == ME_OK && cudaMemcpy(ratio, d_ratio, sizeof(double) * 2 * nhel, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = ME_ECUDA;
    cudaFree(d_hel_out);
    cudaFree(d_me2);
    cudaFree(d_ratio);
    cudaFree(d_all);
    if (rc != ME_OK) return rc;
    short good[128];
    int n = 0;
    for (int i = 0; i < nhel; ++i)
        if (ratio[i] > kFilterThreshold) good[n++] = (short)i;
    if (n == 0) {  // degenerate probe (all zero): keep everything
        for (int i = 0; i < nhel; ++i) good[i] = (short)i;
        n = nhel;
    }
    memcpy(h->hs_mean, ratio + nhel, sizeof(double) * nhel);
    rc = set_good(h, good, n);
    if (rc == ME_OK) h->filtered = 1;
    return rc;
}

int check_finite(const double* d_mom, int64_t n, cudaStream_t st)
{
    unsigned long long* d_bad = nullptr;
    unsigned long long bad = 0;
    if (me::staging_alloc(&d_bad, sizeof(unsigned long long), st) != cudaSuccess) return ME_ENOMEM;
    int rc = ME_OK;
    if (cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), st) != cudaSuccess) rc = ME_ECUDA;
    if (rc == ME_OK) {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 1;
        count_nonfinite<<<nsm * 4, 256, 0, st>>>(d_mom, n, d_bad);
        if (cudaGetLastError() != cudaSuccess) rc = ME_ECUDA;
    }
    if (rc == ME_OK && cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = ME_ECUDA;
    cudaFreeAsync(d_bad, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = ME_ECUDA;
    if (rc == ME_OK && bad) rc = ME_ENONFINITE;
    return rc;
}

}  // namespace

extern "C" {

const char* me_version(void) { return "libme 0.1 (sm_103a)"; }

const char* me_strerror(int status)
{
    switch (status) {
    case ME_OK: return "success";
    case ME_EINVAL: return "invalid argument";
    case ME_ENOMEM: return "out of memory";
    case ME_ECUDA: return "CUDA error";
    case ME_ENOTFILTERED: return "helicities not filtered";
    case ME_ENONFINITE: return "non-finite momenta";
    case ME_ETIMEOUT: return "timeout";
    case ME_ESAMPLER: return "phase-space sampler failed";
    case ME_ETOOLARGE: return "batch exceeds the library's static scratch";
    default: return "unknown status";
    }
}

int me_init(me_handle** hp, const char* process, const double* masses, int nmass, const double* couplings, int ncoup,
            int precision)
{
    if (!hp) return ME_EINVAL;
    *hp = nullptr;
    const ProcDesc* pd = me::find_process(process);
    if (!pd) return ME_EINVAL;
    if (precision < ME_PREC_FP64 || precision > ME_PREC_MIXED64) return ME_EINVAL;
    const bool qcd = pd->family == 1;      // g g -> t t~ + n g: massive tops
    const bool strong = pd->family != 0;   // couplings {alpha_s} (Drell-Yan: electroweak part fixed)
    double mt = qcd ? 173.0 : 0.0;
    if (nmass != 0 || masses) {
        if (!masses || nmass != pd->npar) return ME_EINVAL;
        for (int i = 0; i < nmass; ++i)
            if (!(masses[i] >= 0.0) || !std::isfinite(masses[i])) return ME_EINVAL;
        if (qcd) {
            if (masses[2] != masses[3]) return ME_EINVAL;
            for (int i = 0; i < nmass; ++i)
                if (i != 2 && i != 3 && masses[i] != 0.0) return ME_EINVAL;
            mt = masses[2];
        } else {
            for (int i = 0; i < nmass; ++i)
                if (masses[i] != 0.0) return ME_EINVAL;
        }
    }
    double alpha = strong ? 0.118 : 1.0 / 132.5;
    if (ncoup != 0 || couplings) {
        if (!couplings || ncoup != 1 || !(couplings[0] > 0.0) || !std::isfinite(couplings[0])) return ME_EINVAL;
        alpha = couplings[0];
    }
    me_handle* h = new (std::nothrow) me_handle();
    if (!h) return ME_ENOMEM;
    h->proc = pd;
    h->precision = precision;
    cudaGetDevice(&h->device);
    h->mt = mt;
    h->alpha = alpha;
    h->norm = std::pow(4.0 * M_PI * alpha, pd->coupling_power) / (pd->iden * pd->cden);
    h->nhel = pd->nhel;
    h->gauge_ext = -1;
    if (cudaMalloc(&h->d_hel, sizeof(short) * 128) != cudaSuccess) {
        delete h;
        return ME_ENOMEM;
    }
    if (cudaMalloc(&h->d_hs, sizeof(double) * 256) != cudaSuccess) {
        cudaFree(h->d_hel);
        delete h;
        return ME_ENOMEM;
    }
    short all[128];
    for (int i = 0; i < pd->nhel; ++i) all[i] = (short)i;
    if (set_good(h, all, pd->nhel) != ME_OK) {
        cudaFree(h->d_hel);
        cudaFree(h->d_hs);
        delete h;
        return ME_ECUDA;
    }
    *hp = h;
    return ME_OK;
}

void me_free(me_handle* h)
{
    if (!h) return;
    cudaDeviceSynchronize();
    cudaFree(h->d_hel);
    cudaFree(h->d_hs);
    if (h->pipe_ready) {
        for (int i = 0; i < 2; ++i) {
            cudaStreamDestroy(h->pipe[i]);
            cudaEventDestroy(h->join[i]);
        }
        cudaEventDestroy(h->fork);
    }
    delete h;
}

int me_set_option(me_handle* h, int option, int value)
{
    if (!h) return ME_EINVAL;
    switch (option) {
    case ME_OPT_REQUIRE_FILTER: h->require_filter = value != 0; return ME_OK;
    case ME_OPT_CHECK_FINITE: h->check_finite = value != 0; return ME_OK;
    case ME_OPT_HSAMPLE_UNIFORM:
        h->hs_uniform = value != 0;
        return set_hsample(h);
    case ME_OPT_GAUGE_CHECK:
        if (value < -1 || value >= h->proc->npar) return ME_EINVAL;
        if (value >= 0 && h->proc->ngluon == 0) return ME_EINVAL;
        // not a gluon: t, t~ (2, 3) of g g -> t t~ + n g; u, u~, e+, e- (0..3) of Drell-Yan
        if (value >= 0 && (value == 2 || value == 3 || (h->proc->family == 2 && value < 4))) return ME_EINVAL;
        h->gauge_ext = value;
        return ME_OK;
    default: return ME_EINVAL;
    }
}

int me_info(const me_handle* h, int* npar, int* nhel, int* ncol, int* ndiag, uint64_t* good_mask_words)
{
    if (!h) return ME_EINVAL;
    if (npar) *npar = h->proc->npar;
    if (nhel) *nhel = h->nhel;
    if (ncol) *ncol = h->proc->ncol;
    if (ndiag) *ndiag = h->proc->ndiag;
    if (good_mask_words) {
        good_mask_words[0] = good_mask_words[1] = 0;
        for (int i = 0; i < h->ngood; ++i) good_mask_words[h->good[i] >> 6] |= 1ULL << (h->good[i] & 63);
    }
    return ME_OK;
}

int me_good_helicities(const me_handle* h, int* out, int cap, int* n)
{
    if (!h || (!out && cap > 0)) return ME_EINVAL;
    for (int i = 0; i < h->ngood && i < cap; ++i) out[i] = h->good[i];
    if (n) *n = h->ngood;
    return ME_OK;
}

int me_flops_per_event(const me_handle* h, double* chain_flops, double* colour_flops)
{
    if (!h) return ME_EINVAL;
    if (chain_flops) *chain_flops = (double)h->ngood * (double)h->proc->flops_hel + (double)h->proc->table_flops;
    if (colour_flops) *colour_flops = (double)h->ngood * (double)h->proc->colour_flops_hel;
    return ME_OK;
}

int me_filter_helicities(me_handle* h, const double* momenta, int64_t nevt, int* ngood_out)
{
    if (!h || !momenta || nevt <= 0) return ME_EINVAL;
    const int64_t nprobe = nevt < kMaxProbe ? nevt : kMaxProbe;
    int rc;
    if (is_device_ptr(momenta)) {
        if (cudaDeviceSynchronize() != cudaSuccess) return ME_ECUDA;
        rc = filter_device(h, momenta, nprobe);
    } else {
        const size_t bytes = sizeof(double) * 4 * h->proc->npar * (size_t)nprobe;
        double* d = nullptr;
        if (cudaMalloc(&d, bytes) != cudaSuccess) return ME_ENOMEM;
        rc = cudaMemcpy(d, momenta, bytes, cudaMemcpyHostToDevice) == cudaSuccess ? ME_OK : ME_ECUDA;
        if (rc == ME_OK) rc = filter_device(h, d, nprobe);
        cudaFree(d);
    }
    if (rc == ME_OK && ngood_out) *ngood_out = h->ngood;
    return rc;
}

// Host momenta in, host |M|^2 out: the batch is processed in chunks on the
// handle's two streams, so that the copies of one chunk overlap the evaluation
// of the other (copy engines and SMs work at the same time).  The caller's
// stream orders the call: its earlier work comes first, and it waits for every
// chunk before the call returns.
#ifndef ME_PIPE_CHUNK_LOG2
#define ME_PIPE_CHUNK_LOG2 17  // build option: log2 of the events per host-pipeline chunk
#endif
constexpr int64_t kPipeChunk = int64_t(1) << ME_PIPE_CHUNK_LOG2;

static int sigmakin_host_pipelined(me_handle* h, const double* momenta, int64_t nevt, double* me2, cudaStream_t st)
{
    std::lock_guard<std::mutex> lock(h->pipe_mutex);
    if (!h->pipe_ready) {
        bool ok = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; i < 2 && ok; ++i)
            ok = cudaStreamCreateWithFlags(&h->pipe[i], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&h->join[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return ME_ECUDA;
        }
        h->pipe_ready = true;
    }
    const int64_t per = 4 * (int64_t)h->proc->npar;  // doubles per event
    double *d_mom = nullptr, *d_me2 = nullptr;
    if (me::staging_alloc(&d_mom, sizeof(double) * per * nevt, st) != cudaSuccess) return ME_ENOMEM;
    int rc = ME_OK;
    if (me::staging_alloc(&d_me2, sizeof(double) * nevt, st) != cudaSuccess) rc = ME_ENOMEM;
    if (rc == ME_OK && cudaEventRecord(h->fork, st) != cudaSuccess) rc = ME_ECUDA;
    for (int i = 0; i < 2 && rc == ME_OK; ++i)
        if (cudaStreamWaitEvent(h->pipe[i], h->fork, 0) != cudaSuccess) rc = ME_ECUDA;
    const int64_t chunk = std::max(kPipeChunk, (nevt + 7) / 8);
    for (int64_t c0 = 0, k = 0; c0 < nevt && rc == ME_OK; c0 += chunk, ++k) {
        const int64_t n = std::min(chunk, nevt - c0);
        cudaStream_t s = h->pipe[k & 1];
        if (cudaMemcpyAsync(d_mom + c0 * per, momenta + c0 * per, sizeof(double) * per * n, cudaMemcpyHostToDevice,
                            s) != cudaSuccess) {
            rc = ME_ECUDA;
            break;
        }
        rc = launch_me(h, h->precision, d_mom + c0 * per, n, d_me2 + c0, nullptr, h->d_hel, h->ngood, s);
        if (rc == ME_OK &&
            cudaMemcpyAsync(me2 + c0, d_me2 + c0, sizeof(double) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            rc = ME_ECUDA;
    }
    // join both streams into the caller's before the buffers are released
    for (int i = 0; i < 2; ++i) {
        if (cudaEventRecord(h->join[i], h->pipe[i]) != cudaSuccess || cudaStreamWaitEvent(st, h->join[i], 0) != cudaSuccess) {
            cudaStreamSynchronize(h->pipe[i]);
            if (rc == ME_OK) rc = ME_ECUDA;
        }
    }
    if (d_mom) cudaFreeAsync(d_mom, st);
    if (d_me2) cudaFreeAsync(d_me2, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == ME_OK) rc = ME_ECUDA;
    return rc;
}

static int sigmakin_impl(me_handle* h, const double* momenta, int64_t nevt, double* me2, double* hel_out,
                         cudaStream_t st)
{
    if (!h || nevt < 0) return ME_EINVAL;
    if (nevt == 0) return ME_OK;
    if (!momenta || !me2) return ME_EINVAL;
    const bool dm = is_device_ptr(momenta), dr = is_device_ptr(me2);
    if (hel_out && !(dm && dr && is_device_ptr(hel_out))) return ME_EINVAL;
    if (!h->filtered) {
        if (h->require_filter) return ME_ENOTFILTERED;
        if (dm && cudaStreamSynchronize(st) != cudaSuccess) return ME_ECUDA;
        int rc = me_filter_helicities(h, momenta, nevt, nullptr);
        if (rc != ME_OK) return rc;
    }
    const size_t mbytes = sizeof(double) * 4 * h->proc->npar * (size_t)nevt;
    if (dm && dr) {
        if (h->check_finite) {
            int rc = check_finite(momenta, (int64_t)(mbytes / sizeof(double)), st);
            if (rc != ME_OK) return rc;
        }
        return launch_me(h, h->precision, momenta, nevt, me2, hel_out, h->d_hel, h->ngood, st);
    }
    if (!dm && !dr && !h->check_finite && nevt >= 2 * kPipeChunk) return sigmakin_host_pipelined(h, momenta, nevt, me2, st);
    // other host buffers: stage through stream-ordered device memory, then wait
    double *d_mom = nullptr, *d_me2 = nullptr;
    int rc = ME_OK;
    if (!dm) {
        if (me::staging_alloc(&d_mom, mbytes, st) != cudaSuccess) return ME_ENOMEM;
        if (cudaMemcpyAsync(d_mom, momenta, mbytes, cudaMemcpyHostToDevice, st) != cudaSuccess) rc = ME_ECUDA;
    }
    if (rc == ME_OK && !dr && me::staging_alloc(&d_me2, sizeof(double) * nevt, st) != cudaSuccess) rc = ME_ENOMEM;
    const double* mom_use = dm ? momenta : d_mom;
    double* me2_use = dr ? me2 : d_me2;
    if (rc == ME_OK && h->check_finite) rc = check_finite(mom_use, (int64_t)(mbytes / sizeof(double)), st);
    if (rc == ME_OK) rc = launch_me(h, h->precision, mom_use, nevt, me2_use, nullptr, h->d_hel, h->ngood, st);
    if (rc == ME_OK && !dr &&
        cudaMemcpyAsync(me2, d_me2, sizeof(double) * nevt, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = ME_ECUDA;
    if (d_mom) cudaFreeAsync(d_mom, st);
    if (d_me2) cudaFreeAsync(d_me2, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == ME_OK) rc = ME_ECUDA;
    return rc;
}

int me_sigmakin(me_handle* h, const double* momenta, int64_t nevt, double* me2, void* cuda_stream)
{
    return sigmakin_impl(h, momenta, nevt, me2, nullptr, (cudaStream_t)cuda_stream);
}

int me_sigmakin_hel(me_handle* h, const double* momenta, int64_t nevt, double* me2, double* hel_out,
                    void* cuda_stream)
{
    if (!hel_out) return ME_EINVAL;
    return sigmakin_impl(h, momenta, nevt, me2, hel_out, (cudaStream_t)cuda_stream);
}

int me_sigmakin_sde(me_handle* h, const double* momenta, int64_t nevt, int channel, double* me2, double* weight,
                    void* cuda_stream)
{
    if (!h || nevt < 0 || channel < 0 || channel >= h->proc->ndiag) return ME_EINVAL;
    if (h->proc->family == 2) return ME_EINVAL;  // Drell-Yan: no channel weights (diagrams without line sets)
    if (nevt == 0) return ME_OK;
    if (!momenta || !me2 || !weight || !is_device_ptr(momenta) || !is_device_ptr(me2) || !is_device_ptr(weight))
        return ME_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (!h->filtered) {
        if (h->require_filter) return ME_ENOTFILTERED;
        if (cudaStreamSynchronize(st) != cudaSuccess) return ME_ECUDA;
        int rc = me_filter_helicities(h, momenta, nevt, nullptr);
        if (rc != ME_OK) return rc;
    }
    if (h->check_finite) {
        int rc = check_finite(momenta, nevt * 4 * h->proc->npar, st);
        if (rc != ME_OK) return rc;
    }
    return launch_me(h, h->precision, momenta, nevt, me2, nullptr, h->d_hel, h->ngood, st, weight, channel);
}

int me_sigmakin_hsample(me_handle* h, const double* momenta, int64_t nevt, const double* u, double* me2, int* hel,
                        void* cuda_stream)
{
    if (!h || nevt < 0) return ME_EINVAL;
    if (nevt == 0) return ME_OK;
    if (!momenta || !u || !me2 || !is_device_ptr(momenta) || !is_device_ptr(u) || !is_device_ptr(me2) ||
        (hel && !is_device_ptr(hel)))
        return ME_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (!h->filtered) {
        if (h->require_filter) return ME_ENOTFILTERED;
        if (cudaStreamSynchronize(st) != cudaSuccess) return ME_ECUDA;
        int rc = me_filter_helicities(h, momenta, nevt, nullptr);
        if (rc != ME_OK) return rc;
    }
    if (h->check_finite) {
        int rc = check_finite(momenta, nevt * 4 * h->proc->npar, st);
        if (rc != ME_OK) return rc;
    }
    short* d_hel_ev = nullptr;
    double* d_w_ev = nullptr;
    if (me::staging_alloc(&d_hel_ev, sizeof(short) * nevt, st) != cudaSuccess) return ME_ENOMEM;
    int rc = ME_OK;
    if (me::staging_alloc(&d_w_ev, sizeof(double) * nevt, st) != cudaSuccess) rc = ME_ENOMEM;
    if (rc == ME_OK) {
        hsample_select<<<(unsigned)((nevt + 255) / 256), 256, 0, st>>>(u, nevt, h->d_hs, h->ngood, h->d_hel, d_hel_ev,
                                                                       d_w_ev, hel);
        if (cudaGetLastError() != cudaSuccess) rc = ME_ECUDA;
    }
    if (rc == ME_OK)
        rc = launch_me(h, h->precision, momenta, nevt, me2, nullptr, h->d_hel, 1, st, nullptr, 0, d_hel_ev, d_w_ev);
    if (d_hel_ev) cudaFreeAsync(d_hel_ev, st);
    if (d_w_ev) cudaFreeAsync(d_w_ev, st);
    return rc;
}

int me_hsample_probabilities(const me_handle* h, double* p, int cap, int* n)
{
    if (!h || !n) return ME_EINVAL;
    *n = h->ngood;
    if (p) {
        if (cap < h->ngood) return ME_EINVAL;
        memcpy(p, h->hs_p, sizeof(double) * h->ngood);
    }
    return ME_OK;
}

int me_diagram_lines(const me_handle* h, int diagram, int* masks, int cap, int* n)
{
    if (!h || !n || diagram < 0 || diagram >= h->proc->ndiag || h->proc->family == 2) return ME_EINVAL;
    const int nl = h->proc->diag_nlines[diagram];
    *n = nl;
    if (masks) {
        if (cap < nl) return ME_EINVAL;
        for (int i = 0; i < nl; ++i) masks[i] = h->proc->diag_lines[4 * diagram + i];
    }
    return ME_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Helicity filter that allocates nothing.
//
// Some host programs cannot let a library allocate device memory: they reserve
// the device's memory up front through their own pool (and would see a library
// cudaMalloc fail or fragment that pool), or they run latency-critical loops in
// which cudaMalloc / cudaFree, which may synchronise the whole device, are not
// acceptable.  For them, me_filter_helicities_noalloc runs the same FP64
// per-helicity evaluation and reduction as me_filter_helicities, but keeps its
// scratch (per-event x per-helicity values, per-event totals, per-helicity
// ratios, the list of all helicities) in one fixed array compiled into this
// library instead of allocating it.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchBytes = size_t(4) << 20;  // 4 MiB on every device that loads the library
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_filter_scratch[kStaticScratchBytes];

std::mutex g_scratch_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_filter_scratch on the current device.  In host code the
// array's name is only a host-side stand-in; the runtime maps it to the
// current device's copy here, once per device, and the address is cached.
int scratch_address(void** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return ME_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_filter_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return ME_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return ME_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" int me_filter_helicities_noalloc(me_handle* h, const double* momenta, int64_t nevt, int* ngood_out)
{
    if (!h || !momenta || nevt <= 0) return ME_EINVAL;
    if (!is_device_ptr(momenta)) return ME_EINVAL;  // staging host momenta would need an allocation
    const int nhel = h->nhel;
    const size_t b_hel = align256(sizeof(double) * (size_t)nevt * nhel);
    const size_t b_me2 = align256(sizeof(double) * (size_t)nevt);
    const size_t b_ratio = align256(sizeof(double) * 2 * nhel);
    const size_t b_list = align256(sizeof(short) * nhel);
    const size_t used = b_hel + b_me2 + b_ratio + b_list;
    // the FP64 kernel of the largest process keeps its colour-flow vectors in
    // global memory: they come from the rest of the array, one CTA's worth at
    // least (fewer resident CTAs than a full launch when less is left)
    const size_t per_cta = h->proc->jscratch_per_cta(me::PREC_FP64);
    if ((size_t)nevt > kStaticScratchBytes || used > kStaticScratchBytes || kStaticScratchBytes - used < per_cta)
        return ME_ETOOLARGE;
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != ME_OK) return rc;
    unsigned char* sp = static_cast<unsigned char*>(base);
    double* d_hel_out = reinterpret_cast<double*>(sp);
    double* d_me2 = reinterpret_cast<double*>(sp + b_hel);
    double* d_ratio = reinterpret_cast<double*>(sp + b_hel + b_me2);
    short* d_all = reinterpret_cast<short*>(sp + b_hel + b_me2 + b_ratio);
    // every scratch word read below is written first in this call: the
    // per-helicity values and totals by the |M|^2 kernel, the ratios by the
    // reduction, the helicity list by the copy, the colour-flow vectors by the
    // kernel's own zeroing at the start of every event; nothing needs clearing
    short all[128];
    for (int i = 0; i < nhel; ++i) all[i] = (short)i;
    if (cudaDeviceSynchronize() != cudaSuccess) return ME_ECUDA;
    if (cudaMemcpy(d_all, all, sizeof(short) * nhel, cudaMemcpyHostToDevice) != cudaSuccess) return ME_ECUDA;
    void* d_j = per_cta ? static_cast<void*>(sp + used) : nullptr;
    rc = launch_me(h, me::PREC_FP64, momenta, nevt, d_me2, d_hel_out, d_all, nhel, 0, nullptr, 0, nullptr, nullptr,
                   d_j, per_cta ? kStaticScratchBytes - used : 0);
    if (rc != ME_OK) return rc;
    filter_reduce<<<nhel, 256>>>(d_hel_out, d_me2, (int)nevt, nhel, d_ratio);
    if (cudaGetLastError() != cudaSuccess) return ME_ECUDA;
    double ratio[256];
    if (cudaMemcpy(ratio, d_ratio, sizeof(double) * 2 * nhel, cudaMemcpyDeviceToHost) != cudaSuccess) return ME_ECUDA;
    short good[128];
    int n = 0;
    for (int i = 0; i < nhel; ++i)
        if (ratio[i] > kFilterThreshold) good[n++] = (short)i;
    if (n == 0) {
        for (int i = 0; i < nhel; ++i) good[i] = (short)i;
        n = nhel;
    }
    memcpy(h->hs_mean, ratio + nhel, sizeof(double) * nhel);
    rc = set_good(h, good, n);
    if (rc != ME_OK) return rc;
    h->filtered = 1;
    if (ngood_out) *ngood_out = h->ngood;
    return ME_OK;
}
