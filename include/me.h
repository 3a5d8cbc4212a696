/*
 * libme -- batched tree-level squared matrix elements on GB300 (sm_103a).
 *
 * C ABI of the data-parallel hot path of arXiv:2507.21039: for a batch of
 * phase-space points, the per-event |M|^2 summed over helicities and colours
 * (Sec. 3.1 "Parallel scattering amplitudes"), evaluated by a helicity-amplitude
 * chain and a colour contraction J^+ C J (Sec. 4.1), plus the seeded RAMBO
 * sampler of the standalone application (Sec. 4).  It plays the role of the
 * paper's Bridge / fBridge (Sec. 3.2): create, execute, destroy.
 *
 * Processes (particle order: initial state first):
 *   "ee_mumu"   e-(in) e+(in)  -> mu-  mu+        photon only, massless
 *   "gg_ttx"    g(in)  g(in)   -> t t~            3 diagrams,    2 colour flows
 *   "gg_ttxg"   g g -> t t~ g                     16 diagrams,   6 colour flows
 *   "gg_ttxgg"  g g -> t t~ g g                   123 diagrams,  24 colour flows
 *   "gg_ttxggg" g g -> t t~ g g g                 1240 diagrams, 120 colour flows
 *
 * Returned |M|^2: summed over all helicities and colours, averaged over the
 * initial-state spins (x 1/4) and colours (x 1/64 for gg), divided by n! for n
 * identical final-state gluons.  Couplings are fixed (no running).
 *
 * Conventions for every call:
 *   - momenta are FP64 [nevt][npar][4] row-major, components (E, px, py, pz),
 *     all particles with physical (positive-energy) momenta.  The same bytes as
 *     the paper's Fortran P(0:3, npar, nevt).
 *   - pointers may be host or device memory (detected with
 *     cudaPointerGetAttributes).  With device pointers a call is asynchronous
 *     on `cuda_stream` (a cudaStream_t; NULL = legacy default stream); with any
 *     host pointer the call stages through device memory and returns after the
 *     results are in the caller's buffer.
 *   - the caller owns every buffer it passes; the library never keeps a
 *     pointer to it after the call.  The handle owns its device state.
 *   - temporary device buffers (the staging of host buffers, per-launch
 *     scratch) are stream-ordered allocations from a pool per device that the
 *     library creates on first use and keeps until the process exits; freed
 *     memory stays reserved in it for later calls (at most the largest set of
 *     buffers in flight at once, e.g. about 400 MB after a host-buffer call on
 *     2^20 gg -> t t~ g g events).  While a stream is captured into a graph
 *     they come from the default pool instead.
 *   - every call returns 0 on success or a negative ME_E* code; nothing
 *     throws across the ABI.  nevt == 0 is a no-op returning 0.
 *   - handles are independent; one handle must not be used from two host
 *     threads at the same time.  The global mutable state is the fixed
 *     scratch array of me_filter_helicities_noalloc and that pool.
 */
#ifndef LIBME_ME_H
#define LIBME_ME_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define ME_OK 0
#define ME_EINVAL (-1)        /* null pointer, nevt < 0, unknown process, bad masses/couplings/precision */
#define ME_ENOMEM (-2)        /* a device or host allocation failed */
#define ME_ECUDA (-3)         /* a CUDA runtime call or kernel launch failed */
#define ME_ENOTFILTERED (-4)  /* me_sigmakin before me_filter_helicities with ME_OPT_REQUIRE_FILTER set */
#define ME_ENONFINITE (-5)    /* non-finite momenta found (ME_OPT_CHECK_FINITE) */
#define ME_ETIMEOUT (-6)      /* a bounded wait expired (serving layer) */
#define ME_ESAMPLER (-7)      /* RAMBO: an event needed more than 1000 attempts or Newton failed */
#define ME_ETOOLARGE (-8)     /* me_filter_helicities_noalloc: the probe batch does not fit its fixed scratch */

/* precision modes (Sec. 4.1, Table 1: FP64, FP32, mixed; ME_PREC_MIXED is this library's
   tensor-core variant, ME_PREC_MIXED64 the paper's definition) */
#define ME_PREC_FP64 0   /* chain, colour sum and helicity sum in FP64 */
#define ME_PREC_FP32 1   /* chain and colour sum in FP32; momenta, p^2-m^2 and helicity sum in FP64 */
#define ME_PREC_MIXED 2  /* FP32 chain (FP64 momenta, p^2-m^2), colour sum on BF16 tensor cores
                            with hi/lo split operands and FP32 accumulation where that is
                            faster on GB300 (120 flows; below, FP32 scalar, which measured
                            faster at 24 flows), FP64 helicity sum */
#define ME_PREC_MIXED64 3 /* the paper's mixed mode (Sec. 4.1, Table 1): FP64 chain, the colour-flow
                             amplitudes cast to FP32 for the colour sum, FP64 helicity sum */

typedef struct me_handle me_handle;

/*
 * me_init -- create a handle for one process and precision (the Bridge
 * constructor of Sec. 3.2).
 *   process:   one of the names above.
 *   masses:    nmass == npar external masses in particle order.  gg_ttx*:
 *              gluons 0, t and t~ equal (the top mass, e.g. 173.0).  ee_mumu:
 *              all 0.  NULL with nmass == 0 selects m_t = 173.0.
 *   couplings: {alpha} -- alpha_s for gg_ttx*, alpha_em for ee_mumu; NULL with
 *              ncoup == 0 selects 0.118 / (1/132.5).
 *   precision: ME_PREC_*.
 * The handle starts with all helicities enabled and unfiltered.
 * Errors: ME_EINVAL, ME_ENOMEM, ME_ECUDA.  *h is NULL on error.
 */
int me_init(me_handle** h, const char* process, const double* masses, int nmass, const double* couplings,
            int ncoup, int precision);

/*
 * me_filter_helicities -- find the helicity configurations that contribute
 * ("non-vanishing", Sec. 3.1).  h is kept iff max over the probe events of
 * |M_h|^2 / |M|^2 > 1e-14, computed in FP64 on the first min(nevt, 16384)
 * events of `momenta`.  Synchronous.  Stores the mask in the handle; writes
 * the number of kept helicities to *ngood_out (may be NULL).
 * Errors: ME_EINVAL (null handle/momenta, nevt <= 0), ME_ENOMEM, ME_ECUDA.
 */
int me_filter_helicities(me_handle* h, const double* momenta, int64_t nevt, int* ngood_out);

/*
 * me_filter_helicities_noalloc -- the same filter as me_filter_helicities,
 * for host programs that cannot let a library allocate device memory (they
 * reserve the device's memory up front through their own pool, or run loops in
 * which cudaMalloc / cudaFree, which may synchronise the whole device, are not
 * acceptable).  The paper has no counterpart: this is a deployment variant.
 * It allocates nothing: its scratch is one fixed 4 MiB array inside the
 * library, present on every device that loads the library until the process
 * exits.  The probe events are all nevt events of `momenta`, which must be
 * device memory; scratch needed = 8 * nevt * (nhel + 1) bytes plus a little,
 * so nevt <= 8000 for 64 helicities.  For gg_ttxggg the FP64 kernel also keeps
 * each resident CTA's colour-flow vectors (240 KB) in the array: it runs with as
 * many resident CTAs as the rest of the array holds (about 12 at 1000 probe
 * events, one at 3800; fewer probe events run faster), so nevt <= 3800 there.
 * Larger batches are rejected with ME_ETOOLARGE (pass fewer probe events).
 * The first call on each device looks up that device's copy of the array
 * (cudaGetSymbolAddress) with the device current; make that first call before
 * any stream capture.  All
 * calls share the one array and overwrite it: calls that overlap on the same
 * device (from several host threads) race and must be serialised by the
 * caller.  Synchronous.  Errors: ME_EINVAL (null handle or momenta, host
 * momenta, nevt <= 0), ME_ETOOLARGE, ME_ECUDA.
 */
int me_filter_helicities_noalloc(me_handle* h, const double* momenta, int64_t nevt, int* ngood_out);

/*
 * me_sigmakin -- |M|^2 for nevt events: momenta [nevt][npar][4] -> me2[nevt]
 * (Sec. 3.1 chain + Sec. 4.1 colour algebra + helicity sum).  If the handle has
 * not been filtered it filters on this batch first (synchronously), unless
 * ME_OPT_REQUIRE_FILTER is set, which makes this ME_ENOTFILTERED.  Per-event
 * results do not depend on the batch they are computed in.
 * Errors: ME_EINVAL, ME_ENOTFILTERED, ME_ENONFINITE, ME_ENOMEM, ME_ECUDA.
 */
int me_sigmakin(me_handle* h, const double* momenta, int64_t nevt, double* me2, void* cuda_stream);

/*
 * me_sigmakin_hel -- diagnostic variant: also writes each kept helicity's
 * contribution, hel_out[nevt][ngood] in the order of me_good_helicities, so
 * that sum over the row == me2.  Device pointers only (ME_EINVAL otherwise).
 */
int me_sigmakin_hel(me_handle* h, const double* momenta, int64_t nevt, double* me2, double* hel_out,
                    void* cuda_stream);

/*
 * me_sigmakin_sde -- |M|^2 and the single-diagram-enhancement weight of one
 * integration channel (Sec. 3.2: MadEvent's multi-channel weights, which the
 * event-generation interface keeps): for every event
 *     weight[e] = sum_h |amp_channel|^2 / sum_h sum_d |amp_d|^2,
 * amp_d the amplitude of Feynman diagram d with bare vertex factors (no
 * couplings), summed over the handle's kept helicities; the three Lorentz
 * structures of a four-gluon vertex are amplitudes of one diagram and their
 * |amp|^2 add.  channel: 0 <= channel < ndiag (me_info), the diagram order of
 * me_diagram_lines.  me2 as me_sigmakin computes it, except that both mixed
 * modes evaluate the chain in the precision that carries the weight (FP32 for
 * ME_PREC_MIXED, FP64 for ME_PREC_MIXED64) with a scalar colour sum.
 * momenta, me2, weight: device pointers ([nevt][npar][4], [nevt], [nevt]),
 * owned by the caller.  Filtering as in me_sigmakin.
 * Errors: ME_EINVAL (bad channel, host pointers), ME_ENOTFILTERED,
 * ME_ENONFINITE, ME_ENOMEM, ME_ECUDA.
 */
int me_sigmakin_sde(me_handle* h, const double* momenta, int64_t nevt, int channel, double* me2, double* weight,
                    void* cuda_stream);

/*
 * me_sigmakin_hsample -- helicity sampling instead of the helicity sum (the
 * alternative Sec. 3.1 describes for lockstep execution: here every event
 * keeps its own helicity, which needs no bunching because the external
 * states of both helicities are precomputed per event and only indexed).
 * The kernels are those of me_sigmakin with one helicity per event: the
 * per-event tables of the larger processes are still built for every
 * helicity configuration, so sampling saves the amplitude and colour work.
 * For event e the kept helicity i with cdf[i-1] <= u[e] < cdf[i] is chosen
 * (cdf the cumulative probabilities, last bin up to 1) and
 *     me2[e] = |M_h|^2 / p_h,
 * an unbiased estimator of me_sigmakin's helicity sum; hel[e] = h (the
 * helicity index, bit npar-1-i of h set = particle i has helicity +1).
 * Probabilities (me_hsample_probabilities): adaptive by default,
 * p_i = 0.9 q_i / sum q + 0.1 / ngood with q_i helicity i's mean share of
 * |M|^2 over the filter's probe events; uniform with ME_OPT_HSAMPLE_UNIFORM.
 * u: caller's uniforms in [0, 1) (device, [nevt]); me2 [nevt] and hel [nevt]
 * (may be NULL) on the device.  Filtering as in me_sigmakin.
 * Errors: ME_EINVAL, ME_ENOTFILTERED, ME_ENONFINITE, ME_ENOMEM, ME_ECUDA.
 */
int me_sigmakin_hsample(me_handle* h, const double* momenta, int64_t nevt, const double* u, double* me2, int* hel,
                        void* cuda_stream);

/*
 * me_hsample_probabilities -- the helicity-sampling probability of each kept
 * helicity, in the order of me_good_helicities (p may be NULL: only *n is set;
 * otherwise cap >= *n).  Errors: ME_EINVAL.
 */
int me_hsample_probabilities(const me_handle* h, double* p, int cap, int* n);

/*
 * me_diagram_lines -- identity of Feynman diagram `diagram` (0 <= diagram <
 * ndiag): its internal lines, each as a mask over the external particles
 * (bit i = particle i in the order of the momenta) on the side of the line
 * away from the last particle pair's antifermion (the t~; for e+e- -> mu+mu-
 * the photon line {e-, e+}), sorted ascending.  A tree diagram is fixed by this
 * set.  With masks == NULL only *n is set; otherwise cap must be >= *n
 * (at most npar - 3 lines).  Host-only, no device work.
 * Errors: ME_EINVAL.
 */
int me_diagram_lines(const me_handle* h, int diagram, int* masks, int cap, int* n);

/*
 * me_info -- process sizes: the numbers of external particles, helicity
 * configurations, colour flows (the dimension of the colour matrix of Sec. 4.1)
 * and Feynman diagrams (Sec. 3.1 counts 3 for gg -> t t~), and the helicity mask
 * found by the filter of Sec. 3.1.  Any output pointer may be NULL.
 *   good_mask_words: 2 words; bit h of word h/64 set iff helicity h is kept
 *   (all set before filtering).  nhel <= 128.  Host-only.  Errors: ME_EINVAL.
 */
int me_info(const me_handle* h, int* npar, int* nhel, int* ncol, int* ndiag, uint64_t* good_mask_words);

/* me_good_helicities -- the helicity configurations the filter of Sec. 3.1
 * kept, in ascending order (host array of capacity cap; at most cap are
 * written); *n receives their number.  Helicity index h: particle i has
 * helicity +1 iff bit (npar-1-i) of h is set.  Host-only.  Errors: ME_EINVAL. */
int me_good_helicities(const me_handle* h, int* out, int cap, int* n);

/* me_flops_per_event -- algorithmic work per event of the current mask, as
 * counted by the process generator (the per-event cost the throughput of
 * Sec. 4 divides): chain flops (Sec. 3.1 wavefunctions, currents, amplitudes;
 * FP32/FP64 pipe) and colour quadratic-form flops (Sec. 4.1), each = kept
 * helicities x per-helicity count.  Either pointer may be NULL.  Host-only.
 * Errors: ME_EINVAL. */
int me_flops_per_event(const me_handle* h, double* chain_flops, double* colour_flops);

/* options */
#define ME_OPT_REQUIRE_FILTER 1  /* value 1: me_sigmakin refuses to filter lazily */
#define ME_OPT_CHECK_FINITE 2    /* value 1: reject non-finite momenta (one extra pass, synchronous) */
#define ME_OPT_GAUGE_CHECK 3     /* value = external gluon index: its polarisation is replaced by its
                                    momentum (Ward identity diagnostic); -1 restores normal running */
#define ME_OPT_HSAMPLE_UNIFORM 4 /* value 1: helicity sampling with uniform probabilities over the kept
                                    helicities; 0 (default): adaptive (me_sigmakin_hsample) */
int me_set_option(me_handle* h, int option, int value);

/* me_free -- destroy a handle: the Bridge's destructor of Sec. 3.2 (create,
 * execute, destroy).  Waits for the device to finish (cudaDeviceSynchronize),
 * then releases the handle's device state and streams.  NULL is a no-op.  No
 * status is returned; the handle must not be used afterwards. */
void me_free(me_handle* h);

/* Cuts of the seeded sampler: final-state particle j is subject to the cuts
 * iff bit j of final_mask is set (j counts final-state particles from 0).
 * Each such particle needs pT > ptmin, each such pair Delta R > drmin with
 * Delta R = sqrt(Delta eta^2 + Delta phi^2), eta the pseudorapidity. */
typedef struct me_cuts {
    double ptmin;
    double drmin;
    uint32_t final_mask;
} me_cuts;

/*
 * rambo_sample -- seeded flat phase space (RAMBO, Kleiss-Stirling-Ellis 1986,
 * as in the standalone application of Sec. 4) for events ev0 .. ev0+nevt-1.
 *   masses: npar masses; the two incoming particles are massless and move
 *           along +z and -z with E = sqrt_s / 2.
 *   Random numbers: Philox4x64-10, key (seed, 0), counter (event, attempt,
 *   final particle, 0); one block gives the four uniforms of one final-state
 *   particle, u = ((x >> 11) + 0.5) 2^-53.  Massive particles: Newton solve of
 *   the RAMBO rescaling (|f| <= 1e-14 sqrt_s, at most 50 iterations).  With
 *   cuts, attempt k = 0, 1, ... of the same event until it passes (at most 1000).
 *   momenta_out: [nevt][npar][4]; weights_out (nullable): [nevt] phase-space
 *   weight with (2 pi)^(4-3n) normalisation, -1 for an event that failed.
 *   nfail_out (nullable, host): if given, the call synchronises and stores the
 *   number of failed events; the return is then ME_ESAMPLER if it is > 0.
 * Event i's momenta depend only on (seed, i): any range can be regenerated.
 * Errors: ME_EINVAL (npar < 3 or > 8, masses NULL, sqrt_s <= sum of masses),
 *         ME_ESAMPLER, ME_ENOMEM, ME_ECUDA.
 */
int rambo_sample(uint64_t seed, int64_t ev0, int64_t nevt, double sqrt_s, const double* masses, int npar,
                 const me_cuts* cuts, double* momenta_out, double* weights_out, int64_t* nfail_out,
                 void* cuda_stream);

/* me_strerror -- static description of a status code returned by any call
 * here (the error reporting of the Bridge interface of Sec. 3.2, which returns
 * status codes rather than throwing across the language boundary).  Never NULL;
 * unknown codes give "unknown status".  The string is owned by the library. */
const char* me_strerror(int status);

/* me_version -- library version string (static, owned by the library).  The
 * paper has no counterpart. */
const char* me_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LIBME_ME_H */
