// Staged, descriptor-driven |M|^2 kernel for the largest process
// (arXiv:2507.21039 Sec. 3.1 chain, Sec. 4.1 colour sum, helicity sum).
//
// One CTA per event, NT helicity slots (one thread each, or two threads each
// when J lives in tensor memory: see below).  The helicity-
// recycled table of off-shell objects (see me_kernel_tab.cuh) does not fit in
// shared memory for seven external particles, so the generator cuts the
// amplitudes into stages: each stage first computes, cooperatively and level by
// level, the table objects its amplitudes need that are not yet resident (into
// slots freed by objects whose last reader has passed), then every thread
// evaluates the stage's amplitudes for its helicity from compact descriptors.
// Amplitudes with the same colour vector up to a sign form a colour group:
// their signed sum G is added into the colour-flow vector J once, as +-i G on
// each flow of the group.
//
// Where J lives:
//   * FP32 (default): in tensor memory, accumulated by the tensor cores.  The
//     group sums of one stage (at most 16) form, per helicity, the rows of
//     A = [Re G | Im G] (128 helicities x 16); with the stage's sign matrix B
//     (flow x group, entries +-1 / 0, built by the generator), one stage adds
//     Re J += Im G . B and Im J += Re G . (-B).  G is split exactly into three
//     BF16 parts (8 + 8 + 8 significant bits), B is exact in BF16, the tensor
//     cores accumulate in FP32 in TMEM (columns 0-127 Re J, 128-255 Im J of the
//     thread's lane): six tcgen05.mma (M = 128, N = 128, K = 16) per stage,
//     issued by one thread after the CTA barrier that ends the stage.  J then
//     needs no shared memory, so two CTAs share an SM.  Each helicity has two
//     threads (CTA of 2 NT): the generator splits every stage's amplitudes at
//     a colour-group boundary into two halves of about equal cost; the second
//     thread evaluates the later half and writes its group sums into the later
//     columns of A.  The tensor memory (two CTAs x 256 columns) caps the events
//     in flight per SM at two; the pairs double the warps that hide the
//     latency of the amplitude chain.
//   * FP32, build option ME_INTERP_J_MMA=0: in shared memory, updated flow by
//     flow by each group's last member (one CTA per SM).
//   * FP64: in a global scratch (L2-resident), updated flow by flow; its tables
//     alone fill shared memory.
#pragma once
#include <algorithm>

#include "me_kernel_tab.cuh"
#include "me_pool.h"
#include "me_tmem.cuh"

// Build option ME_INTERP_J_MMA: FP32 colour-flow vector accumulated by the
// tensor cores in tensor memory (1, default) or updated in shared memory (0)
#ifndef ME_INTERP_J_MMA
#define ME_INTERP_J_MMA 1
#endif
// Build option ME_INTERP_HPAIR: with J in tensor memory, two threads per
// helicity share out each stage's amplitudes at a colour-group boundary (1,
// default: twice the warps per SM for the same tensor memory) or one thread
// evaluates them all (0)
#ifndef ME_INTERP_HPAIR
#define ME_INTERP_HPAIR 1
#endif
// Build option ME_INTERP_HPAIR64: the FP64 kernel (J in a global scratch) also
// runs two threads per helicity, each with its own copy of J, summed in the
// colour form (1), or one thread per helicity (0, default: measured on GB300
// for gg -> t t~ g g g, 20.0 k against 19.4 k events/s, for twice the scratch)
#ifndef ME_INTERP_HPAIR64
#define ME_INTERP_HPAIR64 0
#endif
// Build option ME_INTERP_A_MMAJOR: the group-sum operands A in the M-major
// layout (1, default: a warp's 32 rows of one column on distinct banks) or
// K-major (0: the four row groups of a warp on the same banks, 4-way conflicts)
#ifndef ME_INTERP_A_MMAJOR
#define ME_INTERP_A_MMAJOR 1
#endif
// Build option ME_INTERP_PAIRS: amplitudes evaluated two at a time where the
// generator pairs them (1, default) or one at a time with the next one's
// operands loaded ahead (0)
#ifndef ME_INTERP_PAIRS
#define ME_INTERP_PAIRS 1
#endif

namespace me {

constexpr bool kInterpPairs = ME_INTERP_PAIRS != 0;

struct __align__(8) IRound {
    unsigned int task_begin;
    unsigned short ntask;
    unsigned char kind, barrier_after;
};
struct __align__(16) IStage {
    unsigned short round_begin, round_end, amp_begin, amp_end;
    // two threads per helicity: the first evaluates [amp_begin, amp_mid), the
    // second [amp_mid, amp_end) from group update slot_mid on (a group boundary)
    unsigned short amp_mid, slot_mid;
    // 1: the stage's table rounds run beside the previous stage's amplitudes
    // (their slots are not read there); 0: in a phase of their own
    unsigned short ahead;
    // colour terms of the groups before amp_mid (J updated flow by flow: the
    // second thread's first term is stage_term_begin + term_mid)
    unsigned short term_mid;
};
struct __align__(16) IAmp {
    unsigned short op[4];
    unsigned char sup[4];
    unsigned char kind, la, lb, nterm;
};

// codes in the generator's order (gen/interp.py ROUTINES, AMP_KINDS)
enum IRoutine : unsigned char {
    R_VVV1P0_1 = 0, R_VVVV1P0_1, R_VVVV3P0_1, R_VVVV4P0_1, R_FFV1_2, R_FFV1_1, R_FFV1P0_3,
    R_FFV1A_3, R_FFV1A_2, R_FFV1A_1, R_VVV1A_1, R_VVV1A_2, R_VVV1A_3, R_VVVV1A, R_VVVV3A, R_VVVV4A
};
enum IAmpKind : unsigned char { A_FFV1_0 = 0, A_VVV1_0, A_VVVV1_0, A_VVVV3_0, A_VVVV4_0, A_DOTV, A_DOTF };
// IAmp.kind flags above the kind: the amplitude enters its colour group's sum
// with a minus sign (AMP_NEG); the amplitude and the next one have the same
// kind and lie in the same half of the stage (AMP_PAIR)
constexpr unsigned char AMP_NEG = 0x80, AMP_PAIR = 0x40, AMP_KIND_MASK = 0x3f;

template <class P, class T> struct InterpLayout {
    static constexpr size_t mom = 0;
    // T = float: split momenta and FP64 Gram matrix of the FP32 setup (me_kernel.cuh)
    static constexpr size_t pf = mom + P::NPAR * 4 * sizeof(double);
    static constexpr size_t gram = pf + (sizeof(T) == 4 ? P::NPAR * 4 * sizeof(float2) : 0);
    static constexpr size_t lines = gram + (sizeof(T) == 4 ? Gram<P::NPAR>::N * sizeof(double) : 0);
    static constexpr size_t vsup = (lines + P::NLINES * sizeof(Ln<T>) + 15) / 16 * 16;
    static constexpr size_t table = (vsup + (size_t)P::NSUP * P::NT + 15) / 16 * 16;
    static constexpr size_t jsm = table + (size_t)P::TAB * sizeof(Wf<T>);
    // J accumulated by the tensor cores: 128 lanes x (128 + 128) FP32 columns
    static constexpr bool J_MMA = sizeof(T) == 4 && ME_INTERP_J_MMA;
    static constexpr bool J_IN_SMEM = sizeof(T) == 4 && !J_MMA;
    static constexpr uint32_t TMEM_COLS = 256;
    // threads per CTA: one per helicity, or two with J in tensor memory (the
    // second takes the later colour groups of each stage); register budget for
    // two resident CTAs when J is in tensor memory
    static constexpr bool J_GLOBAL = !J_MMA && !J_IN_SMEM;
    static constexpr int NTH = ((J_MMA && ME_INTERP_HPAIR) || (J_GLOBAL && ME_INTERP_HPAIR64)) ? 2 * P::NT : P::NT;
    static constexpr int MIN_CTAS = J_MMA ? 2 : 1;
    // J_MMA operands: six A matrices (BF16 hi / mid / lo of Im G and Re G, 128 x 16
    // each, ABYTES apart) and the stage's sign matrix B (128 flows x 16, 4096 bytes)
    static constexpr bool A_MMAJOR = ME_INTERP_A_MMAJOR != 0;
    static constexpr size_t ABYTES = A_MMAJOR ? kUmmaMn16Bytes : 4096;
    static constexpr uint32_t A_LBO = 128, A_SBO = A_MMAJOR ? kUmmaMn16Sbo : 256;
    static constexpr size_t amat = (jsm + 1023) / 1024 * 1024;
    static constexpr size_t bmat = amat + 6 * ABYTES;
    static constexpr size_t bytes = J_MMA ? bmat + 4096
                                          : jsm + (J_IN_SMEM ? (size_t)P::NCOL * P::NT * sizeof(cx<T>) : 0);
    // colour sum from TMEM: per warp, one half of J (Re, then Im) as [flow][lane]
    // FP32 and 32 floats of row totals, the four warps at once over the (then
    // dead) table
    static constexpr size_t WJ = ((size_t)P::NCOL * 32 * sizeof(float) + 32 * sizeof(float) + 15) / 16 * 16;
    // scalar colour form (FP32 precision): J of a warp as [flow][lane] complex,
    // two warps at a time (the form reads each numerator once for both halves)
    static constexpr size_t WJC = (size_t)P::NCOL * 32 * sizeof(cx<float>);
    static constexpr size_t launch_bytes = bytes;
};

template <class T, int TAB>
__device__ __forceinline__ void run_task(const TabRef<T, TAB>& tab, const Ln<T>* __restrict__ ln, T mt, int kind,
                                         const TabTask& k)
{
    Wf<T> o;
    switch (kind) {
    case R_VVV1P0_1: VVV1P0_1<T>(tab.ld(k.in0), ln[k.la].p, tab.ld(k.in1), ln[k.lb].p, ln[k.lo].inv, o); break;
    case R_VVVV1P0_1: VVVV1P0_1<T>(tab.ld(k.in0), tab.ld(k.in1), tab.ld(k.in2), ln[k.lo].inv, o); break;
    case R_VVVV3P0_1: VVVV3P0_1<T>(tab.ld(k.in0), tab.ld(k.in1), tab.ld(k.in2), ln[k.lo].inv, o); break;
    case R_VVVV4P0_1: VVVV4P0_1<T>(tab.ld(k.in0), tab.ld(k.in1), tab.ld(k.in2), ln[k.lo].inv, o); break;
    case R_FFV1_2: FFV1_2<T>(tab.ld(k.in0), tab.ld(k.in1), ln[k.lo], mt, o); break;
    case R_FFV1_1: FFV1_1<T>(tab.ld(k.in0), tab.ld(k.in1), ln[k.lo], mt, o); break;
    case R_FFV1P0_3: FFV1P0_3<T>(tab.ld(k.in0), tab.ld(k.in1), ln[k.lo].inv, o); break;
    case R_FFV1A_3: FFV1A_3<T>(tab.ld(k.in0), tab.ld(k.in1), o); break;
    case R_FFV1A_2: FFV1A_2<T>(tab.ld(k.in0), tab.ld(k.in1), o); break;
    case R_FFV1A_1: FFV1A_1<T>(tab.ld(k.in0), tab.ld(k.in1), o); break;
    case R_VVV1A_1: VVV1A<1, T>(tab.ld(k.in0), tab.ld(k.in1), ln[k.la].p, ln[k.lb].p, o); break;
    case R_VVV1A_2: VVV1A<2, T>(tab.ld(k.in0), tab.ld(k.in1), ln[k.la].p, ln[k.lb].p, o); break;
    case R_VVV1A_3: VVV1A<3, T>(tab.ld(k.in0), tab.ld(k.in1), ln[k.la].p, ln[k.lb].p, o); break;
    case R_VVVV1A: VVVV1A<T>(tab.ld(k.in0), tab.ld(k.in1), tab.ld(k.in2), o); break;
    case R_VVVV3A: VVVV3A<T>(tab.ld(k.in0), tab.ld(k.in1), tab.ld(k.in2), o); break;
    default: VVVV4A<T>(tab.ld(k.in0), tab.ld(k.in1), tab.ld(k.in2), o); break;
    }
    tab.st(k.out, o);
}

// Three-way exact BF16 split of x (x = hi + mid + lo for finite x in the
// normal range: each part takes the next 8 significant bits)
__device__ __forceinline__ void bf16_split3(float x, __nv_bfloat16& hi, __nv_bfloat16& mid, __nv_bfloat16& lo)
{
    hi = __float2bfloat16_rn(x);
    const float r = x - __bfloat162float(hi);
    mid = __float2bfloat16_rn(r);
    lo = __float2bfloat16_rn(r - __bfloat162float(mid));
}

// TC: colour sum on BF16 tensor cores (T = float); otherwise scalar in C
template <class P, class T, bool TC, class C = T, bool SDE = false>
__global__ void __launch_bounds__(InterpLayout<P, T>::NTH, InterpLayout<P, T>::MIN_CTAS)
    me_kernel_interp(LaunchArgs a, cx<T>* __restrict__ jglobal)
{
    using L = InterpLayout<P, T>;
    constexpr int NTH = L::NTH;
    // (the operand offsets inside are multiples of 1024 from the base; the
    // unswizzled tensor-core operands need 16-byte alignment only)
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NPAR = P::NPAR, NL = P::NLINES, NT = P::NT, NCOL = P::NCOL;
    double* smom = reinterpret_cast<double*>(smem + L::mom);
    Ln<T>* sln = reinterpret_cast<Ln<T>*>(smem + L::lines);
    unsigned char* vsup = smem + L::vsup;
    const TabRef<T, P::TAB> tab{reinterpret_cast<uint4*>(smem + L::table)};
    // this thread's colour-flow vector: J[c] at jp[c * NT] (shared or global
    // memory), or TMEM columns c (Re) and 128 + c (Im) of its lane from tj
    cx<T>* jp = nullptr;
    if constexpr (L::J_IN_SMEM) jp = reinterpret_cast<cx<T>*>(smem + L::jsm) + threadIdx.x;
    else if constexpr (!L::J_MMA)  // one copy per helicity thread (two copies per CTA with helicity pairs)
        jp = jglobal + ((size_t)blockIdx.x * (NTH / NT) + threadIdx.x / NT) * NCOL * NT + (threadIdx.x & (NT - 1));
    __shared__ double red[NTH / 32];
    __shared__ FSum fred[NTH / 32];
    __shared__ double red_sde[SDE ? 2 : 1][NTH / 32];
    __shared__ unsigned char pair_nonfinite[NTH > NT ? NT : 1];  // second thread of a helicity: a group sum was not finite
    constexpr bool F32 = sizeof(T) == 4;
    float2* spf = reinterpret_cast<float2*>(smem + L::pf);
    double* sgram = reinterpret_cast<double*>(smem + L::gram);
    const double m2 = a.mt * a.mt;
    const float mtf = (float)a.mt;
    __shared__ float rowv[NT];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t mma_bar;
    const int tid = threadIdx.x;
    const int h = tid & (NT - 1);  // helicity slot (lane of J in tensor memory)
    const int half = tid / NT;     // 1: the second thread of helicity h
    const bool act = h < a.nlist;
    uint32_t tj = 0;
    uint32_t ncommit = 0;  // tensor-core commits so far (the same count in every thread)
    bool failed = false;   // a wait for the tensor cores ran out: this thread stops waiting
    if constexpr (L::J_MMA) {
        static_assert(NT == 128 && NCOL <= 128, "one TMEM lane per helicity, one column per flow");
        static_assert(P::MAXFLUSH <= 16, "at most 16 colour-group updates per stage (one K = 16 step)");
        static_assert(4 * L::WJ <= (size_t)P::TAB * sizeof(Wf<T>) && 2 * L::WJC <= (size_t)P::TAB * sizeof(Wf<T>),
                      "colour staging exceeds the table");
        if (tid < 32) {
            tmem_alloc(&tmem_base, L::TMEM_COLS);
            tmem_relinquish();
        }
        if (tid == 0) {
            mbar_init(&mma_bar, 1);
            mbar_init_fence();
        }
        // operands start at zero: a slot no group of a stage uses is multiplied by
        // a zero column of B and must hold a finite value
        uint4* z = reinterpret_cast<uint4*>(smem + L::amat);
        for (int i = tid; i < (int)((6 * L::ABYTES + 4096) / 16); i += NTH) z[i] = make_uint4(0u, 0u, 0u, 0u);
        fence_proxy_async_smem();
        tmem_fence_before_sync();
        __syncthreads();
        tmem_fence_after_sync();
        tj = tmem_base + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16);
    }
    // compressed variant index of every operand support for helicity `hel`,
    // stored at this thread's helicity slot h (support particles in descending
    // order = helicity bits from low to high)
    auto variants = [&](int hel) {
        for (int s = 0; s < P::NSUP; ++s) {
            const unsigned m = P::support_mask(s);
            unsigned v = 0, j = 0;
            for (int b = 0; b < NPAR; ++b)
                if ((m >> b) & 1) v |= ((hel >> b) & 1) << j++;
            vsup[s * NT + h] = (unsigned char)v;
        }
    };
    if (!a.hel_ev && half == 0) variants(a.hel_list[act ? h : 0]);
    // wait for the tensor cores' commit number c (its mbarrier phase parity is c & 1)
    auto wait_commit = [&](uint32_t c) {
        if (!failed && !mbar_wait_bounded(&mma_bar, c & 1u, ME_WAIT_LIMIT_CYCLES)) failed = true;
    };

    for (long long e = blockIdx.x; e < a.nevt; e += gridDim.x) {
        if (a.hel_ev && half == 0) variants(a.hel_ev[e]);  // helicity sampling: one helicity per event (nlist = 1)
        const double* g = a.mom + e * NPAR * 4;
        for (int i = tid; i < NPAR * 4; i += NTH) smom[i] = __ldg(g + i);
        if constexpr (!L::J_MMA) {
            for (int c = 0; c < NCOL; ++c) jp[c * NT] = {T(0), T(0)};
        }
        __syncthreads();
        if constexpr (F32) {  // split momenta and FP64 Gram matrix, then lines and external states in FP32
            if constexpr (split_items_one_pass<NPAR, NTH>()) {
                const int it = split_item_of<NPAR>(tid);
                if (it >= 0) split_or_gram<NPAR>(smom, it, spf, sgram);
            } else {
                for (int it = tid; it < 4 * NPAR + Gram<NPAR>::N; it += NTH) split_or_gram<NPAR>(smom, it, spf, sgram);
            }
            __syncthreads();
            for (int it = tid; it < NL + 2 * NPAR; it += NTH) {
                if (it < NL) sln[it] = line_data_split<P>(spf, sgram, it, m2);
                else tab.st(it - NL, ext_wavefunction_split<P>(spf, it - NL, mtf, a.gauge_ext));
            }
        } else {
            for (int it = tid; it < 2 * NPAR + NL; it += NTH) {
                if (it < 2 * NPAR) tab.st(it, ext_wavefunction<P, T>(smom, it, a.mt, a.gauge_ext));
                else sln[it - 2 * NPAR] = line_data<P, T>(smom, it - 2 * NPAR, a.mt);
            }
        }
        __syncthreads();
        const T mt = (T)a.mt;
        T snum = T(0), sden = T(0);
        cx<T> G = {T(0), T(0)};  // open colour group: sum of its amplitudes with their signs
        bool nonfinite = false;   // a group sum was not finite (it enters J as 0; |M|^2 = NaN)
        // table rounds start at the warp after the previous round's last task, so
        // that the many small rounds spread over all warps instead of piling onto the
        // first ones (a warp still runs the tasks of one round only)
        static_assert((NTH & (NTH - 1)) == 0 && NT % 32 == 0, "round rotation assumes a power-of-two CTA of whole warps");
        int rot = 0;
        auto table_rounds = [&](int ts) {  // the table objects that become live in stage ts
            const IStage tst = P::stage(ts);
            for (int r = tst.round_begin; r < tst.round_end; ++r) {
                const IRound rd = P::round(r);
                for (int t = (tid - rot) & (NTH - 1); t < rd.ntask; t += NTH)
                    run_task<T, P::TAB>(tab, sln, mt, rd.kind, ld_task(P::tasks() + rd.task_begin + t));
                rot = (rot + ((rd.ntask + 31) & ~31)) & (NTH - 1);
                if (rd.barrier_after) __syncthreads();
            }
        };
        for (int s = 0; s < P::NSTAGE; ++s) {
            const IStage st = P::stage(s);
            if (!(P::TABLE_AHEAD && st.ahead)) {  // a phase of their own (always for the first stage)
                table_rounds(s);
                __syncthreads();
            }
            int term = P::stage_term_begin(s);
            int slot = 0;  // J_MMA: the stage's next group update (column of A)
            // this thread's amplitudes of the stage: all of them, or one side of the
            // stage's split between the two threads of a helicity
            int amp_lo = st.amp_begin, amp_hi = st.amp_end;
            if constexpr (NTH > NT) {
                if (half == 0) {
                    amp_hi = st.amp_mid;
                } else {
                    amp_lo = st.amp_mid;
                    slot = st.slot_mid;
                    term += st.term_mid;
                }
            }
            if constexpr (L::J_MMA) {
                // the previous stage's tensor-core work has read A and B: they may be rewritten;
                // this stage's sign matrix is copied in while the amplitudes are evaluated
                if (ncommit > 0) wait_commit(ncommit - 1);
                const uint4* bsrc = P::bmat(s);
                uint4* bsm = reinterpret_cast<uint4*>(smem + L::bmat);
                for (int i = tid; i < 256; i += NTH) cp_async16(bsm + i, bsrc + i);
                cp_async_commit();
            }
            // the next stage's table objects, where they may be computed beside
            // these amplitudes (the stage barrier below publishes them)
            if constexpr (P::TABLE_AHEAD) {
                if (s + 1 < P::NSTAGE && P::stage(s + 1).ahead) table_rounds(s + 1);
            }
            // amplitude x of descriptor d with operands w0..w2 (a third operand index of a
            // two-operand kind is 0 with support 0: an external wavefunction entry, read
            // and not used)
            auto opnd = [&](const IAmp& d, int k) { return tab.ld(d.op[k] + vsup[d.sup[k] * NT + h]); };
            auto eval = [&](const IAmp& d, const Wf<T>& w0, const Wf<T>& w1, const Wf<T>& w2) {
                const int kind = d.kind & AMP_KIND_MASK;
                cx<T> x;
                if (kind == A_DOTV) {           // amputated: two-operand contractions
                    x = DOTV<T>(w0, w1);
                } else if (kind == A_DOTF) {
                    x = DOTF<T>(w0, w1);
                } else {
                    switch (kind) {
                    case A_FFV1_0: x = FFV1_0<T>(w0, w1, w2); break;
                    case A_VVV1_0: x = VVV1_0<T>(w0, sln[d.la].p, w1, sln[d.lb].p, w2); break;
                    default: {
                        const Wf<T> w3 = opnd(d, 3);
                        x = kind == A_VVVV1_0 ? VVVV1_0<T>(w0, w1, w2, w3)
                          : kind == A_VVVV3_0 ? VVVV3_0<T>(w0, w1, w2, w3) : VVVV4_0<T>(w0, w1, w2, w3);
                    }
                    }
                }
                return x;
            };
            // x into its colour group's sum; the group's last member adds the group to J
            auto accumulate = [&](const IAmp& d, const cx<T>& x, int ai) {
                if constexpr (SDE) {  // single-diagram enhancement
                    const T w2 = fma(x.re, x.re, x.im * x.im);
                    sden += w2;
                    if (P::diag(ai) == a.sde_channel) snum += w2;
                }
                if (d.kind & AMP_NEG) { G.re -= x.re; G.im -= x.im; }
                else { G.re += x.re; G.im += x.im; }
                // the group's last member: every colour coefficient is +-i, J_c += +-i G
                if (d.nterm) {
                    if constexpr (L::J_MMA) {
                        // row h, column `slot` of the six A matrices: BF16 parts of Im G, Re G
                        float gr = (float)G.re, gi = (float)G.im;
                        if (!(isfinite(gr) && isfinite(gi))) {
                            nonfinite = true;
                            gr = gi = 0.0f;
                        }
                        __nv_bfloat16 q[6];
                        bf16_split3(gi, q[0], q[1], q[2]);
                        bf16_split3(gr, q[3], q[4], q[5]);
                        const uint32_t off = L::A_MMAJOR ? umma_mn16_offset(h, slot) : umma_k16_offset(h, slot);
#pragma unroll
                        for (int m = 0; m < 6; ++m)
                            *reinterpret_cast<__nv_bfloat16*>(smem + L::amat + (size_t)m * L::ABYTES + off) = q[m];
                        ++slot;
                        term += d.nterm;
                    } else {
                        for (int k = 0; k < d.nterm; ++k, ++term) {
                            const unsigned short ct = P::term(term);
                            cx<T>& jc = jp[(ct & 0x7fff) * NT];
                            const cx<T> j = jc;
                            jc = (ct & 0x8000) ? cx<T>{j.re + G.im, j.im - G.re} : cx<T>{j.re - G.im, j.im + G.re};
                        }
                    }
                    G = {T(0), T(0)};
                }
            };
            if constexpr (kInterpPairs) {
                // amplitudes flagged AMP_PAIR and their successor (same kind, same half
                // of the stage) are evaluated together: two independent dependency
                // chains for the scheduler; their operands are loaded at once
                int ai = amp_lo;
                while (ai < amp_hi) {
                    const IAmp d0 = P::amp(ai);
                    const Wf<T> a0 = opnd(d0, 0), a1 = opnd(d0, 1), a2 = opnd(d0, 2);
                    if ((d0.kind & AMP_PAIR) && ai + 1 < amp_hi) {
                        const IAmp d1 = P::amp(ai + 1);
                        const Wf<T> b0 = opnd(d1, 0), b1 = opnd(d1, 1), b2 = opnd(d1, 2);
                        const int kind = d0.kind & AMP_KIND_MASK;
                        cx<T> x0, x1;
                        switch (kind) {
                        case A_FFV1_0:
                            x0 = FFV1_0<T>(a0, a1, a2);
                            x1 = FFV1_0<T>(b0, b1, b2);
                            break;
                        case A_VVV1_0:
                            x0 = VVV1_0<T>(a0, sln[d0.la].p, a1, sln[d0.lb].p, a2);
                            x1 = VVV1_0<T>(b0, sln[d1.la].p, b1, sln[d1.lb].p, b2);
                            break;
                        case A_DOTV:
                            x0 = DOTV<T>(a0, a1);
                            x1 = DOTV<T>(b0, b1);
                            break;
                        case A_DOTF:
                            x0 = DOTF<T>(a0, a1);
                            x1 = DOTF<T>(b0, b1);
                            break;
                        default: {
                            const Wf<T> a3 = opnd(d0, 3), b3 = opnd(d1, 3);
                            if (kind == A_VVVV1_0) {
                                x0 = VVVV1_0<T>(a0, a1, a2, a3);
                                x1 = VVVV1_0<T>(b0, b1, b2, b3);
                            } else if (kind == A_VVVV3_0) {
                                x0 = VVVV3_0<T>(a0, a1, a2, a3);
                                x1 = VVVV3_0<T>(b0, b1, b2, b3);
                            } else {
                                x0 = VVVV4_0<T>(a0, a1, a2, a3);
                                x1 = VVVV4_0<T>(b0, b1, b2, b3);
                            }
                        }
                        }
                        accumulate(d0, x0, ai);
                        accumulate(d1, x1, ai + 1);
                        ai += 2;
                    } else {
                        accumulate(d0, eval(d0, a0, a1, a2), ai);
                        ai += 1;
                    }
                }
            } else {
                // software pipeline: the descriptor and the first three operands of the
                // next amplitude are loaded while the current one is evaluated
                IAmp dn;
                Wf<T> p0, p1, p2;
                auto fetch = [&](int ai) {
                    dn = P::amp(ai);
                    p0 = opnd(dn, 0);
                    p1 = opnd(dn, 1);
                    p2 = opnd(dn, 2);
                };
                if (amp_lo < amp_hi) fetch(amp_lo);
                for (int ai = amp_lo; ai < amp_hi; ++ai) {
                    const IAmp d = dn;
                    const Wf<T> w0 = p0, w1 = p1, w2 = p2;
                    if (ai + 1 < amp_hi) fetch(ai + 1);
                    accumulate(d, eval(d, w0, w1, w2), ai);
                }
            }
            if constexpr (L::J_MMA) {
                cp_async_wait_all();
                fence_proxy_async_smem();  // A and B writes -> the tensor cores' view of shared memory
            }
            __syncthreads();  // stage done: its dead table slots are reused by the next stage
            if constexpr (L::J_MMA) {
                if (tid == 0 && !failed) {
                    tmem_fence_after_sync();
                    const uint64_t bdesc = umma_smem_desc(smem + L::bmat, 128, 256);
                    constexpr uint32_t ID_POS = umma_idesc_bf16_f32(128, 128, false, L::A_MMAJOR);
                    constexpr uint32_t ID_NEG = umma_idesc_bf16_f32(128, 128, true, L::A_MMAJOR);
#pragma unroll
                    for (int m = 0; m < 3; ++m) {  // the first update of an event overwrites J
                        const bool acc = s > 0 || m > 0;
                        umma_bf16(tmem_base, umma_smem_desc(smem + L::amat + (size_t)m * L::ABYTES, L::A_LBO, L::A_SBO),
                                  bdesc, ID_POS, acc);
                        umma_bf16(tmem_base + 128,
                                  umma_smem_desc(smem + L::amat + (size_t)(3 + m) * L::ABYTES, L::A_LBO, L::A_SBO), bdesc,
                                  ID_NEG, acc);
                    }
                    umma_commit(&mma_bar);
                }
                ++ncommit;
            }
        }
        // colour quadratic form sum_ij N_ij Re(conj J_i J_j)
        T v = T(0);
        auto colour_scalar = [&](const cx<T>* jq, int stride) {  // J_c at jq[c * stride], in precision C
            C w = C(0);
            for (int i = 0; i < NCOL; ++i) {
                const cx<T> ji = jq[i * stride];
                C zr = C(0), zi = C(0);
                for (int j = i; j < NCOL; ++j) {
                    const C n = (C)P::cnum2(i, j);
                    const cx<T> jj = jq[j * stride];
                    zr = fma(n, (C)jj.re, zr);
                    zi = fma(n, (C)jj.im, zi);
                }
                w = fma((C)ji.re, zr, fma((C)ji.im, zi, w));
            }
            return (T)w;
        };
        if constexpr (L::J_MMA) {
            wait_commit(ncommit - 1);  // this event's last tensor-core update is in J
            tmem_fence_after_sync();
            if constexpr (NTH > NT) {
                if (half) pair_nonfinite[h] = nonfinite ? 1 : 0;  // read after the barriers below
            }
            // warps 0-3 (lanes 0-127 of tensor memory) form the colour sum over the dead
            // table.  Tensor-core form: all four warps at once, one half of J (Re, then
            // Im) at a time (the form is the sum of the two halves' forms).  Scalar
            // form: two warps at a time, J complex
            const int w = tid >> 5, lane = tid & 31;
            if constexpr (TC) {
                if (w < 4) {
                    unsigned char* stage = smem + L::table + (size_t)w * L::WJ;
                    float* plane = reinterpret_cast<float*>(stage);
                    float* rowt = reinterpret_cast<float*>(stage + (size_t)NCOL * 32 * sizeof(float));
                    T vs = T(0);
#pragma unroll 1
                    for (int hh = 0; hh < 2; ++hh) {
                        for (int c = 0; c < NCOL; c += 16) {
                            uint32_t q[16];
                            tmem_ld_16(tj + 128u * (uint32_t)hh + (uint32_t)c, q);
#pragma unroll
                            for (int k = 0; k < 16; ++k)
                                if (c + k < NCOL) plane[(c + k) * 32 + lane] = __uint_as_float(q[k]);
                        }
                        __syncwarp();
                        vs += colour_tc_plane<NCOL, P::NSPLIT>(plane, P::bfrag(), rowt, lane);
                        __syncwarp();  // the plane is rewritten by the next half
                    }
                    v = vs;
                }
                __syncthreads();
            } else {
                cx<float>* js = reinterpret_cast<cx<float>*>(smem + L::table + (size_t)(w & 1) * L::WJC);
                for (int r = 0; r < 2; ++r) {  // warps 0, 1 then warps 2, 3
                    if ((w >> 1) == r) {
                        for (int c = 0; c < NCOL; c += 16) {
                            uint32_t qr[16], qi[16];
                            tmem_ld_16(tj + (uint32_t)c, qr);
                            tmem_ld_16(tj + 128u + (uint32_t)c, qi);
#pragma unroll
                            for (int k = 0; k < 16; ++k)
                                if (c + k < NCOL)
                                    js[(c + k) * 32 + lane] = {__uint_as_float(qr[k]), __uint_as_float(qi[k])};
                        }
                        __syncwarp();
                        v = colour_scalar(reinterpret_cast<const cx<T>*>(js) + lane, 32);
                    }
                    __syncthreads();
                }
            }
            if constexpr (NTH > NT) {
                if (!half && pair_nonfinite[h]) nonfinite = true;
            }
            if (nonfinite || failed) v = T(NAN);
        } else if constexpr (TC) {
            v = colour_tc_smem<NCOL, NT, P::NSPLIT>(reinterpret_cast<const cx<float>*>(smem + L::jsm), P::bfrag(),
                                                    rowv, tid);
        } else if constexpr (NTH > NT) {
            // J of a helicity is the sum of its two threads' copies (half 1's copy
            // follows half 0's): the first thread forms the colour sum
            __syncthreads();
            if (!half) {
                const cx<T>* j1 = jp + (size_t)NCOL * NT;
                C w = C(0);
                for (int i = 0; i < NCOL; ++i) {
                    const cx<T> ji = {jp[i * NT].re + j1[i * NT].re, jp[i * NT].im + j1[i * NT].im};
                    C zr = C(0), zi = C(0);
                    for (int j = i; j < NCOL; ++j) {
                        const C n = (C)P::cnum2(i, j);
                        zr = fma(n, (C)(jp[j * NT].re + j1[j * NT].re), zr);
                        zi = fma(n, (C)(jp[j * NT].im + j1[j * NT].im), zi);
                    }
                    w = fma((C)ji.re, zr, fma((C)ji.im, zi, w));
                }
                v = (T)w;
            }
        } else {
            v = colour_scalar(jp, NT);
        }
        double acc = 0.0, dn = 0.0, dd = 0.0;
        FSum facc{0.0f, 0.0f};
        if (act) {
            if (half == 0) {  // (the second thread of a helicity holds no colour sum)
                if constexpr (F32) facc.s = (float)v;
                else acc = (double)v;
                if (a.hel_out) a.hel_out[e * a.nlist + h] = (double)v * a.norm;
            }
            if constexpr (SDE) {  // both threads of a helicity: their own amplitudes
                dn = (double)snum;
                dd = (double)sden;
            }
        }
        if constexpr (F32) facc = fsum_warp(facc);
        for (int off = 16; off > 0; off >>= 1) {
            if constexpr (!F32) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if constexpr (SDE) {
                dn += __shfl_xor_sync(0xffffffffu, dn, off);
                dd += __shfl_xor_sync(0xffffffffu, dd, off);
            }
        }
        if ((tid & 31) == 0) {
            if constexpr (F32) fred[tid >> 5] = facc;
            else red[tid >> 5] = acc;
            if constexpr (SDE) {
                red_sde[0][tid >> 5] = dn;
                red_sde[1][tid >> 5] = dd;
            }
        }
        __syncthreads();
        if (tid == 0) {
            double s = 0.0, sn = 0.0, sd = 0.0;
            if constexpr (F32) {  // one conversion per event
                FSum f = fred[0];
                for (int w = 1; w < NTH / 32; ++w) f = fsum_add(f, fred[w]);
                s = (double)f.s + (double)f.c;
            }
            for (int w = 0; w < NTH / 32; ++w) {
                if constexpr (!F32) s += red[w];
                if constexpr (SDE) {
                    sn += red_sde[0][w];
                    sd += red_sde[1][w];
                }
            }
            a.me2[e] = s * a.norm * (a.w_ev ? a.w_ev[e] : 1.0);
            if constexpr (SDE) a.sde_w[e] = sd > 0.0 ? sn / sd : 0.0;
        }
        tmem_fence_before_sync();  // this event's TMEM loads are done before the next event's first update
        __syncthreads();
    }
    if constexpr (L::J_MMA) {
        // the last commit was waited for by every thread (unless a wait ran out:
        // then wait once more, bounded, before the columns are released)
        if (ncommit > 0 && failed) mbar_wait_bounded(&mma_bar, (ncommit - 1) & 1u, ME_WAIT_LIMIT_CYCLES);
        tmem_fence_before_sync();
        __syncthreads();
        if (tid < 32) {
            tmem_fence_after_sync();
            tmem_dealloc(tmem_base, L::TMEM_COLS);
        }
    }
}

// global-memory J scratch of one resident CTA (0 when J stays on chip)
template <class P, class T> constexpr size_t interp_jscratch_per_cta()
{
    using L = InterpLayout<P, T>;
    return L::J_GLOBAL ? sizeof(cx<T>) * (size_t)P::NCOL * P::NT * (L::NTH / P::NT) : 0;
}

// One-time kernel attributes and the number of resident CTAs per SM of the
// persistent grid.  The grid is sized by the occupancy query, which takes the
// kernel's shared-memory carveout preference: ask for the largest carveout, so
// that it counts every CTA that fits the SM's shared memory.
template <class P, class T, bool TC, class C, bool SDE> cudaError_t interp_residency(int& nsm, int& per_sm)
{
    using L = InterpLayout<P, T>;
    static size_t granted = 0;
    cudaError_t e = ensure_smem(me_kernel_interp<P, T, TC, C, SDE>, L::launch_bytes, granted);
    if (e != cudaSuccess) return e;
    static bool carveout = false;
    if (!carveout) {
        e = cudaFuncSetAttribute(me_kernel_interp<P, T, TC, C, SDE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        carveout = true;
    }
    int dev = 0;
    nsm = 0;
    per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, me_kernel_interp<P, T, TC, C, SDE>, L::NTH,
                                                      L::launch_bytes) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    if constexpr (L::J_MMA) per_sm = tmem_kernel_ctas_per_sm(me_kernel_interp<P, T, TC, C, SDE>, L::launch_bytes, L::NTH,
                                                             L::TMEM_COLS);
    return cudaSuccess;
}

// resident CTAs of a full launch (the J scratch it allocates is this x interp_jscratch_per_cta)
template <class P, class T, bool TC = false, class C = T, bool SDE = false> int interp_resident_ctas()
{
    int nsm = 0, per_sm = 0;
    if (interp_residency<P, T, TC, C, SDE>(nsm, per_sm) != cudaSuccess) return 0;
    return nsm * per_sm;
}

template <class P, class T, bool TC = false, class C = T, bool SDE = false> cudaError_t launch_interp(const LaunchArgs& a)
{
    using L = InterpLayout<P, T>;
    static_assert(!TC || sizeof(T) == 4, "tensor-core colour sum is the mixed-precision path");
    static_assert(L::launch_bytes <= 232448, "interpreter shared memory exceeds 227 KB");
    // with J in tensor memory two CTAs share an SM (228 KB; per CTA 1 KB reserved
    // and at most 1.5 KB of static arrays): the generator caps the table for it
    static_assert(!L::J_MMA || 2 * (L::launch_bytes + 1024 + 1536) <= 233472, "two CTAs per SM do not fit");
    if (a.nlist > P::NT) return cudaErrorInvalidValue;
    int nsm = 0, per_sm = 0;
    cudaError_t e = interp_residency<P, T, TC, C, SDE>(nsm, per_sm);
    if (e != cudaSuccess) return e;
    const long long slots = (long long)nsm * per_sm;  // resident CTAs, persistent over events
    long long grid = a.nevt < slots ? a.nevt : slots;
    cx<T>* jg = nullptr;
    bool own = false;
    if constexpr (interp_jscratch_per_cta<P, T>() > 0) {
        constexpr size_t per = interp_jscratch_per_cta<P, T>();
        if (a.jscratch) {  // caller's scratch: fewer resident CTAs if it holds fewer, no allocation
            const long long fit = (long long)(a.jscratch_bytes / per);
            if (fit < 1 || (reinterpret_cast<uintptr_t>(a.jscratch) & 15)) return cudaErrorInvalidValue;
            if (grid > fit) grid = fit;
            jg = static_cast<cx<T>*>(a.jscratch);
        } else {
            e = staging_alloc(&jg, per * (size_t)grid, a.stream);
            if (e != cudaSuccess) return e;
            own = true;
        }
    }
    me_kernel_interp<P, T, TC, C, SDE><<<(unsigned)grid, L::NTH, L::launch_bytes, a.stream>>>(a, jg);
    e = cudaGetLastError();
    if (own) cudaFreeAsync(jg, a.stream);
    return e;
}

}  // namespace me
