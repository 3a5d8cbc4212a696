// Helicity-recycled |M|^2 kernel: one CTA per event (arXiv:2507.21039 Sec. 3.1
// chain, Sec. 4.1 colour sum, helicity sum).
//
//   1. the event's momenta (FP64) are loaded into shared memory;
//   2. per event: the external wavefunctions for both helicities of each
//      particle (in the amplitude precision T) and every line's momentum and
//      1/(p^2 - m^2) (momentum sums and p^2 - m^2 in FP64);
//   3. the off-shell objects (gluon currents, quark-line prefixes/suffixes,
//      pair current) are evaluated once per helicity configuration of their own
//      particles into a shared-memory table, level by level, by all threads;
//   4. each thread takes one good helicity (or several), evaluates that
//      helicity's final amplitudes from table operands into the colour-flow
//      vector J (registers; amplitudes whose colour vectors agree up to a sign
//      are summed first and added into J once), contracts J^+ C J, and
//      accumulates in FP64;
//   5. CTA reduction over helicities -> me2[event].
// The per-thread live state is J plus the operands of the amplitudes in
// flight, so the chain never spills.
#pragma once
#include <type_traits>

#include "me_colour_tc.cuh"
#include "me_kernel.cuh"
#include "me_tmem.cuh"

// Ordering point between amplitudes (a warp barrier, which ptxas does not move
// shared-memory loads across): keeps the operand loads of many amplitudes from
// being hoisted ahead of their use, which would push register pressure past the
// register file and spill.  The generated process struct sets the interval
// (FENCE_F for FP32, FENCE_D for FP64, whose longer dependency chains need
// more cross-amplitude ILP); the build options ME_FENCE_EVERY_F / _D override it.
#define ME_FENCE(T, i)                                                          \
    do {                                                                        \
        if constexpr (((i) + 1) % me::fence_every<T>(FENCE_F, FENCE_D) == 0) \
            __syncwarp();                                                       \
    } while (0)

namespace me {

template <class T> __host__ __device__ constexpr bool is_fp64() { return std::is_same<T, double>::value; }
template <class T> __host__ __device__ constexpr int fence_every(int f, int d)
{
#ifdef ME_FENCE_EVERY_F
    f = ME_FENCE_EVERY_F;
#endif
#ifdef ME_FENCE_EVERY_D
    d = ME_FENCE_EVERY_D;
#endif
    return std::is_same<T, double>::value ? d : f;
}

struct __align__(16) TabTask {
    unsigned short out, in0, in1, in2;
    unsigned char la, lb, lo, pad0;
    unsigned int pad1;
};

__device__ __forceinline__ TabTask ld_task(const TabTask* p)
{
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    TabTask t;
    t.out = (unsigned short)(v.x & 0xffff);
    t.in0 = (unsigned short)(v.x >> 16);
    t.in1 = (unsigned short)(v.y & 0xffff);
    t.in2 = (unsigned short)(v.y >> 16);
    t.la = (unsigned char)(v.z & 0xff);
    t.lb = (unsigned char)((v.z >> 8) & 0xff);
    t.lo = (unsigned char)((v.z >> 16) & 0xff);
    return t;
}

// Tables are stored as planes of 16-byte chunks: chunk c of entry i lives at
// c * TAB + i.  Lanes that read consecutive variants then touch consecutive
// banks (a plain array of 32- or 64-byte entries makes 2- or 4-way conflicts).
// A 16-byte load of a warp is served in phases of 8 lanes, which differ in the
// three lowest helicity bits; the generator numbers an object's variants with
// the highest-numbered support particle (lowest helicity bit) first, so those
// lanes read at most 8 consecutive entries.
template <class T> struct Chunks { static constexpr int N = (int)(sizeof(Wf<T>) / 16); };

template <class T, int TAB> struct TabRef {
    uint4* base;
    __device__ __forceinline__ Wf<T> ld(int i) const
    {
        Wf<T> w;
        uint4* dst = reinterpret_cast<uint4*>(&w);
#pragma unroll
        for (int c = 0; c < Chunks<T>::N; ++c) dst[c] = base[c * TAB + i];
        return w;
    }
    __device__ __forceinline__ void st(int i, const Wf<T>& w) const
    {
        const uint4* src = reinterpret_cast<const uint4*>(&w);
#pragma unroll
        for (int c = 0; c < Chunks<T>::N; ++c) base[c * TAB + i] = src[c];
    }
};

// per-event shared memory: FP64 momenta; for T = float the split momenta and
// the Gram matrix (FP32 setup, see me_kernel.cuh); lines; table
template <class P, class T> __host__ __device__ constexpr size_t tab_pf_offset()
{
    return (size_t)P::NPAR * 4 * sizeof(double);
}
template <class P, class T> __host__ __device__ constexpr size_t tab_gram_offset()
{
    return tab_pf_offset<P, T>() + (std::is_same<T, float>::value ? (size_t)P::NPAR * 4 * sizeof(float2) : 0);
}
template <class P, class T> __host__ __device__ constexpr size_t tab_line_offset()
{
    return tab_gram_offset<P, T>() + (std::is_same<T, float>::value ? (size_t)Gram<P::NPAR>::N * sizeof(double) : 0);
}
template <class P, class T> __host__ __device__ constexpr size_t tab_table_offset()
{
    return (tab_line_offset<P, T>() + (size_t)P::NLINES * sizeof(Ln<T>) + 15) / 16 * 16;
}
template <class P, class T> __host__ __device__ constexpr size_t tab_smem_bytes()
{
    return tab_table_offset<P, T>() + (size_t)P::TAB * sizeof(Wf<T>);
}

// TC: colour sum on the tensor cores (T = float, NCOL >= 24, one helicity per
// thread: nlist <= NT); otherwise the scalar quadratic form in precision T.
// EPC events share a CTA (NT threads each, own shared-memory region); CTA-wide
// barriers keep their warps at the same point of the amplitude code, so they
// share instruction-cache lines and overlap each other's long-latency FP64 work.
// Build option ME_TAB_TC_FROM_SMEM: tensor-core colour sum from a shared-memory
// copy of J (1) or from J in registers (0)
#ifndef ME_TAB_TC_FROM_SMEM
#define ME_TAB_TC_FROM_SMEM 1
#endif

template <class P, class T> __host__ __device__ constexpr int tab_epc() { return is_fp64<T>() ? P::EPC_D : P::EPC_F; }

// Build option ME_TAB_TC_UMMA: the tensor-core colour sum of a CTA of 128
// helicity rows as tcgen05.mma with the result in TMEM (1, default where the
// colour numerators are exact in BF16 and at most 32 flows), or as per-warp
// mma.sync (0)
#ifndef ME_TAB_TC_UMMA
#define ME_TAB_TC_UMMA 1
#endif
template <class P, class T, bool TC> __host__ __device__ constexpr bool tab_umma()
{
    if constexpr (!TC) {
        return false;
    } else {
        return ME_TAB_TC_UMMA && P::NCOL <= 32 && !P::NSPLIT && P::NT * tab_epc<P, T>() == 128 &&
               tab_epc<P, T>() == 2 && (size_t)P::TAB * sizeof(Wf<T>) >= 4 * 4096;
    }
}
constexpr uint32_t kTabUmmaCols = 64;  // TMEM columns: Re rows' results 0-31, Im rows' 32-63

// Colour form J^+ N J of the CTA's 128 helicity rows (thread = row = TMEM
// lane) on the tensor cores with tcgen05.mma (Sec. 4.1 colour algebra):
//   * each thread writes its row of A: Re J and Im J split exactly into BF16
//     hi + lo (16 significant bits of each FP32 value), flows 0..31 (zero past
//     NCOL) as two K = 16 operand images per matrix -- eight 4096-byte images,
//     four in each event slot's table region, which is dead at this point;
//   * one thread issues Y_re = (Re J)_hi N + (Re J)_lo N and the same for Im
//     (M = 128, N = 32, K = 16, eight MMAs; N exact in BF16, FP32 accumulation
//     in TMEM columns 0-31 and 32-63) and commits them to the mbarrier;
//   * every thread waits (bounded), reads its row of Y from TMEM and returns
//     Re J . Y_re + Im J . Y_im with its own FP32 J.
// The caller has passed a CTA barrier after the last table read.  Returns NaN
// for the thread if a wait ran out (`failed` then stays set).
template <class P, class T, class JT>
__device__ __forceinline__ float colour_umma(const JT& J, unsigned char* smem_all, const unsigned char* cn_smem,
                                             uint32_t tmem_base, uint64_t* bar, uint32_t& ncommit, bool& failed)
{
    constexpr int NCOL = P::NCOL;
    // image j = 2 m + ks (m: 0 Re hi, 1 Re lo, 2 Im hi, 3 Im lo; ks: K step) of event slot j / 4
    auto img = [&](int m, int ks) -> unsigned char* {
        const int j = 2 * m + ks;
        return smem_all + (size_t)(j >> 2) * tab_smem_bytes<P, T>() + tab_table_offset<P, T>() + (size_t)(j & 3) * 4096;
    };
    auto jre = [&](int f) { return f < NCOL ? (float)J[f < NCOL ? f : 0].re : 0.0f; };
    auto jim = [&](int f) { return f < NCOL ? (float)J[f < NCOL ? f : 0].im : 0.0f; };
    const int row = threadIdx.x;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
        for (int kc = 0; kc < 2; ++kc) {  // 8 flows = one 16-byte chunk of the row per matrix
            uint32_t w[4][4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int f = 16 * ks + 8 * kc + 2 * q;
                split2(jre(f), jre(f + 1), w[0][q], w[1][q]);
                split2(jim(f), jim(f + 1), w[2][q], w[3][q]);
            }
            const uint32_t off = umma_k16_offset(row, 8 * kc);
#pragma unroll
            for (int m = 0; m < 4; ++m)
                *reinterpret_cast<uint4*>(img(m, ks) + off) = make_uint4(w[m][0], w[m][1], w[m][2], w[m][3]);
        }
    fence_proxy_async_smem();
    __syncthreads();
    if (row == 0 && !failed) {
        tmem_fence_after_sync();
        constexpr uint32_t ID = umma_idesc_bf16_f32(128, 32, false);
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const uint64_t bdesc = umma_smem_desc(cn_smem + 1024 * ks, 128, 256);
#pragma unroll
            for (int m = 0; m < 4; ++m)  // the first MMA into each result overwrites it
                umma_bf16(tmem_base + (m < 2 ? 0u : 32u), umma_smem_desc(img(m, ks), 128, 256), bdesc, ID,
                          ks > 0 || (m & 1));
        }
        umma_commit(bar);
    }
    if (!failed && !mbar_wait_bounded(bar, ncommit & 1u, ME_WAIT_LIMIT_CYCLES)) failed = true;
    ++ncommit;
    tmem_fence_after_sync();
    const uint32_t tl = tmem_base + ((uint32_t)(32 * (row >> 5)) << 16);
    uint32_t y[4][16];
#pragma unroll
    for (int c = 0; c < 4; ++c) tmem_ld_16(tl + 16u * (uint32_t)c, y[c]);
    float v = 0.0f;
#pragma unroll
    for (int c = 0; c < NCOL; ++c)
        v = fmaf(jre(c), __uint_as_float(y[c >> 4][c & 15]), fmaf(jim(c), __uint_as_float(y[2 + (c >> 4)][c & 15]), v));
    return failed ? __int_as_float(0x7fc00000) : v;
}

template <class P, class T, bool TC, class C = T, bool SDE = false>
__global__ void __launch_bounds__(P::NT * tab_epc<P, T>(), is_fp64<T>() ? P::MIN_CTAS_D : P::MIN_CTAS_F)
    me_kernel_tab(LaunchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_all[];
    constexpr int NPAR = P::NPAR, NL = P::NLINES, NT = P::NT, EPC = tab_epc<P, T>();
    const int grp = threadIdx.x / NT;      // event slot of this thread within the CTA
    const int tid = threadIdx.x - grp * NT;
    unsigned char* smem = smem_all + grp * tab_smem_bytes<P, T>();
    double* smom = reinterpret_cast<double*>(smem);
    Ln<T>* sln = reinterpret_cast<Ln<T>*>(smem + tab_line_offset<P, T>());
    const TabRef<T, P::TAB> tab{reinterpret_cast<uint4*>(smem + tab_table_offset<P, T>())};
    __shared__ double red[EPC][NT / 32 > 0 ? NT / 32 : 1];
    __shared__ FSum fred[EPC][NT / 32 > 0 ? NT / 32 : 1];
    __shared__ double red_sde[SDE ? EPC : 1][2][NT / 32 > 0 ? NT / 32 : 1];
    constexpr bool F32 = !is_fp64<T>();
    float2* spf = reinterpret_cast<float2*>(smem + tab_pf_offset<P, T>());
    double* sgram = reinterpret_cast<double*>(smem + tab_gram_offset<P, T>());
    const double m2 = a.mt * a.mt;
    const float mtf = (float)a.mt;
    // tcgen05 colour sum: the numerators (B operand) in shared memory once per
    // CTA, 64 TMEM columns, one mbarrier for the MMAs' completion
    constexpr bool UMMA = tab_umma<P, T, TC>();
    __shared__ __align__(16) unsigned char cn_smem[UMMA ? 2048 : 16];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t mma_bar;
    uint32_t ncommit = 0;  // MMA commits so far (the same in every thread)
    bool failed = false;   // a wait for the tensor cores ran out
    if constexpr (UMMA) {
        if (threadIdx.x < 32) {
            tmem_alloc(&tmem_base, kTabUmmaCols);
            tmem_relinquish();
        }
        if (threadIdx.x == 0) {
            mbar_init(&mma_bar, 1);
            mbar_init_fence();
        }
        for (int i = threadIdx.x; i < 128; i += blockDim.x) reinterpret_cast<uint4*>(cn_smem)[i] = __ldg(P::umma_cn() + i);
        fence_proxy_async_smem();
        tmem_fence_before_sync();
        __syncthreads();
        tmem_fence_after_sync();
    }

    for (long long e0 = (long long)blockIdx.x * EPC; e0 < a.nevt; e0 += (long long)gridDim.x * EPC) {
        const long long e = e0 + grp;
        const bool live = e < a.nevt;      // a ragged last CTA still takes part in every barrier
        // (a1) momenta
        if (live) {
            const double* g = a.mom + e * NPAR * 4;
            if ((reinterpret_cast<uintptr_t>(g) & 15) == 0) {
                if (tid < NPAR * 2)
                    reinterpret_cast<double2*>(smom)[tid] = __ldg(reinterpret_cast<const double2*>(g) + tid);
            } else {
                for (int i = tid; i < NPAR * 4; i += NT) smom[i] = __ldg(g + i);
            }
        }
        __syncthreads();
        // (a2, a3 denominators) per-event data; external wavefunctions are the
        // first 2*NPAR table entries
        if constexpr (F32) {
            // split momenta and FP64 Gram matrix, then lines and external states in FP32
            if (live) {
                if constexpr (split_items_one_pass<NPAR, NT>()) {
                    const int it = split_item_of<NPAR>(tid);
                    if (it >= 0) split_or_gram<NPAR>(smom, it, spf, sgram);
                } else {
                    for (int it = tid; it < 4 * NPAR + Gram<NPAR>::N; it += NT) split_or_gram<NPAR>(smom, it, spf, sgram);
                }
            }
            __syncthreads();
            if (live) {
                for (int it = tid; it < NL + P::NEXT; it += NT) {
                    if (it < NL) sln[it] = line_data_split<P>(spf, sgram, it, m2);
                    else if (it < NL + 2 * NPAR) tab.st(it - NL, ext_wavefunction_split<P>(spf, it - NL, mtf, a.gauge_ext));
                    else tab.st(2 * NPAR, ew_coefficients<T>(smom));  // Drell-Yan: entry 2 NPAR
                }
            }
        } else if (live) {
            for (int it = tid; it < P::NEXT + NL; it += NT) {
                if (it < 2 * NPAR) tab.st(it, ext_wavefunction<P, T>(smom, it, a.mt, a.gauge_ext));
                else if (it < P::NEXT) tab.st(2 * NPAR, ew_coefficients<T>(smom));  // Drell-Yan: entry 2 NPAR
                else sln[it - P::NEXT] = line_data<P, T>(smom, it - P::NEXT, a.mt);
            }
        }
        __syncthreads();
        // (a3) off-shell objects for every helicity configuration of their support
        // (a dead slot computes on whatever its shared memory holds; nothing is stored)
        if constexpr (!P::STAGED) {
            P::template tables<T>(tab, sln, (T)a.mt, tid);
            __syncthreads();
        }
        // (a4-a6) amplitudes per good helicity, colour sum, FP64 accumulation.
        // Every lane runs every pass (lanes past the end of the list evaluate a
        // real helicity and discard it), so the warp and CTA barriers inside
        // the amplitude code are always reached by every thread.  A staged
        // process computes its table objects stage by stage between its
        // amplitudes, in one pass (nlist <= NT).
        double acc = 0.0, snum = 0.0, sden = 0.0;
        FSum facc{0.0f, 0.0f};
        for (int base = 0; base < a.nlist; base += NT) {
            const int i = base + tid;
            const bool act = live && i < a.nlist;
            // helicity sampling: one helicity per event (nlist = 1)
            const int h = a.hel_ev ? a.hel_ev[live ? e : 0] : a.hel_list[i < a.nlist ? i : 0];
            cx<T> J[P::NCOL];
#pragma unroll
            for (int c = 0; c < P::NCOL; ++c) J[c] = {T(0), T(0)};
            SdeAcc<T> sde{T(0), T(0), a.sde_channel};
            if constexpr (P::STAGED) P::template staged<T, SDE>(tab, sln, (T)a.mt, tid, h, J, sde);
            else P::template amps<T, SDE>(tab, h, sln, J, sde);
            T v;
            if constexpr (UMMA) {
                __syncthreads();  // single pass (nlist <= NT): the tables are dead, reuse them as staging
                v = colour_umma<P, T>(J, smem_all, cn_smem, tmem_base, &mma_bar, ncommit, failed);
            } else if constexpr (TC) {
                __syncthreads();  // single pass (nlist <= NT): the tables are dead, reuse them as staging
#if ME_TAB_TC_FROM_SMEM
                // J leaves the registers first ([flow][lane] FP32 per warp), so the
                // tensor-core phase does not hold it next to its fragments
                constexpr size_t WJ = (size_t)P::NCOL * 32 * sizeof(cx<float>) + 32 * sizeof(float);
                static_assert((size_t)(NT / 32) * WJ <= (size_t)P::TAB * sizeof(Wf<T>), "staging exceeds the table");
                unsigned char* stage = smem + tab_table_offset<P, T>() + (tid >> 5) * WJ;
                cx<float>* js = reinterpret_cast<cx<float>*>(stage);
#pragma unroll
                for (int c = 0; c < P::NCOL; ++c) js[c * 32 + (tid & 31)] = J[c];
                __syncwarp();
                v = colour_tc_smem<P::NCOL, 32, P::NSPLIT>(js, P::bfrag(),
                                                           reinterpret_cast<float*>(stage + (size_t)P::NCOL * 32 * sizeof(cx<float>)),
                                                           tid & 31);
#else
                unsigned char* stage = smem + tab_table_offset<P, T>() + (tid >> 5) * TcShape<P::NCOL>::WARP_BYTES;
                v = colour_tc_warp<P::NCOL, P::NSPLIT>(J, stage, P::bfrag(), tid & 31);
#endif
            } else {
                v = colour_as<P, T, C>(J);
            }
            if (!P::hel_allowed(h)) v = T(0);  // vanishes exactly; its table variants were not computed
            if (act) {
                if constexpr (F32) facc = fsum_add(facc, FSum{(float)v, 0.0f});
                else acc += (double)v;
                if constexpr (SDE) {
                    snum += (double)sde.num;
                    sden += (double)sde.den;
                }
                if (a.hel_out) a.hel_out[e * a.nlist + i] = (double)v * a.norm;
            }
        }
        // (events of fewer than 32 threads share a warp: reduce within each event's lanes)
        constexpr int W = NT < 32 ? NT : 32;
        static_assert((W & (W - 1)) == 0, "threads per event: a power of two below 32, or whole warps");
        if constexpr (F32) facc = fsum_warp<W>(facc);
        for (int off = W / 2; off > 0; off >>= 1) {
            if constexpr (!F32) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if constexpr (SDE) {
                snum += __shfl_xor_sync(0xffffffffu, snum, off);
                sden += __shfl_xor_sync(0xffffffffu, sden, off);
            }
        }
        if constexpr (NT > 32) {
            if ((tid & 31) == 0) {
                if constexpr (F32) fred[grp][tid >> 5] = facc;
                else red[grp][tid >> 5] = acc;
                if constexpr (SDE) {
                    red_sde[grp][0][tid >> 5] = snum;
                    red_sde[grp][1][tid >> 5] = sden;
                }
            }
            __syncthreads();
            if (tid == 0 && live) {
                double s = 0.0, sn = 0.0, sd = 0.0;
                if constexpr (F32) {  // one conversion per event
                    FSum f = fred[grp][0];
                    for (int w = 1; w < NT / 32; ++w) f = fsum_add(f, fred[grp][w]);
                    s = (double)f.s + (double)f.c;
                }
                for (int w = 0; w < NT / 32; ++w) {
                    if constexpr (!F32) s += red[grp][w];
                    if constexpr (SDE) {
                        sn += red_sde[grp][0][w];
                        sd += red_sde[grp][1][w];
                    }
                }
                a.me2[e] = s * a.norm * (a.w_ev ? a.w_ev[e] : 1.0);
                if constexpr (SDE) a.sde_w[e] = sd > 0.0 ? sn / sd : 0.0;
            }
        } else {
            if constexpr (F32) acc = (double)facc.s + (double)facc.c;
            if (tid == 0 && live) {
                a.me2[e] = acc * a.norm * (a.w_ev ? a.w_ev[e] : 1.0);
                if constexpr (SDE) a.sde_w[e] = sden > 0.0 ? snum / sden : 0.0;
            }
        }
        if constexpr (UMMA) tmem_fence_before_sync();  // TMEM reads done before the next events' MMAs
        __syncthreads();  // shared memory is reused by the next events
    }
    if constexpr (UMMA) {
        if (ncommit > 0 && failed) mbar_wait_bounded(&mma_bar, (ncommit - 1) & 1u, ME_WAIT_LIMIT_CYCLES);
        tmem_fence_before_sync();
        __syncthreads();
        if (threadIdx.x < 32) {
            tmem_fence_after_sync();
            tmem_dealloc(tmem_base, kTabUmmaCols);
        }
    }
}


template <class P, class T, bool TC = false, class C = T, bool SDE = false> cudaError_t launch_tab(const LaunchArgs& a)
{
    {
        constexpr int EPC = tab_epc<P, T>();
        constexpr size_t smem = tab_smem_bytes<P, T>() * EPC;
        if (P::STAGED && a.nlist > P::NT) return cudaErrorInvalidValue;
        if constexpr (TC)
            static_assert((P::NT / 32) * TcShape<P::NCOL>::WARP_BYTES <= P::TAB * sizeof(Wf<T>),
                          "tensor-core staging must fit in the table region");
        static size_t granted = 0;
        cudaError_t e = ensure_smem(me_kernel_tab<P, T, TC, C, SDE>, smem, granted);
        if (e != cudaSuccess) return e;
        const long long ctas = (a.nevt + EPC - 1) / EPC;
        long long grid = ctas < 0x7fffffffLL ? ctas : 0x7fffffffLL;
        if constexpr (tab_umma<P, T, TC>()) {
            // persistent: TMEM is allocated once per CTA, which then loops over event pairs
            static int resident = 0;
            if (!resident) {
                int dev = 0, nsm = 0;
                cudaGetDevice(&dev);
                cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
                resident = std::max(1, nsm) *
                           tmem_kernel_ctas_per_sm(me_kernel_tab<P, T, TC, C, SDE>, smem, P::NT * EPC, (int)kTabUmmaCols);
            }
            if (grid > resident) grid = resident;
        }
        me_kernel_tab<P, T, TC, C, SDE><<<(unsigned)grid, P::NT * EPC, smem, a.stream>>>(a);
        return cudaGetLastError();
    }
}

// Mixed precision: FP32 chain; colour sum on BF16 tensor cores for 24 or more
// colour flows when every thread holds one helicity, FP32 scalar otherwise.
template <class P, class T, bool TC, class C, bool SDE> cudaError_t launch_interp(const LaunchArgs& a);

// Build option ME_MIXED_TC_MIN_NCOL: smallest colour basis whose mixed-precision
// colour sum runs on the tensor cores.  Default 120, the crossover measured on
// GB300: at 24 flows (gg -> t t~ g g, J in registers, 0.65 k FMA per helicity)
// the FP32 scalar form is faster than either tensor-core form (20.2 ms per 2^20
// events against 21.5 ms with mma.sync and 22.8 ms with tcgen05.mma); at 120
// flows the tensor cores pay (gg -> t t~ ggg: 674 ms against 847 ms per 2^18).
#ifndef ME_MIXED_TC_MIN_NCOL
#define ME_MIXED_TC_MIN_NCOL 120
#endif
template <class P> cudaError_t launch_mixed(const LaunchArgs& a)
{
    if constexpr (P::IS_INTERP) {
        if constexpr (P::NCOL >= ME_MIXED_TC_MIN_NCOL) return launch_interp<P, float, true, float, false>(a);
        else return launch_interp<P, float, false, float, false>(a);
    } else if constexpr (P::IS_TAB) {
        if constexpr (P::NCOL >= ME_MIXED_TC_MIN_NCOL) {
            if (a.nlist <= P::NT) return launch_tab<P, float, true>(a);
        }
        return launch_tab<P, float, false>(a);
    } else {
        return launch_scalar<P, float>(a);
    }
}

}  // namespace me
