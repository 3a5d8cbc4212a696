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
//      vector J (registers), contracts J^+ C J, and accumulates in FP64;
//   5. CTA reduction over helicities -> me2[event].
// The per-thread live state is J plus the operands of the amplitudes in
// flight, so the chain never spills.
#pragma once
#include <type_traits>

#include "me_colour_tc.cuh"
#include "me_kernel.cuh"

// Ordering point between amplitudes (a warp barrier, which ptxas does not move
// shared-memory loads across): keeps the operand loads of many amplitudes from
// being hoisted ahead of their use, which would push register pressure past the
// register file and spill.  The generated process struct sets the interval
// (FENCE_F for FP32, FENCE_P for packed FP32x2, FENCE_D for FP64: the longer
// FP64 and packed dependency chains need more cross-amplitude ILP); the build
// options ME_FENCE_EVERY_F / _P / _D override it.
//
// Every ME_CTA_SYNC amplitudes (0: never) the whole CTA meets at a barrier, so
// that all its warps execute the same short stretch of the straight-line
// amplitude code.  The amplitude code is only ever called in CTA-uniform
// control flow.
#ifndef ME_CTA_SYNC
#define ME_CTA_SYNC 0
#endif
#define ME_FENCE(T, i)                                                                        \
    do {                                                                                      \
        if constexpr (ME_CTA_SYNC > 0 && ((i) + 1) % (ME_CTA_SYNC > 0 ? ME_CTA_SYNC : 1) == 0) \
            __syncthreads();                                                                  \
        else if constexpr (((i) + 1) % me::fence_every<T>(FENCE_F, FENCE_P, FENCE_D) == 0)    \
            __syncwarp();                                                                     \
    } while (0)

namespace me {

template <class T> __host__ __device__ constexpr bool is_fp64() { return std::is_same<T, double>::value; }
template <class T> __host__ __device__ constexpr int fence_every(int f, int p, int d)
{
#ifdef ME_FENCE_EVERY_F
    f = ME_FENCE_EVERY_F;
#endif
#ifdef ME_FENCE_EVERY_P
    p = ME_FENCE_EVERY_P;
#endif
#ifdef ME_FENCE_EVERY_D
    d = ME_FENCE_EVERY_D;
#endif
    return std::is_same<T, double>::value ? d : std::is_same<T, f2>::value ? p : f;
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

template <class P, class T> __host__ __device__ constexpr size_t tab_line_offset()
{
    return (size_t)P::NPAR * 4 * sizeof(double);
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
template <class P, class T> __host__ __device__ constexpr int tab_epc() { return is_fp64<T>() ? P::EPC_D : P::EPC_F; }

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
    __shared__ double red_sde[SDE ? EPC : 1][2][NT / 32 > 0 ? NT / 32 : 1];

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
        if (live) {
            for (int it = tid; it < 2 * NPAR + NL; it += NT) {
                if (it < 2 * NPAR) tab.st(it, ext_wavefunction<P, T>(smom, it, a.mt, a.gauge_ext));
                else sln[it - 2 * NPAR] = line_data<P, T>(smom, it - 2 * NPAR, a.mt);
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
            if constexpr (TC) {
                __syncthreads();  // single pass (nlist <= NT): the tables are dead, reuse them as staging
                unsigned char* stage = smem + tab_table_offset<P, T>() + (tid >> 5) * TcShape<P::NCOL>::WARP_BYTES;
                v = colour_tc_warp<P::NCOL, P::NSPLIT>(J, stage, P::bfrag(), tid & 31);
            } else {
                v = colour_as<P, T, C>(J);
            }
            if (act) {
                acc += (double)v;
                if constexpr (SDE) {
                    snum += (double)sde.num;
                    sden += (double)sde.den;
                }
                if (a.hel_out) a.hel_out[e * a.nlist + i] = (double)v * a.norm;
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if constexpr (SDE) {
                snum += __shfl_xor_sync(0xffffffffu, snum, off);
                sden += __shfl_xor_sync(0xffffffffu, sden, off);
            }
        }
        if constexpr (NT > 32) {
            if ((tid & 31) == 0) {
                red[grp][tid >> 5] = acc;
                if constexpr (SDE) {
                    red_sde[grp][0][tid >> 5] = snum;
                    red_sde[grp][1][tid >> 5] = sden;
                }
            }
            __syncthreads();
            if (tid == 0 && live) {
                double s = 0.0, sn = 0.0, sd = 0.0;
                for (int w = 0; w < NT / 32; ++w) {
                    s += red[grp][w];
                    if constexpr (SDE) {
                        sn += red_sde[grp][0][w];
                        sd += red_sde[grp][1][w];
                    }
                }
                a.me2[e] = s * a.norm * (a.w_ev ? a.w_ev[e] : 1.0);
                if constexpr (SDE) a.sde_w[e] = sd > 0.0 ? sn / sd : 0.0;
            }
        } else {
            if (tid == 0 && live) {
                a.me2[e] = acc * a.norm * (a.w_ev ? a.w_ev[e] : 1.0);
                if constexpr (SDE) a.sde_w[e] = sden > 0.0 ? snum / sden : 0.0;
            }
        }
        __syncthreads();  // shared memory is reused by the next events
    }
}


// ---------------------------------------------------------------------------
// Event-pair kernel (FP32 and mixed precision): one CTA evaluates two events in
// lock step with packed FP32x2 arithmetic (T = f2, lane 0 = event e, lane 1 =
// event e + 1).  The two events' tables are interleaved component by component,
// so a 16-byte shared-memory load delivers two packed operands, and every
// arithmetic instruction of the table and amplitude phases does the work of
// two events.  The external wavefunctions and line data are computed per event
// in FP32 (denominators formed in FP64) and then packed.  The colour sum runs
// per event: scalar FP32, or the BF16 tensor-core form (TC).
// ---------------------------------------------------------------------------
template <class P> struct PairLayout {
    static constexpr size_t mom = 0;                                           // [2][NPAR][4] double
    static constexpr size_t lines = mom + 2 * (size_t)P::NPAR * 4 * sizeof(double);
    static constexpr size_t table = (lines + (size_t)P::NLINES * sizeof(Ln<f2>) + 15) / 16 * 16;
    static constexpr size_t bytes = table + (size_t)P::TAB * sizeof(Wf<f2>);
};

__device__ __forceinline__ Wf<f2> pack_wf(const Wf<float>& a, const Wf<float>& b)
{
    Wf<f2> o;
#pragma unroll
    for (int k = 0; k < 4; ++k) o.c[k] = {f2::pack(a.c[k].re, b.c[k].re), f2::pack(a.c[k].im, b.c[k].im)};
    return o;
}

template <class P, bool TC>
__global__ void __launch_bounds__(P::NT * P::PPC, P::MIN_CTAS_P) me_kernel_pair(LaunchArgs a)
{
    using L = PairLayout<P>;
    extern __shared__ __align__(16) unsigned char smem_all[];
    constexpr int NPAR = P::NPAR, NL = P::NLINES, NT = P::NT, PPC = P::PPC;
    const int grp = threadIdx.x / NT;  // event pair of this thread within the CTA
    const int tid = threadIdx.x - grp * NT;
    unsigned char* smem = smem_all + grp * L::bytes;
    double* smom = reinterpret_cast<double*>(smem + L::mom);
    Ln<f2>* sln = reinterpret_cast<Ln<f2>*>(smem + L::lines);
    const TabRef<f2, P::TAB> tab{reinterpret_cast<uint4*>(smem + L::table)};
    __shared__ double red[PPC][2][NT / 32 > 0 ? NT / 32 : 1];

    for (long long q0 = (long long)blockIdx.x * PPC; 2 * q0 < a.nevt; q0 += (long long)gridDim.x * PPC) {
        const long long e0 = 2 * (q0 + grp);
        // a dead pair (past the end) and the missing half of a ragged last pair
        // evaluate a real event and store nothing; every thread reaches every barrier
        const bool live0 = e0 < a.nevt, live1 = e0 + 1 < a.nevt;
        const long long s0 = live0 ? e0 : a.nevt - 1, s1 = live1 ? e0 + 1 : s0;
        // (a1) momenta of both events
        for (int i = tid; i < 2 * NPAR * 4; i += NT) {
            const long long e = i < NPAR * 4 ? s0 : s1;
            smom[i] = __ldg(a.mom + e * NPAR * 4 + (i % (NPAR * 4)));
        }
        __syncthreads();
        // (a2, a3 denominators) per event in FP32, then packed
        for (int it = tid; it < 2 * NPAR + NL; it += NT) {
            if (it < 2 * NPAR) {
                tab.st(it, pack_wf(ext_wavefunction<P, float>(smom, it, a.mt, a.gauge_ext),
                                   ext_wavefunction<P, float>(smom + NPAR * 4, it, a.mt, a.gauge_ext)));
            } else {
                const Ln<float> l0 = line_data<P, float>(smom, it - 2 * NPAR, a.mt);
                const Ln<float> l1 = line_data<P, float>(smom + NPAR * 4, it - 2 * NPAR, a.mt);
                Ln<f2> o;
#pragma unroll
                for (int mu = 0; mu < 4; ++mu) o.p[mu] = f2::pack(l0.p[mu], l1.p[mu]);
                o.inv = f2::pack(l0.inv, l1.inv);
                sln[it - 2 * NPAR] = o;
            }
        }
        __syncthreads();
        // (a3) off-shell objects for every helicity configuration of their support
        if constexpr (!P::STAGED) {
            P::template tables<f2>(tab, sln, f2((float)a.mt), tid);
            __syncthreads();
        }
        // (a4-a6) amplitudes per good helicity (uniform passes, see me_kernel_tab)
        double acc0 = 0.0, acc1 = 0.0;
        for (int base = 0; base < a.nlist; base += NT) {
            const int i = base + tid;
            const bool act = i < a.nlist;
            const int h = a.hel_list[act ? i : 0];
            cx<f2> J[P::NCOL];
#pragma unroll
            for (int c = 0; c < P::NCOL; ++c) J[c] = {f2(0), f2(0)};
            SdeAcc<f2> sde{f2(0), f2(0), 0};   // unused: the pair kernel computes no enhancement weights
            if constexpr (P::STAGED) P::template staged<f2, false>(tab, sln, f2((float)a.mt), tid, h, J, sde);
            else P::template amps<f2, false>(tab, h, sln, J, sde);
            float v0, v1;
            if constexpr (TC) {
                __syncthreads();  // single pass (nlist <= NT): the tables are dead, reuse them as staging
                unsigned char* stage = smem + L::table + (tid >> 5) * TcShape<P::NCOL>::WARP_BYTES;
                cx<float> Je[P::NCOL];
#pragma unroll
                for (int c = 0; c < P::NCOL; ++c) Je[c] = {J[c].re.lo(), J[c].im.lo()};
                v0 = colour_tc_warp<P::NCOL, P::NSPLIT>(Je, stage, P::bfrag(), tid & 31);
#pragma unroll
                for (int c = 0; c < P::NCOL; ++c) Je[c] = {J[c].re.hi(), J[c].im.hi()};
                v1 = colour_tc_warp<P::NCOL, P::NSPLIT>(Je, stage, P::bfrag(), tid & 31);
            } else {
                const f2 v = P::template colour<f2>(J);
                v0 = v.lo();
                v1 = v.hi();
            }
            if (act) {
                acc0 += (double)v0;
                acc1 += (double)v1;
                if (a.hel_out) {
                    if (live0) a.hel_out[e0 * a.nlist + i] = (double)v0 * a.norm;
                    if (live1) a.hel_out[(e0 + 1) * a.nlist + i] = (double)v1 * a.norm;
                }
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            acc0 += __shfl_xor_sync(0xffffffffu, acc0, off);
            acc1 += __shfl_xor_sync(0xffffffffu, acc1, off);
        }
        if constexpr (NT > 32) {
            if ((tid & 31) == 0) {
                red[grp][0][tid >> 5] = acc0;
                red[grp][1][tid >> 5] = acc1;
            }
            __syncthreads();
            if (tid < 2 && (tid == 0 ? live0 : live1)) {
                double s = 0.0;
                for (int w = 0; w < NT / 32; ++w) s += red[grp][tid][w];
                a.me2[e0 + tid] = s * a.norm;
            }
        } else {
            if (tid == 0) {
                if (live0) a.me2[e0] = acc0 * a.norm;
                if (live1) a.me2[e0 + 1] = acc1 * a.norm;
            }
        }
        __syncthreads();  // shared memory is reused by the next pairs
    }
}

template <class P, bool TC> cudaError_t launch_pair(const LaunchArgs& a)
{
    constexpr size_t smem = PairLayout<P>::bytes * P::PPC;
    if (P::STAGED && a.nlist > P::NT) return cudaErrorInvalidValue;
    if constexpr (TC)
        static_assert((P::NT / 32) * TcShape<P::NCOL>::WARP_BYTES <= P::TAB * sizeof(Wf<f2>),
                      "tensor-core staging must fit in the table region");
    static size_t granted = 0;
    cudaError_t e = ensure_smem(me_kernel_pair<P, TC>, smem, granted);
    if (e != cudaSuccess) return e;
    const long long pairs = (a.nevt + 1) / 2;
    const long long ctas = (pairs + P::PPC - 1) / P::PPC;
    const long long grid = ctas < 0x7fffffffLL ? ctas : 0x7fffffffLL;
    me_kernel_pair<P, TC><<<(unsigned)grid, P::NT * P::PPC, smem, a.stream>>>(a);
    return cudaGetLastError();
}

template <class P, class T, bool TC = false, class C = T, bool SDE = false> cudaError_t launch_tab(const LaunchArgs& a)
{
    if constexpr (!is_fp64<T>() && std::is_same<C, T>::value && !SDE && P::PAIR_F) {
        if (!a.hel_ev) return launch_pair<P, TC>(a);  // the pair kernel shares each helicity between two events
    }
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
        const long long grid = ctas < 0x7fffffffLL ? ctas : 0x7fffffffLL;
        me_kernel_tab<P, T, TC, C, SDE><<<(unsigned)grid, P::NT * EPC, smem, a.stream>>>(a);
        return cudaGetLastError();
    }
}

// Mixed precision: FP32 chain; colour sum on BF16 tensor cores for 24 or more
// colour flows when every thread holds one helicity, FP32 scalar otherwise.
template <class P, class T, bool TC, class C, bool SDE> cudaError_t launch_interp(const LaunchArgs& a);

// Build option ME_MIXED_TC_MIN_NCOL: smallest colour basis whose mixed-precision
// colour sum runs on the tensor cores (default 24).
#ifndef ME_MIXED_TC_MIN_NCOL
#define ME_MIXED_TC_MIN_NCOL 24
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
