// Staged, descriptor-driven |M|^2 kernel for the largest process
// (arXiv:2507.21039 Sec. 3.1 chain, Sec. 4.1 colour sum, helicity sum).
//
// One CTA of NT threads per event, one helicity per thread.  The helicity-
// recycled table of off-shell objects (see me_kernel_tab.cuh) does not fit in
// shared memory for seven external particles, so the generator cuts the
// amplitudes into stages: each stage first computes, cooperatively and level by
// level, the table objects its amplitudes need that are not yet resident (into
// slots freed by objects whose last reader has passed), then every thread
// evaluates the stage's amplitudes for its helicity from compact descriptors
// and adds them into its colour-flow vector J.  J lives in shared memory in
// FP32 and in a global scratch (L2-resident) in FP64, whose tables alone fill
// shared memory.
#pragma once
#include "me_kernel_tab.cuh"

namespace me {

struct __align__(8) IRound {
    unsigned int task_begin;
    unsigned short ntask;
    unsigned char kind, barrier_after;
};
struct __align__(8) IStage {
    unsigned short round_begin, round_end, amp_begin, amp_end;
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

template <class P, class T> struct InterpLayout {
    static constexpr size_t mom = 0;
    static constexpr size_t lines = mom + P::NPAR * 4 * sizeof(double);
    static constexpr size_t vsup = (lines + P::NLINES * sizeof(Ln<T>) + 15) / 16 * 16;
    static constexpr size_t table = (vsup + (size_t)P::NSUP * P::NT + 15) / 16 * 16;
    static constexpr size_t jsm = table + (size_t)P::TAB * sizeof(Wf<T>);
    static constexpr bool J_IN_SMEM = sizeof(T) == 4;
    static constexpr size_t bytes = jsm + (J_IN_SMEM ? (size_t)P::NCOL * P::NT * sizeof(cx<T>) : 0);
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

// TC: colour sum on BF16 tensor cores (T = float); otherwise scalar in C
template <class P, class T, bool TC, class C = T, bool SDE = false>
__global__ void __launch_bounds__(P::NT) me_kernel_interp(LaunchArgs a, cx<T>* __restrict__ jglobal)
{
    using L = InterpLayout<P, T>;
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NPAR = P::NPAR, NL = P::NLINES, NT = P::NT, NCOL = P::NCOL;
    double* smom = reinterpret_cast<double*>(smem + L::mom);
    Ln<T>* sln = reinterpret_cast<Ln<T>*>(smem + L::lines);
    unsigned char* vsup = smem + L::vsup;
    const TabRef<T, P::TAB> tab{reinterpret_cast<uint4*>(smem + L::table)};
    // this thread's colour-flow vector: J[c] at jp[c * NT]
    cx<T>* jp = L::J_IN_SMEM ? reinterpret_cast<cx<T>*>(smem + L::jsm) + threadIdx.x
                             : jglobal + (size_t)blockIdx.x * NCOL * NT + threadIdx.x;
    __shared__ double red[NT / 32];
    __shared__ double red_sde[SDE ? 2 : 1][NT / 32];
    __shared__ float rowv[NT];
    const int tid = threadIdx.x;
    const bool act = tid < a.nlist;
    // compressed variant index of every operand support for helicity h
    // (support particles in descending order = helicity bits from low to high)
    auto variants = [&](int h) {
        for (int s = 0; s < P::NSUP; ++s) {
            const unsigned m = P::support_mask(s);
            unsigned v = 0, j = 0;
            for (int b = 0; b < NPAR; ++b)
                if ((m >> b) & 1) v |= ((h >> b) & 1) << j++;
            vsup[s * NT + tid] = (unsigned char)v;
        }
    };
    if (!a.hel_ev) variants(a.hel_list[act ? tid : 0]);

    for (long long e = blockIdx.x; e < a.nevt; e += gridDim.x) {
        if (a.hel_ev) variants(a.hel_ev[e]);  // helicity sampling: one helicity per event (nlist = 1)
        const double* g = a.mom + e * NPAR * 4;
        for (int i = tid; i < NPAR * 4; i += NT) smom[i] = __ldg(g + i);
        for (int c = 0; c < NCOL; ++c) jp[c * NT] = {T(0), T(0)};
        __syncthreads();
        for (int it = tid; it < 2 * NPAR + NL; it += NT) {
            if (it < 2 * NPAR) tab.st(it, ext_wavefunction<P, T>(smom, it, a.mt, a.gauge_ext));
            else sln[it - 2 * NPAR] = line_data<P, T>(smom, it - 2 * NPAR, a.mt);
        }
        __syncthreads();
        const T mt = (T)a.mt;
        T snum = T(0), sden = T(0);
        for (int s = 0; s < P::NSTAGE; ++s) {
            const IStage st = P::stage(s);
            for (int r = st.round_begin; r < st.round_end; ++r) {
                const IRound rd = P::round(r);
                for (int t = tid; t < rd.ntask; t += NT) run_task<T, P::TAB>(tab, sln, mt, rd.kind, ld_task(P::tasks() + rd.task_begin + t));
                if (rd.barrier_after) __syncthreads();
            }
            __syncthreads();
            int term = P::stage_term_begin(s);
            for (int ai = st.amp_begin; ai < st.amp_end; ++ai) {
                const IAmp d = P::amp(ai);
                const Wf<T> w0 = tab.ld(d.op[0] + vsup[d.sup[0] * NT + tid]);
                const Wf<T> w1 = tab.ld(d.op[1] + vsup[d.sup[1] * NT + tid]);
                cx<T> x;
                if (d.kind == A_DOTV) {         // amputated: two-operand contractions
                    x = DOTV<T>(w0, w1);
                } else if (d.kind == A_DOTF) {
                    x = DOTF<T>(w0, w1);
                } else {
                    const Wf<T> w2 = tab.ld(d.op[2] + vsup[d.sup[2] * NT + tid]);
                    switch (d.kind) {
                    case A_FFV1_0: x = FFV1_0<T>(w0, w1, w2); break;
                    case A_VVV1_0: x = VVV1_0<T>(w0, sln[d.la].p, w1, sln[d.lb].p, w2); break;
                    default: {
                        const Wf<T> w3 = tab.ld(d.op[3] + vsup[d.sup[3] * NT + tid]);
                        x = d.kind == A_VVVV1_0 ? VVVV1_0<T>(w0, w1, w2, w3)
                          : d.kind == A_VVVV3_0 ? VVVV3_0<T>(w0, w1, w2, w3) : VVVV4_0<T>(w0, w1, w2, w3);
                    }
                    }
                }
                if constexpr (SDE) {  // single-diagram enhancement
                    const T w2 = fma(x.re, x.re, x.im * x.im);
                    sden += w2;
                    if (P::diag(ai) == a.sde_channel) snum += w2;
                }
                // every colour coefficient is +-i: J_c += +-i x
                for (int k = 0; k < d.nterm; ++k, ++term) {
                    const unsigned short ct = P::term(term);
                    cx<T>& jc = jp[(ct & 0x7fff) * NT];
                    const cx<T> j = jc;
                    jc = (ct & 0x8000) ? cx<T>{j.re + x.im, j.im - x.re} : cx<T>{j.re - x.im, j.im + x.re};
                }
            }
            __syncthreads();  // stage done: its dead table slots are reused by the next stage
        }
        // colour quadratic form sum_ij N_ij Re(conj J_i J_j)
        T v = T(0);
        if constexpr (TC) {
            v = colour_tc_smem<NCOL, NT, P::NSPLIT>(reinterpret_cast<const cx<float>*>(smem + L::jsm), P::bfrag(),
                                                    rowv, tid);
        } else {
            C w = C(0);
            for (int i = 0; i < NCOL; ++i) {
                const cx<T> ji = jp[i * NT];
                C zr = C(0), zi = C(0);
                for (int j = i; j < NCOL; ++j) {
                    const C n = (C)P::cnum2(i, j);
                    const cx<T> jj = jp[j * NT];
                    zr = fma(n, (C)jj.re, zr);
                    zi = fma(n, (C)jj.im, zi);
                }
                w = fma((C)ji.re, zr, fma((C)ji.im, zi, w));
            }
            v = (T)w;
        }
        double acc = 0.0, dn = 0.0, dd = 0.0;
        if (act) {
            acc = (double)v;
            if constexpr (SDE) {
                dn = (double)snum;
                dd = (double)sden;
            }
            if (a.hel_out) a.hel_out[e * a.nlist + tid] = (double)v * a.norm;
        }
        for (int off = 16; off > 0; off >>= 1) {
            acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if constexpr (SDE) {
                dn += __shfl_xor_sync(0xffffffffu, dn, off);
                dd += __shfl_xor_sync(0xffffffffu, dd, off);
            }
        }
        if ((tid & 31) == 0) {
            red[tid >> 5] = acc;
            if constexpr (SDE) {
                red_sde[0][tid >> 5] = dn;
                red_sde[1][tid >> 5] = dd;
            }
        }
        __syncthreads();
        if (tid == 0) {
            double s = 0.0, sn = 0.0, sd = 0.0;
            for (int w = 0; w < NT / 32; ++w) {
                s += red[w];
                if constexpr (SDE) {
                    sn += red_sde[0][w];
                    sd += red_sde[1][w];
                }
            }
            a.me2[e] = s * a.norm * (a.w_ev ? a.w_ev[e] : 1.0);
            if constexpr (SDE) a.sde_w[e] = sd > 0.0 ? sn / sd : 0.0;
        }
        __syncthreads();
    }
}

template <class P, class T, bool TC = false, class C = T, bool SDE = false> cudaError_t launch_interp(const LaunchArgs& a)
{
    using L = InterpLayout<P, T>;
    static_assert(!TC || sizeof(T) == 4, "tensor-core colour sum is the mixed-precision path");
    static_assert(L::bytes <= 232448, "interpreter shared memory exceeds 227 KB");
    if (a.nlist > P::NT) return cudaErrorInvalidValue;
    static size_t granted = 0;
    cudaError_t e = ensure_smem(me_kernel_interp<P, T, TC, C, SDE>, L::bytes, granted);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, me_kernel_interp<P, T, TC, C, SDE>, P::NT, L::bytes) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const long long slots = (long long)nsm * per_sm;  // resident CTAs, persistent over events
    const long long grid = a.nevt < slots ? a.nevt : slots;
    cx<T>* jg = nullptr;
    if constexpr (!L::J_IN_SMEM) {
        e = cudaMallocAsync(&jg, sizeof(cx<T>) * (size_t)grid * P::NCOL * P::NT, a.stream);
        if (e != cudaSuccess) return e;
    }
    me_kernel_interp<P, T, TC, C, SDE><<<(unsigned)grid, P::NT, L::bytes, a.stream>>>(a, jg);
    e = cudaGetLastError();
    if (jg) cudaFreeAsync(jg, a.stream);
    return e;
}

}  // namespace me
