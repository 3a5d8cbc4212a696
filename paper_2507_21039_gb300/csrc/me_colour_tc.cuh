// Colour contraction J^+ C J on BF16 tensor cores (mixed precision, Sec. 4.1 of
// arXiv:2507.21039: the colour algebra is an inner product with an integer
// colour matrix, which tolerates reduced-precision arithmetic).
//
// For one warp (32 lanes = 32 helicities of one event), the 64 rows
// {Re J_lane, Im J_lane} form A [64 x K]; C = N / D with integer numerators N.
// Y = A N is a dense GEMM on the tensor cores: A is split as A_hi + A_lo
// (both BF16; |A - A_hi - A_lo| <= 2^-18 |A|), N is exact in BF16 when every
// numerator has at most 8 significant bits (24 flows) and is split N_hi + N_lo
// otherwise (120 flows); products accumulate in FP32 (mma.sync m16n8k16).
// Each lane then forms Re J.Y_re + Im J.Y_im with its own FP32 J.
// Staging: per warp, 2 BF16 planes of 32 rows x (K + 8) for one half (Re or
// Im), reused for the FP32 Y rows; the kernel places it over the table memory,
// which is dead once every lane has finished its amplitudes.
#pragma once
#include <cuda_bf16.h>

#include "me_kernel.cuh"

namespace me {

template <int NCOL> struct TcShape {
    static constexpr int KP = (NCOL + 15) / 16 * 16;   // K padded to the MMA k-step
    static constexpr int NP = (NCOL + 7) / 8 * 8;      // N padded to the MMA n-tile
    static constexpr int KS = KP / 16, NT8 = NP / 8;
    static constexpr int RS = KP + 8;                  // BF16 row stride (elements) of a staging plane
    static constexpr int YS = NP + 4;                  // FP32 row stride of the Y rows
    static constexpr size_t PLANE = 32 * RS * 2;       // bytes of one BF16 plane
    static constexpr size_t WARP_BYTES = (2 * PLANE > 32 * YS * 4 ? 2 * PLANE : 32 * YS * 4);
};

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void split2(float x, float y, uint32_t& hi, uint32_t& lo)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x - hf.x, y - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// bfrag: [KS][NT8][32 lanes] uint2 fragments of N_hi, then (if NSPLIT) of N_lo
template <int NCOL, bool NSPLIT>
__device__ __forceinline__ float colour_tc_warp(const cx<float> (&J)[NCOL], unsigned char* __restrict__ stage,
                                                const uint2* __restrict__ bfrag, int lane)
{
    using S = TcShape<NCOL>;
    uint32_t* hi = reinterpret_cast<uint32_t*>(stage);
    uint32_t* lo = reinterpret_cast<uint32_t*>(stage + S::PLANE);
    float* Y = reinterpret_cast<float*>(stage);
    const int g = lane >> 2, t = lane & 3;
    float total = 0.0f;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        // this lane's row of A for the half: Re J (half 0) or Im J (half 1)
#pragma unroll
        for (int c = 0; c < S::KP / 2; ++c) {
            const float x = 2 * c < NCOL ? (half ? J[2 * c].im : J[2 * c].re) : 0.0f;
            const float y = 2 * c + 1 < NCOL ? (half ? J[2 * c + 1].im : J[2 * c + 1].re) : 0.0f;
            uint32_t h2, l2;
            split2(x, y, h2, l2);
            hi[lane * (S::RS / 2) + c] = h2;
            lo[lane * (S::RS / 2) + c] = l2;
        }
        __syncwarp();
        float acc[2][S::NT8][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < S::NT8; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.0f;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int r0 = 16 * mt + g, r1 = r0 + 8;
#pragma unroll
            for (int ks = 0; ks < S::KS; ++ks) {
                const int c0 = (16 * ks + 2 * t) / 2, c1 = c0 + 4;
                const uint32_t ah0 = hi[r0 * (S::RS / 2) + c0], ah1 = hi[r1 * (S::RS / 2) + c0];
                const uint32_t ah2 = hi[r0 * (S::RS / 2) + c1], ah3 = hi[r1 * (S::RS / 2) + c1];
                const uint32_t al0 = lo[r0 * (S::RS / 2) + c0], al1 = lo[r1 * (S::RS / 2) + c0];
                const uint32_t al2 = lo[r0 * (S::RS / 2) + c1], al3 = lo[r1 * (S::RS / 2) + c1];
#pragma unroll
                for (int nt = 0; nt < S::NT8; ++nt) {
                    const uint2 b = __ldg(bfrag + (ks * S::NT8 + nt) * 32 + lane);
                    mma_bf16(acc[mt][nt], ah0, ah1, ah2, ah3, b.x, b.y);
                    mma_bf16(acc[mt][nt], al0, al1, al2, al3, b.x, b.y);
                    if constexpr (NSPLIT) {
                        const uint2 bl = __ldg(bfrag + (S::KS * S::NT8 + ks * S::NT8 + nt) * 32 + lane);
                        mma_bf16(acc[mt][nt], ah0, ah1, ah2, ah3, bl.x, bl.y);
                    }
                }
            }
        }
        __syncwarp();  // all fragments read: the planes become the Y rows
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < S::NT8; ++nt) {
                const int r0 = 16 * mt + g, c = 8 * nt + 2 * t;
                Y[r0 * S::YS + c] = acc[mt][nt][0];
                Y[r0 * S::YS + c + 1] = acc[mt][nt][1];
                Y[(r0 + 8) * S::YS + c] = acc[mt][nt][2];
                Y[(r0 + 8) * S::YS + c + 1] = acc[mt][nt][3];
            }
        __syncwarp();
        float s = 0.0f;
#pragma unroll
        for (int c = 0; c < NCOL; ++c) s = fmaf(half ? J[c].im : J[c].re, Y[lane * S::YS + c], s);
        total += s;
        __syncwarp();  // before the next half overwrites the staging area
    }
    return total;
}

}  // namespace me

namespace me {

// Tensor-core colour quadratic form, one warp, J read from shared memory
// through el(c, thread, half) (flow c of that thread's Re J for half 0, Im J
// for half 1; halves H0 <= half < H1).  Per warp: rows = its 32 threads' Re J
// or Im J; A fragments are built straight from shared memory (BF16 hi/lo
// split), Y = A N accumulates in FP32 over the K steps of each n-tile, and each
// fragment entry Y[row][n] is immediately multiplied by J_row[n].  Returns this
// thread's own share of J^+ N J (rows are summed within quads, then handed to
// their owners through `rowv`, one float per thread of the CTA).
template <int NCOL, bool NSPLIT, int H0, int H1, class F>
__device__ __forceinline__ float colour_tc_rows(F el, const uint2* __restrict__ bfrag, float* __restrict__ rowv,
                                                int tid)
{
    using S = TcShape<NCOL>;
    const int lane = tid & 31, wbase = tid & ~31;
    const int g = lane >> 2, t = lane & 3;
    float own = 0.0f;
#pragma unroll 1
    for (int half = H0; half < H1; ++half) {
        float rsum[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};  // [mt][row g / g+8]
#pragma unroll 1
        for (int mt = 0; mt < 2; ++mt) {
            const int l0 = wbase + 16 * mt + g, l1 = l0 + 8;  // threads owning rows g and g+8
            uint32_t ahi[S::KS][4], alo[S::KS][4];
#pragma unroll
            for (int ks = 0; ks < S::KS; ++ks) {
                const int c0 = 16 * ks + 2 * t;
                float v[8];
                const int cols[4] = {c0, c0 + 1, c0 + 8, c0 + 9};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    v[q] = cols[q] < NCOL ? el(cols[q], l0, half) : 0.0f;
                    v[4 + q] = cols[q] < NCOL ? el(cols[q], l1, half) : 0.0f;
                }
                split2(v[0], v[1], ahi[ks][0], alo[ks][0]);  // row g,   k = c0, c0+1
                split2(v[4], v[5], ahi[ks][1], alo[ks][1]);  // row g+8, k = c0, c0+1
                split2(v[2], v[3], ahi[ks][2], alo[ks][2]);  // row g,   k = c0+8, c0+9
                split2(v[6], v[7], ahi[ks][3], alo[ks][3]);  // row g+8, k = c0+8, c0+9
            }
#pragma unroll 1
            for (int nt = 0; nt < S::NT8; ++nt) {
                float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int ks = 0; ks < S::KS; ++ks) {
                    const uint2 b = __ldg(bfrag + (ks * S::NT8 + nt) * 32 + lane);
                    mma_bf16(acc, ahi[ks][0], ahi[ks][1], ahi[ks][2], ahi[ks][3], b.x, b.y);
                    mma_bf16(acc, alo[ks][0], alo[ks][1], alo[ks][2], alo[ks][3], b.x, b.y);
                    if constexpr (NSPLIT) {
                        const uint2 bl = __ldg(bfrag + (S::KS * S::NT8 + ks * S::NT8 + nt) * 32 + lane);
                        mma_bf16(acc, ahi[ks][0], ahi[ks][1], ahi[ks][2], ahi[ks][3], bl.x, bl.y);
                    }
                }
                const int n0 = 8 * nt + 2 * t;
                if (n0 < NCOL) {
                    rsum[mt][0] = fmaf(acc[0], el(n0, l0, half), rsum[mt][0]);
                    rsum[mt][1] = fmaf(acc[2], el(n0, l1, half), rsum[mt][1]);
                }
                if (n0 + 1 < NCOL) {
                    rsum[mt][0] = fmaf(acc[1], el(n0 + 1, l0, half), rsum[mt][0]);
                    rsum[mt][1] = fmaf(acc[3], el(n0 + 1, l1, half), rsum[mt][1]);
                }
            }
        }
        // row totals: sum the 4 threads of each quad, then hand each row to its owner
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                float x = rsum[mt][r];
                x += __shfl_xor_sync(0xffffffffu, x, 1);
                x += __shfl_xor_sync(0xffffffffu, x, 2);
                rsum[mt][r] = x;
            }
        if (t == 0) {
            rowv[wbase + g] = rsum[0][0];
            rowv[wbase + g + 8] = rsum[0][1];
            rowv[wbase + 16 + g] = rsum[1][0];
            rowv[wbase + 24 + g] = rsum[1][1];
        }
        __syncwarp();
        own += rowv[tid];
        __syncwarp();
    }
    return own;
}


// J held in shared memory as jsm[c * NT + thread] (FP32 complex), both halves
template <int NCOL, int NT, bool NSPLIT>
__device__ __forceinline__ float colour_tc_smem(const cx<float>* __restrict__ jsm, const uint2* __restrict__ bfrag,
                                                float* __restrict__ rowv, int tid)
{
    const float* jf = reinterpret_cast<const float*>(jsm);
    return colour_tc_rows<NCOL, NSPLIT, 0, 2>([jf](int c, int l, int half) { return jf[2 * (c * NT + l) + half]; },
                                              bfrag, rowv, tid);
}

// one half of J (Re or Im: its share of the form) held per warp as
// plane[c * 32 + lane] (FP32); rowv: 32 floats of the warp
template <int NCOL, bool NSPLIT>
__device__ __forceinline__ float colour_tc_plane(const float* __restrict__ plane, const uint2* __restrict__ bfrag,
                                                 float* __restrict__ rowv, int lane)
{
    return colour_tc_rows<NCOL, NSPLIT, 0, 1>([plane](int c, int l, int) { return plane[c * 32 + (l & 31)]; }, bfrag,
                                              rowv, lane);
}

}  // namespace me
