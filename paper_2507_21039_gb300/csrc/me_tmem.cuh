// Tensor memory (TMEM) as per-thread storage on sm_100-family GPUs.
//
// TMEM is 128 lanes x 512 columns of 32-bit cells per SM, next to the tensor
// cores and separate from shared memory.  A CTA allocates a power-of-two number
// of columns (one warp issues the allocation and, at the end, the release);
// warp w of the CTA reaches lanes 32 (w % 4) .. 32 (w % 4) + 31, and in the
// 32x32b access shape lane i of the warp reads or writes TMEM lane
// 32 (w % 4) + i.  An address is (lane << 16) | column.  Loads and stores are
// asynchronous: a load's registers are valid after tcgen05.wait::ld, and a
// thread's stores are complete (visible to its later loads) after
// tcgen05.wait::st.  Every access here is warp-collective (.sync.aligned): the
// whole warp executes it with the same address.
#pragma once
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

// Bound on each wait for the tensor cores (clock cycles, about a second):
// a wait that runs out marks the thread's events as failed (|M|^2 = NaN) and
// the kernel stops waiting instead of hanging the GPU
#ifndef ME_WAIT_LIMIT_CYCLES
#define ME_WAIT_LIMIT_CYCLES (1LL << 31)
#endif

namespace me {

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"((uint32_t)__cvta_generic_to_shared(dst)), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols) : "memory");
}

// ordering of TMEM accesses across a CTA barrier
__device__ __forceinline__ void tmem_fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// eight loads of two columns each at addr[q] (after this thread's earlier
// stores have completed); the values are valid on return
__device__ __forceinline__ void tmem_ld_8x2(const uint32_t (&addr)[8], uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.wait::st.sync.aligned;\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%16];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%2, %3}, [%17];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%4, %5}, [%18];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%6, %7}, [%19];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%8, %9}, [%20];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%10, %11}, [%21];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%12, %13}, [%22];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%14, %15}, [%23];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(addr[0]), "r"(addr[1]), "r"(addr[2]), "r"(addr[3]), "r"(addr[4]), "r"(addr[5]), "r"(addr[6]),
          "r"(addr[7])
        : "memory");
}

// sixteen consecutive columns from addr (after this thread's earlier stores)
__device__ __forceinline__ void tmem_ld_16(uint32_t addr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.wait::st.sync.aligned;\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(addr)
        : "memory");
}

__device__ __forceinline__ void tmem_st_2(uint32_t addr, uint32_t a, uint32_t b)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" :: "r"(addr), "r"(a), "r"(b) : "memory");
}

// sixteen consecutive columns from addr set to zero
__device__ __forceinline__ void tmem_zero_16(uint32_t addr)
{
    const uint32_t z = 0u;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1};"
        :: "r"(addr), "r"(z) : "memory");
}

// ---------------------------------------------------------------------------
// tcgen05.mma with operands in shared memory and the accumulator in TMEM.
//
// Operand layout (both A [M x K] and B [N x K], K-major, no swizzle): the
// matrix is cut into core matrices of 8 rows x 16 bytes (8 BF16 along K),
// each stored as 128 contiguous bytes (row r at byte 16 r).  Core matrix
// (row group i, K group j) starts at i * SBO + j * LBO.  Here LBO = 128 and
// SBO = 256 for a K = 16 operand: the two K groups of a row group are adjacent,
// row groups follow each other.  Element (row, k) of a K = 16 operand is at
// byte (row / 8) * 256 + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr uint32_t umma_k16_offset(int row, int k)
{
    return (uint32_t)((row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// M-major (MN-major) K = 16 operand for an M = 128 A written one element per
// thread and column: the 8 consecutive rows of a K row form 16 contiguous bytes,
// the 8 K rows of a core matrix follow at 16-byte pitch (128 bytes), the two K
// groups at LBO = 128 and the 16 row groups at SBO = 272.  The 16 bytes of
// padding per row group put the four row groups a warp writes for one column on
// different banks (with SBO = 256 they would share the same four).  Element
// (row, k) is at byte (row / 8) * 272 + (k / 8) * 128 + (k % 8) * 16 + (row % 8) * 2,
// inside 16 * 272 = 4352 bytes; read with strides 128 and 272 in either role
// every access stays inside them.
constexpr uint32_t kUmmaMn16Sbo = 272, kUmmaMn16Bytes = 16 * kUmmaMn16Sbo;
__host__ __device__ constexpr uint32_t umma_mn16_offset(int row, int k)
{
    return (uint32_t)((row >> 3) * kUmmaMn16Sbo + (k >> 3) * 128 + (k & 7) * 16 + (row & 7) * 2);
}
static_assert(umma_mn16_offset(1, 0) == 2 && umma_mn16_offset(0, 1) == 16 && umma_mn16_offset(0, 8) == 128 &&
                  umma_mn16_offset(8, 0) == 272 && umma_mn16_offset(127, 15) + 2 <= kUmmaMn16Bytes,
              "M-major operand layout");
static_assert(15 * 128 + 272 + 128 <= kUmmaMn16Bytes, "strides read in swapped roles stay inside the operand");

// shared-memory matrix descriptor: start address, leading-dimension (K)
// byte offset, stride-dimension (M/N) byte offset, each in 16-byte units;
// bit 46 set (descriptor version of the sm_100 family); no swizzle, base offset 0
__device__ __forceinline__ uint64_t umma_smem_desc(const void* smem_ptr, uint32_t lbo, uint32_t sbo)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem_ptr);
    return (uint64_t)((a >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9, 10-12 = 1), B optionally negated (bit 14), A K-major or
// M-major (bit 15 = 0 / 1), B K-major (bit 16 = 0), N / 8 at bits 17-22,
// M / 16 at bits 24-28
__host__ __device__ constexpr uint32_t umma_idesc_bf16_f32(int m, int n, bool neg_b, bool a_m_major = false)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (neg_b ? (1u << 14) : 0u) | (a_m_major ? (1u << 15) : 0u) |
           ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// D[tmem] (+)= A * B for one M x N x 16 step, issued by a single thread;
// accumulate = false overwrites D
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          bool accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

// the mbarrier at `bar` receives one arrival once every tcgen05.mma this
// thread issued before has completed
__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"((uint32_t)__cvta_generic_to_shared(bar)) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"((uint32_t)__cvta_generic_to_shared(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// generic-proxy shared-memory writes of this thread become visible to the
// async proxy (the tensor cores reading operands)
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16-byte copy global -> shared that completes in the background
// (cp.async; both addresses 16-byte aligned), and the wait for this thread's copies
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                 :: "r"((uint32_t)__cvta_generic_to_shared(smem_dst)), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"((uint32_t)__cvta_generic_to_shared(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Wait for the completion of the phase with the given parity, for at most
// `limit` clock cycles.  Returns false if the limit passed first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// Resident CTAs per SM of a kernel that allocates `tmem_cols` TMEM columns
// per CTA.  The occupancy query counts one CTA per SM for such a kernel; the
// SM takes another CTA once the resident one has given up its allocation
// permit (our kernels do right after allocating), so the residency is what
// shared memory, registers and the 512 TMEM columns allow.  (1 on failure.)
template <class K> int tmem_kernel_ctas_per_sm(K kernel, size_t dyn_smem, int threads, int tmem_cols)
{
    int dev = 0, smem_sm = 0, reserved = 0;
    cudaFuncAttributes fa{};
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, kernel) != cudaSuccess || fa.numRegs <= 0) {
        cudaGetLastError();
        return 1;
    }
    const int by_smem = (int)((size_t)smem_sm / (dyn_smem + fa.sharedSizeBytes + (size_t)reserved));
    const int regs = (fa.numRegs + 7) / 8 * 8;
    const int by_regs = 65536 / (regs * threads);
    return std::max(1, std::min({by_smem, by_regs, 2048 / threads, 512 / tmem_cols}));
}

}  // namespace me
