// Two FP32 lanes in one 64-bit register, computed with the packed FP32x2
// instructions of sm_100-class SMs (add / sub / mul / fma .rn.f32x2): one
// instruction performs the same IEEE single-precision operation for two events,
// which halves the issue slots and the instruction fetch of the FP32 chain.
//
// f2 is used as the amplitude type T of the HELAS routines (helas.cuh): the
// generic routines compile unchanged; the complex helpers below are overloads
// that avoid separate negations, which the packed instruction set lacks.
// Each lane's result is bitwise what the scalar FP32 instruction gives for the
// same operation sequence.
#pragma once
#include <cuda_runtime.h>

namespace me {

// The operators are hidden friends (found by argument-dependent lookup only),
// so they never compete with the scalar fma / operators for float and double.
struct f2 {
    unsigned long long v;
    f2() = default;
    __device__ __forceinline__ explicit f2(float x) { asm("mov.b64 %0, {%1, %1};" : "=l"(v) : "f"(x)); }
    __device__ __forceinline__ explicit f2(int x) : f2((float)x) {}
    __device__ __forceinline__ static f2 pack(float lo, float hi)
    {
        f2 r;
        asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
        return r;
    }
    __device__ __forceinline__ float lo() const
    {
        float a, b;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
        return a;
    }
    __device__ __forceinline__ float hi() const
    {
        float a, b;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
        return b;
    }

    __device__ __forceinline__ friend f2 operator+(f2 a, f2 b)
    {
        f2 r;
        asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
        return r;
    }
    __device__ __forceinline__ friend f2 operator-(f2 a, f2 b)
    {
        f2 r;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
        return r;
    }
    __device__ __forceinline__ friend f2 operator*(f2 a, f2 b)
    {
        f2 r;
        asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
        return r;
    }
    __device__ __forceinline__ friend f2 fma(f2 a, f2 b, f2 c)
    {
        f2 r;
        asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
        return r;
    }
    // sign flip of both lanes (an integer operation on the sign bits)
    __device__ __forceinline__ friend f2 operator-(f2 a)
    {
        f2 r;
        r.v = a.v ^ 0x8000000080000000ull;
        return r;
    }
    __device__ __forceinline__ friend f2& operator+=(f2& a, f2 b) { return a = a + b; }
    __device__ __forceinline__ friend f2& operator-=(f2& a, f2 b) { return a = a - b; }
};

}  // namespace me
