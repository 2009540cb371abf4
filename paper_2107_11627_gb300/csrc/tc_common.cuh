// Helpers shared by the tcgen05 kernels: bounded mbarrier waits with a CTA
// abort flag, and packing of two FP32 values into a 16-bit operand pair.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "tc_ptx.cuh"

namespace p2s {
namespace tcc {

// Two FP32 values -> one 32-bit word of FP16 (fmt 0) or BF16 (fmt 1), RNE.
__device__ __forceinline__ uint32_t pack2(float a, float b, int fmt) {
    if (fmt == 1) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// (a0 + b0, a1 + b1) as one packed FP32 pair add (each sum rounded as a plain add)
__device__ __forceinline__ void add2(float a0, float a1, float b0, float b1, float &s0, float &s1) {
    asm("{\n.reg .b64 p, q, r;\nmov.b64 p, {%2, %3};\nmov.b64 q, {%4, %5};\nadd.rn.f32x2 r, p, q;\n"
        "mov.b64 {%0, %1}, r;\n}\n"
        : "=f"(s0), "=f"(s1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// (c0, c1) += (a, a) * (b0, b1) as one packed FP32 pair FMA (each lane rounded as fmaf)
__device__ __forceinline__ void fma2_bcast(float a, float b0, float b1, float &c0, float &c1) {
    asm("{\n.reg .b64 p, q, r;\nmov.b64 p, {%2, %2};\nmov.b64 q, {%3, %4};\nmov.b64 r, {%0, %1};\n"
        "fma.rn.f32x2 r, p, q, r;\nmov.b64 {%0, %1}, r;\n}\n"
        : "+f"(c0), "+f"(c1)
        : "f"(a), "f"(b0), "f"(b1));
}

// max(a, 0), max(b, 0) -> one 32-bit word, in one conversion instruction (the
// value max(x, 0) rounded as pack2 rounds it)
__device__ __forceinline__ uint32_t pack2_relu(float a, float b, int fmt) {
    uint32_t r;
    if (fmt == 1)
        asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
    else
        asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
    return r;
}

// g0, g1 rounded to FP16 into one word: g0 in the low half, g1 in the high
__device__ __forceinline__ uint32_t pack_f16x2(float g0, float g1) {
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(g1), "f"(g0));
    return r;
}

// c0 += lo(x) * g, c1 += hi(x) * g with FP16 operands (x a word of two FP16
// values, g the low or high half of `gw`) and FP32 accumulation.  The product
// of two FP16 values is exact in FP32, so each is rounded once, exactly like an
// fmaf of the widened operands.
template <bool GHI>
__device__ __forceinline__ void fma_mix_x2(uint32_t x, uint32_t gw, float &c0, float &c1) {
    if (GHI)
        asm("{\n.reg .b16 xl, xh, gl, gh;\nmov.b32 {xl, xh}, %2;\nmov.b32 {gl, gh}, %3;\n"
            "fma.rn.f32.f16 %0, xl, gh, %0;\nfma.rn.f32.f16 %1, xh, gh, %1;\n}\n"
            : "+f"(c0), "+f"(c1) : "r"(x), "r"(gw));
    else
        asm("{\n.reg .b16 xl, xh, gl, gh;\nmov.b32 {xl, xh}, %2;\nmov.b32 {gl, gh}, %3;\n"
            "fma.rn.f32.f16 %0, xl, gl, %0;\nfma.rn.f32.f16 %1, xh, gl, %1;\n}\n"
            : "+f"(c0), "+f"(c1) : "r"(x), "r"(gw));
}

// c += lo(x) * g, as fma_mix_x2 for one value
template <bool GHI>
__device__ __forceinline__ void fma_mix_x1(uint32_t x, uint32_t gw, float &c) {
    if (GHI)
        asm("{\n.reg .b16 xl, xh, gl, gh;\nmov.b32 {xl, xh}, %1;\nmov.b32 {gl, gh}, %2;\n"
            "fma.rn.f32.f16 %0, xl, gh, %0;\n}\n"
            : "+f"(c) : "r"(x), "r"(gw));
    else
        asm("{\n.reg .b16 xl, xh, gl, gh;\nmov.b32 {xl, xh}, %1;\nmov.b32 {gl, gh}, %2;\n"
            "fma.rn.f32.f16 %0, xl, gl, %0;\n}\n"
            : "+f"(c) : "r"(x), "r"(gw));
}

// a += g * (x, x) as one packed FP16 FMA, x the low (XHI false) or high half of the
// word `x`: both halves of `a` accumulate in FP16, each rounded once per FMA.
template <bool XHI>
__device__ __forceinline__ void hfma2_bcast(uint32_t &a, uint32_t g, uint32_t x) {
    if (XHI)
        asm("{\n.reg .b16 xl, xh;\n.reg .b32 xb;\nmov.b32 {xl, xh}, %2;\nmov.b32 xb, {xh, xh};\n"
            "fma.rn.f16x2 %0, %1, xb, %0;\n}\n"
            : "+r"(a) : "r"(g), "r"(x));
    else
        asm("{\n.reg .b16 xl, xh;\n.reg .b32 xb;\nmov.b32 {xl, xh}, %2;\nmov.b32 xb, {xl, xl};\n"
            "fma.rn.f16x2 %0, %1, xb, %0;\n}\n"
            : "+r"(a) : "r"(g), "r"(x));
}

// c0 += lo(a), c1 += hi(a): an FP16 pair added into two FP32 sums (each an exact
// product by 1.0 and one FP32 rounding, i.e. a plain FP32 add)
__device__ __forceinline__ void flush_f16x2(uint32_t a, float &c0, float &c1) {
    asm("{\n.reg .b16 al, ah, one;\nmov.b32 {al, ah}, %2;\nmov.b16 one, 0x3C00;\n"
        "fma.rn.f32.f16 %0, al, one, %0;\nfma.rn.f32.f16 %1, ah, one, %1;\n}\n"
        : "+f"(c0), "+f"(c1) : "r"(a));
}

// v0, v1 (FP32) as E4M3 hi/lo pairs: hi = e4m3(v), lo = e4m3(v - hi) (the difference is
// exact in FP32), both rounded to nearest even and saturated at +-448.  Each result is
// two bytes: v0's in the low byte, v1's in the high byte.
__device__ __forceinline__ void e4m3_hi_lo(float v0, float v1, uint16_t &hi, uint16_t &lo) {
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %2, %1;" : "=h"(hi) : "f"(v0), "f"(v1));
    uint32_t h2;
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"(hi));
    const float2 hv = __half22float2(*reinterpret_cast<const __half2 *>(&h2));
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %2, %1;" : "=h"(lo) : "f"(v0 - hv.x), "f"(v1 - hv.y));
}

struct Ctl {
    volatile int *abort;
    int *status;
};

// Bounded wait (about 2 s at 2 GHz); on timeout flags the CTA and the status
// word.  Once the CTA is flagged every wait returns false at once, so all
// roles run their (data-independent) loops to the end and meet at teardown.
// Each try may suspend the thread for up to 20 us (it resumes when the phase
// completes), so a waiting thread takes no issue slots from working warps.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, const Ctl &ctl, int code,
                                         long long limit = 4000000000ll) {
    if (ptx::mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (ptx::mbar_try_hint(bar, parity, 20000u)) return true;
        if (*ctl.abort) return false;
        if (clock64() - t0 > limit) {
            *ctl.abort = 1;
            atomicOr(ctl.status, code);
            return false;
        }
    }
}

// Bounded wait that ignores the abort flag: lets issued copies and MMAs land
// before the CTA's shared and tensor memory are released.
__device__ __forceinline__ void drain_bar(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!ptx::mbar_try(bar, parity) && clock64() - t0 < 4000000000ll) {
    }
}

}  // namespace tcc
}  // namespace p2s
