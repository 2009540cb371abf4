// Host-side 16-bit operand encoding shared by the tensor-core weight and basis images:
// FP16 (fmt 0) or BF16 (fmt 1), round to nearest even.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace p2s {

__host__ inline uint16_t to_half_bits(double v, int fmt) {
    if (fmt == 1) {
        const __nv_bfloat16_raw r = __float2bfloat16_rn((float)v);
        return r.x;
    }
    const __half_raw r = __float2half_rn((float)v);
    return r.x;
}

__host__ inline double from_half_bits(uint16_t u, int fmt) {
    if (fmt == 1) {
        __nv_bfloat16_raw r;
        r.x = u;
        return (double)__bfloat162float(__nv_bfloat16(r));
    }
    __half_raw r;
    r.x = u;
    return (double)__half2float(__half(r));
}

}  // namespace p2s
