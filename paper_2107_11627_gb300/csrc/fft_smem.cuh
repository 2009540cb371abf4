// Radix-2 Stockham FFT of a batch of rows held in shared memory (used by the
// field filters and by the FFT blur variant).
#pragma once

#include <cuda_runtime.h>

namespace p2s {
namespace fftsm {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// R rows of length N (power of two) in `a`, ping-ponging with `b`; natural
// order in and out, unnormalised.  All threads of the block take part.
// Returns the buffer that holds the result.  tw[m] = exp(-2 pi i m / N).
__device__ __forceinline__ float2 *fft_rows(float2 *a, float2 *b, const float2 *tw, int N, int R, bool inverse) {
    const int half = N >> 1;
    for (int ns = 1; ns < N; ns <<= 1) {
        const int tstep = N / (2 * ns);
        for (int idx = threadIdx.x; idx < R * half; idx += blockDim.x) {
            const int r = idx / half, j = idx - r * half;
            const int k = j & (ns - 1);
            const float2 v0 = a[r * N + j];
            float2 w = tw[k * tstep];
            if (inverse) w.y = -w.y;
            const float2 v1 = cmul(a[r * N + j + half], w);
            const int d = ((j - k) << 1) + k;
            b[r * N + d] = make_float2(v0.x + v1.x, v0.y + v1.y);
            b[r * N + d + ns] = make_float2(v0.x - v1.x, v0.y - v1.y);
        }
        __syncthreads();
        float2 *t = a;
        a = b;
        b = t;
    }
    return a;
}

// The same transform with N = 2^LOGN known at compile time: index arithmetic
// by shifts and masks, stages unrolled.  Same butterflies in the same order.
template <int LOGN>
__device__ __forceinline__ float2 *fft_rows_t(float2 *a, float2 *b, const float2 *tw, int R, bool inverse) {
    constexpr int N = 1 << LOGN, HALF = N >> 1;
#pragma unroll
    for (int s = 0; s < LOGN; ++s) {
        const int ns = 1 << s;
        const int tshift = LOGN - 1 - s;  // twiddle stride N / (2 ns)
        for (int idx = threadIdx.x; idx < R * HALF; idx += blockDim.x) {
            const int r = idx >> (LOGN - 1), j = idx & (HALF - 1);
            const int k = j & (ns - 1);
            const float2 v0 = a[r * N + j];
            float2 w = tw[k << tshift];
            if (inverse) w.y = -w.y;
            const float2 v1 = cmul(a[r * N + j + HALF], w);
            const int d = ((j - k) << 1) + k;
            b[r * N + d] = make_float2(v0.x + v1.x, v0.y + v1.y);
            b[r * N + d + ns] = make_float2(v0.x - v1.x, v0.y - v1.y);
        }
        __syncthreads();
        float2 *t = a;
        a = b;
        b = t;
    }
    return a;
}

// fft_rows with a compile-time length for the common sizes.
__device__ __forceinline__ float2 *fft_rows_any(float2 *a, float2 *b, const float2 *tw, int N, int R, bool inverse) {
    switch (N) {
        case 32: return fft_rows_t<5>(a, b, tw, R, inverse);
        case 64: return fft_rows_t<6>(a, b, tw, R, inverse);
        case 128: return fft_rows_t<7>(a, b, tw, R, inverse);
        case 256: return fft_rows_t<8>(a, b, tw, R, inverse);
        case 512: return fft_rows_t<9>(a, b, tw, R, inverse);
        default: return fft_rows(a, b, tw, N, R, inverse);
    }
}

}  // namespace fftsm
}  // namespace p2s
