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

// Radix-4 Stockham passes (radix-2 for the last when log2 N is odd): the same
// transform as fft_rows in half the passes and barriers.  A pass of span ns
// reads a[j + q N/4] (q = 0..3), twiddles them by w^(q k N / (4 ns)) with
// k = j mod ns, takes the 4-point DFT and writes b[4 (j - k) + k + p ns].
template <int LOGN>
__device__ __forceinline__ float2 *fft_rows_r4(float2 *a, float2 *b, const float2 *tw, int R, bool inverse) {
    constexpr int N = 1 << LOGN, Q = N >> 2, HALF = N >> 1;
    // w^m for 0 <= m < N from the table of m < N/2 (w^(m + N/2) = -w^m)
    auto wpow = [&](int m) -> float2 {
        float2 w = tw[m & (HALF - 1)];
        if (m & HALF) w = make_float2(-w.x, -w.y);
        if (inverse) w.y = -w.y;
        return w;
    };
    int ns = 1;
#pragma unroll
    for (int st = 0; st < LOGN / 2; ++st, ns <<= 2) {
        const int tshift = LOGN - 2 - 2 * st;  // N / (4 ns) = 2^tshift
        for (int idx = threadIdx.x; idx < R * Q; idx += blockDim.x) {
            const int r = idx >> (LOGN - 2), j = idx & (Q - 1);
            const int k = j & (ns - 1);
            const float2 *ar = a + r * N;
            const float2 v0 = ar[j];
            const float2 v1 = cmul(ar[j + Q], wpow((k << tshift)));
            const float2 v2 = cmul(ar[j + 2 * Q], wpow((2 * k) << tshift));
            const float2 v3 = cmul(ar[j + 3 * Q], wpow((3 * k) << tshift));
            const float2 s02 = make_float2(v0.x + v2.x, v0.y + v2.y), d02 = make_float2(v0.x - v2.x, v0.y - v2.y);
            const float2 s13 = make_float2(v1.x + v3.x, v1.y + v3.y), d13 = make_float2(v1.x - v3.x, v1.y - v3.y);
            // forward: y1 = d02 - i d13, y3 = d02 + i d13 (inverse: signs of i swapped)
            const float2 id13 = inverse ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);
            float2 *br = b + r * N + 4 * (j - k) + k;
            br[0] = make_float2(s02.x + s13.x, s02.y + s13.y);
            br[ns] = make_float2(d02.x + id13.x, d02.y + id13.y);
            br[2 * ns] = make_float2(s02.x - s13.x, s02.y - s13.y);
            br[3 * ns] = make_float2(d02.x - id13.x, d02.y - id13.y);
        }
        __syncthreads();
        float2 *t = a;
        a = b;
        b = t;
    }
    if (LOGN & 1) {  // last pass radix 2, span N / 2
        for (int idx = threadIdx.x; idx < R * HALF; idx += blockDim.x) {
            const int r = idx >> (LOGN - 1), j = idx & (HALF - 1);
            const float2 v0 = a[r * N + j];
            float2 w = tw[j];
            if (inverse) w.y = -w.y;
            const float2 v1 = cmul(a[r * N + j + HALF], w);
            b[r * N + j] = make_float2(v0.x + v1.x, v0.y + v1.y);
            b[r * N + j + HALF] = make_float2(v0.x - v1.x, v0.y - v1.y);
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
        case 32: return fft_rows_r4<5>(a, b, tw, R, inverse);
        case 64: return fft_rows_r4<6>(a, b, tw, R, inverse);
        case 128: return fft_rows_r4<7>(a, b, tw, R, inverse);
        case 256: return fft_rows_r4<8>(a, b, tw, R, inverse);
        case 512: return fft_rows_r4<9>(a, b, tw, R, inverse);
        default: return fft_rows(a, b, tw, N, R, inverse);
    }
}

}  // namespace fftsm
}  // namespace p2s
