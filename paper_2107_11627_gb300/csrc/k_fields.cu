// Anchor-grid Zernike fields (Sec. 3.4): counter-based white noise, Fourier
// filtering on the torus, inter-mode colouring by chol(R_Z) (Sec. 2.2).
//
// The filter sqrt(C) of the wrapped Gaussian covariance is separable, so the
// 2-D filtering is a batch of 1-D circular filters along rows, then along
// columns.  Each 1-D filter is FFT -> real gain -> inverse FFT in shared
// memory, with two real rows packed into one complex sequence (the gain is
// real and even, so the two results come back in the real and imaginary
// parts).  Only the A_w columns of the row pass and the A_h rows of the
// column pass that the anchors use are kept.
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "fft_smem.cuh"
#include "p2s_internal.h"

namespace p2s {

namespace {

constexpr int kThreads = 256;
constexpr int kFftElems = 2048;  // complex elements per ping-pong buffer (32 KB per CTA: several CTAs per SM)

struct U4 {
    uint32_t x, y, z, w;
};

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the two 32x32->64-bit
// multiplies, key bumped by the Weyl constants after every round.
__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// -2 ln u for u = (w + 1/2) 2^-32, accurate near u = 1 through log1p of 1 - u.
__device__ __forceinline__ float neg2log_u(uint32_t w) {
    const float two_m32 = 2.3283064365386963e-10f;
    if (w < 0x80000000u) return -2.0f * logf(((float)w + 0.5f) * two_m32);
    const float v = ((float)(0xFFFFFFFFu - w) + 0.5f) * two_m32;
    return -2.0f * log1pf(-v);
}

// Box-Muller pair from two words: r = sqrt(-2 ln u_a), angle 2 pi u_b.  The
// quadrant comes exactly from the top two bits of w_b, the rest through sincospi.
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float *z0, float *z1) {
    const float r = sqrtf(neg2log_u(wa));
    const float x = ((float)(wb & 0x3FFFFFFFu) + 0.5f) * 4.656612873077393e-10f;  // (0, 1/2)
    float sn, cs;
    sincospif(x, &sn, &cs);
    float c, s;
    switch (wb >> 30) {
        case 0: c = cs; s = sn; break;
        case 1: c = -sn; s = cs; break;
        case 2: c = -cs; s = -sn; break;
        default: c = sn; s = -cs; break;
    }
    *z0 = r * c;
    *z1 = r * s;
}

// Four normals of quad q of stream (seed, mode).
__device__ __forceinline__ void normals4(unsigned long long seed, int mode, uint32_t q, float z[4]) {
    U4 w = philox4x32_10(U4{q, (uint32_t)mode, 0u, 0u}, (uint32_t)seed, (uint32_t)(seed >> 32));
    box_muller(w.x, w.y, &z[0], &z[1]);
    box_muller(w.z, w.w, &z[2], &z[3]);
}

__global__ void noise_kernel(unsigned long long seed, int mode, long long n, float *out) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (4 * q >= n) return;
    float z[4];
    normals4(seed, mode, (uint32_t)q, z);
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (4 * q + i < n) out[4 * q + i] = z[i];
}

using fftsm::cmul;
using fftsm::fft_rows_any;

// Row pass: white noise rows (y0, y0+1) packed as one complex row, filtered
// along x; columns [0, Aw) of both rows go to t[frame][mode][y][x].
__global__ void __launch_bounds__(kThreads) row_filter_kernel(FrameBatch fb, int Fh, int Fw, int Aw, int rows_per_cta,
                                                              const float2 *__restrict__ tw,
                                                              const float *__restrict__ gain,
                                                              const int *__restrict__ kernel_of_mode, float *t) {
    extern __shared__ float2 smem[];
    const int mode = blockIdx.y, frame = blockIdx.z;
    const int R = rows_per_cta;  // complex rows = row pairs
    float2 *buf0 = smem, *buf1 = smem + R * Fw, *stw = smem + 2 * R * Fw;
    float *sg = (float *)(stw + (Fw / 2 > 0 ? Fw / 2 : 1));
    const float *g = gain + (size_t)kernel_of_mode[mode] * Fw;
    for (int i = threadIdx.x; i < Fw / 2; i += blockDim.x) stw[i] = tw[i];
    for (int i = threadIdx.x; i < Fw; i += blockDim.x) sg[i] = g[i];
    const int y_base = blockIdx.x * R * 2;  // first torus row of this CTA
    const int n_rows = min(2 * R, Fh - y_base);
    const unsigned long long seed = fb.seed[frame];
    const int lgF = __ffs(Fw) - 1;
    // noise: samples [y_base*Fw, (y_base+n_rows)*Fw) of stream (seed, mode), quad by quad
    const int q0 = (y_base * Fw) >> 2, q1 = ((y_base + n_rows) * Fw + 3) >> 2;
    for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        float z[4];
        normals4(seed, mode, (uint32_t)q, z);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int s = 4 * q + i - y_base * Fw;
            if (s < 0 || s >= n_rows * Fw) continue;
            const int row = s >> lgF, x = s & (Fw - 1);  // Fw is a power of two
            float *dst = (float *)&buf0[(row >> 1) * Fw + x];
            dst[row & 1] = z[i];
        }
    }
    if (n_rows & 1)  // odd tail (Fh is a power of two, so only when Fh == 1)
        for (int x = threadIdx.x; x < Fw; x += blockDim.x) buf0[(n_rows >> 1) * Fw + x].y = 0.0f;
    __syncthreads();
    const int Rk = (n_rows + 1) >> 1;
    float2 *res = fft_rows_any(buf0, buf1, stw, Fw, Rk, false);
    for (int i = threadIdx.x; i < Rk * Fw; i += blockDim.x) {
        const float gg = sg[i & (Fw - 1)];
        res[i].x *= gg;
        res[i].y *= gg;
    }
    __syncthreads();
    float2 *other = res == buf0 ? buf1 : buf0;
    res = fft_rows_any(res, other, stw, Fw, Rk, true);
    float *tf = t + ((size_t)frame * kModes + mode) * Fh * Aw;
    for (int i = threadIdx.x; i < n_rows * Aw; i += blockDim.x) {
        const int row = i / Aw, x = i - row * Aw;
        const float2 v = res[(row >> 1) * Fw + x];
        tf[(size_t)(y_base + row) * Aw + x] = (row & 1) ? v.y : v.x;
    }
}

// Column pass: columns (x0, x0+1) of t packed as one complex column, filtered
// along y; rows [0, Ah) go to f[frame][mode][y][x].
__global__ void __launch_bounds__(kThreads) col_filter_kernel(int Fh, int Ah, int Aw, int cols_per_cta,
                                                              const float2 *__restrict__ tw,
                                                              const float *__restrict__ gain,
                                                              const int *__restrict__ kernel_of_mode,
                                                              const float *__restrict__ t, float *f) {
    extern __shared__ float2 smem[];
    const int mode = blockIdx.y, frame = blockIdx.z;
    const int R = cols_per_cta;
    float2 *buf0 = smem, *buf1 = smem + R * Fh, *stw = smem + 2 * R * Fh;
    float *sg = (float *)(stw + (Fh / 2 > 0 ? Fh / 2 : 1));
    const float *g = gain + (size_t)kernel_of_mode[mode] * Fh;
    for (int i = threadIdx.x; i < Fh / 2; i += blockDim.x) stw[i] = tw[i];
    for (int i = threadIdx.x; i < Fh; i += blockDim.x) sg[i] = g[i];
    const int x_base = blockIdx.x * R * 2;
    const int n_cols = min(2 * R, Aw - x_base);
    const int Rk = (n_cols + 1) >> 1;
    const float *tf = t + ((size_t)frame * kModes + mode) * Fh * Aw;
    const int lgF = __ffs(Fh) - 1;
    for (int i = threadIdx.x; i < Rk * Fh; i += blockDim.x) {
        const int c = i >> lgF, y = i & (Fh - 1);
        const int x = x_base + 2 * c;
        const float re = tf[(size_t)y * Aw + x];
        const float im = (2 * c + 1 < n_cols) ? tf[(size_t)y * Aw + x + 1] : 0.0f;
        buf0[c * Fh + y] = make_float2(re, im);
    }
    __syncthreads();
    float2 *res = fft_rows_any(buf0, buf1, stw, Fh, Rk, false);
    for (int i = threadIdx.x; i < Rk * Fh; i += blockDim.x) {
        const float gg = sg[i & (Fh - 1)];  // Fh is a power of two
        res[i].x *= gg;
        res[i].y *= gg;
    }
    __syncthreads();
    float2 *other = res == buf0 ? buf1 : buf0;
    res = fft_rows_any(res, other, stw, Fh, Rk, true);
    float *ff = f + ((size_t)frame * kModes + mode) * Ah * Aw;
    for (int i = threadIdx.x; i < n_cols * Ah; i += blockDim.x) {
        const int cc = i / Ah, y = i - cc * Ah;
        const float2 v = res[(cc >> 1) * Fh + y];
        ff[(size_t)y * Aw + x_base + cc] = (cc & 1) ? v.y : v.x;
    }
}

// ---- one kernel per field: both filter passes with warp-register FFTs ----------
//
// A warp transforms one complex sequence of N = 32 P points, lane l holding
// elements l + 32 i (i < P): a P-point DFT in the thread, the twiddle
// w_N^(l k1), then a 32-point DFT across the lanes by five radix-2 shuffle
// stages (decimation in frequency), which leaves X[k1 + P bitrev5(l)] in lane l,
// register k1.  The gain is real, so the spectrum is multiplied in that order
// and the inverse runs the same steps backwards (decimation in time from
// bit-reversed input), ending in natural order: no reordering pass at all.
// tw[m] = exp(-2 pi i m / N) for m < N / 2 (shared memory), w^(m + N/2) = -w^m.

__device__ __forceinline__ float2 tw_at(const float2 *tw, int m, int N, bool inverse) {
    float2 w = tw[m & (N / 2 - 1)];
    if (m & (N / 2)) w = make_float2(-w.x, -w.y);
    if (inverse) w.y = -w.y;
    return w;
}

// v[i] <- sum_k v[k] w_P^(i k) (w_P = exp(-+2 pi i / P)), P >= 2 a power of two, by an
// iterative radix-2 decimation in time on the bit-reversed order; N is the table's length.
template <int P>
__device__ __forceinline__ void dft_in_thread_pow2(float2 (&v)[P], const float2 *tw, int N, bool inverse) {
    float2 a[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
        int r = 0;
#pragma unroll
        for (int b = 1; b < P; b <<= 1) r = (r << 1) | ((i / b) & 1);
        a[r] = v[i];
    }
#pragma unroll
    for (int len = 2; len <= P; len <<= 1)
#pragma unroll
        for (int i0 = 0; i0 < P; i0 += len)
#pragma unroll
            for (int j = 0; j < len / 2; ++j) {
                const float2 w = tw_at(tw, j * (N / len), N, inverse);
                const float2 x0 = a[i0 + j], x1 = cmul(a[i0 + j + len / 2], w);
                a[i0 + j] = make_float2(x0.x + x1.x, x0.y + x1.y);
                a[i0 + j + len / 2] = make_float2(x0.x - x1.x, x0.y - x1.y);
            }
#pragma unroll
    for (int i = 0; i < P; ++i) v[i] = a[i];
}

// the same for any power of two P (P = 1: nothing to do)
template <int P>
__device__ __forceinline__ void dft_in_thread(float2 (&v)[P], const float2 *tw, int N, bool inverse) {
    if constexpr (P > 1) dft_in_thread_pow2<P>(v, tw, N, inverse);
}

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

template <int P>
__device__ __forceinline__ void warp_fft_fwd(float2 (&v)[P], const float2 *tw, int lane) {
    constexpr int N = 32 * P;
    dft_in_thread<P>(v, tw, N, false);
#pragma unroll
    for (int k1 = 1; k1 < P; ++k1) v[k1] = cmul(v[k1], tw_at(tw, lane * k1, N, false));
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        const bool hi = lane & h;
        const float2 w = tw_at(tw, (lane & (h - 1)) * (N / (2 * h)), N, false);
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) {
            const float2 o = shfl_xor2(v[k1], h);
            v[k1] = hi ? cmul(make_float2(o.x - v[k1].x, o.y - v[k1].y), w)
                       : make_float2(v[k1].x + o.x, v[k1].y + o.y);
        }
    }
}

template <int P>
__device__ __forceinline__ void warp_fft_inv(float2 (&v)[P], const float2 *tw, int lane) {
    constexpr int N = 32 * P;
#pragma unroll
    for (int h = 1; h <= 16; h <<= 1) {
        const bool hi = lane & h;
        const float2 w = tw_at(tw, (lane & (h - 1)) * (N / (2 * h)), N, true);
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) {
            const float2 o = shfl_xor2(v[k1], h);
            if (hi) {
                const float2 t = cmul(v[k1], w);
                v[k1] = make_float2(o.x - t.x, o.y - t.y);
            } else {
                const float2 t = cmul(o, w);
                v[k1] = make_float2(v[k1].x + t.x, v[k1].y + t.y);
            }
        }
    }
#pragma unroll
    for (int k1 = 1; k1 < P; ++k1) v[k1] = cmul(v[k1], tw_at(tw, lane * k1, N, true));
    dft_in_thread<P>(v, tw, N, true);
}

__device__ __forceinline__ int bitrev5(int l) { return (int)(__brev((unsigned)l) >> 27); }

constexpr int kFieldWarps = 8;

// Row pass (white noise rows (2 r, 2 r + 1) packed as one complex row, filtered along x,
// columns [0, Aw) kept in shared memory), then column pass (columns (2 c, 2 c + 1) of that
// block filtered along y, rows [0, Ah) to f[frame][mode][y][x]).  One CTA per (mode, frame);
// the same arithmetic as row_filter_kernel and col_filter_kernel.
// Frames of one launch may differ in their anchor grids (one torus for all): each has its
// own Ah x Aw and output block, and `pitch` is odd and at least every frame's Aw.
template <int PW, int PH>
__global__ void __launch_bounds__(32 * kFieldWarps, (PW <= 4 && PH <= 4) ? 4 : 1) field_kernel(FrameBatch fb, FieldFrames geo, int pitch,
                                                                  const float2 *__restrict__ twx,
                                                                  const float *__restrict__ gainx,
                                                                  const float2 *__restrict__ twy,
                                                                  const float *__restrict__ gainy,
                                                                  const int *__restrict__ kernel_of_mode) {
    constexpr int Fw = 32 * PW, Fh = 32 * PH;
    extern __shared__ float sfm[];
    float *tb = sfm;                                   // [Fh][pitch]: the row pass's columns < Aw
    float *stage = tb + Fh * pitch;                    // [warps][2 Fw]: a row pair of white noise
    float *gx = stage + kFieldWarps * 2 * Fw, *gy = gx + Fw;
    float2 *tx = (float2 *)(gy + Fh), *ty = tx + Fw / 2;
    const int mode = blockIdx.x, frame = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Ah = geo.ah[frame], Aw = geo.aw[frame];
    const int kk = kernel_of_mode[mode];
    for (int i = threadIdx.x; i < Fw; i += blockDim.x) gx[i] = gainx[(size_t)kk * Fw + i];
    for (int i = threadIdx.x; i < Fh; i += blockDim.x) gy[i] = gainy[(size_t)kk * Fh + i];
    for (int i = threadIdx.x; i < Fw / 2; i += blockDim.x) tx[i] = twx[i];
    for (int i = threadIdx.x; i < Fh / 2; i += blockDim.x) ty[i] = twy[i];
    __syncthreads();
    const unsigned long long seed = fb.seed[frame];
    float *st = stage + warp * 2 * Fw;
    for (int rp = warp; rp < Fh / 2; rp += kFieldWarps) {
        // noise: samples [2 rp Fw, (2 rp + 2) Fw) of stream (seed, mode), quad by quad
        const uint32_t q0 = (uint32_t)(2 * rp * Fw) >> 2;
        for (int qq = lane; qq < Fw / 2; qq += 32) {
            float z[4];
            normals4(seed, mode, q0 + qq, z);
#pragma unroll
            for (int i = 0; i < 4; ++i) st[4 * qq + i] = z[i];
        }
        __syncwarp();
        float2 v[PW];
#pragma unroll
        for (int i = 0; i < PW; ++i) v[i] = make_float2(st[lane + 32 * i], st[Fw + lane + 32 * i]);
        __syncwarp();
        warp_fft_fwd<PW>(v, tx, lane);
        const int kb = PW * bitrev5(lane);
#pragma unroll
        for (int k1 = 0; k1 < PW; ++k1) {
            const float g = gx[k1 + kb];
            v[k1] = make_float2(v[k1].x * g, v[k1].y * g);
        }
        warp_fft_inv<PW>(v, tx, lane);
#pragma unroll
        for (int i = 0; i < PW; ++i) {
            const int x = lane + 32 * i;
            if (x < Aw) {
                tb[(2 * rp) * pitch + x] = v[i].x;
                tb[(2 * rp + 1) * pitch + x] = v[i].y;
            }
        }
    }
    __syncthreads();
    float *ff = geo.f[frame] + (size_t)mode * Ah * Aw;
    for (int cp = warp; 2 * cp < Aw; cp += kFieldWarps) {
        const int x0 = 2 * cp;
        const bool two = x0 + 1 < Aw;
        float2 v[PH];
#pragma unroll
        for (int i = 0; i < PH; ++i) {
            const int y = lane + 32 * i;
            v[i] = make_float2(tb[y * pitch + x0], two ? tb[y * pitch + x0 + 1] : 0.0f);
        }
        warp_fft_fwd<PH>(v, ty, lane);
        const int kb = PH * bitrev5(lane);
#pragma unroll
        for (int k1 = 0; k1 < PH; ++k1) {
            const float g = gy[k1 + kb];
            v[k1] = make_float2(v[k1].x * g, v[k1].y * g);
        }
        warp_fft_inv<PH>(v, ty, lane);
#pragma unroll
        for (int i = 0; i < PH; ++i) {
            const int y = lane + 32 * i;
            if (y < Ah) {
                ff[(size_t)y * Aw + x0] = v[i].x;
                if (two) ff[(size_t)y * Aw + x0 + 1] = v[i].y;
            }
        }
    }
}

// alpha(a) = (D/r0)^(5/6) L f(a): slot 0 (piston) = 0, slot l+1 = mode l + 2.
// A block colours 128 consecutive anchors of one frame into shared memory (row pitch 37,
// so that the per-anchor writes fall in distinct banks), then writes their alpha rows,
// one contiguous run of 128 x 36 floats, with consecutive threads on consecutive floats.
constexpr int kColourAnchors = 128;
constexpr int kColourPitch = kAlphaStride + 1;

__global__ void __launch_bounds__(kColourAnchors) colour_kernel(FrameBatch fb, FieldFrames geo,
                                                                const float *__restrict__ L) {
    __shared__ float sL[kModes * kModes];
    __shared__ float so[kColourAnchors * kColourPitch];
    for (int i = threadIdx.x; i < kModes * kModes; i += blockDim.x) sL[i] = L[i];
    __syncthreads();
    const int frame = blockIdx.y;
    const int A = geo.ah[frame] * geo.aw[frame];
    const int a0 = blockIdx.x * kColourAnchors;
    if (a0 >= A) return;
    const int na = min(kColourAnchors, A - a0);
    const int t = threadIdx.x;
    if (t < na) {
        const float *ff = geo.f[frame] + a0 + t;
        float v[kModes];
#pragma unroll
        for (int l = 0; l < kModes; ++l) v[l] = ff[(size_t)l * A];
        const float sc = fb.scale[frame];
        float *o = so + t * kColourPitch;
        o[0] = 0.0f;
#pragma unroll
        for (int j = 0; j < kModes; ++j) {
            float acc = 0.0f;
#pragma unroll
            for (int l = 0; l <= j; ++l) acc = fmaf(sL[j * kModes + l], v[l], acc);
            o[j + 1] = sc * acc;
        }
    }
    __syncthreads();
    float *out = geo.alpha[frame] + (size_t)a0 * kAlphaStride;
    for (int e = t; e < na * kAlphaStride; e += blockDim.x) {
        const int a = e / kAlphaStride;
        out[e] = so[a * kColourPitch + (e - a * kAlphaStride)];
    }
}

}  // namespace

p2s_status launch_noise(unsigned long long seed, int mode, int Fh, int Fw, float *out, cudaStream_t st) {
    const long long n = (long long)Fh * Fw;
    const long long quads = (n + 3) / 4;
    noise_kernel<<<(unsigned)((quads + 255) / 256), 256, 0, st>>>(seed, mode, n, out);
    P2S_CUDA(cudaGetLastError());
    return P2S_OK;
}

// The one-kernel filter for tori of 32 .. 256 points per axis whose row-pass block fits
// in shared memory; false: use the two-pass kernels.
template <int PW, int PH>
static p2s_status launch_field_pw_ph(const FrameBatch &fb, const FieldFrames &geo, int pitch, size_t smem,
                                     const FilterTable *tw, const FilterTable *th, const int *kom, cudaStream_t st) {
    P2S_CUDA(cudaFuncSetAttribute(field_kernel<PW, PH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    field_kernel<PW, PH><<<dim3(kModes, fb.n), 32 * kFieldWarps, smem, st>>>(fb, geo, pitch, tw->twiddle, tw->gain,
                                                                             th->twiddle, th->gain, kom);
    P2S_CUDA(cudaGetLastError());
    return P2S_OK;
}

template <int PW>
static p2s_status launch_field_pw(int PH, const FrameBatch &fb, const FieldFrames &geo, int pitch, size_t smem,
                                  const FilterTable *tw, const FilterTable *th, const int *kom, cudaStream_t st) {
    switch (PH) {
        case 1: return launch_field_pw_ph<PW, 1>(fb, geo, pitch, smem, tw, th, kom, st);
        case 2: return launch_field_pw_ph<PW, 2>(fb, geo, pitch, smem, tw, th, kom, st);
        case 4: return launch_field_pw_ph<PW, 4>(fb, geo, pitch, smem, tw, th, kom, st);
        default: return launch_field_pw_ph<PW, 8>(fb, geo, pitch, smem, tw, th, kom, st);
    }
}

// The one-kernel filter serves tori of 32 .. 256 points per axis whose row-pass block
// (Fh rows of the widest anchor grid, Aw_max) fits in shared memory.
static bool field_kernel_fits(int Fh, int Fw, int Ah_max, int Aw_max, int *pitch, size_t *smem) {
    auto ok_len = [](int F) { return F == 32 || F == 64 || F == 128 || F == 256; };
    if (!ok_len(Fw) || !ok_len(Fh) || Aw_max > Fw || Ah_max > Fh) return false;
    *pitch = Aw_max | 1;  // odd: the column pass reads 32 rows of one column without bank conflicts
    *smem = ((size_t)Fh * *pitch + (size_t)kFieldWarps * 2 * Fw + Fw + Fh) * sizeof(float) +
            (size_t)(Fw / 2 + Fh / 2) * sizeof(float2);
    return *smem <= 160 * 1024;
}
static bool field_kernel_fits(const FieldGeom &g, int *pitch, size_t *smem) {
    return field_kernel_fits(g.Fh, g.Fw, g.Ah, g.Aw, pitch, smem);
}

// filter (one kernel) and colour over frames of one torus, each with its own anchor grid
static p2s_status run_field_group(p2s_ctx *ctx, int Fh, int Fw, const FrameBatch &fb, const FieldFrames &geo,
                                  int pitch, size_t fsmem, cudaStream_t st) {
    const FilterTable *th = nullptr, *tw = nullptr;
    p2s_status s = filter_table(ctx, Fh, &th);
    if (s != P2S_OK) return s;
    if ((s = filter_table(ctx, Fw, &tw)) != P2S_OK) return s;
    double cells = 0.0;
    int max_a = 0;
    for (int k = 0; k < fb.n; ++k) {
        cells += (double)geo.ah[k] * geo.aw[k];
        max_a = std::max(max_a, geo.ah[k] * geo.aw[k]);
    }
    {
        ProfScope pf(ctx, st, "fields_filter", 0.0, cells * kModes * 4);
        const int PW = Fw / 32, PH = Fh / 32;
        p2s_status rs;
        switch (PW) {
            case 1: rs = launch_field_pw<1>(PH, fb, geo, pitch, fsmem, tw, th, ctx->d_kernel_of_mode, st); break;
            case 2: rs = launch_field_pw<2>(PH, fb, geo, pitch, fsmem, tw, th, ctx->d_kernel_of_mode, st); break;
            case 4: rs = launch_field_pw<4>(PH, fb, geo, pitch, fsmem, tw, th, ctx->d_kernel_of_mode, st); break;
            default: rs = launch_field_pw<8>(PH, fb, geo, pitch, fsmem, tw, th, ctx->d_kernel_of_mode, st); break;
        }
        if (rs != P2S_OK) return rs;
    }
    dim3 grid_a((max_a + kColourAnchors - 1) / kColourAnchors, fb.n);
    ProfScope pa(ctx, st, "fields_colour", cells * kModes * (kModes + 1), cells * (kModes + kAlphaStride) * 4);
    colour_kernel<<<grid_a, kColourAnchors, 0, st>>>(fb, geo, ctx->d_L);
    P2S_CUDA(cudaGetLastError());
    return P2S_OK;
}

bool fields_group_ok(const p2s_ctx *ctx, int Fh, int Fw, int Ah_max, int Aw_max) {
    int pitch = 0;
    size_t smem = 0;
    return ctx->field_method == 0 && field_kernel_fits(Fh, Fw, Ah_max, Aw_max, &pitch, &smem);
}

p2s_status launch_fields_group(p2s_ctx *ctx, int Fh, int Fw, const FrameBatch &fb, const FieldFrames &geo,
                               cudaStream_t st) {
    if (fb.n <= 0) return P2S_OK;
    int ah_max = 0, aw_max = 0;
    for (int k = 0; k < fb.n; ++k) {
        ah_max = std::max(ah_max, geo.ah[k]);
        aw_max = std::max(aw_max, geo.aw[k]);
    }
    int pitch = 0;
    size_t fsmem = 0;
    if (ctx->field_method != 0 || !field_kernel_fits(Fh, Fw, ah_max, aw_max, &pitch, &fsmem)) {
        set_error("mixed anchor grids need the one-kernel Fourier filter");
        return P2S_EINVAL;
    }
    return run_field_group(ctx, Fh, Fw, fb, geo, pitch, fsmem, st);
}

size_t fields_scratch_bytes(const FieldGeom &g, int n) {
    const size_t t = (size_t)n * kModes * g.Fh * g.Aw * sizeof(float);
    const size_t f = (size_t)n * kModes * g.Ah * g.Aw * sizeof(float);
    return ((t + 255) & ~(size_t)255) + f;
}

// Dense anchor draw (Sec. 3.4): f = chol(Sigma) w over the anchors, Sigma the
// unwrapped Gaussian correlation, evaluated through its Kronecker factors as
// f = L_y W L_x^T (W: white noise of stream (seed, mode) row-major over the
// anchors).  One CTA per (mode, frame); W and L_y W in shared memory.
__global__ void __launch_bounds__(kThreads) dense_field_kernel(FrameBatch fb, int Ah, int Aw,
                                                               const float *__restrict__ Ly,
                                                               const float *__restrict__ Lx,
                                                               const int *__restrict__ kernel_of_mode, float *f) {
    extern __shared__ float sdf[];
    const int mode = blockIdx.x, frame = blockIdx.y;
    const int A = Ah * Aw;
    float *W = sdf, *T = sdf + A;
    const unsigned long long seed = fb.seed[frame];
    for (int q = threadIdx.x; 4 * q < A; q += blockDim.x) {
        float z[4];
        normals4(seed, mode, (uint32_t)q, z);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (4 * q + i < A) W[4 * q + i] = z[i];
    }
    __syncthreads();
    const int kk = kernel_of_mode[mode];
    const float *ly = Ly + (size_t)kk * Ah * Ah, *lx = Lx + (size_t)kk * Aw * Aw;
    for (int e = threadIdx.x; e < A; e += blockDim.x) {  // T = L_y W (L_y lower triangular)
        const int i = e / Aw, j = e - i * Aw;
        float acc = 0.f;
        for (int k = 0; k <= i; ++k) acc = fmaf(__ldg(ly + (size_t)i * Ah + k), W[k * Aw + j], acc);
        T[e] = acc;
    }
    __syncthreads();
    float *ff = f + ((size_t)frame * kModes + mode) * A;
    for (int e = threadIdx.x; e < A; e += blockDim.x) {  // F = T L_x^T
        const int i = e / Aw, j = e - i * Aw;
        float acc = 0.f;
        for (int m = 0; m <= j; ++m) acc = fmaf(T[i * Aw + m], __ldg(lx + (size_t)j * Aw + m), acc);
        ff[e] = acc;
    }
}

// lower Cholesky factor (FP32) of the 1-D unwrapped Gaussian correlation over
// n anchors for every kernel, [n_kernels][n][n], built in FP64 on the host
static p2s_status dense_factor(p2s_ctx *ctx, int n, const float **out) {
    auto it = ctx->dense_L.find(n);
    if (it != ctx->dense_L.end()) {
        *out = (const float *)it->second;
        return P2S_OK;
    }
    std::vector<float> Lf((size_t)ctx->n_kernels * n * n, 0.f);
    std::vector<double> C((size_t)n * n);
    for (int kk = 0; kk < ctx->n_kernels; ++kk) {
        const double ell = ctx->ell[kk], s = ctx->s;
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < n; ++k) {
                const double d = (i - k) * s;
                C[(size_t)i * n + k] = std::exp(-d * d / (2.0 * ell * ell));
            }
        // Cholesky-Banachiewicz, row by row
        for (int i = 0; i < n; ++i)
            for (int k = 0; k <= i; ++k) {
                double acc = C[(size_t)i * n + k];
                for (int m = 0; m < k; ++m) acc -= C[(size_t)i * n + m] * C[(size_t)k * n + m];
                if (i == k) {
                    if (acc <= 0.0) {
                        set_error("anchor correlation matrix of %d points is not positive definite (ell / spacing too "
                                  "large for the dense draw)", n);
                        return P2S_EINVAL;
                    }
                    C[(size_t)i * n + i] = std::sqrt(acc);
                } else {
                    C[(size_t)i * n + k] = acc / C[(size_t)k * n + k];
                }
            }
        for (int i = 0; i < n; ++i)
            for (int k = 0; k <= i; ++k) Lf[((size_t)kk * n + i) * n + k] = (float)C[(size_t)i * n + k];
    }
    void *d = nullptr;
    if (cudaMalloc(&d, Lf.size() * sizeof(float)) != cudaSuccess) {
        set_error("no memory for the dense-draw factors");
        return P2S_ENOMEM;
    }
    P2S_CUDA(cudaMemcpy(d, Lf.data(), Lf.size() * sizeof(float), cudaMemcpyHostToDevice));
    ctx->dense_L[n] = d;
    *out = (const float *)d;
    return P2S_OK;
}

p2s_status dense_prepare(p2s_ctx *ctx, const FieldGeom &g) {
    const float *a, *b;
    p2s_status s = dense_factor(ctx, g.Ah, &a);
    return s == P2S_OK ? dense_factor(ctx, g.Aw, &b) : s;
}

p2s_status launch_fields(p2s_ctx *ctx, const FieldGeom &g, const FrameBatch &fb, float *alpha, void *scratch,
                         cudaStream_t st) {
    if (fb.n <= 0) return P2S_OK;
    // every frame on the same anchor grid: f [frame][mode][Ah][Aw] after the row-pass scratch,
    // alpha [frame][Ah][Aw][kAlphaStride]
    auto uniform_geo = [&](float *f) {
        FieldFrames geo;
        for (int k = 0; k < fb.n; ++k) {
            geo.ah[k] = g.Ah;
            geo.aw[k] = g.Aw;
            geo.f[k] = f + (size_t)k * kModes * g.Ah * g.Aw;
            geo.alpha[k] = alpha + (size_t)k * g.Ah * g.Aw * kAlphaStride;
        }
        return geo;
    };
    if (ctx->field_method == 1) {
        if (g.Ah > 128 || g.Aw > 128) {
            set_error("the dense anchor draw supports at most 128 anchors per axis");
            return P2S_EUNSUPPORTED;
        }
        const float *Ly = nullptr, *Lx = nullptr;
        p2s_status s0 = dense_factor(ctx, g.Ah, &Ly);
        if (s0 == P2S_OK) s0 = dense_factor(ctx, g.Aw, &Lx);
        if (s0 != P2S_OK) return s0;
        const size_t t_bytes = (size_t)fb.n * kModes * g.Fh * g.Aw * sizeof(float);
        float *f = (float *)((char *)scratch + ((t_bytes + 255) & ~(size_t)255));
        const int A = g.Ah * g.Aw;
        const size_t smem = (size_t)2 * A * sizeof(float);
        P2S_CUDA(cudaFuncSetAttribute(dense_field_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        {
            ProfScope pd(ctx, st, "fields_dense", (double)fb.n * kModes * A * (g.Ah + g.Aw), (double)fb.n * kModes * A * 4);
            dense_field_kernel<<<dim3(kModes, fb.n), kThreads, smem, st>>>(fb, g.Ah, g.Aw, Ly, Lx,
                                                                           ctx->d_kernel_of_mode, f);
            P2S_CUDA(cudaGetLastError());
        }
        dim3 grid_a((A + kColourAnchors - 1) / kColourAnchors, fb.n);
        ProfScope pa(ctx, st, "fields_colour", (double)fb.n * A * kModes * (kModes + 1),
                     (double)fb.n * A * (kModes + kAlphaStride) * 4);
        colour_kernel<<<grid_a, kColourAnchors, 0, st>>>(fb, uniform_geo(f), ctx->d_L);
        P2S_CUDA(cudaGetLastError());
        return P2S_OK;
    }
    const FilterTable *th = nullptr, *tw = nullptr;
    p2s_status s = filter_table(ctx, g.Fh, &th);
    if (s != P2S_OK) return s;
    if ((s = filter_table(ctx, g.Fw, &tw)) != P2S_OK) return s;
    float *t = (float *)scratch;
    const size_t t_bytes = (size_t)fb.n * kModes * g.Fh * g.Aw * sizeof(float);
    float *f = (float *)((char *)scratch + ((t_bytes + 255) & ~(size_t)255));
    int pitch = 0;
    size_t fsmem = 0;
    if (field_kernel_fits(g, &pitch, &fsmem)) return run_field_group(ctx, g.Fh, g.Fw, fb, uniform_geo(f), pitch, fsmem, st);

    // rows: R row pairs per CTA, R * Fw <= kFftElems
    int R = kFftElems / g.Fw;
    if (R < 1) R = 1;
    if (R > (g.Fh + 1) / 2) R = (g.Fh + 1) / 2;
    size_t smem = (size_t)2 * R * g.Fw * sizeof(float2) + (size_t)(g.Fw / 2 > 0 ? g.Fw / 2 : 1) * sizeof(float2) +
                  (size_t)g.Fw * sizeof(float);
    P2S_CUDA(cudaFuncSetAttribute(row_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid_r((g.Fh + 2 * R - 1) / (2 * R), kModes, fb.n);
    ProfScope pr(ctx, st, "fields_row_filter", 0.0, (double)fb.n * kModes * g.Fh * g.Aw * 4);
    row_filter_kernel<<<grid_r, kThreads, smem, st>>>(fb, g.Fh, g.Fw, g.Aw, R, tw->twiddle, tw->gain,
                                                       ctx->d_kernel_of_mode, t);
    P2S_CUDA(cudaGetLastError());

    int Rc = kFftElems / g.Fh;
    if (Rc < 1) Rc = 1;
    if (Rc > (g.Aw + 1) / 2) Rc = (g.Aw + 1) / 2;
    smem = (size_t)2 * Rc * g.Fh * sizeof(float2) + (size_t)(g.Fh / 2 > 0 ? g.Fh / 2 : 1) * sizeof(float2) +
           (size_t)g.Fh * sizeof(float);
    P2S_CUDA(cudaFuncSetAttribute(col_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid_c((g.Aw + 2 * Rc - 1) / (2 * Rc), kModes, fb.n);
    ProfScope pc(ctx, st, "fields_col_filter", 0.0,
                 (double)fb.n * kModes * (g.Fh * g.Aw + g.Ah * g.Aw) * 4);
    col_filter_kernel<<<grid_c, kThreads, smem, st>>>(g.Fh, g.Ah, g.Aw, Rc, th->twiddle, th->gain,
                                                       ctx->d_kernel_of_mode, t, f);
    P2S_CUDA(cudaGetLastError());

    const int A = g.Ah * g.Aw;
    dim3 grid_a((A + kColourAnchors - 1) / kColourAnchors, fb.n);
    ProfScope pa(ctx, st, "fields_colour", (double)fb.n * A * kModes * (kModes + 1),
                 (double)fb.n * A * (kModes + kAlphaStride) * 4);
    colour_kernel<<<grid_a, kColourAnchors, 0, st>>>(fb, uniform_geo(f), ctx->d_L);
    P2S_CUDA(cudaGetLastError());
    return P2S_OK;
}

}  // namespace p2s
