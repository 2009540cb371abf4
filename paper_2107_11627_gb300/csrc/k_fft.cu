// Batched-FFT evaluation of the scatter blur (Sec. 3.1), the comparison
// variant of the direct basis contraction:
//     y_c = sum_k h_k * (beta_k . x_c)  =  IDFT( sum_k DFT(h_k) DFT(beta_k . x_c) )
// on an Fh x Fw torus with Fh, Fw the powers of two >= H + 32, W + 32, so
// that no tap wraps into the kept H x W window ("same" output, zeros outside
// the image).  FP32 throughout, beta from the FP32 network.
//
//   1. beta [H][W][K] -> [K][H][W] (tiled transpose);
//   2. row pass: two real fields (k, c) per complex FFT of each image row,
//      separated into half spectra, written transposed Z[field][u][row];
//   3. column pass, one frequency column u per CTA: for every k, the three
//      channels' columns are transformed and multiplied by the basis spectrum
//      Hk[k][u][v], accumulating Y_c in registers; then Y_c is transformed
//      back and written Y[c][u][row];
//   4. final row pass: two real output rows per complex inverse FFT, scaled
//      by 1 / (Fh Fw), cropped to W.
// The basis spectra Hk (h_k placed with its centre tap at the origin) are
// made once per torus size by the same row and column kernels.
#include <cmath>
#include <vector>

#include "fft_smem.cuh"
#include "p2s_internal.h"

namespace p2s {
namespace fftb {

using fftsm::cmul;
using fftsm::fft_rows;

constexpr int kThreads = 256;
constexpr int kMaxF = 2048;
constexpr int kRowElems = 4096;  // complex elements per row-pass ping-pong buffer (>= 2 rows of 2048)

// ---- 1. beta [H][W][K] -> [K][H][W] -------------------------------------------
__global__ void transpose_beta(const float *__restrict__ in, float *__restrict__ out, int npx, int K) {
    __shared__ float t[32][33];
    const int p0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int p = p0 + i, k = k0 + threadIdx.x;
        t[i][threadIdx.x] = (p < npx && k < K) ? in[(size_t)p * K + k] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int k = k0 + i, p = p0 + threadIdx.x;
        if (k < K && p < npx) out[(size_t)k * npx + p] = t[threadIdx.x][i];
    }
}

// ---- 2. row pass ----------------------------------------------------------------
// Source of real row values: frame fields (beta_k x_c, field = k * C + c) or
// basis taps (field = k; row rho holds tap row ty with (ty - 16) mod Fh = rho).
struct RowSrc {
    int mode;  // 0: frame, 1: basis
    const float *betaT;  // [K][H][W]
    const float *x;      // [H][W][C]
    const float *H;      // basis FP32 [K][th * tw]
    int Hh, Ww, C, K, th, tw;
};

__device__ __forceinline__ float row_value(const RowSrc &s, int field, int row, int j, int Fw, int Fh) {
    if (s.mode == 0) {
        if (row >= s.Hh || j >= s.Ww) return 0.f;
        const int k = field / s.C, c = field - k * s.C;
        return s.betaT[((size_t)k * s.Hh + row) * s.Ww + j] * s.x[((size_t)row * s.Ww + j) * s.C + c];
    }
    // basis: tap (ty, tx) sits at ((ty - th/2) mod Fh, (tx - tw/2) mod Fw)
    const int ty = (row + s.th / 2) % Fh, tx = (j + s.tw / 2) % Fw;
    if (ty >= s.th || tx >= s.tw) return 0.f;
    return s.H[(size_t)field * s.th * s.tw + ty * s.tw + tx];
}

// grid (field pairs, row blocks); out Z[field][u][row], u in [0, Fw/2], rows [0, n_rows)
__global__ void __launch_bounds__(kThreads) row_r2c(RowSrc src, int n_fields, int n_rows, int Fh, int Fw, int RB,
                                                    const float2 *__restrict__ tw, float2 *__restrict__ Z) {
    extern __shared__ float2 sm[];
    float2 *a = sm, *b = sm + RB * Fw, *stw = sm + 2 * RB * Fw;
    for (int i = threadIdx.x; i < Fw / 2; i += blockDim.x) stw[i] = tw[i];
    const int fa = 2 * blockIdx.x, fb = fa + 1;
    const int r0 = blockIdx.y * RB;
    for (int i = threadIdx.x; i < RB * Fw; i += blockDim.x) {
        const int rr = i / Fw, j = i - rr * Fw, row = r0 + rr;
        float va = 0.f, vb = 0.f;
        if (row < n_rows) {
            va = row_value(src, fa, row, j, Fw, Fh);
            if (fb < n_fields) vb = row_value(src, fb, row, j, Fw, Fh);
        }
        a[i] = make_float2(va, vb);
    }
    __syncthreads();
    float2 *res = fft_rows(a, b, stw, Fw, RB, false);
    const int nu = Fw / 2 + 1;
    for (int i = threadIdx.x; i < nu * RB; i += blockDim.x) {
        const int u = i / RB, rr = i - u * RB, row = r0 + rr;
        if (row >= n_rows) continue;
        const float2 z = res[rr * Fw + u], zc = res[rr * Fw + ((Fw - u) & (Fw - 1))];
        // A = (Z(u) + conj Z(-u)) / 2, B = (Z(u) - conj Z(-u)) / 2i
        const float2 A = make_float2(0.5f * (z.x + zc.x), 0.5f * (z.y - zc.y));
        const float2 B = make_float2(0.5f * (z.y + zc.y), -0.5f * (z.x - zc.x));
        Z[((size_t)fa * nu + u) * n_rows + row] = A;
        if (fb < n_fields) Z[((size_t)fb * nu + u) * n_rows + row] = B;
    }
}

// ---- basis column pass: Hk[k][u][v] = column FFT of Z[k][u][*] over Fh rows ----
__global__ void __launch_bounds__(kThreads) col_basis(const float2 *__restrict__ Z, int Fh, int nu,
                                                      const float2 *__restrict__ twh, float2 *__restrict__ Hk) {
    extern __shared__ float2 sm[];
    float2 *a = sm, *b = sm + Fh, *stw = sm + 2 * Fh;
    for (int i = threadIdx.x; i < Fh / 2; i += blockDim.x) stw[i] = twh[i];
    const int u = blockIdx.x, k = blockIdx.y;
    const float2 *src = Z + ((size_t)k * nu + u) * Fh;
    for (int i = threadIdx.x; i < Fh; i += blockDim.x) a[i] = src[i];
    __syncthreads();
    float2 *res = fft_rows(a, b, stw, Fh, 1, false);
    float2 *dst = Hk + ((size_t)k * nu + u) * Fh;
    for (int i = threadIdx.x; i < Fh; i += blockDim.x) dst[i] = res[i];
}

// ---- 3. frame column pass: Y_c[u][row] = IDFT_v( sum_k DFT_v(Z[k,c][u][*]) Hk[k][u][v] ) ----
template <int C>
__global__ void __launch_bounds__(kThreads) col_mac(const float2 *__restrict__ Z, const float2 *__restrict__ Hk,
                                                    int K, int Hh, int Fh, int nu, const float2 *__restrict__ twh,
                                                    float2 *__restrict__ Y) {
    extern __shared__ float2 sm[];
    float2 *a = sm, *b = sm + C * Fh, *stw = sm + 2 * C * Fh;
    for (int i = threadIdx.x; i < Fh / 2; i += blockDim.x) stw[i] = twh[i];
    const int u = blockIdx.x;
    constexpr int kPer = kMaxF / kThreads;  // accumulators per thread and channel
    float2 acc[C][kPer];
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int q = 0; q < kPer; ++q) acc[c][q] = make_float2(0.f, 0.f);
    for (int k = 0; k < K; ++k) {
        __syncthreads();  // the previous k's buffers are no longer read
        for (int i = threadIdx.x; i < C * Fh; i += blockDim.x) {
            const int c = i / Fh, v = i - c * Fh;
            a[i] = v < Hh ? Z[((size_t)(k * C + c) * nu + u) * Hh + v] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const float2 *res = fft_rows(a, b, stw, Fh, C, false);
        const float2 *hk = Hk + ((size_t)k * nu + u) * Fh;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int v = threadIdx.x + q * kThreads;
            if (v < Fh) {
                const float2 h = __ldg(hk + v);
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float2 z = res[c * Fh + v];
                    acc[c][q].x += z.x * h.x - z.y * h.y;
                    acc[c][q].y += z.x * h.y + z.y * h.x;
                }
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int v = threadIdx.x + q * kThreads;
        if (v < Fh)
#pragma unroll
            for (int c = 0; c < C; ++c) a[c * Fh + v] = acc[c][q];
    }
    __syncthreads();
    const float2 *res = fft_rows(a, b, stw, Fh, C, true);
    for (int i = threadIdx.x; i < C * Hh; i += blockDim.x) {
        const int c = i / Hh, row = i - c * Hh;
        Y[((size_t)c * nu + u) * Hh + row] = res[c * Fh + row];
    }
}

// ---- 4. final row pass: two output rows per complex inverse FFT ---------------
// Rows are numbered over (c, row): pair p covers flat rows 2p, 2p + 1.
template <int C>
__global__ void __launch_bounds__(kThreads) row_c2r(const float2 *__restrict__ Y, int Hh, int Ww, int Fw, int nu,
                                                    int RB, float scale, const float2 *__restrict__ tw,
                                                    float *__restrict__ y) {
    extern __shared__ float2 sm[];
    float2 *a = sm, *b = sm + RB * Fw, *stw = sm + 2 * RB * Fw;
    for (int i = threadIdx.x; i < Fw / 2; i += blockDim.x) stw[i] = tw[i];
    const int n_flat = C * Hh;
    const int p0 = blockIdx.x * RB;  // first row pair
    for (int i = threadIdx.x; i < RB * Fw; i += blockDim.x) {
        const int rr = i / Fw, uu = i - rr * Fw;
        const int fa = 2 * (p0 + rr), fb = fa + 1;
        // Hermitian extension: Y(Fw - u) = conj Y(u)
        const bool hi = uu >= nu;
        const int u = hi ? Fw - uu : uu;
        float2 ya = make_float2(0.f, 0.f), yb = make_float2(0.f, 0.f);
        if (fa < n_flat) {
            const int c = fa / Hh, row = fa - c * Hh;
            ya = Y[((size_t)c * nu + u) * Hh + row];
        }
        if (fb < n_flat) {
            const int c = fb / Hh, row = fb - c * Hh;
            yb = Y[((size_t)c * nu + u) * Hh + row];
        }
        if (hi) {
            ya.y = -ya.y;
            yb.y = -yb.y;
        }
        a[i] = make_float2(ya.x - yb.y, ya.y + yb.x);  // Ya + i Yb
    }
    __syncthreads();
    const float2 *res = fft_rows(a, b, stw, Fw, RB, true);
    for (int i = threadIdx.x; i < RB * Ww; i += blockDim.x) {
        const int rr = i / Ww, j = i - rr * Ww;
        const int fa = 2 * (p0 + rr), fb = fa + 1;
        const float2 z = res[rr * Fw + j];
        if (fa < n_flat) {
            const int c = fa / Hh, row = fa - c * Hh;
            y[((size_t)row * Ww + j) * C + c] = z.x * scale;
        }
        if (fb < n_flat) {
            const int c = fb / Hh, row = fb - c * Hh;
            y[((size_t)row * Ww + j) * C + c] = z.y * scale;
        }
    }
}

int pow2_at_least(int v) {
    int f = 1;
    while (f < v) f <<= 1;
    return f;
}

float2 *twiddles(p2s_ctx *ctx, int F) {
    auto it = ctx->fft_tw.find(F);
    if (it != ctx->fft_tw.end()) return (float2 *)it->second;
    std::vector<float2> tw(F / 2 > 0 ? F / 2 : 1);
    for (int m = 0; m < F / 2; ++m) {
        const double a = 2.0 * M_PI * m / F;
        tw[m] = make_float2((float)std::cos(a), (float)-std::sin(a));
    }
    void *d = nullptr;
    if (cudaMalloc(&d, tw.size() * sizeof(float2)) != cudaSuccess) return nullptr;
    cudaMemcpy(d, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
    ctx->fft_tw[F] = d;
    return (float2 *)d;
}

}  // namespace fftb

using namespace fftb;

// Basis spectra for an Fh x Fw torus, cached in the context.
static p2s_status basis_spectra(p2s_ctx *ctx, int Fh, int Fw, const float2 **out, cudaStream_t st) {
    const long long key = (long long)Fh * 65536 + Fw;
    auto it = ctx->fft_basis.find(key);
    if (it != ctx->fft_basis.end()) {
        *out = (const float2 *)it->second;
        return P2S_OK;
    }
    float2 *twh = twiddles(ctx, Fh), *tww = twiddles(ctx, Fw);
    if (!twh || !tww) {
        set_error("twiddle table allocation failed");
        return P2S_ENOMEM;
    }
    const int nu = Fw / 2 + 1, K = ctx->K;
    void *Hk = nullptr, *Z = nullptr;
    if (cudaMalloc(&Hk, (size_t)K * nu * Fh * sizeof(float2)) != cudaSuccess) {
        set_error("no memory for the basis spectra");
        return P2S_ENOMEM;
    }
    P2S_CUDA(cudaMallocAsync(&Z, (size_t)K * nu * Fh * sizeof(float2), st));
    RowSrc src{1, nullptr, nullptr, ctx->d_H32, 0, 0, 1, K, ctx->th, ctx->tw};
    const int RB = kRowElems / Fw;
    const size_t smem_r = (2 * (size_t)RB * Fw + Fw / 2) * sizeof(float2);
    P2S_CUDA(cudaFuncSetAttribute(row_r2c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_r));
    row_r2c<<<dim3((K + 1) / 2, (Fh + RB - 1) / RB), kThreads, smem_r, st>>>(src, K, Fh, Fh, Fw, RB, tww, (float2 *)Z);
    P2S_CUDA(cudaGetLastError());
    const size_t smem_c = (2 * (size_t)Fh + Fh / 2) * sizeof(float2);
    col_basis<<<dim3(nu, K), kThreads, smem_c, st>>>((const float2 *)Z, Fh, nu, twh, (float2 *)Hk);
    P2S_CUDA(cudaGetLastError());
    cudaFreeAsync(Z, st);
    ctx->fft_basis[key] = Hk;
    *out = (const float2 *)Hk;
    return P2S_OK;
}

p2s_status launch_blur_fft(p2s_ctx *ctx, int H, int W, int C, int n, const float *const *xw, const float *beta,
                           float *const *y, cudaStream_t st) {
    if (n <= 0) return P2S_OK;
    if (C != 1 && C != 3) {
        set_error("C must be 1 or 3");
        return P2S_EINVAL;
    }
    const int Fh = pow2_at_least(H + ctx->th - 1), Fw = pow2_at_least(W + ctx->tw - 1);
    if (Fh > kMaxF || Fw > kMaxF || Fw * 2 > kRowElems * 2) {
        set_error("FFT blur supports frames up to %d pixels per side minus the taps", kMaxF);
        return P2S_EUNSUPPORTED;
    }
    const float2 *Hk = nullptr;
    p2s_status s0 = basis_spectra(ctx, Fh, Fw, &Hk, st);
    if (s0 != P2S_OK) return s0;
    const float2 *twh = twiddles(ctx, Fh), *tww = twiddles(ctx, Fw);
    const int K = ctx->K, nu = Fw / 2 + 1, npx = H * W;
    const size_t b_bytes = (size_t)K * npx * sizeof(float);
    const size_t z_bytes = (size_t)K * C * nu * H * sizeof(float2);
    const size_t y_bytes = (size_t)C * nu * H * sizeof(float2);
    char *buf = nullptr;
    P2S_CUDA(cudaMallocAsync((void **)&buf, b_bytes + z_bytes + y_bytes + 1024, st));
    float *betaT = (float *)buf;
    float2 *Z = (float2 *)(buf + ((b_bytes + 255) & ~(size_t)255));
    float2 *Y = (float2 *)((char *)Z + ((z_bytes + 255) & ~(size_t)255));
    const int RB = kRowElems / Fw;
    const size_t smem_r = (2 * (size_t)RB * Fw + Fw / 2) * sizeof(float2);
    const size_t smem_c = (2 * (size_t)C * Fh + Fh / 2) * sizeof(float2);
    P2S_CUDA(cudaFuncSetAttribute(row_r2c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_r));
    const double flops = 2.0 * ctx->K * ctx->T * (double)npx;  // the direct form's work, for comparison
    for (int i = 0; i < n; ++i) {
        {
            ProfScope pr(ctx, st, "blur_fft_rows", flops, (double)npx * (C * 4.0 + K * 8.0) + (double)z_bytes);
            transpose_beta<<<dim3((npx + 31) / 32, (K + 31) / 32), dim3(32, 8), 0, st>>>(beta + (size_t)i * npx * K,
                                                                                        betaT, npx, K);
            RowSrc src{0, betaT, xw[i], nullptr, H, W, C, K, 0, 0};
            row_r2c<<<dim3((K * C + 1) / 2, (H + RB - 1) / RB), kThreads, smem_r, st>>>(src, K * C, H, Fh, Fw, RB, tww,
                                                                                          Z);
        }
        ProfScope pr(ctx, st, "blur_fft_cols", 0.0, (double)z_bytes + (double)K * nu * Fh * 8.0 + (double)npx * C * 4.0);
        if (C == 3) {
            P2S_CUDA(cudaFuncSetAttribute(col_mac<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
            col_mac<3><<<nu, kThreads, smem_c, st>>>(Z, Hk, K, H, Fh, nu, twh, Y);
            P2S_CUDA(cudaFuncSetAttribute(row_c2r<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_r));
            row_c2r<3><<<(C * H / 2 + 1 + RB - 1) / RB, kThreads, smem_r, st>>>(Y, H, W, Fw, nu, RB,
                                                                                 1.0f / ((float)Fh * Fw), tww, y[i]);
        } else {
            P2S_CUDA(cudaFuncSetAttribute(col_mac<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
            col_mac<1><<<nu, kThreads, smem_c, st>>>(Z, Hk, K, H, Fh, nu, twh, Y);
            P2S_CUDA(cudaFuncSetAttribute(row_c2r<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_r));
            row_c2r<1><<<(C * H / 2 + 1 + RB - 1) / RB, kThreads, smem_r, st>>>(Y, H, W, Fw, nu, RB,
                                                                                 1.0f / ((float)Fh * Fw), tww, y[i]);
        }
        P2S_CUDA(cudaGetLastError());
    }
    cudaFreeAsync(buf, st);
    return P2S_OK;
}

}  // namespace p2s
