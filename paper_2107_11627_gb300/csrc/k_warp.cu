// Tilt warp (Sec. 2.2, Sec. 3.3): the tilt coefficients alpha_2, alpha_3,
// bilinearly interpolated from the anchors (Sec. 3.4), displace each pixel
// by d = kappa (alpha_3, alpha_2) (rows, columns); the warped frame is the
// backward bilinear sample x_w(p) = x(p - d(p)) with coordinates clamped to
// the frame.  The sample position is kept as integer pixel + FP32 offset.
#include "p2s_internal.h"

namespace p2s {

namespace {

struct WarpPtrs {
    const float *in[kMaxBatch];
    float *out[kMaxBatch];
};

template <int C>
__global__ void __launch_bounds__(256) warp_kernel(WarpPtrs ptr, int H, int W, int s, float inv_s, int Aw, int A,
                                                   float kappa, const float *__restrict__ alpha) {
    const int frame = blockIdx.y;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (long long)H * W) return;
    const int i = (int)(p / W), j = (int)(p - (long long)i * W);
    const int ay = i / s, ax = j / s;
    const float fy = (float)(i - ay * s) * inv_s, fx = (float)(j - ax * s) * inv_s;
    const float *a = alpha + ((size_t)frame * A + (size_t)ay * Aw + ax) * kAlphaStride;
    const float *b = a + (size_t)Aw * kAlphaStride;
    // slot 1 = alpha_2 (x tilt), slot 2 = alpha_3 (y tilt)
    const float a2 = (1.0f - fy) * ((1.0f - fx) * a[1] + fx * a[kAlphaStride + 1]) +
                     fy * ((1.0f - fx) * b[1] + fx * b[kAlphaStride + 1]);
    const float a3 = (1.0f - fy) * ((1.0f - fx) * a[2] + fx * a[kAlphaStride + 2]) +
                     fy * ((1.0f - fx) * b[2] + fx * b[kAlphaStride + 2]);
    const float lim = (float)(H + W);
    const float ty = fminf(fmaxf(-kappa * a3, -lim), lim);
    const float tx = fminf(fmaxf(-kappa * a2, -lim), lim);
    const float iy = floorf(ty), ix = floorf(tx);
    const float wy = ty - iy, wx = tx - ix;
    const int y0 = i + (int)iy, x0 = j + (int)ix;
    const int y0c = min(max(y0, 0), H - 1), y1c = min(max(y0 + 1, 0), H - 1);
    const int x0c = min(max(x0, 0), W - 1), x1c = min(max(x0 + 1, 0), W - 1);
    const float *x = ptr.in[frame];
    const float *r0 = x + (size_t)y0c * W * C, *r1 = x + (size_t)y1c * W * C;
    float *o = ptr.out[frame] + (size_t)p * C;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float top = (1.0f - wx) * __ldg(r0 + x0c * C + c) + wx * __ldg(r0 + x1c * C + c);
        const float bot = (1.0f - wx) * __ldg(r1 + x0c * C + c) + wx * __ldg(r1 + x1c * C + c);
        o[c] = (1.0f - wy) * top + wy * bot;
    }
}

}  // namespace

p2s_status launch_warp(const p2s_ctx *ctx, const FieldGeom &g, int n, const float *const *in, const float *alpha,
                       float *const *out, int C, cudaStream_t st) {
    if (n <= 0) return P2S_OK;
    if (n > kMaxBatch) {
        set_error("warp batch larger than %d", kMaxBatch);
        return P2S_EINVAL;
    }
    WarpPtrs ptr;
    for (int i = 0; i < n; ++i) {
        ptr.in[i] = in[i];
        ptr.out[i] = out[i];
    }
    const long long npx = (long long)g.H * g.W;
    dim3 grid((unsigned)((npx + 255) / 256), n);
    const float inv_s = 1.0f / (float)g.s;
    ProfScope pr(ctx, st, "warp", 0.0, (double)n * npx * C * 4 * 2);
    if (C == 3)
        warp_kernel<3><<<grid, 256, 0, st>>>(ptr, g.H, g.W, g.s, inv_s, g.Aw, g.Ah * g.Aw, (float)ctx->kappa, alpha);
    else
        warp_kernel<1><<<grid, 256, 0, st>>>(ptr, g.H, g.W, g.s, inv_s, g.Aw, g.Ah * g.Aw, (float)ctx->kappa, alpha);
    P2S_CUDA(cudaGetLastError());
    return P2S_OK;
}

}  // namespace p2s
