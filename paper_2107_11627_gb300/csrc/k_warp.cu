// Tilt warp (Sec. 2.2, Sec. 3.3): the tilt coefficients alpha_2, alpha_3,
// bilinearly interpolated from the anchors (Sec. 3.4), displace each pixel
// by d = kappa (alpha_3, alpha_2) (rows, columns); the warped frame is the
// backward bilinear sample x_w(p) = x(p - d(p)) with coordinates clamped to
// the frame.  The sample position is kept as integer pixel + FP32 offset.
#include <algorithm>

#include "p2s_internal.h"

namespace p2s {

namespace {

// frames of one launch: input, output, anchors ([Ah][Aw][36]), size, first block
struct WarpTable {
    const float *in[kMaxBatch];
    float *out[kMaxBatch];
    const float *alpha[kMaxBatch];
    int H[kMaxBatch], W[kMaxBatch], Aw[kMaxBatch], b0[kMaxBatch];
    int nf;
};

// ONE_SIZE: frames of one size on a 2-D grid (blockIdx.y the frame, the size read from
// entry 0); else a 1-D grid, each block finding its frame by binary search over the
// frames' first blocks.
template <int C, bool ONE_SIZE>
__global__ void __launch_bounds__(256) warp_kernel(const __grid_constant__ WarpTable t, int s, float inv_s,
                                                   float kappa) {
    int frame = (int)blockIdx.y, blk = (int)blockIdx.x;
    if (!ONE_SIZE) {
        int hi = t.nf - 1;
        while (frame < hi) {
            const int mid = (frame + hi + 1) >> 1;
            if (blk >= t.b0[mid]) frame = mid;
            else hi = mid - 1;
        }
        blk -= t.b0[frame];
    }
    const int f0 = ONE_SIZE ? 0 : frame;
    const int H = t.H[f0], W = t.W[f0], Aw = t.Aw[f0];
    const long long p = (long long)blk * blockDim.x + threadIdx.x;
    if (p >= (long long)H * W) return;
    const int i = (int)(p / W), j = (int)(p - (long long)i * W);
    const int ay = i / s, ax = j / s;
    const float fy = (float)(i - ay * s) * inv_s, fx = (float)(j - ax * s) * inv_s;
    const float *a = t.alpha[frame] + ((size_t)ay * Aw + ax) * kAlphaStride;
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
    const float *x = t.in[frame];
    const float *r0 = x + (size_t)y0c * W * C, *r1 = x + (size_t)y1c * W * C;
    float *o = t.out[frame] + (size_t)p * C;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float top = (1.0f - wx) * __ldg(r0 + x0c * C + c) + wx * __ldg(r0 + x1c * C + c);
        const float bot = (1.0f - wx) * __ldg(r1 + x0c * C + c) + wx * __ldg(r1 + x1c * C + c);
        o[c] = (1.0f - wy) * top + wy * bot;
    }
}

}  // namespace

p2s_status launch_warp_frames(const p2s_ctx *ctx, const WarpFrame *frames, int n, int C, cudaStream_t st) {
    if (n <= 0) return P2S_OK;
    if (n > kMaxBatch) {
        set_error("warp batch larger than %d", kMaxBatch);
        return P2S_EINVAL;
    }
    WarpTable t;
    long long blocks = 0;
    double px = 0.0;
    bool uniform = true;
    for (int i = 0; i < n; ++i) {
        const WarpFrame &f = frames[i];
        t.in[i] = f.in;
        t.out[i] = f.out;
        t.alpha[i] = f.alpha;
        t.H[i] = f.H;
        t.W[i] = f.W;
        t.Aw[i] = (f.W - 1) / ctx->s + 2;
        t.b0[i] = (int)std::min(blocks, 0x7fffffffll);
        uniform = uniform && f.H == frames[0].H && f.W == frames[0].W;
        blocks += ((long long)f.H * f.W + 255) / 256;
        px += (double)f.H * f.W;
    }
    t.nf = n;
    if (blocks == 0) return P2S_OK;
    if (blocks > 0x7fffffffll) {
        set_error("warp batch too large");
        return P2S_EINVAL;
    }
    // one size: a 2-D grid of one frame's blocks by the frames; else the blocks of all
    // frames in a row
    const dim3 grid = uniform ? dim3((unsigned)(blocks / n), (unsigned)n) : dim3((unsigned)blocks, 1);
    const float inv_s = 1.0f / (float)ctx->s, kappa = (float)ctx->kappa;
    ProfScope pr(ctx, st, "warp", 0.0, px * C * 4 * 2);
    if (uniform) {
        if (C == 3) warp_kernel<3, true><<<grid, 256, 0, st>>>(t, ctx->s, inv_s, kappa);
        else warp_kernel<1, true><<<grid, 256, 0, st>>>(t, ctx->s, inv_s, kappa);
    } else {
        if (C == 3) warp_kernel<3, false><<<grid, 256, 0, st>>>(t, ctx->s, inv_s, kappa);
        else warp_kernel<1, false><<<grid, 256, 0, st>>>(t, ctx->s, inv_s, kappa);
    }
    P2S_CUDA(cudaGetLastError());
    return P2S_OK;
}

p2s_status launch_warp(const p2s_ctx *ctx, const FieldGeom &g, int n, const float *const *in, const float *alpha,
                       float *const *out, int C, cudaStream_t st) {
    if (n <= 0) return P2S_OK;
    if (n > kMaxBatch) {
        set_error("warp batch larger than %d", kMaxBatch);
        return P2S_EINVAL;
    }
    WarpFrame fr[kMaxBatch];
    for (int i = 0; i < n; ++i) fr[i] = WarpFrame{in[i], out[i], alpha + (size_t)i * g.Ah * g.Aw * kAlphaStride, g.H, g.W};
    return launch_warp_frames(ctx, fr, n, C, st);
}

}  // namespace p2s
