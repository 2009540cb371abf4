// Plain FP32 path on the CUDA cores: the P2S network (Sec. 3.3) and the basis
// blur (Sec. 3.1, Eq. 3-5) without tensor cores.
#include "p2s_internal.h"

namespace p2s {

namespace {

constexpr int kMlpThreads = 64;  // pixels per network block
constexpr int kMaxWidth = 128;
// Shared memory of the plain network kernel: the weight image plus two activation
// buffers [kMaxWidth][kMlpThreads]; the image is limited by what is left of 227 KiB.
constexpr size_t kMlpActBytes = 2ull * kMaxWidth * kMlpThreads * 4;
constexpr size_t kMlpSmemLimit = 227 * 1024;

struct MlpLayers {
    int n;
    int in[4], out[4];
    int w_off[4], b_off[4];  // float offsets into the shared weight image
    int relu[4];
};

// One thread per pixel.  Weights (transposed, [in][out]) and biases live in
// shared memory; activations in per-thread shared columns; each layer's
// outputs accumulate in registers over the inputs in order.
__global__ void __launch_bounds__(kMlpThreads) mlp_simt_kernel(MlpLayers lay, int total_w, int n_frames, int H,
                                                              int W, int s, float inv_s, int Aw, int A,
                                                              const float *__restrict__ wimg,
                                                              const float *__restrict__ alpha, float *beta) {
    extern __shared__ float sm[];
    float *sw = sm;                                    // weights + biases
    float *bufA = sm + total_w;                        // [kMaxWidth][kMlpThreads]
    float *bufB = bufA + kMaxWidth * kMlpThreads;      // [kMaxWidth][kMlpThreads]
    for (int i = threadIdx.x; i < total_w; i += blockDim.x) sw[i] = wimg[i];
    __syncthreads();
    const int tid = threadIdx.x;
    const long long npx = (long long)H * W;
    const long long nblk = (npx * n_frames + kMlpThreads - 1) / kMlpThreads;
    const int K = lay.out[lay.n - 1];
    for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const long long gp = blk * kMlpThreads + tid;  // global pixel over the batch
        const bool valid = gp < npx * n_frames;
        if (valid) {
            const int frame = (int)(gp / npx);
            const long long p = gp - (long long)frame * npx;
            const int i = (int)(p / W), j = (int)(p - (long long)i * W);
            const int ay = i / s, ax = j / s;
            const float fy = (float)(i - ay * s) * inv_s, fx = (float)(j - ax * s) * inv_s;
            const float *a = alpha + ((size_t)frame * A + (size_t)ay * Aw + ax) * kAlphaStride;
            const float *b = a + (size_t)Aw * kAlphaStride;
            for (int m = 0; m < kHiModes; ++m) {  // slots 3..35 = J 4..36
                const int sl = m + 3;
                bufA[m * kMlpThreads + tid] = (1.0f - fy) * ((1.0f - fx) * a[sl] + fx * a[kAlphaStride + sl]) +
                                              fy * ((1.0f - fx) * b[sl] + fx * b[kAlphaStride + sl]);
            }
        } else {
            for (int m = 0; m < kHiModes; ++m) bufA[m * kMlpThreads + tid] = 0.0f;
        }
        float *in = bufA, *outb = bufB;
        for (int l = 0; l < lay.n; ++l) {
            const int fi = lay.in[l], fo = lay.out[l];
            const float *wt = sw + lay.w_off[l];
            const float *bb = sw + lay.b_off[l];
            float acc[kMaxWidth];
#pragma unroll
            for (int o = 0; o < kMaxWidth; ++o) acc[o] = 0.0f;
            for (int ii = 0; ii < fi; ++ii) {
                const float v = in[ii * kMlpThreads + tid];
                const float *wr = wt + ii * fo;
#pragma unroll
                for (int o = 0; o < kMaxWidth; ++o)
                    if (o < fo) acc[o] = fmaf(wr[o], v, acc[o]);
            }
#pragma unroll
            for (int o = 0; o < kMaxWidth; ++o)
                if (o < fo) {
                    float h = acc[o] + bb[o];
                    if (lay.relu[l]) h = fmaxf(h, 0.0f);
                    outb[o * kMlpThreads + tid] = h;
                }
            float *t = in;
            in = outb;
            outb = t;
        }
        __syncthreads();
        // coalesced write of beta [pixel][K] for the block's pixels
        const long long base = blk * kMlpThreads;
        for (int e = tid; e < kMlpThreads * K; e += kMlpThreads) {
            const int px = e / K, k = e - px * K;
            if (base + px < npx * n_frames) beta[(base + px) * K + k] = in[k * kMlpThreads + px];
        }
        __syncthreads();
    }
}

struct BlurPtrs {
    const float *x[kMaxBatch];
    float *y[kMaxBatch];
};

constexpr int kTile = 16;      // 16 x 16 pixels per block
constexpr int kTapChunk = 32;  // taps of H staged per pass

// Gather (Eq. 5): one thread per OUTPUT pixel q, its beta in registers,
// y_c[q] = sum_t (sum_k beta[q,k] H[k,t]) x_c[q - o(t)].
template <int KP, int C>
__global__ void __launch_bounds__(kTile *kTile) blur_gather_simt(BlurPtrs ptr, int H, int W, int K, int th, int tw,
                                                                 const float *__restrict__ Ht,
                                                                 const float *__restrict__ beta) {
    extern __shared__ float sm[];
    const int frame = blockIdx.z;
    const int r0 = blockIdx.y * kTile, c0 = blockIdx.x * kTile;
    const int xr = kTile + th - 1, xc = kTile + tw - 1;
    float *xs = sm;                                  // [C][xr][xc]
    float *hs = sm + ((C * xr * xc + 3) & ~3);       // [kTapChunk][KP], 16-byte aligned
    const float *x = ptr.x[frame];
    for (int e = threadIdx.x; e < C * xr * xc; e += blockDim.x) {
        const int c = e / (xr * xc), rem = e - c * xr * xc, rr = rem / xc, cc = rem - rr * xc;
        const int gy = r0 + rr - th / 2, gx = c0 + cc - tw / 2;
        xs[e] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? x[((size_t)gy * W + gx) * C + c] : 0.0f;
    }
    const int ly = threadIdx.x / kTile, lx = threadIdx.x % kTile;
    const int gy = r0 + ly, gx = c0 + lx;
    const bool inside = gy < H && gx < W;
    float bq[KP];
    const float *bp = beta + (((size_t)frame * H + (inside ? gy : 0)) * W + (inside ? gx : 0)) * K;
#pragma unroll
    for (int k = 0; k < KP; ++k) bq[k] = (inside && k < K) ? bp[k] : 0.0f;
    float acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = 0.0f;
    const int T = th * tw;
    for (int t0 = 0; t0 < T; t0 += kTapChunk) {
        const int nt = min(kTapChunk, T - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < nt * KP; e += blockDim.x) {
            const int t = e / KP, k = e - t * KP;
            hs[e] = k < K ? Ht[(size_t)(t0 + t) * K + k] : 0.0f;
        }
        __syncthreads();
        for (int t = 0; t < nt; ++t) {
            const float4 *hv = (const float4 *)(hs + t * KP);
            float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
#pragma unroll
            for (int k4 = 0; k4 < KP / 4; ++k4) {
                const float4 h4 = hv[k4];
                g0 = fmaf(bq[4 * k4 + 0], h4.x, g0);
                g1 = fmaf(bq[4 * k4 + 1], h4.y, g1);
                g2 = fmaf(bq[4 * k4 + 2], h4.z, g2);
                g3 = fmaf(bq[4 * k4 + 3], h4.w, g3);
            }
            const float g = (g0 + g1) + (g2 + g3);
            const int tt = t0 + t, ty = tt / tw, tx = tt - ty * tw;  // o(t) = (ty - th/2, tx - tw/2)
            const int sy = ly + th - 1 - ty, sx = lx + tw - 1 - tx;    // tile index of q - o(t)
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] = fmaf(g, xs[(c * xr + sy) * xc + sx], acc[c]);
        }
    }
    if (inside) {
        float *y = ptr.y[frame] + ((size_t)gy * W + gx) * C;
#pragma unroll
        for (int c = 0; c < C; ++c) y[c] = acc[c];
    }
}

// Scatter: one thread per SOURCE pixel p, its beta in registers; each tap's
// contribution G[p,t] x_c[p] lands in a shared accumulator tile covering the
// block's pixels plus the PSF halo; the tile is then added to y (zeroed
// beforehand) with global atomics, which also merges overlapping halos.
template <int KP, int C>
__global__ void __launch_bounds__(kTile *kTile) blur_scatter_simt(BlurPtrs ptr, int H, int W, int K, int th, int tw,
                                                                  const float *__restrict__ Ht,
                                                                  const float *__restrict__ beta) {
    extern __shared__ float sm[];
    const int frame = blockIdx.z;
    const int r0 = blockIdx.y * kTile, c0 = blockIdx.x * kTile;
    const int ar = kTile + th - 1, ac = kTile + tw - 1;
    float *as = sm;                                  // [C][ar][ac] accumulator
    float *hs = sm + ((C * ar * ac + 3) & ~3);       // [kTapChunk][KP], 16-byte aligned
    for (int e = threadIdx.x; e < C * ar * ac; e += blockDim.x) as[e] = 0.0f;
    const int ly = threadIdx.x / kTile, lx = threadIdx.x % kTile;
    const int gy = r0 + ly, gx = c0 + lx;
    const bool inside = gy < H && gx < W;
    float bq[KP];
    const float *bp = beta + (((size_t)frame * H + (inside ? gy : 0)) * W + (inside ? gx : 0)) * K;
#pragma unroll
    for (int k = 0; k < KP; ++k) bq[k] = (inside && k < K) ? bp[k] : 0.0f;
    float xv[C];
    const float *x = ptr.x[frame];
#pragma unroll
    for (int c = 0; c < C; ++c) xv[c] = inside ? x[((size_t)gy * W + gx) * C + c] : 0.0f;
    const int T = th * tw;
    for (int t0 = 0; t0 < T; t0 += kTapChunk) {
        const int nt = min(kTapChunk, T - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < nt * KP; e += blockDim.x) {
            const int t = e / KP, k = e - t * KP;
            hs[e] = k < K ? Ht[(size_t)(t0 + t) * K + k] : 0.0f;
        }
        __syncthreads();
        if (!inside) continue;
        for (int t = 0; t < nt; ++t) {
            const float4 *hv = (const float4 *)(hs + t * KP);
            float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
#pragma unroll
            for (int k4 = 0; k4 < KP / 4; ++k4) {
                const float4 h4 = hv[k4];
                g0 = fmaf(bq[4 * k4 + 0], h4.x, g0);
                g1 = fmaf(bq[4 * k4 + 1], h4.y, g1);
                g2 = fmaf(bq[4 * k4 + 2], h4.z, g2);
                g3 = fmaf(bq[4 * k4 + 3], h4.w, g3);
            }
            const float g = (g0 + g1) + (g2 + g3);
            const int tt = t0 + t, ty = tt / tw, tx = tt - ty * tw;
            const int dy = ly + ty, dx = lx + tx;  // tile index of p + o(t)
#pragma unroll
            for (int c = 0; c < C; ++c) atomicAdd(&as[(c * ar + dy) * ac + dx], g * xv[c]);
        }
    }
    __syncthreads();
    float *y = ptr.y[frame];
    for (int e = threadIdx.x; e < C * ar * ac; e += blockDim.x) {
        const int c = e / (ar * ac), rem = e - c * ar * ac, rr = rem / ac, cc = rem - rr * ac;
        const int oy = r0 + rr - th / 2, ox = c0 + cc - tw / 2;
        if (oy >= 0 && oy < H && ox >= 0 && ox < W) atomicAdd(&y[((size_t)oy * W + ox) * C + c], as[e]);
    }
}

template <int KP, int C>
p2s_status launch_blur_kp(int H, int W, int K, int th, int tw, int n, const BlurPtrs &ptr, const float *Ht,
                          const float *beta, p2s_blur_form form, cudaStream_t st) {
    dim3 grid((W + kTile - 1) / kTile, (H + kTile - 1) / kTile, n);
    const size_t smem =
        ((((size_t)C * (kTile + th - 1) * (kTile + tw - 1) + 3) & ~(size_t)3) + (size_t)kTapChunk * KP) * sizeof(float);
    if (form == P2S_GATHER) {
        P2S_CUDA(cudaFuncSetAttribute(blur_gather_simt<KP, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        blur_gather_simt<KP, C><<<grid, kTile * kTile, smem, st>>>(ptr, H, W, K, th, tw, Ht, beta);
    } else {
        P2S_CUDA(cudaFuncSetAttribute(blur_scatter_simt<KP, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        blur_scatter_simt<KP, C><<<grid, kTile * kTile, smem, st>>>(ptr, H, W, K, th, tw, Ht, beta);
    }
    P2S_CUDA(cudaGetLastError());
    return P2S_OK;
}

template <int C>
p2s_status launch_blur_c(int H, int W, int K, int th, int tw, int n, const BlurPtrs &ptr, const float *Ht,
                         const float *beta, p2s_blur_form form, cudaStream_t st) {
    if (K <= 32) return launch_blur_kp<32, C>(H, W, K, th, tw, n, ptr, Ht, beta, form, st);
    if (K <= 64) return launch_blur_kp<64, C>(H, W, K, th, tw, n, ptr, Ht, beta, form, st);
    return launch_blur_kp<128, C>(H, W, K, th, tw, n, ptr, Ht, beta, form, st);
}

}  // namespace

// Weight image layout of the plain network kernel: per layer W^T [in][out] then the
// bias padded to 4 floats.  Returns the image size in floats and the shared memory
// the kernel needs (the image plus two activation buffers).
static p2s_status mlp_simt_layout(const p2s_ctx *ctx, MlpLayers *lay, int *floats, size_t *smem) {
    if (ctx->n_layers > 4) {
        set_error("plain network path supports at most 4 layers");
        return P2S_EUNSUPPORTED;
    }
    lay->n = ctx->n_layers;
    int off = 0;
    for (int l = 0; l < lay->n; ++l) {
        lay->in[l] = ctx->dims[l];
        lay->out[l] = ctx->dims[l + 1];
        lay->w_off[l] = off;
        off += lay->in[l] * lay->out[l];
        lay->b_off[l] = off;
        off += (lay->out[l] + 3) & ~3;
        lay->relu[l] = l + 1 < lay->n;
    }
    *floats = off;
    *smem = (size_t)off * 4 + kMlpActBytes;
    if (*smem > kMlpSmemLimit) {
        set_error("network too large for the plain path (%zu bytes of shared memory)", *smem);
        return P2S_EUNSUPPORTED;
    }
    return P2S_OK;
}

// Fills the weight image `wimg` (device, `floats` long) from the context's per-layer
// copies and launches the kernel over n frames, all on stream `st`.
static p2s_status mlp_simt_run(const p2s_ctx *ctx, const MlpLayers &lay, int floats, size_t smem, const FieldGeom &g,
                               int n, float *wimg, const float *alpha, float *beta, cudaStream_t st) {
    for (int l = 0; l < lay.n; ++l) {
        P2S_CUDA(cudaMemcpyAsync(wimg + lay.w_off[l], ctx->d_Wt32[l], (size_t)lay.in[l] * lay.out[l] * 4,
                                 cudaMemcpyDeviceToDevice, st));
        P2S_CUDA(cudaMemcpyAsync(wimg + lay.b_off[l], ctx->d_b32[l], (size_t)lay.out[l] * 4, cudaMemcpyDeviceToDevice,
                                 st));
    }
    P2S_CUDA(cudaFuncSetAttribute(mlp_simt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const long long nblk = ((long long)g.H * g.W * n + kMlpThreads - 1) / kMlpThreads;
    const int grid = (int)(nblk < 2LL * sms ? nblk : 2LL * sms);
    double macs = 0.0;
    for (int l = 0; l < lay.n; ++l) macs += (double)lay.in[l] * lay.out[l];
    const double npx = (double)g.H * g.W * n;
    ProfScope pr(ctx, st, "mlp_fp32", 2.0 * macs * npx, npx * ctx->K * 4);
    mlp_simt_kernel<<<grid, kMlpThreads, smem, st>>>(lay, floats, n, g.H, g.W, g.s, 1.0f / g.s, g.Aw, g.Ah * g.Aw,
                                                     wimg, alpha, beta);
    P2S_CUDA(cudaGetLastError());
    return P2S_OK;
}

p2s_status launch_mlp_simt(const p2s_ctx *ctx, const FieldGeom &g, int n, const float *alpha, float *beta,
                           cudaStream_t st) {
    if (n <= 0) return P2S_OK;
    MlpLayers lay;
    int floats = 0;
    size_t smem = 0;
    p2s_status rc = mlp_simt_layout(ctx, &lay, &floats, &smem);
    if (rc != P2S_OK) return rc;
    // The weight image is assembled once per call from the per-layer device copies.
    float *wimg = nullptr;
    P2S_CUDA(cudaMallocAsync((void **)&wimg, (size_t)floats * 4, st));
    rc = mlp_simt_run(ctx, lay, floats, smem, g, n, wimg, alpha, beta, st);
    cudaFreeAsync(wimg, st);
    return rc;
}

p2s_status launch_blur_simt(const p2s_ctx *ctx, int H, int W, int C, int n, const float *const *xw,
                            const float *beta, float *const *y, p2s_blur_form form, cudaStream_t st) {
    if (n <= 0) return P2S_OK;
    if (n > kMaxBatch) {
        set_error("blur batch larger than %d", kMaxBatch);
        return P2S_EINVAL;
    }
    BlurPtrs ptr;
    for (int i = 0; i < n; ++i) {
        ptr.x[i] = xw[i];
        ptr.y[i] = y[i];
        if (form != P2S_GATHER) P2S_CUDA(cudaMemsetAsync(y[i], 0, (size_t)H * W * C * sizeof(float), st));
    }
    const double npx = (double)H * W * n;
    ProfScope pr(ctx, st, form == P2S_GATHER ? "blur_gather_fp32" : "blur_scatter_fp32",
                 npx * 2.0 * ctx->T * (ctx->K + C), npx * (2.0 * C + ctx->K) * 4);
    if (C == 3) return launch_blur_c<3>(H, W, ctx->K, ctx->th, ctx->tw, n, ptr, ctx->d_Ht32, beta, form, st);
    return launch_blur_c<1>(H, W, ctx->K, ctx->th, ctx->tw, n, ptr, ctx->d_Ht32, beta, form, st);
}

}  // namespace p2s

// ---- allocation-free variant of the FP32 network stage ---------------------
//
// Some callers cannot allocate device memory at the moment they want to run
// the network: code that runs under a fixed, pre-reserved memory budget, or a
// host thread that must not enter the CUDA allocator (for example while it
// records work that has to stay free of allocations).  p2s_stage_mlp
// assembles the network's weight image in a buffer it allocates per call;
// this variant assembles it in a file-scope device array instead, so the call
// allocates nothing.  Every GPU that loads the library holds the array until
// the process exits.

#include <mutex>

namespace p2s {
namespace {

// Weight image limit of the variant: the largest image the plain network kernel can
// stage in shared memory, (227 KiB - 64 KiB of activation buffers) / 4 = 41,728 floats
// (163 KiB).
constexpr int kNoAllocWeightFloats = (int)((kMlpSmemLimit - kMlpActBytes) / 4);
static __device__ __align__(256) float g_noalloc_weights[kNoAllocWeightFloats];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
float *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the array on `dev` (the current device).  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device with cudaGetSymbolAddress and cached.
p2s_status noalloc_weights_on(int dev, float **out) {
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("device ordinal %d out of range for the allocation-free scratch", dev);
        return P2S_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_weights);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress of the allocation-free scratch failed: %s", cudaGetErrorString(e));
            return P2S_ECUDA;
        }
        g_noalloc_ptr[dev] = (float *)p;
    }
    *out = g_noalloc_ptr[dev];
    return P2S_OK;
}

}  // namespace
}  // namespace p2s

extern "C" p2s_status p2s_stage_mlp_noalloc(p2s_ctx *ctx, int H, int W, const float *alpha, float *beta,
                                            void *stream) {
    using namespace p2s;
    if (!ctx || !alpha || !beta) {
        set_error("ctx, alpha and beta must be non-NULL");
        return P2S_EINVAL;
    }
    if (ctx->prec != P2S_FP32) {
        set_error("the allocation-free network stage serves FP32 contexts only");
        return P2S_EUNSUPPORTED;
    }
    FieldGeom g;
    p2s_status st = geometry(ctx, H, W, &g);
    if (st != P2S_OK) return st;
    MlpLayers lay;
    int floats = 0;
    size_t smem = 0;
    // Size check first: an image beyond the array is the caller's argument error.
    {
        int off = 0;
        for (int l = 0; l < ctx->n_layers; ++l) off += ctx->dims[l] * ctx->dims[l + 1] + ((ctx->dims[l + 1] + 3) & ~3);
        if (off > kNoAllocWeightFloats) {
            set_error("network weights need %d floats; the allocation-free scratch holds %d", off,
                      kNoAllocWeightFloats);
            return P2S_EINVAL;
        }
    }
    if ((st = mlp_simt_layout(ctx, &lay, &floats, &smem)) != P2S_OK) return st;
    int dev = -1;
    P2S_CUDA(cudaGetDevice(&dev));
    if (dev != ctx->device) {
        set_error("current device %d is not the context's device %d", dev, ctx->device);
        return P2S_EINVAL;
    }
    float *wimg = nullptr;
    if ((st = noalloc_weights_on(dev, &wimg)) != P2S_OK) return st;
    // The image is rewritten in full by every call; the padding floats after
    // each bias block are never read, so nothing needs clearing.
    return mlp_simt_run(ctx, lay, floats, smem, g, 1, wimg, alpha, beta, (cudaStream_t)stream);
}
