// The P2S network (Sec. 3.3) on the tensor cores as its own persistent
// kernel, writing beta in the 16-bit operand layout of the scatter blur.
//
// Work unit: 128 consecutive pixels of one image row (one TMEM lane each).
// Per unit: alpha_4..36 bilinear from the anchors (Sec. 3.4) -> layer 1
// (A from shared memory) -> ReLU -> layer 2 (A from TMEM, in place) -> ReLU
// -> layer 3 -> beta, rounded to the operand type and stored as
//     beta16[frame][row][g][col][8],  g = k / 8 (14 groups, K padded to 112),
// i.e. one 16-byte run of 8 consecutive k per (pixel, group).  The last
// layer's bias is left out; with `ones` set, entries k = K, K + 1 hold 1.0
// so that a basis carrying the bias PSF as an exact hi/lo pair of rows K,
// K + 1 adds it back in FP32-equivalent precision.  Entries beyond are 0.
//
// Two units are in flight per CTA: TMEM columns [256 s, 256 s + 256) belong
// to slot s, whose activations alternate between two 128-column regions.
// Roles: warp 0 issues the MMAs (one thread), warp 1 loads the weights once,
// warps 2..9 form two groups of four (one warp per TMEM lane quadrant), group
// s converting the units of slot s.  Every wait is bounded.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstring>

#include "p2s_internal.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace p2s {
namespace net {

using tcc::Ctl;
using tcc::drain_bar;
using tcc::pack2;
using tcc::wait_bar;

constexpr int kTile = 128;
constexpr int kThreads = 320;
constexpr int kK1 = 48;                    // layer-1 depth: 33 modes padded
constexpr int kGroups = 14;                // beta16 k-groups of 8 (K padded to 112)
constexpr int kA1Bytes = kTile * kK1 * 2;  // [6 k-groups][128 rows][16 B]
constexpr int kMaxItems = 6;
constexpr int kMaxAx = kTile + 1;           // anchor columns a 128-pixel unit touches (spacing 1)
constexpr int kRowBytes = (kMaxAx * kHiModes * 4 + 127) & ~127;  // interpolated anchor row, per group
static_assert(kRowBytes % 128 == 0 && kA1Bytes % 1024 == 0, "shared-memory offsets stay 16-byte aligned");

struct Params {
    const float *alpha;
    uint4 *beta16;
    const uint8_t *wstream;
    const float *bias;  // b1 [h1p], b2 [h2p]
    int *status;
    int n, H, W, s, Ah, Aw;
    float inv_s;
    int K, h1p, h2p, n3, ab_fmt, per, ones;
    int tiles_x, tiles_total;
    uint32_t wbytes;
    uint32_t item_off[kMaxItems], item_bytes[kMaxItems], item_n[kMaxItems], item_k[kMaxItems], item_soff[kMaxItems];
};

// barriers
enum Bar { kW = 0, kA1 = 1, kD1 = 3, kA2 = 5, kD2 = 7, kA3 = 9, kD3 = 11, kDone = 13, kNBar = 14 };

__host__ __device__ constexpr uint32_t colR0(int s) { return 256u * s; }
__host__ __device__ constexpr uint32_t colR1(int s) { return 256u * s + 128u; }

__global__ void __launch_bounds__(kThreads, 1) net_kernel(const __grid_constant__ Params p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = ptx::smem_u32(sm);
    const uint32_t offA1 = (p.wbytes + 1023) & ~1023u;
    const uint32_t offRow = offA1 + 2 * kA1Bytes;
    const uint32_t offBias = offRow + 2 * kRowBytes;
    const uint32_t offBar = offBias + (uint32_t)(p.h1p + p.h2p) * 4;
    const uint32_t offMisc = offBar + kNBar * 8;
    float *sbias = (float *)(sm + offBias);
    uint32_t *tmem_holder = (uint32_t *)(sm + offMisc);
    volatile int *abort_flag = (volatile int *)(sm + offMisc + 4);
    const uint32_t bar0 = sbase + offBar;
    auto BAR = [&](int i) { return bar0 + 8u * (uint32_t)i; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Ctl ctl{abort_flag, p.status};

    if (threadIdx.x == 0) {
        *abort_flag = 0;
        ptx::mbar_init(BAR(kW), 1);
        for (int s = 0; s < 2; ++s) {
            ptx::mbar_init(BAR(kA1 + s), 4);
            ptx::mbar_init(BAR(kD1 + s), 1);
            ptx::mbar_init(BAR(kA2 + s), 4);
            ptx::mbar_init(BAR(kD2 + s), 1);
            ptx::mbar_init(BAR(kA3 + s), 4);
            ptx::mbar_init(BAR(kD3 + s), 1);
        }
        ptx::mbar_init(BAR(kDone), 1);
        ptx::mbar_fence_init();
    }
    for (int i = threadIdx.x; i < p.h1p + p.h2p; i += blockDim.x) sbias[i] = p.bias[i];
    if (warp == 0) ptx::tmem_alloc(ptx::smem_u32(tmem_holder), 512);
    ptx::fence_before();
    __syncthreads();
    ptx::fence_after();
    const uint32_t tmem = *tmem_holder;
    const int n_local = p.tiles_total > (int)blockIdx.x ? (p.tiles_total - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp == 1) {
        // ---------------- weights, once ----------------
        if (lane == 0 && n_local > 0) {
            ptx::mbar_arrive_tx(BAR(kW), p.wbytes);
            for (int i = 0; i < 3 * p.per; ++i)
                ptx::bulk_g2s(sbase + p.item_soff[i], p.wstream + p.item_off[i], p.item_bytes[i], BAR(kW));
            drain_bar(BAR(kW), 0);
        }
    } else if (warp == 0) {
        // ---------------- MMA issuer ----------------
        if (lane == 0 && n_local > 0) {
            const bool wok = wait_bar(BAR(kW), 0, ctl, 1);
            ptx::fence_after();
            const int ready[3] = {kA1, kA2, kA3};
            const int done[3] = {kD1, kD2, kD3};
            for (int i0 = 0; i0 < n_local; i0 += 2) {
                for (int L = 0; L < 3; ++L) {
                    for (int j = i0; j < i0 + 2 && j < n_local; ++j) {
                        const int s = j & 1;
                        const uint32_t ph = (uint32_t)(j >> 1) & 1u;
                        const bool rdy = wait_bar(BAR(ready[L] + s), ph, ctl, 2);
                        ptx::fence_after();
                        if (rdy && wok) {
                            const uint32_t d = tmem + (L == 1 ? colR1(s) : colR0(s));
                            for (int w = 0; w < p.per; ++w) {
                                const int it = L * p.per + w;
                                const uint32_t n = p.item_n[it];
                                const int ksteps = (int)p.item_k[it] / 16;
                                const uint32_t idesc = ptx::idesc_f16(p.ab_fmt, (int)n);
                                const uint64_t bd = ptx::smem_desc(sbase + p.item_soff[it], n * 16, 128);
                                if (L == 0) {
                                    const uint64_t ad = ptx::smem_desc(sbase + offA1 + s * kA1Bytes, kTile * 16, 128);
                                    for (int ks = 0; ks < ksteps; ++ks)
                                        ptx::mma_ss(d, ad + (uint64_t)(ks * 2 * kTile), bd + (uint64_t)(ks * 2 * n), idesc,
                                                    (w > 0 || ks > 0) ? 1u : 0u);
                                } else {
                                    const uint32_t a = tmem + (L == 1 ? colR0(s) : colR1(s));
                                    for (int ks = 0; ks < ksteps; ++ks)
                                        ptx::mma_ts(d, a + ks * 8, bd + (uint64_t)(ks * 2 * n), idesc,
                                                    (w > 0 || ks > 0) ? 1u : 0u);
                                }
                            }
                        }
                        ptx::mma_commit(BAR(done[L] + s));
                    }
                }
            }
            // every MMA has completed before tensor memory is released
            ptx::mma_commit(BAR(kDone));
            drain_bar(BAR(kDone), 0);
        }
    } else {
        // ---------------- two groups of four converting warps ----------------
        const int grp = (warp - 2) >> 2;
        const int quad = warp & 3;
        const int m = quad * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
        const uint32_t r0 = lane_base + colR0(grp), r1 = lane_base + colR1(grp);
        uint8_t *a1 = sm + offA1 + grp * kA1Bytes;
        for (int i = grp; i < n_local; i += 2) {
            const uint32_t ph = (uint32_t)(i >> 1) & 1u;
            const int tile = (int)blockIdx.x + i * (int)gridDim.x;
            const int per_frame = p.H * p.tiles_x;
            const int f = tile / per_frame;
            const int rem = tile - f * per_frame;
            const int row = rem / p.tiles_x;
            const int col = (rem - row * p.tiles_x) * kTile + m;
            bool ok = true;
            // ---- layer-1 operand: alpha_4..36 at (row, col), bilinear from the anchors.
            //      The group first interpolates the two anchor rows at this image row
            //      (shared by all 128 pixels), then each pixel interpolates along x. ----
            {
                float *arow = (float *)(sm + offRow + grp * kRowBytes);
                const int c0 = col - m;
                const int ay = row / p.s;
                const float fy = (float)(row - ay * p.s) * p.inv_s;
                const int ax0 = min(c0, p.W - 1) / p.s;
                const int nax = min(min(c0 + kTile - 1, p.W - 1) / p.s + 2, p.Aw) - ax0;
                const float *a = p.alpha + ((size_t)f * p.Ah * p.Aw + (size_t)ay * p.Aw + ax0) * kAlphaStride;
                const float *b = a + (size_t)p.Aw * kAlphaStride;
                for (int e = m; e < nax * kHiModes; e += kTile) {
                    const int ax = e / kHiModes, k = e - ax * kHiModes;
                    const int off = ax * kAlphaStride + k + 3;
                    arow[e] = (1.0f - fy) * __ldg(a + off) + fy * __ldg(b + off);
                }
                ptx::named_bar(2 + grp, kTile);
                const int gj = min(col, p.W - 1);
                const int ax = gj / p.s - ax0;
                const float fx = (float)(gj - (ax + ax0) * p.s) * p.inv_s;
                const float *r0p = arow + ax * kHiModes;
                const float *r1p = r0p + (ax + 1 < nax ? kHiModes : 0);
                float v[kK1];
#pragma unroll
                for (int k = 0; k < kK1; ++k) v[k] = k < kHiModes ? (1.0f - fx) * r0p[k] + fx * r1p[k] : 0.f;
#pragma unroll
                for (int g = 0; g < kK1 / 8; ++g) {
                    uint4 u;
                    u.x = pack2(v[8 * g + 0], v[8 * g + 1], p.ab_fmt);
                    u.y = pack2(v[8 * g + 2], v[8 * g + 3], p.ab_fmt);
                    u.z = pack2(v[8 * g + 4], v[8 * g + 5], p.ab_fmt);
                    u.w = pack2(v[8 * g + 6], v[8 * g + 7], p.ab_fmt);
                    *(uint4 *)(a1 + g * (kTile * 16) + m * 16) = u;
                }
                ptx::fence_proxy_async();
                ptx::fence_before();
                // every pixel has read the anchor row before the group's next unit rewrites it
                ptx::named_bar(2 + grp, kTile);
                if (lane == 0) ptx::mbar_arrive(BAR(kA1 + grp));
            }
            // ---- layers 1, 2: D -> bias, ReLU -> packed activations in place ----
            const int done[2] = {kD1, kD2};
            const int ready[2] = {kA2, kA3};
            const uint32_t dreg[2] = {r0, r1};
            const int width[2] = {p.h1p, p.h2p};
            const int boff[2] = {0, p.h1p};
#pragma unroll 1
            for (int L = 0; L < 2; ++L) {
                ok = __all_sync(0xffffffffu, wait_bar(BAR(done[L] + grp), ph, ctl, 4) && ok);
                ptx::fence_after();
                if (ok) {
                    // TMEM loads double-buffered: chunk q + 1 is in flight while q converts
                    const int nq = width[L] / 32;
                    uint32_t d[2][32];
                    ptx::tmem_ld32(dreg[L], d[0]);
#pragma unroll 1
                    for (int q = 0; q < nq; q += 2) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int qq = q + h;
                            if (qq < nq) {
                                ptx::tmem_wait_ld_dep(d[h]);
                                if (qq + 1 < nq) ptx::tmem_ld32(dreg[L] + 32 * (qq + 1), d[h ^ 1]);
                                const float4 *bv = (const float4 *)(sbias + boff[L] + 32 * qq);
                                uint32_t u[16];
#pragma unroll
                                for (int j = 0; j < 8; ++j) {
                                    const float4 bb = bv[j];
                                    const float h0 = fmaxf(__uint_as_float(d[h][4 * j]) + bb.x, 0.f);
                                    const float h1 = fmaxf(__uint_as_float(d[h][4 * j + 1]) + bb.y, 0.f);
                                    const float h2 = fmaxf(__uint_as_float(d[h][4 * j + 2]) + bb.z, 0.f);
                                    const float h3 = fmaxf(__uint_as_float(d[h][4 * j + 3]) + bb.w, 0.f);
                                    u[2 * j] = pack2(h0, h1, p.ab_fmt);
                                    u[2 * j + 1] = pack2(h2, h3, p.ab_fmt);
                                }
                                const uint32_t(&u0)[8] = *reinterpret_cast<const uint32_t(*)[8]>(&u[0]);
                                const uint32_t(&u1)[8] = *reinterpret_cast<const uint32_t(*)[8]>(&u[8]);
                                ptx::tmem_st8(dreg[L] + 16 * qq, u0);
                                ptx::tmem_st8(dreg[L] + 16 * qq + 8, u1);
                            }
                        }
                    }
                }
                ptx::tmem_wait_st();
                ptx::fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(BAR(ready[L] + grp));
            }
            // ---- layer 3: beta (no bias) -> 16-bit groups of 8 in global memory ----
            ok = __all_sync(0xffffffffu, wait_bar(BAR(kD3 + grp), ph, ctl, 8) && ok);
            ptx::fence_after();
            const bool store = ok && f < p.n && col < p.W;
            uint4 *dst = p.beta16 + ((size_t)(f * p.H + row) * kGroups) * p.W + col;
            uint32_t d[2][16];
            if (ok) ptx::tmem_ld16(r0, d[0]);
#pragma unroll 1
            for (int q = 0; q < kGroups / 2; q += 2) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int qq = q + h;
                    if (qq < kGroups / 2) {
                        if (ok) {
                            ptx::tmem_wait_ld_dep(d[h]);
                            if (qq + 1 < kGroups / 2 && 16 * (qq + 1) < p.n3) ptx::tmem_ld16(r0 + 16 * (qq + 1), d[h ^ 1]);
                        }
                        float v[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int k = 16 * qq + j;
                            v[j] = k < p.K ? __uint_as_float(d[h][j])
                                           : ((p.ones && (k == p.K || k == p.K + 1)) ? 1.0f : 0.0f);
                        }
                        if (store) {
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                uint4 u;
                                u.x = pack2(v[8 * e + 0], v[8 * e + 1], p.ab_fmt);
                                u.y = pack2(v[8 * e + 2], v[8 * e + 3], p.ab_fmt);
                                u.z = pack2(v[8 * e + 4], v[8 * e + 5], p.ab_fmt);
                                u.w = pack2(v[8 * e + 6], v[8 * e + 7], p.ab_fmt);
                                dst[(size_t)(2 * qq + e) * p.W] = u;
                            }
                        }
                    }
                }
            }
            if (ok) ptx::tmem_wait_ld();
            // D3 fully read before this slot's next layer-1 result lands in r0
            ptx::fence_before();
        }
    }
    // ---------------- teardown ----------------
    ptx::fence_before();
    __syncthreads();
    if (warp == 0) {
        ptx::fence_after();
        ptx::tmem_dealloc(tmem, 512);
    }
}

// beta FP32 [n][H][W][K] -> beta16 (no bias fold: entries k >= K are 0)
__global__ void pack16_kernel(const float *__restrict__ beta, uint4 *__restrict__ out, long long npx, int W, int K,
                              int fmt) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (pixel, group)
    if (i >= npx * kGroups) return;
    const long long px = i / kGroups;
    const int g = (int)(i - px * kGroups);
    const long long rowf = px / W;  // frame * H + row
    const int col = (int)(px - rowf * W);
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int k = 8 * g + j;
        v[j] = k < K ? __ldg(beta + px * K + k) : 0.f;
    }
    uint4 u;
    u.x = pack2(v[0], v[1], fmt);
    u.y = pack2(v[2], v[3], fmt);
    u.z = pack2(v[4], v[5], fmt);
    u.w = pack2(v[6], v[7], fmt);
    out[(rowf * kGroups + g) * W + col] = u;
}

}  // namespace net

using namespace net;

size_t beta16_bytes(int H, int W, int n) { return (size_t)n * H * W * kGroups * 16; }

int net_smem_bytes(const p2s_ctx *ctx) {
    uint32_t w = 0;
    const Item16 *it = (const Item16 *)ctx->tc_items.data();
    for (int i = 0; i < ctx->tc.n_mlp; ++i) w += it[i].bytes;
    const uint32_t offA1 = (w + 1023) & ~1023u;
    return (int)(offA1 + 2 * kA1Bytes + 2 * kRowBytes + (ctx->tc.h1p + ctx->tc.h2p) * 4 + kNBar * 8 + 16 + 1024);
}

p2s_status launch_net16(p2s_ctx *ctx, const FieldGeom &g, int n, const float *alpha, void *beta16, int ones,
                        int *status, cudaStream_t st) {
    if (n <= 0) return P2S_OK;
    p2s_status s0 = tc_prepare(ctx);
    if (s0 != P2S_OK) return s0;
    Params p;
    std::memset(&p, 0, sizeof p);
    p.alpha = alpha;
    p.beta16 = (uint4 *)beta16;
    p.wstream = (const uint8_t *)ctx->tc.d_H;
    p.bias = ctx->tc.d_bias;
    p.status = status;
    p.n = n;
    p.H = g.H;
    p.W = g.W;
    p.s = g.s;
    p.Ah = g.Ah;
    p.Aw = g.Aw;
    p.inv_s = 1.0f / (float)g.s;
    p.K = ctx->K;
    p.h1p = ctx->tc.h1p;
    p.h2p = ctx->tc.h2p;
    p.n3 = ctx->tc.n3;
    p.ab_fmt = ctx->tc.fmt;
    p.per = ctx->tc.split ? 2 : 1;
    p.ones = ones;
    p.tiles_x = (g.W + kTile - 1) / kTile;
    p.tiles_total = p.tiles_x * g.H * n;
    const Item16 *it = (const Item16 *)ctx->tc_items.data();
    uint32_t soff = 0;
    for (int i = 0; i < 3 * p.per; ++i) {
        p.item_off[i] = it[i].offset;
        p.item_bytes[i] = it[i].bytes;
        p.item_n[i] = it[i].n;
        p.item_k[i] = it[i].k;
        p.item_soff[i] = soff;
        soff += it[i].bytes;
    }
    p.wbytes = soff;
    const int smem = net_smem_bytes(ctx);
    if (smem > 227 * 1024) {
        set_error("network weights too large for the tensor-core network kernel (%d B of shared memory)", smem);
        return P2S_EUNSUPPORTED;
    }
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const int grid = p.tiles_total < sms ? p.tiles_total : sms;
    const double npx = (double)g.H * g.W * n;
    double macs = 0.0;
    for (int l = 0; l < 3; ++l) macs += (double)ctx->dims[l] * ctx->dims[l + 1];
    ProfScope pr(ctx, st, "net_tc", 2.0 * macs * npx, npx * kGroups * 16.0);
    P2S_CUDA(cudaFuncSetAttribute(net_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    net_kernel<<<grid, kThreads, smem, st>>>(p);
    P2S_CUDA(cudaGetLastError());
    return P2S_OK;
}

p2s_status launch_pack16(p2s_ctx *ctx, int H, int W, int n, const float *beta, void *beta16, cudaStream_t st) {
    p2s_status s0 = tc_prepare(ctx);
    if (s0 != P2S_OK) return s0;
    const long long npx = (long long)n * H * W;
    const long long work = npx * kGroups;
    if (work == 0) return P2S_OK;
    ProfScope pr(ctx, st, "pack_beta16", 0.0, npx * (ctx->K * 4.0 + kGroups * 16.0));
    pack16_kernel<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(beta, (uint4 *)beta16, npx, W, ctx->K, ctx->tc.fmt);
    P2S_CUDA(cudaGetLastError());
    return P2S_OK;
}

}  // namespace p2s
