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
// Two units are in flight per CTA, one per slot.  A slot owns 192 TMEM
// columns: D of the current layer in [0, 128), the next layer's 16-bit A
// operand in [128, 192), so no conversion writes over columns still being
// read.  Roles: warp 0 issues the MMAs (one thread, serving whichever slot is
// ready), warp 1 loads the weights once, warps 2..17 form two slots of eight
// converting warps, two per TMEM lane quadrant, each taking half of every
// layer's columns.  A CTA takes a contiguous run of units ordered row-fastest
// within a 128-column block, so consecutive units share anchor rows (L1 hits).
// Every wait is bounded.
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
constexpr int kConvWarps = 8;               // per slot: two per TMEM lane quadrant
constexpr int kConv = 32 * kConvWarps;      // converting threads per slot
constexpr int kThreads = 64 + 2 * kConv;    // + MMA warp + weight-loader warp
constexpr int kK1 = 48;                     // layer-1 depth: 33 modes padded
constexpr int kGroups = 14;                 // beta16 k-groups of 8 (K padded to 112)
constexpr int kA1Bytes = kTile * kK1 * 2;   // [6 k-groups][128 rows][16 B]
constexpr int kMaxItems = 6;
constexpr int kMaxAx = kTile + 1;           // anchor columns a 128-pixel unit touches (spacing 1)
constexpr int kRowBytes = (kMaxAx * kHiModes * 4 + 127) & ~127;  // interpolated anchor row, per slot
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
    int tiles_x, tiles_total, per_cta;
    uint32_t wbytes;
    uint32_t item_off[kMaxItems], item_bytes[kMaxItems], item_n[kMaxItems], item_k[kMaxItems], item_soff[kMaxItems];
};

// barriers
enum Bar { kW = 0, kA1 = 1, kD1 = 3, kA2 = 5, kD2 = 7, kA3 = 9, kD3 = 11, kDone = 13, kNBar = 14 };

__host__ __device__ constexpr uint32_t colD(int s) { return 256u * s; }         // 128 columns
__host__ __device__ constexpr uint32_t colA(int s) { return 256u * s + 128u; }  // 64 columns

template <int FMT>  // operand type: 0 FP16, 1 BF16
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
            ptx::mbar_init(BAR(kA1 + s), kConvWarps);
            ptx::mbar_init(BAR(kD1 + s), 1);
            ptx::mbar_init(BAR(kA2 + s), kConvWarps);
            ptx::mbar_init(BAR(kD2 + s), 1);
            ptx::mbar_init(BAR(kA3 + s), kConvWarps);
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
    const int u_base = (int)blockIdx.x * p.per_cta;
    const int n_local = max(0, min(p.per_cta, p.tiles_total - u_base));

    if (warp == 1) {
        // ---------------- weights, once ----------------
        if (lane == 0 && n_local > 0) {
            ptx::mbar_arrive_tx(BAR(kW), p.wbytes);
            for (int i = 0; i < 3 * p.per; ++i)
                ptx::bulk_g2s(sbase + p.item_soff[i], p.wstream + p.item_off[i], p.item_bytes[i], BAR(kW));
            drain_bar(BAR(kW), 0);
        }
    } else if (warp == 0) {
        // ---------------- MMA issuer: next layer of whichever slot is ready ----------------
        if (lane == 0 && n_local > 0) {
            const bool wok = wait_bar(BAR(kW), 0, ctl, 1);
            ptx::fence_after();
            int js[2] = {0, 1}, Ls[2] = {0, 0};
            long long t0 = clock64();
            while (js[0] < n_local || js[1] < n_local) {
                bool prog = false;
                for (int s = 0; s < 2; ++s) {
                    if (js[s] >= n_local) continue;
                    const int L = Ls[s];
                    const bool aborted = *abort_flag != 0;
                    const int rdy = L == 0 ? kA1 : (L == 1 ? kA2 : kA3);
                    const int dn = L == 0 ? kD1 : (L == 1 ? kD2 : kD3);
                    if (!aborted && !ptx::mbar_test(BAR(rdy + s), (uint32_t)(js[s] >> 1) & 1u)) continue;
                    ptx::fence_after();
                    if (!aborted && wok) {
                        const uint32_t d = tmem + colD(s);
                        for (int w = 0; w < p.per; ++w) {
                            const int it = L * p.per + w;
                            const uint32_t n = p.item_n[it];
                            const int ksteps = (int)p.item_k[it] / 16;
                            const uint32_t idesc = ptx::idesc_f16(FMT, (int)n);
                            const uint64_t bd = ptx::smem_desc(sbase + p.item_soff[it], n * 16, 128);
                            if (L == 0) {
                                const uint64_t ad = ptx::smem_desc(sbase + offA1 + s * kA1Bytes, kTile * 16, 128);
                                for (int ks = 0; ks < ksteps; ++ks)
                                    ptx::mma_ss(d, ad + (uint64_t)(ks * 2 * kTile), bd + (uint64_t)(ks * 2 * n), idesc,
                                                (w > 0 || ks > 0) ? 1u : 0u);
                            } else {
                                const uint32_t a = tmem + colA(s);
                                for (int ks = 0; ks < ksteps; ++ks)
                                    ptx::mma_ts(d, a + ks * 8, bd + (uint64_t)(ks * 2 * n), idesc,
                                                (w > 0 || ks > 0) ? 1u : 0u);
                            }
                        }
                    }
                    ptx::mma_commit(BAR(dn + s));
                    if (++Ls[s] == 3) {
                        Ls[s] = 0;
                        js[s] += 2;
                    }
                    prog = true;
                }
                if (prog) {
                    t0 = clock64();
                } else if (clock64() - t0 > 4000000000ll) {
                    *abort_flag = 1;
                    atomicOr(p.status, 2);
                }
            }
            // every MMA has completed before tensor memory is released
            ptx::mma_commit(BAR(kDone));
            drain_bar(BAR(kDone), 0);
        }
    } else {
        // ---------------- two slots of eight converting warps ----------------
        const int e = warp - 2;
        const int slot = e / kConvWarps;
        const int half = (e % kConvWarps) >> 2;  // which half of each layer's columns
        const int quad = warp & 3;
        const int m = quad * 32 + lane;
        const int tid = threadIdx.x - 64 - slot * kConv;
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
        const uint32_t dcol = lane_base + colD(slot), acol = lane_base + colA(slot);
        uint8_t *a1 = sm + offA1 + slot * kA1Bytes;
        float *arow = (float *)(sm + offRow + slot * kRowBytes);
        const int per_frame = p.H * p.tiles_x;
        for (int i = slot; i < n_local; i += 2) {
            const uint32_t ph = (uint32_t)(i >> 1) & 1u;
            const int u = u_base + i;
            const int f = u / per_frame;
            const int rem = u - f * per_frame;
            const int tcol = rem / p.H;
            const int row = rem - tcol * p.H;
            const int c0 = tcol * kTile;
            const int col = c0 + m;
            bool ok = true;
            // ---- layer-1 operand: alpha_4..36 at (row, col), bilinear from the anchors.
            //      The slot first interpolates the two anchor rows at this image row
            //      (shared by all 128 pixels), then each pixel interpolates along x. ----
            {
                const int ay = row / p.s;
                const float fy = (float)(row - ay * p.s) * p.inv_s;
                const int ax0 = min(c0, p.W - 1) / p.s;
                const int nax = min(min(c0 + kTile - 1, p.W - 1) / p.s + 2, p.Aw) - ax0;
                const float *a = p.alpha + ((size_t)f * p.Ah * p.Aw + (size_t)ay * p.Aw + ax0) * kAlphaStride;
                const float *b = a + (size_t)p.Aw * kAlphaStride;
                // every pixel has read the previous unit's anchor row
                ptx::named_bar(2 + slot, kConv);
                for (int e2 = tid; e2 < nax * kHiModes; e2 += kConv) {
                    const int ax = e2 / kHiModes, k = e2 - ax * kHiModes;
                    const int off = ax * kAlphaStride + k + 3;
                    arow[e2] = (1.0f - fy) * __ldg(a + off) + fy * __ldg(b + off);
                }
                ptx::named_bar(2 + slot, kConv);
                const int gj = min(col, p.W - 1);
                const int ax = gj / p.s - ax0;
                const float fx = (float)(gj - (ax + ax0) * p.s) * p.inv_s;
                const float *r0p = arow + ax * kHiModes;
                const float *r1p = r0p + (ax + 1 < nax ? kHiModes : 0);
                // this warp's 24 of the 48 inputs (k-groups 3 half .. 3 half + 2)
                float v[kK1 / 2];
#pragma unroll
                for (int k = 0; k < kK1 / 2; ++k) {
                    const int kk = (kK1 / 2) * half + k;
                    v[k] = kk < kHiModes ? (1.0f - fx) * r0p[kk] + fx * r1p[kk] : 0.f;
                }
#pragma unroll
                for (int g = 0; g < kK1 / 16; ++g) {
                    uint4 q;
                    q.x = pack2(v[8 * g + 0], v[8 * g + 1], FMT);
                    q.y = pack2(v[8 * g + 2], v[8 * g + 3], FMT);
                    q.z = pack2(v[8 * g + 4], v[8 * g + 5], FMT);
                    q.w = pack2(v[8 * g + 6], v[8 * g + 7], FMT);
                    *(uint4 *)(a1 + ((kK1 / 16) * half + g) * (kTile * 16) + m * 16) = q;
                }
                ptx::fence_proxy_async();
                ptx::fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(BAR(kA1 + slot));
            }
            // ---- layers 1, 2: D -> bias, ReLU -> packed activations (the next A) ----
#pragma unroll 1
            for (int L = 0; L < 2; ++L) {
                const int width = L ? p.h2p : p.h1p, boff = L ? p.h1p : 0;
                ok = __all_sync(0xffffffffu, wait_bar(BAR((L ? kD2 : kD1) + slot), ph, ctl, 4) && ok);
                ptx::fence_after();
                // columns [64 half, 64 half + 64) of D, 32 per TMEM load
                const int ncol = ok ? max(0, min(64, width - 64 * half)) : 0;
#pragma unroll 1
                for (int c32 = 0; c32 < ncol; c32 += 32) {
                    uint32_t d[32];
                    ptx::tmem_ld32(dcol + 64 * half + c32, d);
                    ptx::tmem_wait_ld_dep(d);
#pragma unroll
                    for (int qq = 0; qq < 2; ++qq) {
                        const float4 *bv = (const float4 *)(sbias + boff + 64 * half + c32 + 16 * qq);
                        uint32_t w8[8];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float4 bb = bv[j];
                            const float h0 = fmaxf(__uint_as_float(d[16 * qq + 4 * j]) + bb.x, 0.f);
                            const float h1 = fmaxf(__uint_as_float(d[16 * qq + 4 * j + 1]) + bb.y, 0.f);
                            const float h2 = fmaxf(__uint_as_float(d[16 * qq + 4 * j + 2]) + bb.z, 0.f);
                            const float h3 = fmaxf(__uint_as_float(d[16 * qq + 4 * j + 3]) + bb.w, 0.f);
                            w8[2 * j] = pack2(h0, h1, FMT);
                            w8[2 * j + 1] = pack2(h2, h3, FMT);
                        }
                        ptx::tmem_st8(acol + 32 * half + c32 / 2 + 8 * qq, w8);
                    }
                }
                ptx::tmem_wait_st();
                ptx::fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(BAR((L ? kA3 : kA2) + slot));
            }
            // ---- layer 3: beta (no bias) -> 16-bit groups of 8 in global memory;
            //      this warp stores k-groups [7 half, 7 half + 7) ----
            ok = __all_sync(0xffffffffu, wait_bar(BAR(kD3 + slot), ph, ctl, 8) && ok);
            ptx::fence_after();
            const bool store = ok && f < p.n && col < p.W;
            uint4 *dst = p.beta16 + ((size_t)(f * p.H + row) * kGroups) * p.W + col;
            const int g0 = (kGroups / 2) * half;
#pragma unroll 1
            for (int c32 = 0; c32 < 64; c32 += 32) {  // groups g0 + c32 / 8 .. + 3 (7 in all)
                uint32_t d[32];
                if (ok) {
                    ptx::tmem_ld32(dcol + 8 * g0 + c32, d);
                    ptx::tmem_wait_ld_dep(d);
                }
                if (store) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int g = g0 + c32 / 8 + q;
                        if (g < g0 + kGroups / 2) {
                            float v[8];
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const int k = 8 * g + j;
                                v[j] = k < p.K ? __uint_as_float(d[8 * q + j])
                                               : ((p.ones && (k == p.K || k == p.K + 1)) ? 1.0f : 0.0f);
                            }
                            uint4 w4;
                            w4.x = pack2(v[0], v[1], FMT);
                            w4.y = pack2(v[2], v[3], FMT);
                            w4.z = pack2(v[4], v[5], FMT);
                            w4.w = pack2(v[6], v[7], FMT);
                            dst[(size_t)g * p.W] = w4;
                        }
                    }
                }
            }
            // D3 fully read before this slot's next layer-1 result lands in its D columns
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
    // contiguous runs of units per CTA (row-fastest order inside a column block)
    p.per_cta = (p.tiles_total + sms - 1) / sms;
    const int grid = (p.tiles_total + p.per_cta - 1) / p.per_cta;
    const double npx = (double)g.H * g.W * n;
    double macs = 0.0;
    for (int l = 0; l < 3; ++l) macs += (double)ctx->dims[l] * ctx->dims[l + 1];
    ProfScope pr(ctx, st, "net_tc", 2.0 * macs * npx, npx * kGroups * 16.0);
    if (p.ab_fmt == 1) {
        P2S_CUDA(cudaFuncSetAttribute(net_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        net_kernel<1><<<grid, kThreads, smem, st>>>(p);
    } else {
        P2S_CUDA(cudaFuncSetAttribute(net_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        net_kernel<0><<<grid, kThreads, smem, st>>>(p);
    }
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
