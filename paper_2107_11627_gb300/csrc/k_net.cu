// The P2S network (Sec. 3.3) on the tensor cores as its own persistent
// kernel, writing beta in the 16-bit operand layout that the blur-only
// tensor-core kernels (gather and scatter) read.
//
// Work unit: 128 consecutive pixels of one image row (one TMEM lane each).
// Per unit: alpha_4..36 bilinear from the anchors (Sec. 3.4) -> layer 1 ->
// ReLU -> layer 2 -> ReLU -> layer 3 (every A operand from shared memory) ->
// beta, rounded to the operand type and stored as
//     beta16[frame][row][g][col][8],  g = k / 8 (14 groups, K padded to 112),
// i.e. one 16-byte run of 8 consecutive k per (pixel, group).  The last
// layer's bias is left out; with `ones` set, entries k = K, K + 1 hold 1.0
// so that a basis carrying the bias PSF as an exact hi/lo pair of rows K,
// K + 1 adds it back in FP32-equivalent precision.  Entries beyond are 0.
//
// Up to four units are in flight per CTA, one per slot: every layer's A
// operand sits in the slot's 32 KB of shared memory (A1, then A2, then A3 in
// the same buffer), so a slot needs only the 128 TMEM columns of its D.  The
// slot count is the largest that fits the weights and anchor rows in shared
// memory (4 for FP16 weights at anchor spacing 8, 2 for the BF16 hi/lo pair).
// Roles: one MMA-issuing thread per slot (warp 0 also loads the weights, warps
// 4 NS + s issue for slots s >= 1): a single thread issues an MMA only every
// 76-100 cycles, several threads keep the tensor core busy.  Four converting
// warps per slot, one per TMEM lane quadrant (warps 1 .. 4 NS).  A CTA takes a contiguous run of units ordered
// row-fastest within a 128-column block, so consecutive units share anchor
// rows (L1 hits).  Every wait is bounded.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
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
constexpr int kMaxSlots = 4;
constexpr int kThreads = kMaxSlots * 160;        // per slot: four converting warps and one MMA warp
constexpr int kK1 = 48;                         // layer-1 depth: 33 modes padded
constexpr int kGroups = 14;                     // beta16 k-groups of 8 (K padded to 112)
constexpr int kGroups8 = 16;                    // FP8 beta: 8 hi + 8 lo groups of 16 k (K padded to 128)
constexpr int kABytes = kTile * 128 * 2;        // A operand of one slot: [16 k-groups][128 rows][16 B]
constexpr int kMaxItems = 6;

// One frame of a launch: its anchors ([Ah][Aw][36]), its beta block, its size, and the
// index of its first unit (units run frame by frame, column block by column block, row-fastest).
struct Frame {
    const float *alpha;
    uint4 *beta;
    int H, W, Aw, pitch, tiles_x, u0;
};

struct Params {
    Frame fr[kMaxBatch];
    int nf;
    const uint8_t *wstream;
    const float *bias;  // b1 [h1p], b2 [h2p]
    int *status;
    int s;
    float inv_s;
    int K, h1p, h2p, n3, ab_fmt, per, ones, perm;
    const float *scale8;  // non-null: write beta as E4M3 hi/lo pairs, beta_k multiplied by scale8[k]
    int tiles_total, per_cta, nslots;
    uint32_t wbytes, offA, offRow, rowBytes, offBias, offBar, offMisc;
    uint32_t item_off[kMaxItems], item_bytes[kMaxItems], item_n[kMaxItems], item_k[kMaxItems], item_soff[kMaxItems];
};

// barriers: kW, then per slot {A1, D1, A2, D2, A3, D3}, then kDone
enum Bar { kW = 0, kSlotBar0 = 1, kDone = 1 + 6 * kMaxSlots, kNBar = kDone + 1 };
__host__ __device__ constexpr int barA(int s, int L) { return kSlotBar0 + 6 * s + 2 * L; }      // operand L ready
__host__ __device__ constexpr int barD(int s, int L) { return kSlotBar0 + 6 * s + 2 * L + 1; }  // D of layer L done

// A unit's place in the batch and the anchors it interpolates from: rows ay
// (a) and ay + 1 (b) of frame f's anchor grid, columns ax0 .. ax0 + nax - 1.
struct UnitGeom {
    int f, row, c0, ax0, nax;
    float fy;
    const float *a, *b;
};

// the frame of unit u, searched forward from frame f (a slot's units only increase)
__device__ __forceinline__ int frame_of(const Params &p, int u, int f) {
    while (f + 1 < p.nf && u >= p.fr[f + 1].u0) ++f;
    return f;
}

__device__ __forceinline__ UnitGeom unit_geom(const Params &p, int u, int f) {
    UnitGeom g;
    const Frame &F = p.fr[f];
    g.f = f;
    const int rem = u - F.u0;
    const int tcol = rem / F.H;
    g.row = rem - tcol * F.H;
    g.c0 = tcol * kTile;
    const int ay = g.row / p.s;
    g.fy = (float)(g.row - ay * p.s) * p.inv_s;
    g.ax0 = min(g.c0, F.W - 1) / p.s;
    g.nax = min(min(g.c0 + kTile - 1, F.W - 1) / p.s + 2, F.Aw) - g.ax0;
    g.a = F.alpha + ((size_t)ay * F.Aw + g.ax0) * kAlphaStride;
    g.b = g.a + (size_t)F.Aw * kAlphaStride;
    return g;
}

// element e2 of an interpolated anchor row (anchor e2 / 33, mode 4 + e2 % 33)
// as an offset from the row's first anchor
__device__ __forceinline__ int anchor_off(int e2) {
    const int ax = e2 / kHiModes, k = e2 - ax * kHiModes;
    return ax * kAlphaStride + k + 3;
}

constexpr int kPre = 5;  // anchor-row elements per thread loaded one unit ahead (covers 18 anchors)
constexpr int kRowStride = 36;  // floats per interpolated anchor in shared memory (33 modes, 16-byte rows)

// shared-memory index of element e2 (anchor e2 / 33, mode e2 % 33) of an interpolated anchor row
__device__ __forceinline__ int arow_idx(int e2) {
    const int ax = e2 / kHiModes;
    return ax * kRowStride + (e2 - ax * kHiModes);
}

template <int FMT>  // operand type: 0 FP16, 1 BF16
__global__ void __launch_bounds__(kThreads, 1) net_kernel(const __grid_constant__ Params p) {
    extern __shared__ uint8_t smem_raw[];
    // aligned by pointer arithmetic on the __shared__ array, so that the compiler still
    // knows every access through `sm` is to shared memory (ld/st.shared, not generic)
    uint8_t *sm = smem_raw + ((1024u - (uint32_t)((uintptr_t)smem_raw & 1023u)) & 1023u);
    const uint32_t sbase = ptx::smem_u32(sm);
    float *sbias = (float *)(sm + p.offBias);
    uint32_t *tmem_holder = (uint32_t *)(sm + p.offMisc);
    volatile int *abort_flag = (volatile int *)(sm + p.offMisc + 4);
    const uint32_t bar0 = sbase + p.offBar;
    auto BAR = [&](int i) { return bar0 + 8u * (uint32_t)i; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NS = p.nslots;
    Ctl ctl{abort_flag, p.status};
    const int u_base = (int)blockIdx.x * p.per_cta;
    const int n_local = max(0, min(p.per_cta, p.tiles_total - u_base));
    const int n_issuers = min(NS, n_local);  // slots with work

    if (threadIdx.x == 0) {
        *abort_flag = 0;
        ptx::mbar_init(BAR(kW), 1);
        for (int s = 0; s < NS; ++s)
            for (int L = 0; L < 3; ++L) {
                ptx::mbar_init(BAR(barA(s, L)), 4);
                ptx::mbar_init(BAR(barD(s, L)), 1);
            }
        ptx::mbar_init(BAR(kDone), n_issuers > 0 ? n_issuers : 1);
        ptx::mbar_fence_init();
    }
    for (int i = threadIdx.x; i < p.h1p + p.h2p; i += blockDim.x) sbias[i] = p.bias[i];
    if (warp == 0) ptx::tmem_alloc(ptx::smem_u32(tmem_holder), 512);
    ptx::fence_before();
    __syncthreads();
    ptx::fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0 || warp > 4 * NS) {
        // ---------------- MMA issuer of one slot (warp 0: slot 0, and the weights) ----------------
        const int s = warp == 0 ? 0 : warp - 4 * NS;
        if (lane == 0 && s < n_issuers) {
            if (s == 0) {
                ptx::mbar_arrive_tx(BAR(kW), p.wbytes);
                for (int i = 0; i < 3 * p.per; ++i)
                    ptx::bulk_g2s(sbase + p.item_soff[i], p.wstream + p.item_off[i], p.item_bytes[i], BAR(kW));
            }
            const bool wok = wait_bar(BAR(kW), 0, ctl, 1);
            ptx::fence_after();
            const uint32_t d = tmem + 128u * s;
            const uint64_t ad = ptx::smem_desc(sbase + p.offA + s * kABytes, kTile * 16, 128);
            for (int i = s; i < n_local; i += NS) {
                const uint32_t ph = (uint32_t)(i / NS) & 1u;
#pragma unroll 1
                for (int L = 0; L < 3; ++L) {
                    const bool rdy = wait_bar(BAR(barA(s, L)), ph, ctl, 2);
                    ptx::fence_after();
                    if (rdy && wok) {
                        for (int w = 0; w < p.per; ++w) {
                            const int it = L * p.per + w;
                            const uint32_t n = p.item_n[it];
                            const int ksteps = (int)p.item_k[it] / 16;
                            const uint32_t idesc = ptx::idesc_f16(FMT, (int)n);
                            const uint64_t bd = ptx::smem_desc(sbase + p.item_soff[it], n * 16, 128);
                            for (int ks = 0; ks < ksteps; ++ks)
                                ptx::mma_ss(d, ad + (uint64_t)(ks * 2 * kTile), bd + (uint64_t)(ks * 2 * n), idesc,
                                            (w > 0 || ks > 0) ? 1u : 0u);
                        }
                    }
                    ptx::mma_commit(BAR(barD(s, L)));
                }
            }
            // every copy and MMA has completed before shared and tensor memory are released
            ptx::mma_commit(BAR(kDone));
            drain_bar(BAR(kDone), 0);
        }
    } else if (warp <= 4 * NS) {
        // ---------------- converting warps: slot (warp - 1) / 4, one per lane quadrant ----------------
        const int slot = (warp - 1) >> 2;
        const int quad = warp & 3;
        const int m = quad * 32 + lane;
        const int tid = threadIdx.x - 32 - slot * 128;
        const uint32_t dcol = tmem + ((uint32_t)(quad * 32) << 16) + 128u * slot;
        uint8_t *abuf = sm + p.offA + slot * kABytes;
        float *arow = (float *)(sm + p.offRow + slot * p.rowBytes);
        // the slot's current frame (units increase along the loop)
        int fcur = frame_of(p, u_base + slot, 0);
        // the first kPre elements per thread of the slot's next unit's anchor row, interpolated
        // at its image row: loaded and formed while the current unit waits for its layer-1 result
        float pi[kPre];
        if (slot < n_local) {
            const UnitGeom g = unit_geom(p, u_base + slot, fcur);
#pragma unroll
            for (int q = 0; q < kPre; ++q) {
                const int e2 = tid + 128 * q;
                if (e2 < g.nax * kHiModes) {
                    const int off = anchor_off(e2);
                    pi[q] = (1.0f - g.fy) * __ldg(g.a + off) + g.fy * __ldg(g.b + off);
                }
            }
        }
        for (int i = slot; i < n_local; i += NS) {
            const uint32_t ph = (uint32_t)(i / NS) & 1u;
            const int u = u_base + i;
            fcur = frame_of(p, u, fcur);
            const UnitGeom g = unit_geom(p, u, fcur);
            const Frame &F = p.fr[fcur];
            const int row = g.row, c0 = g.c0;
            const int col = c0 + m;
            bool ok = true;
            // ---- layer-1 operand: alpha_4..36 at (row, col), bilinear from the anchors.
            //      The slot first interpolates the two anchor rows at this image row
            //      (shared by all 128 pixels), then each pixel interpolates along x. ----
            {
                const float fy = g.fy;
                const int ax0 = g.ax0, nax = g.nax;
                // every pixel has read the previous unit's anchor row
                ptx::named_bar(1 + slot, 128);
#pragma unroll
                for (int q = 0; q < kPre; ++q) {
                    const int e2 = tid + 128 * q;
                    if (e2 < nax * kHiModes) arow[arow_idx(e2)] = pi[q];
                }
                for (int e2 = tid + 128 * kPre; e2 < nax * kHiModes; e2 += 128) {
                    const int off = anchor_off(e2);
                    arow[arow_idx(e2)] = (1.0f - fy) * __ldg(g.a + off) + fy * __ldg(g.b + off);
                }
                ptx::named_bar(1 + slot, 128);
                const int gj = min(col, F.W - 1);
                const int ax = gj / p.s - ax0;
                const float fx = (float)(gj - (ax + ax0) * p.s) * p.inv_s;
                const float4 *r0p = (const float4 *)(arow + ax * kRowStride);
                const float4 *r1p = r0p + (ax + 1 < nax ? kRowStride / 4 : 0);
#pragma unroll
                for (int g = 0; g < kK1 / 8; ++g) {
                    float v[8];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int k4 = 2 * g + h;  // modes 4 k4 .. 4 k4 + 3
                        float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
                        if (4 * k4 < kHiModes) {
                            a0 = r0p[k4];
                            a1 = r1p[k4];
                        }
                        const float e[4][2] = {{a0.x, a1.x}, {a0.y, a1.y}, {a0.z, a1.z}, {a0.w, a1.w}};
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int k = 4 * k4 + j;  // column 33 = 1: the weight image carries b1 there
                            v[4 * h + j] = k < kHiModes ? (1.0f - fx) * e[j][0] + fx * e[j][1] : (k == kHiModes ? 1.f : 0.f);
                        }
                    }
                    uint4 q;
                    q.x = pack2(v[0], v[1], FMT);
                    q.y = pack2(v[2], v[3], FMT);
                    q.z = pack2(v[4], v[5], FMT);
                    q.w = pack2(v[6], v[7], FMT);
                    *(uint4 *)(abuf + g * (kTile * 16) + m * 16) = q;
                }
                ptx::fence_proxy_async();
                ptx::fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(BAR(barA(slot, 0)));
            }
            if (i + NS < n_local) {
                const UnitGeom gn = unit_geom(p, u + NS, frame_of(p, u + NS, fcur));
#pragma unroll
                for (int q = 0; q < kPre; ++q) {
                    const int e2 = tid + 128 * q;
                    if (e2 < gn.nax * kHiModes) {
                        const int off = anchor_off(e2);
                        pi[q] = (1.0f - gn.fy) * __ldg(gn.a + off) + gn.fy * __ldg(gn.b + off);
                    }
                }
            }
            // ---- layers 1, 2: D -> bias, ReLU -> packed activations (the next A, same buffer) ----
#pragma unroll 1
            for (int L = 0; L < 2; ++L) {
                const int width = L ? p.h2p : p.h1p, boff = L ? p.h1p : 0;
                ok = __all_sync(0xffffffffu, wait_bar(BAR(barD(slot, L)), ph, ctl, 4) && ok);
                ptx::fence_after();
#pragma unroll 1
                for (int c32 = 0; ok && c32 < width; c32 += 32) {
                    uint32_t d[32];
                    ptx::tmem_ld32(dcol + c32, d);
                    ptx::tmem_wait_ld_dep(d);
                    const float4 *bv = (const float4 *)(sbias + boff + c32);
#pragma unroll
                    for (int g = 0; g < 4; ++g) {  // k-group c32 / 8 + g
                        uint32_t w4[4];
                        if (L == 0) {  // b1 came through the tensor core (operand column 33)
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                w4[j] = tcc::pack2_relu(__uint_as_float(d[8 * g + 2 * j]), __uint_as_float(d[8 * g + 2 * j + 1]),
                                                        FMT);
                        } else {
#pragma unroll
                            for (int j = 0; j < 2; ++j) {
                                const float4 bb = bv[2 * g + j];
                                float h0, h1, h2, h3;
                                tcc::add2(__uint_as_float(d[8 * g + 4 * j]), __uint_as_float(d[8 * g + 4 * j + 1]), bb.x,
                                          bb.y, h0, h1);
                                tcc::add2(__uint_as_float(d[8 * g + 4 * j + 2]), __uint_as_float(d[8 * g + 4 * j + 3]),
                                          bb.z, bb.w, h2, h3);
                                w4[2 * j] = tcc::pack2_relu(h0, h1, FMT);  // ReLU in the conversion
                                w4[2 * j + 1] = tcc::pack2_relu(h2, h3, FMT);
                            }
                        }
                        *(uint4 *)(abuf + (c32 / 8 + g) * (kTile * 16) + m * 16) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
                    }
                }
                ptx::fence_proxy_async();
                ptx::fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(BAR(barA(slot, L + 1)));
            }
            // ---- layer 3: beta (no bias) -> 16-bit groups of 8 in global memory ----
            ok = __all_sync(0xffffffffu, wait_bar(BAR(barD(slot, 2)), ph, ctl, 8) && ok);
            ptx::fence_after();
            const bool store = ok && col < F.W;
            const int pos = p.perm ? (col & ~31) + 8 * (col & 3) + ((col & 31) >> 2) : col;
            if (p.scale8) {
                // FP8: k = 0 .. 127 (entries K, K + 1 are the bias columns, 1 before scaling, and
                // k >= K + 2 have scale 0), 16 groups: hi bytes of k = 16 g .. 16 g + 15 in group g,
                // lo bytes in group 8 + g
                uint4 *dst8 = F.beta + ((size_t)row * kGroups8) * F.pitch + pos;
#pragma unroll 1
                for (int c32 = 0; ok && c32 < 128; c32 += 32) {
                    uint32_t d[32];
                    ptx::tmem_ld32(dcol + c32, d);
                    ptx::tmem_wait_ld_dep(d);
                    if (store) {
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            uint32_t hw[4], lw[4];
#pragma unroll
                            for (int jj = 0; jj < 8; ++jj) {  // k = c32 + 16 q + 2 jj, + 1
                                float v2[2];
#pragma unroll
                                for (int e = 0; e < 2; ++e) {
                                    const int k = c32 + 16 * q + 2 * jj + e;
                                    const float raw = k < p.K ? __uint_as_float(d[16 * q + 2 * jj + e])
                                                              : ((k == p.K || k == p.K + 1) ? 1.0f : 0.0f);
                                    v2[e] = raw * __ldg(p.scale8 + k);
                                }
                                uint16_t hi, lo;
                                tcc::e4m3_hi_lo(v2[0], v2[1], hi, lo);
                                if (jj & 1) {
                                    hw[jj >> 1] |= (uint32_t)hi << 16;
                                    lw[jj >> 1] |= (uint32_t)lo << 16;
                                } else {
                                    hw[jj >> 1] = hi;
                                    lw[jj >> 1] = lo;
                                }
                            }
                            const int g = c32 / 16 + q;
                            dst8[(size_t)g * F.pitch] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                            dst8[(size_t)(8 + g) * F.pitch] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                        }
                    }
                }
                ptx::fence_before();
                continue;
            }
            uint4 *dst = F.beta + ((size_t)row * kGroups) * F.pitch + pos;
#pragma unroll 1
            for (int c32 = 0; ok && c32 < 8 * kGroups; c32 += 32) {  // columns 112..127 are read, unused
                uint32_t d[32];
                ptx::tmem_ld32(dcol + c32, d);
                ptx::tmem_wait_ld_dep(d);
                if (store) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int g = c32 / 8 + q;
                        if (g < kGroups) {
                            float v[8];
                            if (8 * g + 8 <= p.K) {  // every group below K: the values as they are
#pragma unroll
                                for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(d[8 * q + j]);
                            } else {
#pragma unroll
                                for (int j = 0; j < 8; ++j) {
                                    const int k = 8 * g + j;
                                    v[j] = k < p.K ? __uint_as_float(d[8 * q + j])
                                                   : ((p.ones && (k == p.K || k == p.K + 1)) ? 1.0f : 0.0f);
                                }
                            }
                            uint4 w4;
                            w4.x = pack2(v[0], v[1], FMT);
                            w4.y = pack2(v[2], v[3], FMT);
                            w4.z = pack2(v[4], v[5], FMT);
                            w4.w = pack2(v[6], v[7], FMT);
                            dst[(size_t)g * F.pitch] = w4;
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
                              int fmt, int perm, int pitch) {
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
    const int pos = perm ? (col & ~31) + 8 * (col & 3) + ((col & 31) >> 2) : col;
    out[(rowf * kGroups + g) * pitch + pos] = u;
}

// FP32 beta [n][H][W][K] -> the FP8 hi/lo layout [row][16][W][16 B] (beta_k times
// scale8[k]; k >= K zero: the given beta already includes the last layer's bias).
__global__ void pack8_kernel(const float *__restrict__ beta, uint4 *__restrict__ out, long long npx, int W, int K,
                             const float *__restrict__ scale8) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (pixel, group of 16 k)
    if (i >= npx * 8) return;
    const long long px = i / 8;
    const int g = (int)(i - px * 8);
    const long long rowf = px / W;  // frame * H + row
    const int col = (int)(px - rowf * W);
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
        float v2[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int k = 16 * g + 2 * jj + e;
            v2[e] = k < K ? __ldg(beta + px * K + k) * __ldg(scale8 + k) : 0.f;
        }
        uint16_t hi, lo;
        tcc::e4m3_hi_lo(v2[0], v2[1], hi, lo);
        if (jj & 1) {
            hw[jj >> 1] |= (uint32_t)hi << 16;
            lw[jj >> 1] |= (uint32_t)lo << 16;
        } else {
            hw[jj >> 1] = hi;
            lw[jj >> 1] = lo;
        }
    }
    out[(rowf * kGroups8 + g) * W + col] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    out[(rowf * kGroups8 + 8 + g) * W + col] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

}  // namespace net

using namespace net;

size_t beta8_bytes(int H, int W, int n) { return (size_t)n * H * W * kGroups8 * 16; }

p2s_status launch_pack8(p2s_ctx *ctx, int H, int W, int n, const float *beta, void *beta8, cudaStream_t st) {
    p2s_status s0 = tc_prepare(ctx);
    if (s0 != P2S_OK) return s0;
    if (!ctx->tc.d_scale8) {
        set_error("the FP8 operand layout exists for FP8 contexts only");
        return P2S_EUNSUPPORTED;
    }
    const long long npx = (long long)n * H * W;
    if (npx == 0) return P2S_OK;
    ProfScope pr(ctx, st, "pack_beta8", 0.0, npx * (ctx->K * 4.0 + kGroups8 * 16.0));
    pack8_kernel<<<(unsigned)((npx * 8 + 255) / 256), 256, 0, st>>>(beta, (uint4 *)beta8, npx, W, ctx->K,
                                                                      ctx->tc.d_scale8);
    P2S_CUDA(cudaGetLastError());
    return P2S_OK;
}

size_t beta16_bytes(int H, int W, int n, int perm) { return (size_t)n * H * beta16_pitch(W, perm) * kGroups * 16; }

// Shared-memory layout of the network kernel for a geometry; returns the
// bytes needed and fills the offsets and the slot count (0 if nothing fits).
static int net_layout(const p2s_ctx *ctx, int s, int W, Params *p) {
    uint32_t w = 0;
    const Item16 *it = (const Item16 *)ctx->tc_items.data();
    for (int i = 0; i < ctx->tc.n_mlp; ++i) w += it[i].bytes;
    const int max_ax = std::min((kTile - 1) / s + 3, (W - 1) / s + 2);
    const uint32_t row_bytes = ((uint32_t)max_ax * kRowStride * 4 + 127) & ~127u;
    const uint32_t fixed_tail = (uint32_t)(ctx->tc.h1p + ctx->tc.h2p) * 4 + kNBar * 8 + 16 + 1024;
    const uint32_t offA = (w + 1023) & ~1023u;
    int ns = kMaxSlots;
    while (ns > 0 && offA + ns * (kABytes + row_bytes) + fixed_tail > 227u * 1024u) --ns;
    p->nslots = ns;
    p->offA = offA;
    p->rowBytes = row_bytes;
    p->offRow = offA + ns * kABytes;
    p->offBias = p->offRow + ns * row_bytes;
    p->offBar = (p->offBias + (uint32_t)(ctx->tc.h1p + ctx->tc.h2p) * 4 + 7) & ~7u;
    p->offMisc = p->offBar + kNBar * 8;
    return (int)(p->offMisc + 16 + 1024);
}

p2s_status launch_net16_frames(p2s_ctx *ctx, const NetFrame *frames, int n, int ones, int perm, int *status,
                               cudaStream_t st) {
    if (n <= 0) return P2S_OK;
    if (n > kMaxBatch) {
        set_error("network batch larger than %d frames", kMaxBatch);
        return P2S_EINVAL;
    }
    p2s_status s0 = tc_prepare(ctx);
    if (s0 != P2S_OK) return s0;
    Params p;
    std::memset(&p, 0, sizeof p);
    p.scale8 = ctx->prec == P2S_FP8E4M3 ? ctx->tc.d_scale8 : nullptr;  // FP8: the hi/lo layout (perm 0)
    if (p.scale8 && perm) {
        set_error("the FP8 beta layout has natural column order");
        return P2S_EUNSUPPORTED;
    }
    int units = 0, w_max = 1;
    double npx = 0.0;
    for (int i = 0; i < n; ++i) {
        const NetFrame &q = frames[i];
        Frame &F = p.fr[i];
        F.alpha = q.alpha;
        F.beta = (uint4 *)q.beta;
        F.H = q.H;
        F.W = q.W;
        F.Aw = (q.W - 1) / ctx->s + 2;
        F.pitch = beta16_pitch(q.W, perm);
        F.tiles_x = (q.W + kTile - 1) / kTile;
        F.u0 = units;
        units += F.tiles_x * q.H;
        w_max = std::max(w_max, q.W);
        npx += (double)q.H * q.W;
    }
    p.nf = n;
    p.wstream = (const uint8_t *)ctx->tc.d_H;
    p.bias = ctx->tc.d_bias;
    p.status = status;
    p.s = ctx->s;
    p.inv_s = 1.0f / (float)ctx->s;
    p.K = ctx->K;
    p.h1p = ctx->tc.h1p;
    p.h2p = ctx->tc.h2p;
    p.n3 = ctx->tc.n3;
    p.ab_fmt = ctx->tc.fmt;
    p.per = ctx->tc.split ? 2 : 1;
    p.ones = ones;
    p.perm = perm;
    p.tiles_total = units;
    if (units == 0) return P2S_OK;
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
    const int smem = net_layout(ctx, ctx->s, w_max, &p);
    if (p.nslots < 1) {
        set_error("network weights too large for the tensor-core network kernel (%u B)", p.wbytes);
        return P2S_EUNSUPPORTED;
    }
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    // contiguous runs of units per CTA (row-fastest order inside a column block)
    p.per_cta = (p.tiles_total + sms - 1) / sms;
    const int grid = (p.tiles_total + p.per_cta - 1) / p.per_cta;
    double macs = 0.0;
    for (int l = 0; l < 3; ++l) macs += (double)ctx->dims[l] * ctx->dims[l + 1];
    ProfScope pr(ctx, st, "net_tc", 2.0 * macs * npx, npx * (p.scale8 ? kGroups8 : kGroups) * 16.0);
    if (p.ab_fmt == 1) {
        P2S_CUDA(cudaFuncSetAttribute(net_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        net_kernel<1><<<grid, 160 * p.nslots, smem, st>>>(p);
    } else {
        P2S_CUDA(cudaFuncSetAttribute(net_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        net_kernel<0><<<grid, 160 * p.nslots, smem, st>>>(p);
    }
    P2S_CUDA(cudaGetLastError());
    return P2S_OK;
}

p2s_status launch_net16(p2s_ctx *ctx, const FieldGeom &g, int n, const float *alpha, void *beta16, int ones, int perm,
                        int *status, cudaStream_t st) {
    const size_t fbytes = ctx->prec == P2S_FP8E4M3 ? beta8_bytes(g.H, g.W, 1) : beta16_bytes(g.H, g.W, 1, perm);
    NetFrame fr[kMaxBatch];
    for (int i0 = 0; i0 < n; i0 += kMaxBatch) {
        const int nb = std::min(kMaxBatch, n - i0);
        for (int k = 0; k < nb; ++k)
            fr[k] = NetFrame{alpha + (size_t)(i0 + k) * g.Ah * g.Aw * kAlphaStride,
                             (char *)beta16 + (size_t)(i0 + k) * fbytes, g.H, g.W};
        p2s_status s0 = launch_net16_frames(ctx, fr, nb, ones, perm, status, st);
        if (s0 != P2S_OK) return s0;
    }
    return P2S_OK;
}

p2s_status launch_pack16(p2s_ctx *ctx, int H, int W, int n, const float *beta, void *beta16, int perm,
                         cudaStream_t st) {
    p2s_status s0 = tc_prepare(ctx);
    if (s0 != P2S_OK) return s0;
    const long long npx = (long long)n * H * W;
    const long long work = npx * kGroups;
    if (work == 0) return P2S_OK;
    ProfScope pr(ctx, st, "pack_beta16", 0.0, npx * (ctx->K * 4.0 + kGroups * 16.0));
    pack16_kernel<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(beta, (uint4 *)beta16, npx, W, ctx->K, ctx->tc.fmt, perm,
                                                                 beta16_pitch(W, perm));
    P2S_CUDA(cudaGetLastError());
    return P2S_OK;
}

}  // namespace p2s
