// Tensor-core path (tcgen05, sm_103a): the P2S network (Sec. 3.3) and the
// basis blur (Sec. 3.1, Eq. 5) fused in one persistent kernel.
//
// Work unit: a tile of 128 output columns x 32 output rows of one frame,
// processed two rows at a time.  Per row pair:
//   network   three tcgen05.mma layers per row (M = 128 pixels), activations
//             kept in tensor memory between layers (A operand from TMEM);
//   beta      written into TMEM as the A operand of the contraction, with
//             two extra "one" columns that pick up the last layer's bias,
//             folded into the basis as an exact hi/lo pair of rows;
//   G = beta H  chunk by chunk into TMEM (N = 96: 3 tap columns x 32 tap
//             rows; the last tap row as a final N = 48 chunk);
//   gather    y_c[q] += G[q, t] x_c[q - o(t)] on the CUDA cores: each thread
//             owns one output column of the row pair, walks a tap column with
//             a 33-row window of x in registers (x staged in shared memory as
//             FP16 RGB in 8 bytes, widened to FP32 on load: 2/3 of the FP32
//             staging traffic, the contraction's largest shared-memory stream),
//             accumulates in FP32.
// Roles: warps 0 and 10 issue MMAs (one thread each, one output row each: a
// single issuing thread caps tcgen05.mma at one per ~76 cycles), warp 1 streams weights and basis
// chunks into a 3-slot shared-memory ring with 1-D bulk copies, warps 2..9
// (two per TMEM lane quadrant) convert between layers and run the gather;
// the two halves take alternate chunks, each with its own TMEM buffer.
// Every wait is bounded; a timeout sets the status word and the kernel
// drains and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>

#include "half_bits.h"
#include "p2s_internal.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace p2s {
namespace tc {

constexpr int kStrip = 128;                    // output columns per tile (TMEM lanes)
constexpr int kHalo = 16;                      // 33 x 33 taps
constexpr int kTaps = 2 * kHalo + 1;
constexpr int kTC = kStrip + 2 * kHalo;        // x tile columns
constexpr int kKP = 112;                       // padded contraction depth
constexpr int kKSteps = kKP / 16;
constexpr int kMainN = 96;                     // main chunk width
constexpr int kMainChunks = 11;                // 33 tap columns / 3
constexpr int kChunks = kMainChunks + 1;       // + the last tap row
constexpr int kLastN = 48;
constexpr int kSlot = 32768;
constexpr int kSlots = 3;
constexpr int kThreads = 352;  // + the second MMA warp (warp 10, row 1)
constexpr int kMmaWarp1 = 10;
constexpr int kEpi = 256;

// tensor-memory column map (512 columns allocated)
__host__ __device__ constexpr uint32_t colA1(int r) { return r ? 24u : 0u; }
__host__ __device__ constexpr uint32_t colD1(int r) { return r ? 256u : 128u; }  // A2 in place
__host__ __device__ constexpr uint32_t colD2(int r) { return r ? 0u : 384u; }    // A3 in place
__host__ __device__ constexpr uint32_t colD3(int r) { return r ? 256u : 128u; }
__host__ __device__ constexpr uint32_t colBeta(int r) { return r ? 56u : 0u; }
__host__ __device__ constexpr uint32_t colDB(int h) { return h ? 320u : 128u; }  // contraction, 2 rows x 96

enum Mode { kFull = 0, kMlpOnly = 1, kBlurOnly = 2 };

struct Item {
    uint32_t offset, bytes, n, k;
};

struct Params {
    TcFrame fr[kMaxTcFrames];  // per-frame pointers and geometry; tiles numbered frame by frame
    int n_frames;
    const float *beta_in;
    float *beta_out;
    const uint8_t *stream;
    const float *bias;  // b1 [h1p], b2 [h2p]
    const float *b3;    // [K]
    int *status;
    int C, s;
    float inv_s;
    int K, h1p, h2p, n3;
    int mode, fold, ab_fmt, split;
    int tiles_total;
    int n_mlp_items;
    Item item[6 + kChunks];  // network items (hi[,lo] per layer), then chunks
};

// shared-memory layout
constexpr int kOffRing = 0;
// ring full/empty, network stage handshakes, contraction buffer full/empty
enum Bar { kFull0 = 0, kEmpty0 = 3, kA1b = 6, kD1b, kA2b, kD2b, kA3b, kD3b, kBetab, kDFull0 = 13, kDEmpty0 = 15, kNBar = 17 };

// Tile shape: 128 output columns x BAND output rows (BAND = 16 or 32); the x
// tile with its halo is (BAND + 32) x 160 FP32 pixels in shared memory.
template <int BAND>
struct Lay {
    static constexpr int TR = BAND + 2 * kHalo;                  // x tile rows
    static constexpr int OffX = kOffRing + kSlots * kSlot;       // uint2 [TR][kTC]: (R, G, B, 0) as FP16
    static constexpr int OffBias = OffX + TR * kTC * 8;          // 256 floats
    static constexpr int OffXchg = OffBias + 256 * 4;            // [128][6] floats
    static constexpr int OffBar = OffXchg + kStrip * 6 * 4;      // mbarriers
    static constexpr int OffMisc = OffBar + kNBar * 8;           // tmem base, abort flag
    static constexpr int SmemBytes = OffMisc + 16 + 1024;        // + alignment slack
    static_assert(SmemBytes <= 227 * 1024, "shared memory budget");
};

using tcc::Ctl;
using tcc::drain_bar;
using tcc::pack2;
using tcc::wait_bar;

static_assert(sizeof(Params) <= 32000, "kernel parameter block (frame table) exceeds the 32 KB limit");

// frame of a global tile index (frames are laid out one after another)
__device__ __forceinline__ int frame_of(const Params &p, int tile) {
    int lo = 0, hi = p.n_frames - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.fr[mid].tile_base <= tile)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <int C, int BAND>
__global__ void __launch_bounds__(kThreads, 1) fused_kernel(const __grid_constant__ Params p) {
    using L = Lay<BAND>;
    extern __shared__ uint8_t smem_raw[];
    // aligned by pointer arithmetic on the __shared__ array, so that the compiler still
    // knows every access through `sm` is to shared memory (ld/st.shared, not generic)
    uint8_t *sm = smem_raw + ((1024u - (uint32_t)((uintptr_t)smem_raw & 1023u)) & 1023u);
    const uint32_t sbase = ptx::smem_u32(sm);
    uint2 *x16 = (uint2 *)(sm + L::OffX);
    float *sbias = (float *)(sm + L::OffBias);
    float *xchg = (float *)(sm + L::OffXchg);
    const uint32_t bar0 = sbase + L::OffBar;
    uint32_t *tmem_holder = (uint32_t *)(sm + L::OffMisc);
    volatile int *abort_flag = (volatile int *)(sm + L::OffMisc + 4);
    auto BAR = [&](int i) { return bar0 + 8u * (uint32_t)i; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Ctl ctl{abort_flag, p.status};

    if (threadIdx.x == 0) {
        *abort_flag = 0;
        for (int i = 0; i < kSlots; ++i) {
            ptx::mbar_init(BAR(kFull0 + i), 1);
            ptx::mbar_init(BAR(kEmpty0 + i), 2);  // one commit per MMA thread
        }
        ptx::mbar_init(BAR(kA1b), 8);
        ptx::mbar_init(BAR(kD1b), 2);
        ptx::mbar_init(BAR(kA2b), 8);
        ptx::mbar_init(BAR(kD2b), 2);
        ptx::mbar_init(BAR(kA3b), 8);
        ptx::mbar_init(BAR(kD3b), 2);  // D barriers: one commit per MMA thread
        ptx::mbar_init(BAR(kBetab), 8);
        ptx::mbar_init(BAR(kDFull0), 2);
        ptx::mbar_init(BAR(kDFull0 + 1), 2);
        ptx::mbar_init(BAR(kDEmpty0), 8);
        ptx::mbar_init(BAR(kDEmpty0 + 1), 8);
        ptx::mbar_fence_init();
    }
    for (int i = threadIdx.x; i < p.h1p + p.h2p; i += blockDim.x) sbias[i] = p.bias[i];
    if (warp == 0) ptx::tmem_alloc(ptx::smem_u32(tmem_holder), 512);
    ptx::fence_before();
    __syncthreads();
    ptx::fence_after();
    const uint32_t tmem = *tmem_holder;
    const uint32_t idesc_n96 = ptx::idesc_f16(p.ab_fmt, kMainN);
    const uint32_t idesc_n48 = ptx::idesc_f16(p.ab_fmt, kLastN);
    const bool do_mlp = p.mode != kBlurOnly, do_blur = p.mode != kMlpOnly;
    const int items_per_pair = (do_mlp ? p.n_mlp_items : 0) + (do_blur ? kChunks : 0);

    auto n_pairs_of = [&](int tile) {
        const TcFrame &F = p.fr[frame_of(p, tile)];
        const int ty = (tile - F.tile_base) / F.tiles_x;
        const int rows = min(BAND, F.H - ty * BAND);
        return (rows + 1) >> 1;
    };

    if (warp == 1) {
        // ---------------- producer: weights and basis chunks into the ring ----------------
        if (lane == 0) {
            uint32_t it = 0;
            for (int tile = blockIdx.x; tile < p.tiles_total; tile += gridDim.x) {
                const int npair = n_pairs_of(tile);
                for (int rp = 0; rp < npair; ++rp) {
                    for (int j = 0; j < items_per_pair; ++j) {
                        const int id = (do_mlp && j < p.n_mlp_items) ? j : 6 + (j - (do_mlp ? p.n_mlp_items : 0));
                        const Item itm = p.item[id];
                        const uint32_t slot = it % kSlots;
                        if (!wait_bar(BAR(kEmpty0 + slot), ((it / kSlots) & 1) ^ 1, ctl, 1)) continue;
                        ptx::mbar_arrive_tx(BAR(kFull0 + slot), itm.bytes);
                        ptx::bulk_g2s(sbase + kOffRing + slot * kSlot, p.stream + itm.offset, itm.bytes,
                                      BAR(kFull0 + slot));
                        ++it;
                    }
                }
            }
            // every issued copy must land before the CTA's shared memory is released
            for (uint32_t k = (it > (uint32_t)kSlots ? it - kSlots : 0); k < it; ++k)
                drain_bar(BAR(kFull0 + k % kSlots), (k / kSlots) & 1);
        }
    } else if (warp == 0 || warp == kMmaWarp1) {
        // ---------------- MMA issuers: warp 0 row 0, warp 10 row 1 ----------------
        // One thread issues an MMA about every 76-100 cycles whatever its size; a
        // thread per row, each on its own accumulators, keeps the tensor core busy.
        if (lane == 0) {
            const int row = warp == 0 ? 0 : 1;
            uint32_t it = 0, pairs = 0, uses[2] = {0, 0};
            // next ring item: wait until it has landed; returns its shared address (0 if aborted)
            auto take = [&](uint32_t &slot) -> uint32_t {
                slot = it % kSlots;
                const bool ok = wait_bar(BAR(kFull0 + slot), (it / kSlots) & 1, ctl, 2);
                ++it;
                return ok ? sbase + kOffRing + slot * kSlot : 0u;
            };
            const int per = p.split ? 2 : 1;
            for (int tile = blockIdx.x; tile < p.tiles_total; tile += gridDim.x) {
                const int npair = n_pairs_of(tile);
                for (int rp = 0; rp < npair; ++rp, ++pairs) {
                    const uint32_t ph = pairs & 1;
                    if (do_mlp) {
                        const uint32_t a_reg[3][2] = {{colA1(0), colA1(1)}, {colD1(0), colD1(1)}, {colD2(0), colD2(1)}};
                        const uint32_t d_reg[3][2] = {{colD1(0), colD1(1)}, {colD2(0), colD2(1)}, {colD3(0), colD3(1)}};
                        const int ready[3] = {kA1b, kA2b, kA3b};
                        const int done[3] = {kD1b, kD2b, kD3b};
                        for (int L = 0; L < 3; ++L) {
                            const bool rdy = wait_bar(BAR(ready[L]), ph, ctl, 4);
                            ptx::fence_after();
                            for (int w = 0; w < per; ++w) {
                                const Item itm = p.item[L * per + w];
                                uint32_t slot;
                                const uint32_t sa = take(slot);
                                if (rdy && sa) {
                                    ptx::fence_after();
                                    const uint32_t idesc = ptx::idesc_f16(p.ab_fmt, (int)itm.n);
                                    const int ksteps = (int)itm.k / 16;
                                    const uint64_t bd = ptx::smem_desc(sa, itm.n * 16, 128);
                                    const uint64_t bstep = (uint64_t)(2 * itm.n);  // 2 core-matrix columns, 16-byte units
                                    const uint32_t d = tmem + d_reg[L][row], a = tmem + a_reg[L][row];
                                    for (int ks = 0; ks < ksteps; ++ks)
                                        ptx::mma_ts(d, a + ks * 8, bd + ks * bstep, idesc, (w > 0 || ks > 0) ? 1u : 0u);
                                }
                                ptx::mma_commit(BAR(kEmpty0 + slot));
                            }
                            ptx::mma_commit(BAR(done[L]));
                        }
                    }
                    const bool brdy = wait_bar(BAR(kBetab), ph, ctl, 8);
                    ptx::fence_after();
                    if (do_blur) {
                        for (int c = 0; c < kChunks; ++c) {
                            const int h = c & 1;
                            uint32_t slot;
                            const uint32_t sa = take(slot);
                            const bool free_buf = wait_bar(BAR(kDEmpty0 + h), (uses[h] & 1) ^ 1, ctl, 16);
                            ptx::fence_after();
                            if (brdy && sa && free_buf) {
                                const uint32_t n = p.item[6 + c].n;
                                const uint32_t idesc = (n == (uint32_t)kMainN) ? idesc_n96 : idesc_n48;
                                const uint64_t bd = ptx::smem_desc(sa, n * 16, 128);
                                const uint64_t bstep = (uint64_t)(2 * n);
                                const uint32_t d = tmem + colDB(h) + row * kMainN, a = tmem + colBeta(row);
#pragma unroll
                                for (int ks = 0; ks < kKSteps; ++ks)
                                    ptx::mma_ts(d, a + ks * 8, bd + ks * bstep, idesc, ks > 0 ? 1u : 0u);
                            }
                            ptx::mma_commit(BAR(kEmpty0 + slot));
                            ptx::mma_commit(BAR(kDFull0 + h));
                            ++uses[h];
                        }
                    }
                }
            }
        }
    } else {
        // ---------------- epilogue: 8 warps, two per TMEM lane quadrant ----------------
        const int e = warp - 2;
        const int half = e >> 2;               // 0: warps 2-5, 1: warps 6-9
        const int quad = warp & 3;             // TMEM lane quadrant of this warp
        const int col = quad * 32 + lane;      // output column within the strip
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
        const int tid_e = threadIdx.x - 64;    // 0..255
        uint32_t pairs = 0, uses = 0;
        for (int tile = blockIdx.x; tile < p.tiles_total; tile += gridDim.x) {
            const int frame = frame_of(p, tile);
            const TcFrame &F = p.fr[frame];
            const int lt = tile - F.tile_base;
            const int ty = lt / F.tiles_x, tx = lt - ty * F.tiles_x;
            const int r_band = ty * BAND, c0 = tx * kStrip;
            const int npair = n_pairs_of(tile);
            if (do_blur) {
                ptx::named_bar(1, kEpi);  // previous tile fully consumed
                const float *x = F.xw;
                for (int i = tid_e; i < L::TR * kTC; i += kEpi) {
                    const int tr = i / kTC, tcol = i - tr * kTC;
                    const int gr = r_band - kHalo + tr, gc = c0 - kHalo + tcol;
                    float r = 0.f, g = 0.f, b = 0.f;
                    if (gr >= 0 && gr < F.H && gc >= 0 && gc < F.W) {
                        const float *px = x + ((size_t)gr * F.W + gc) * C;
                        r = __ldg(px);
                        if (C == 3) {
                            g = __ldg(px + 1);
                            b = __ldg(px + 2);
                        }
                    }
                    const __half2 rg = __floats2half2_rn(r, g), b0 = __floats2half2_rn(b, 0.f);
                    x16[i] = make_uint2(*reinterpret_cast<const uint32_t *>(&rg), *reinterpret_cast<const uint32_t *>(&b0));
                }
                ptx::named_bar(1, kEpi);
            }
            for (int rp = 0; rp < npair; ++rp, ++pairs) {
                const uint32_t ph = pairs & 1;
                bool ok = true;
                const int row = r_band + 2 * rp + half;  // this half's row for network stages
                const bool col_ok = c0 + col < F.W, row_ok = row < F.H;
                if (do_mlp) {
                    // ---- network input: alpha_4..36 at (row, col), bilinear from the anchors ----
                    {
                        const int gi = min(row, F.H - 1), gj = min(c0 + col, F.W - 1);
                        const int ay = gi / p.s, ax = gj / p.s;
                        const float fy = (float)(gi - ay * p.s) * p.inv_s, fx = (float)(gj - ax * p.s) * p.inv_s;
                        const float *a = F.alpha + ((size_t)ay * F.Aw + ax) * kAlphaStride;
                        const float *b = a + (size_t)F.Aw * kAlphaStride;
                        float v[48];
#pragma unroll
                        for (int m = 0; m < 48; ++m) {
                            if (m < kHiModes) {
                                const int sl = m + 3;
                                v[m] = (1.0f - fy) * ((1.0f - fx) * __ldg(a + sl) + fx * __ldg(a + kAlphaStride + sl)) +
                                       fy * ((1.0f - fx) * __ldg(b + sl) + fx * __ldg(b + kAlphaStride + sl));
                            } else {
                                v[m] = 0.f;
                            }
                        }
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            uint32_t u[8];
#pragma unroll
                            for (int j = 0; j < 8; ++j) u[j] = pack2(v[16 * q + 2 * j], v[16 * q + 2 * j + 1], p.ab_fmt);
                            ptx::tmem_st8(lane_base + colA1(half) + 8 * q, u);
                        }
                        ptx::tmem_wait_st();
                        ptx::fence_before();
                        __syncwarp();
                        if (lane == 0) ptx::mbar_arrive(BAR(kA1b));
                    }
                    // ---- layers 1, 2: D -> bias, ReLU -> packed activations in place ----
                    const int done[2] = {kD1b, kD2b};
                    const int ready[2] = {kA2b, kA3b};
                    const uint32_t dreg[2] = {colD1(half), colD2(half)};
                    const int width[2] = {p.h1p, p.h2p};
                    const int boff[2] = {0, p.h1p};
                    for (int L = 0; L < 2; ++L) {
                        ok = __all_sync(0xffffffffu, wait_bar(BAR(done[L]), ph, ctl, 32) && ok);
                        ptx::fence_after();
                        for (int q = 0; ok && q < width[L] / 32; ++q) {
                            uint32_t d[32];
                            ptx::tmem_ld32(lane_base + dreg[L] + 32 * q, d);
                            ptx::tmem_wait_ld();
                            uint32_t u[16];
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const float h0 = __uint_as_float(d[2 * j]) + sbias[boff[L] + 32 * q + 2 * j];
                                const float h1 = __uint_as_float(d[2 * j + 1]) + sbias[boff[L] + 32 * q + 2 * j + 1];
                                u[j] = tcc::pack2_relu(h0, h1, p.ab_fmt);  // ReLU in the conversion
                            }
                            const uint32_t (&u0)[8] = *reinterpret_cast<const uint32_t(*)[8]>(&u[0]);
                            const uint32_t (&u1)[8] = *reinterpret_cast<const uint32_t(*)[8]>(&u[8]);
                            ptx::tmem_st8(lane_base + dreg[L] + 16 * q, u0);
                            ptx::tmem_st8(lane_base + dreg[L] + 16 * q + 8, u1);
                        }
                        ptx::tmem_wait_st();
                        ptx::fence_before();
                        __syncwarp();
                        if (lane == 0) ptx::mbar_arrive(BAR(ready[L]));
                    }
                    // ---- layer 3: beta = D3 (+ b3 folded into the basis) ----
                    ok = __all_sync(0xffffffffu, wait_bar(BAR(kD3b), ph, ctl, 64) && ok);
                    ptx::fence_after();
                    if (ok) {
                        float v[kKP];
#pragma unroll
                        for (int q = 0; q < kKP / 16; ++q) {
                            uint32_t d[16];
                            if (16 * q < p.n3) {
                                ptx::tmem_ld16(lane_base + colD3(half) + 16 * q, d);
                                ptx::tmem_wait_ld();
                            } else {
#pragma unroll
                                for (int j = 0; j < 16; ++j) d[j] = 0u;
                            }
#pragma unroll
                            for (int j = 0; j < 16; ++j) v[16 * q + j] = __uint_as_float(d[j]);
                        }
                        if (p.mode == kMlpOnly) {
                            if (row_ok && col_ok) {
                                float *o = p.beta_out + ((size_t)row * F.W + c0 + col) * p.K;
#pragma unroll
                                for (int k = 0; k < kKP; ++k)
                                    if (k < p.K) o[k] = v[k] + __ldg(p.b3 + k);
                            }
                        } else {
#pragma unroll
                            for (int k = 0; k < kKP; ++k)
                                if (k >= p.K) v[k] = (p.fold && (k == p.K || k == p.K + 1)) ? 1.0f : 0.0f;
#pragma unroll
                            for (int q = 0; q < kKP / 16; ++q) {
                                uint32_t u[8];
#pragma unroll
                                for (int j = 0; j < 8; ++j) u[j] = pack2(v[16 * q + 2 * j], v[16 * q + 2 * j + 1], p.ab_fmt);
                                ptx::tmem_st8(lane_base + colBeta(half) + 8 * q, u);
                            }
                            ptx::tmem_wait_st();
                        }
                    }
                    ptx::fence_before();
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(BAR(kBetab));
                } else {
                    // blur alone: beta of (row, col) from global, no bias fold
                    const int gi = min(row, F.H - 1), gj = min(c0 + col, F.W - 1);
                    const float *bp = p.beta_in + ((size_t)gi * F.W + gj) * p.K;
                    for (int q = 0; q < kKP / 16; ++q) {
                        uint32_t u[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int k0 = 16 * q + 2 * j;
                            const float a0 = k0 < p.K ? __ldg(bp + k0) : 0.f;
                            const float a1 = k0 + 1 < p.K ? __ldg(bp + k0 + 1) : 0.f;
                            u[j] = pack2(a0, a1, p.ab_fmt);
                        }
                        ptx::tmem_st8(lane_base + colBeta(half) + 8 * q, u);
                    }
                    ptx::tmem_wait_st();
                    ptx::fence_before();
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(BAR(kBetab));
                }
                if (!do_blur) continue;
                // ---- contraction chunks: every warp takes every chunk; half h covers
                //      tap rows [16h, 16h + 16) of each tap column (the last tap row:
                //      tap columns [17h, 17h + 17 - h)) ----
                float acc[2][3];
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) acc[i][ch] = 0.f;
                const int jlo = 16 - 16 * half;  // first window row (relative to tile row 2rp + 1)
                for (int c = 0; c < kChunks; ++c) {
                    const int b = c & 1;
                    const uint32_t buf = lane_base + colDB(b);
                    const bool got = __all_sync(0xffffffffu, wait_bar(BAR(kDFull0 + b), (uses >> b) & 1 ? 1u : 0u, ctl, 128));
                    // uses holds one parity bit per buffer
                    uses ^= (1u << b);
                    ok = ok && got;
                    ptx::fence_after();
                    if (!got) {
                    } else if (c < kMainChunks) {
#pragma unroll 1
                        for (int u3 = 0; u3 < 3; ++u3) {
                            const int txx = 3 * c + u3;  // tap column 0..32
                            // G of this tap column; loading the next one ahead would keep two
                            // copies live across the unroll-1 loop (register moves per tap)
                            uint32_t g0[16], g1[16];
                            ptx::tmem_ld16(buf + 32 * u3 + 16 * half, g0);
                            ptx::tmem_ld16(buf + kMainN + 32 * u3 + 16 * half, g1);
                            float wr[17], wg[17], wb[17];
                            const int base = (2 * rp + 1 + jlo) * kTC + col + 32 - txx;
#pragma unroll
                            for (int m = 0; m < 17; ++m) {
                                const uint2 v = x16[base + m * kTC];
                                const float2 rg = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
                                wr[m] = rg.x;
                                wg[m] = rg.y;
                                wb[m] = (C == 3) ? __low2float(*reinterpret_cast<const __half2 *>(&v.y)) : 0.f;
                            }
                            ptx::tmem_wait_ld_dep(g0);
                            ptx::tmem_wait_ld_dep(g1);
                            float a[16], bb[16];
#pragma unroll
                            for (int t = 0; t < 16; ++t) {
                                a[t] = __uint_as_float(g0[t]);
                                bb[t] = __uint_as_float(g1[t]);
                            }
#pragma unroll
                            for (int t = 0; t < 16; ++t) {
                                // tap row ty = 16 half + t: window rows 15 - t (row 0), 16 - t (row 1)
                                acc[0][0] = fmaf(a[t], wr[15 - t], acc[0][0]);
                                acc[1][0] = fmaf(bb[t], wr[16 - t], acc[1][0]);
                                if (C == 3) {
                                    acc[0][1] = fmaf(a[t], wg[15 - t], acc[0][1]);
                                    acc[0][2] = fmaf(a[t], wb[15 - t], acc[0][2]);
                                    acc[1][1] = fmaf(bb[t], wg[16 - t], acc[1][1]);
                                    acc[1][2] = fmaf(bb[t], wb[16 - t], acc[1][2]);
                                }
                            }
                        }
                        ptx::tmem_wait_ld();
                    } else {
                        // last tap row (dy = +16): source tile rows 2rp + i
                        uint32_t g0[17], g1[17];
                        ptx::tmem_ld16(buf + 17 * half, *reinterpret_cast<uint32_t(*)[16]>(&g0[0]));
                        ptx::tmem_ld16(buf + kMainN + 17 * half, *reinterpret_cast<uint32_t(*)[16]>(&g1[0]));
                        ptx::tmem_ld1(buf + 17 * half + 16, g0[16]);
                        ptx::tmem_ld1(buf + kMainN + 17 * half + 16, g1[16]);
                        ptx::tmem_wait_ld();
                        const int ntx = half ? 16 : 17;
#pragma unroll
                        for (int q = 0; q < 17; ++q) {
                            if (q < ntx) {
                                const int txx = 17 * half + q;
                                const int i0 = (2 * rp) * kTC + col + 32 - txx, i1 = i0 + kTC;
                                const float a = __uint_as_float(g0[q]), b2 = __uint_as_float(g1[q]);
                                const uint2 v0 = x16[i0], v1 = x16[i1];
                                const float2 rg0 = __half22float2(*reinterpret_cast<const __half2 *>(&v0.x));
                                const float2 rg1 = __half22float2(*reinterpret_cast<const __half2 *>(&v1.x));
                                acc[0][0] = fmaf(a, rg0.x, acc[0][0]);
                                acc[1][0] = fmaf(b2, rg1.x, acc[1][0]);
                                if (C == 3) {
                                    acc[0][1] = fmaf(a, rg0.y, acc[0][1]);
                                    acc[0][2] = fmaf(a, __low2float(*reinterpret_cast<const __half2 *>(&v0.y)), acc[0][2]);
                                    acc[1][1] = fmaf(b2, rg1.y, acc[1][1]);
                                    acc[1][2] = fmaf(b2, __low2float(*reinterpret_cast<const __half2 *>(&v1.y)), acc[1][2]);
                                }
                            }
                        }
                    }
                    ptx::fence_before();
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(BAR(kDEmpty0 + b));
                }
                // ---- combine the halves, write the row pair ----
                if (half == 1) {
#pragma unroll
                    for (int i = 0; i < 2; ++i)
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) xchg[col * 6 + i * 3 + ch] = acc[i][ch];
                }
                ptx::named_bar(2, kEpi);
                if (half == 0 && ok) {
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const int orow = r_band + 2 * rp + i;
                        if (orow < F.H && col_ok) {
                            float *o = F.y + ((size_t)orow * F.W + c0 + col) * C;
#pragma unroll
                            for (int ch = 0; ch < C; ++ch) o[ch] = acc[i][ch] + xchg[col * 6 + i * 3 + ch];
                        }
                    }
                }
                ptx::named_bar(2, kEpi);
            }
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


// canonical K-major, no swizzle: (n, k) -> byte offset; rows N (multiple of 8)
__host__ inline size_t canon(int n, int k, int N) { return (size_t)(k / 8) * (N * 16) + (n / 8) * 128 + (n % 8) * 16 + (k % 8) * 2; }

}  // namespace tc

using namespace tc;

static int round16(int v) { return (v + 15) & ~15; }
static int round32(int v) { return (v + 31) & ~31; }

// FP8 E4M3 (OCP definition: 4 exponent bits, bias 7, 3 fraction bits, subnormals
// down to 2^-9, largest finite 448, no infinities): round to nearest even,
// saturating at +-448, as cvt.rn.satfinite.e4m3x2 does on the device.
static uint8_t e4m3_bits(double v) {
    const uint8_t sign = v < 0 ? 0x80 : 0;
    const double a = std::fabs(v);
    if (!(a < 448.0)) return sign | 0x7e;  // 448 = 1.75 * 2^8 (0x7f would be NaN)
    if (a == 0.0) return sign;
    int e;
    std::frexp(a, &e);  // a = m 2^e, m in [0.5, 1): unbiased exponent e - 1
    int E = e - 1;
    if (E < -6) {  // subnormal: quantum 2^-9
        const int q = (int)std::nearbyint(std::ldexp(a, 9));
        return sign | (uint8_t)q;  // q == 8 is the smallest normal, bits 0x08, as wanted
    }
    int q = (int)std::nearbyint(std::ldexp(a, 3 - E));  // in [8, 16]
    if (q == 16) {
        q = 8;
        ++E;
    }
    if (E > 8 || (E == 8 && q > 14)) return sign | 0x7e;
    return sign | (uint8_t)(((E + 7) << 3) | (q - 8));
}
static double e4m3_value(uint8_t b) {
    const int f = (b >> 3) & 15, m = b & 7;
    const double v = f == 0 ? std::ldexp((double)m, -9) : std::ldexp((double)(8 + m), f - 10);
    return (b & 0x80) ? -v : v;
}

// The FP8 contraction's operands (P2S_FP8E4M3).  Per basis row k a power of two
// 2^b_k brings max_t |H_k,t| into [120, 240); beta_k is multiplied by 2^(c - b_k)
// so that every product keeps the common factor 2^c, removed after the tap sums.
// c is the largest exponent that keeps 4 |beta_k| below 240 for every k over 2048
// seeded draws of alpha at D/r0 = 6 (the strongest turbulence of the workloads)
// pushed through the network (without the last bias, which is folded into the
// basis as rows K, K + 1).  Each scaled row and the scaled beta are split into an
// E4M3 hi/lo pair; G = b_hi H_hi + b_lo H_hi + b_hi H_lo in FP32.
static p2s_status fp8_prepare(p2s_ctx *ctx, const std::vector<double> &hb) {
    const int K = ctx->K, T = ctx->T;
    constexpr int KP8 = 128;
    if (K + 2 > KP8) {
        set_error("FP8 contraction needs K <= %d", KP8 - 2);
        return P2S_EUNSUPPORTED;
    }
    auto exp_for = [](double m, double target) {  // largest b with m 2^b < target
        if (!(m > 0.0)) return 0;
        int b = (int)std::floor(std::log2(target / m));
        while (std::ldexp(m, b) >= target) --b;
        return b;
    };
    // rows of the scaled basis: K rows of H, then the bias PSF hb and its remainder
    std::vector<double> rows((size_t)(K + 2) * T, 0.0);
    std::vector<int> bexp(K + 2, 0);
    for (int k = 0; k < K; ++k) {
        double m = 0.0;
        for (int t = 0; t < T; ++t) m = std::max(m, std::fabs(ctx->H[(size_t)k * T + t]));
        bexp[k] = exp_for(m, 240.0);
        for (int t = 0; t < T; ++t) rows[(size_t)k * T + t] = std::ldexp(ctx->H[(size_t)k * T + t], bexp[k]);
    }
    {
        double m = 0.0;
        for (int t = 0; t < T; ++t) m = std::max(m, std::fabs(hb[t]));
        bexp[K] = exp_for(m, 240.0);
        std::vector<double> rem(T);
        double mr = 0.0;
        for (int t = 0; t < T; ++t) {
            const double v = std::ldexp(hb[t], bexp[K]);
            const uint8_t hi = e4m3_bits(v);
            const uint8_t lo = e4m3_bits(v - e4m3_value(hi));
            rows[(size_t)K * T + t] = v;
            rem[t] = hb[t] - std::ldexp(e4m3_value(hi) + e4m3_value(lo), -bexp[K]);
            mr = std::max(mr, std::fabs(rem[t]));
        }
        bexp[K + 1] = mr > 0.0 ? exp_for(mr, 240.0) : bexp[K];
        for (int t = 0; t < T; ++t) rows[(size_t)(K + 1) * T + t] = std::ldexp(rem[t], bexp[K + 1]);
    }
    // beta range: alpha_4..36 = 6^(5/6) L z, z ~ N(0, I) (Box-Muller on a seeded 64-bit LCG)
    std::vector<double> bmax(K, 0.0);
    {
        uint64_t st = 0x9E3779B97F4A7C15ull;
        auto unif = [&]() {
            st = st * 6364136223846793005ull + 1442695040888963407ull;
            return ((double)(st >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        };
        const int NM = kModes;  // 35 modes J = 2..36; the network takes J = 4..36
        std::vector<double> z(NM), a(NM), h0, h1;
        const double sc = std::pow(6.0, 5.0 / 6.0);
        for (int sidx = 0; sidx < 2048; ++sidx) {
            for (int i = 0; i < NM; i += 2) {
                const double r = std::sqrt(-2.0 * std::log(unif())), th = 2.0 * M_PI * unif();
                z[i] = r * std::cos(th);
                if (i + 1 < NM) z[i + 1] = r * std::sin(th);
            }
            for (int i = 0; i < NM; ++i) {
                double acc = 0.0;
                for (int l = 0; l <= i; ++l) acc += ctx->L64[(size_t)i * NM + l] * z[l];
                a[i] = sc * acc;
            }
            h0.assign(a.begin() + 2, a.end());
            for (int l = 0; l < ctx->n_layers; ++l) {
                const int fi = ctx->dims[l], fo = ctx->dims[l + 1];
                h1.assign(fo, 0.0);
                for (int o = 0; o < fo; ++o) {
                    double acc = l + 1 < ctx->n_layers ? ctx->b[l][o] : 0.0;
                    for (int i = 0; i < fi; ++i) acc += ctx->W[l][(size_t)o * fi + i] * h0[i];
                    h1[o] = (l + 1 < ctx->n_layers) ? std::max(acc, 0.0) : acc;
                }
                h0.swap(h1);
            }
            for (int k = 0; k < K; ++k) bmax[k] = std::max(bmax[k], std::fabs(h0[k]));
        }
    }
    int c = 1 << 20;
    for (int k = 0; k < K; ++k) c = std::min(c, exp_for(4.0 * bmax[k], 240.0) + bexp[k]);
    if (c == (1 << 20)) c = 0;
    // the bias columns carry 2^(c - b) exactly: keep that exponent inside E4M3's normal range
    for (int k = K; k < K + 2; ++k) {
        const int s = c - bexp[k];
        const int sc = s > 8 ? 8 : (s < -6 ? -6 : s);
        if (sc != s) {
            for (int t = 0; t < T; ++t) rows[(size_t)k * T + t] = std::ldexp(rows[(size_t)k * T + t], (c - sc) - bexp[k]);
            bexp[k] = c - sc;
        }
    }
    std::vector<float> scale(KP8, 0.f);
    for (int k = 0; k < K + 2; ++k) scale[k] = (float)std::ldexp(1.0, c - bexp[k]);
    // images: per chunk the hi image then the lo image, canonical K-major 8-bit layout
    // (core matrices of 8 rows x 16 bytes), chunk columns as in the split gather
    auto canon8 = [](int n, int k, int N) { return (size_t)(k / 16) * (N * 16) + (n / 8) * 128 + (n % 8) * 16 + (k % 16); };
    std::vector<uint8_t> buf;
    auto add = [&](int ci, int N, auto tap_of) {
        const size_t img = (size_t)N * KP8;
        const size_t off = buf.size();
        buf.resize(off + 2 * img, 0);
        for (int n = 0; n < N; ++n) {
            const int t = tap_of(n);
            for (int k = 0; k < K + 2 && t >= 0; ++k) {
                const double v = rows[(size_t)k * T + t];
                const uint8_t hi = e4m3_bits(v);
                buf[off + canon8(n, k, N)] = hi;
                buf[off + img + canon8(n, k, N)] = e4m3_bits(v - e4m3_value(hi));
            }
        }
        ctx->tc.item8_off[ci] = (uint32_t)off;
        ctx->tc.item8_bytes[ci] = (uint32_t)(2 * img);
        ctx->tc.item8_n[ci] = (uint32_t)N;
    };
    for (int ci = 0; ci < kMainChunks; ++ci)
        add(ci, kMainN, [&](int n) { return (n % 32) * kTaps + 3 * ci + n / 32; });
    add(kMainChunks, kLastN, [&](int n) { return n < kTaps ? (kTaps - 1) * kTaps + n : -1; });
    void *d = nullptr;
    float *ds = nullptr;
    if (cudaMalloc(&d, buf.size()) != cudaSuccess || cudaMalloc(&ds, KP8 * sizeof(float)) != cudaSuccess) {
        cudaFree(d);
        set_error("device allocation failed for the FP8 operands");
        return P2S_ENOMEM;
    }
    P2S_CUDA(cudaMemcpy(d, buf.data(), buf.size(), cudaMemcpyHostToDevice));
    P2S_CUDA(cudaMemcpy(ds, scale.data(), KP8 * sizeof(float), cudaMemcpyHostToDevice));
    ctx->tc.d_H8 = d;
    ctx->tc.d_scale8 = ds;
    ctx->tc.inv_c8 = (float)std::ldexp(1.0, -c);
    return P2S_OK;
}

// Pack the network weights and the basis chunks into one stream of B images.
p2s_status tc_prepare(p2s_ctx *ctx) {
    if (ctx->tc.ready) return P2S_OK;
    const int fmt = ctx->prec == P2S_BF16 ? 1 : 0;
    const int split = ctx->prec == P2S_BF16 ? 1 : 0;
    if (ctx->n_layers != 3 || ctx->th != kTaps || ctx->tw != kTaps || ctx->K > kKP - 2 || ctx->dims[1] > 128 ||
        ctx->dims[2] > 128) {
        set_error("tensor-core path needs 3 layers (widths <= 128), 33x33 taps and K <= %d", kKP - 2);
        return P2S_EUNSUPPORTED;
    }
    const int K = ctx->K, T = ctx->T;
    const int h1p = round32(ctx->dims[1]), h2p = round32(ctx->dims[2]), n3 = round16(K);
    std::vector<uint8_t> buf;
    std::vector<Item> items;
    auto add_image = [&](int N, int Kd, auto value) {
        Item it{(uint32_t)buf.size(), (uint32_t)(N * Kd * 2), (uint32_t)N, (uint32_t)Kd};
        buf.resize(buf.size() + it.bytes, 0);
        uint8_t *base = buf.data() + it.offset;
        for (int n = 0; n < N; ++n)
            for (int k = 0; k < Kd; ++k) {
                const uint16_t u = value(n, k);
                std::memcpy(base + canon(n, k, N), &u, 2);
            }
        items.push_back(it);
    };
    // network: layer l weights W[l] [out][in] as B = [N = out][K = in]
    const int ins[3] = {kHiModes, ctx->dims[1], ctx->dims[2]};
    const int inp[3] = {48, h1p, h2p};
    const int outs[3] = {ctx->dims[1], ctx->dims[2], K};
    const int outp[3] = {h1p, h2p, n3};
    for (int l = 0; l < 3; ++l) {
        const std::vector<double> &W = ctx->W[l];
        // layer 1 also carries b1 in input column 33 (one of the padding columns up to 48): the
        // network kernel sets that operand column to 1 and the tensor core adds the bias; the
        // fused kernel leaves it 0 and adds b1 itself
        auto w_at = [&](int n, int k) -> double {
            if (n >= outs[l]) return 0.0;
            if (k < ins[l]) return W[(size_t)n * ins[l] + k];
            return (l == 0 && k == kHiModes) ? ctx->b[0][n] : 0.0;
        };
        add_image(outp[l], inp[l], [&](int n, int k) { return to_half_bits(w_at(n, k), fmt); });
        if (split)
            add_image(outp[l], inp[l], [&](int n, int k) {
                const double v = w_at(n, k);
                return to_half_bits(v - from_half_bits(to_half_bits(v, fmt), fmt), fmt);
            });
    }
    const int n_mlp = (int)items.size();
    while (items.size() < 6) items.push_back(Item{0, 0, 0, 0});
    // folded bias PSF h_b = sum_k b3_k H_k as an exact hi/lo pair of rows K, K+1
    std::vector<double> hb(T, 0.0);
    for (int k = 0; k < K; ++k)
        for (int t = 0; t < T; ++t) hb[t] += ctx->b[2][k] * ctx->H[(size_t)k * T + t];
    auto basis_row = [&](int k, int t) -> uint16_t {
        if (k < K) return to_half_bits(ctx->H[(size_t)k * T + t], fmt);
        const uint16_t hi = to_half_bits(hb[t], fmt);
        if (k == K) return hi;
        if (k == K + 1) return to_half_bits(hb[t] - from_half_bits(hi, fmt), fmt);
        return 0;
    };
    for (int c = 0; c < kMainChunks; ++c)
        add_image(kMainN, kKP, [&](int n, int k) {
            const int u = n / 32, ty = n % 32, tx = 3 * c + u;
            return basis_row(k, ty * kTaps + tx);
        });
    add_image(kLastN, kKP, [&](int n, int k) { return n < kTaps ? basis_row(k, (kTaps - 1) * kTaps + n) : (uint16_t)0; });
    // The same chunks for the split gather kernel (k_gather.cu), columns ordered for
    // its 16x256b TMEM fragments: column n = 8 B + 2 j + e, 8-column block B.
    //   main chunk c: B = 6 m + 2 u + v -> tap column 3 c + u, tap row 16 m + 4 j + 2 v + e
    //   last chunk:   B = 3 m + b       -> tap row 32, tap column 24 m + 6 j + 2 b + e (0 beyond 32)
    for (int c = 0; c < kMainChunks; ++c)
        add_image(kMainN, kKP, [&](int n, int k) {
            const int B = n / 8, j = (n % 8) / 2, e = n % 2;
            const int m = B / 6, u = (B % 6) / 2, v = B % 2;
            return basis_row(k, (16 * m + 4 * j + 2 * v + e) * kTaps + 3 * c + u);
        });
    add_image(kLastN, kKP, [&](int n, int k) {
        const int B = n / 8, j = (n % 8) / 2, e = n % 2;
        const int tx = 24 * (B / 3) + 6 * j + 2 * (B % 3) + e;
        return tx < kTaps ? basis_row(k, (kTaps - 1) * kTaps + tx) : (uint16_t)0;
    });
    // The packed-FP16 gather kernel (k_gather_h2.cu): tap-row-major chunks whose second
    // output row reads the image one tap row (32 N-rows) further in.
    //   main chunk c: N-row n -> tap row 3 c + n / 32 - 1 (zero outside 0 .. 32), tap column n % 32
    //   last chunk:   n < 32 -> tap row 32, tap column n; n < 65 -> tap row n - 32, tap column 32
    for (int c = 0; c < kMainChunks; ++c)
        add_image(128, kKP, [&](int n, int k) {
            const int ty = 3 * c + n / 32 - 1, tx = n % 32;
            return (ty >= 0 && ty < kTaps) ? basis_row(k, ty * kTaps + tx) : (uint16_t)0;
        });
    add_image(80, kKP, [&](int n, int k) {
        if (n < 32) return basis_row(k, (kTaps - 1) * kTaps + n);
        if (n < 32 + kTaps) return basis_row(k, (n - 32) * kTaps + kTaps - 1);
        return (uint16_t)0;
    });
    std::vector<float> bias(h1p + h2p, 0.f);
    for (int o = 0; o < ctx->dims[1]; ++o) bias[o] = (float)ctx->b[0][o];
    for (int o = 0; o < ctx->dims[2]; ++o) bias[h1p + o] = (float)ctx->b[1][o];
    std::vector<float> b3(K);
    for (int k = 0; k < K; ++k) b3[k] = (float)ctx->b[2][k];
    void *dstream = nullptr;
    float *dbias = nullptr;
    if (cudaMalloc(&dstream, buf.size()) != cudaSuccess ||
        cudaMalloc(&dbias, (bias.size() + b3.size()) * sizeof(float)) != cudaSuccess) {
        cudaFree(dstream);
        set_error("device allocation failed for tensor-core operands");
        return P2S_ENOMEM;
    }
    P2S_CUDA(cudaMemcpy(dstream, buf.data(), buf.size(), cudaMemcpyHostToDevice));
    P2S_CUDA(cudaMemcpy(dbias, bias.data(), bias.size() * 4, cudaMemcpyHostToDevice));
    P2S_CUDA(cudaMemcpy(dbias + bias.size(), b3.data(), b3.size() * 4, cudaMemcpyHostToDevice));
    ctx->tc.d_H = dstream;
    ctx->tc.d_bias = dbias;
    ctx->tc.H_bytes = buf.size();
    static_assert(sizeof(Item) == 16, "item layout");
    ctx->tc_items.assign((const uint8_t *)items.data(), (const uint8_t *)(items.data() + items.size()));
    ctx->tc.n_mlp = n_mlp;
    ctx->tc.h1p = h1p;
    ctx->tc.h2p = h2p;
    ctx->tc.n3 = n3;
    ctx->tc.fmt = fmt;
    ctx->tc.split = split;
    if (ctx->prec == P2S_FP8E4M3) {
        p2s_status s8 = fp8_prepare(ctx, hb);
        if (s8 != P2S_OK) return s8;
    }
    ctx->tc.ready = 1;
    return P2S_OK;
}

int tc_smem_bytes() { return Lay<32>::SmemBytes; }

static p2s_status launch_tc_chunk(p2s_ctx *ctx, int mode, const TcFrame *frames, int n, int C, const float *beta_in,
                                  float *beta_out, int *status, cudaStream_t st);

p2s_status launch_tc(p2s_ctx *ctx, int mode, const TcFrame *frames, int n, int C, const float *beta_in,
                     float *beta_out, int *status, cudaStream_t st) {
    if (n <= 0) return P2S_OK;
    if ((mode != kTcFull) && n != 1) {
        set_error("the network-only and blur-only tensor-core stages take one frame");
        return P2S_EINVAL;
    }
    p2s_status s0 = tc_prepare(ctx);
    if (s0 != P2S_OK) return s0;
    for (int i0 = 0; i0 < n; i0 += kMaxTcFrames) {
        const int nb = n - i0 < kMaxTcFrames ? n - i0 : kMaxTcFrames;
        s0 = launch_tc_chunk(ctx, mode, frames + i0, nb, C, beta_in, beta_out, status, st);
        if (s0 != P2S_OK) return s0;
    }
    return P2S_OK;
}

static p2s_status launch_tc_chunk(p2s_ctx *ctx, int mode, const TcFrame *frames, int n, int C, const float *beta_in,
                                  float *beta_out, int *status, cudaStream_t st) {
    thread_local Params p;  // large (frame table); copied into the launch by value
    std::memset(&p, 0, sizeof p);
    const int band = ctx->tc.band_rows == 16 ? 16 : 32;
    int tiles = 0;
    double npx = 0.0;
    for (int i = 0; i < n; ++i) {
        TcFrame f = frames[i];
        f.tiles_x = (f.W + kStrip - 1) / kStrip;
        f.tiles_y = (f.H + band - 1) / band;
        f.tile_base = tiles;
        tiles += f.tiles_x * f.tiles_y;
        npx += (double)f.H * f.W;
        p.fr[i] = f;
    }
    p.n_frames = n;
    p.beta_in = beta_in;
    p.beta_out = beta_out;
    p.stream = (const uint8_t *)ctx->tc.d_H;
    p.bias = ctx->tc.d_bias;
    p.b3 = ctx->tc.d_bias + ctx->tc.h1p + ctx->tc.h2p;
    p.status = status;
    p.C = C;
    p.s = ctx->s;
    p.inv_s = 1.0f / (float)ctx->s;
    p.K = ctx->K;
    p.h1p = ctx->tc.h1p;
    p.h2p = ctx->tc.h2p;
    p.n3 = ctx->tc.n3;
    p.mode = mode;
    p.fold = mode == kFull ? 1 : 0;
    p.ab_fmt = ctx->tc.fmt;
    p.split = ctx->tc.split;
    p.tiles_total = tiles;
    p.n_mlp_items = ctx->tc.n_mlp;
    std::memcpy(p.item, ctx->tc_items.data(), sizeof(p.item));
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const int grid = p.tiles_total < sms ? p.tiles_total : sms;
    double macs_net = 0.0;
    for (int l = 0; l < 3; ++l) macs_net += (double)ctx->dims[l] * ctx->dims[l + 1];
    const double flops = mode == kBlurOnly   ? 2.0 * ctx->K * ctx->T * npx
                         : mode == kMlpOnly ? 2.0 * macs_net * npx
                                            : 2.0 * (ctx->K * ctx->T + macs_net) * npx;
    ProfScope pr(ctx, st, mode == kFull ? "fused_tc_gather" : mode == kMlpOnly ? "mlp_tc" : "blur_tc_gather", flops,
                 npx * C * 8.0);
    auto go = [&](auto kern, int smem) -> p2s_status {
        P2S_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        kern<<<grid, kThreads, smem, st>>>(p);
        return P2S_OK;
    };
    p2s_status ls;
    if (band == 16)
        ls = C == 3 ? go(fused_kernel<3, 16>, Lay<16>::SmemBytes) : go(fused_kernel<1, 16>, Lay<16>::SmemBytes);
    else
        ls = C == 3 ? go(fused_kernel<3, 32>, Lay<32>::SmemBytes) : go(fused_kernel<1, 32>, Lay<32>::SmemBytes);
    if (ls != P2S_OK) return ls;
    P2S_CUDA(cudaGetLastError());
    return P2S_OK;
}

}  // namespace p2s
