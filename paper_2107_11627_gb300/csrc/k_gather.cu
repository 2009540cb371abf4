// Blur-only tensor-core gather (Sec. 3.1, Eq. 5) reading beta from the
// network kernel's 16-bit operand layout: the split alternative to the fused
// kernel, chosen by P2S_OPT_GATHER_SPLIT.
//
// With the network out of the kernel, the tap accumulation gets four warps
// per TMEM lane quadrant (16 accumulating warps) instead of two: each takes a
// quarter of the tap rows of every chunk (8), with its own window of x.  x is
// staged as vertical pixel pairs, so a window of 9 rows costs five 16-byte
// loads per tap column.  Per row pair of a 128 x 32 tile:
//   producer  beta rows (2 x 14 runs of 16-byte groups) into a staging buffer
//             with 1-D bulk copies, basis chunks into a 2-slot ring;
//   warps of groups 0, 1 move their row's beta from the staging buffer into
//             TMEM (the A operand), then everyone accumulates;
//   MMA       G = beta H chunk by chunk (N = 96: 3 tap columns x 32 tap rows,
//             then N = 48 for the last tap row), two TMEM buffers;
//   gather    y_c[q] += G[q, t] x_c[q - o(t)], x staged as FP16 RGB and G
//             rounded to FP16, so each product is one fma.rn.f32.f16 (FP16
//             operands, FP32 accumulation, no conversion of x); the four
//             groups' partial sums are added through shared memory and written.
// Every wait is bounded.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstring>

#include "p2s_internal.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace p2s {
namespace gs {

using tcc::Ctl;
using tcc::drain_bar;
using tcc::wait_bar;

constexpr int kStrip = 128;
constexpr int kBand = 32;
constexpr int kHalo = 16;
constexpr int kTR = kBand + 2 * kHalo;
constexpr int kTC = kStrip + 2 * kHalo;
constexpr int kKSteps = 7;
constexpr int kMainN = 96;
constexpr int kMainChunks = 11;
constexpr int kChunks = kMainChunks + 1;
constexpr int kSlot = 32768;
constexpr int kSlots = 2;
constexpr int kGroups = 14;                       // beta16 k-groups
constexpr int kGroups8 = 16;                      // FP8 beta: 8 hi + 8 lo groups of 16 k
constexpr int kGroupsEpi = 4;                     // accumulating groups of 4 warps
constexpr int kEpi = 128 * kGroupsEpi;            // 512
constexpr int kThreads = 64 + kEpi + 32;          // 608: + the second MMA warp (row 1)
constexpr int kMmaWarp1 = (64 + kEpi) / 32;       // 18
constexpr int kXPairs = kTR / 2 + 1;              // x tile rows (2 j - 1, 2 j), j = 0 .. 32
constexpr int kBetaRow = kGroups8 * kStrip * 16;  // 32,768 B per staged row (the FP8 layout's 16 groups)

// beta of output row r in TMEM: 56 columns of 16-bit values (K = 112), or 64 of E4M3
// (hi in the first 32, lo in the next 32; K = 128)
template <bool F8>
__host__ __device__ constexpr uint32_t colBeta(int r) { return r ? (F8 ? 64u : 56u) : 0u; }
__host__ __device__ constexpr uint32_t colDB(int h) { return h ? 320u : 128u; }

constexpr int kOffRing = 0;
constexpr int kOffX = kOffRing + kSlots * kSlot;           // uint4 [kXPairs][kTC]: two FP16 RGB pixels
constexpr int kOffBeta = kOffX + kXPairs * kTC * 16;       // [2 rows][14][128][16 B]
constexpr int kOffXchg = kOffBeta + 2 * kBetaRow;          // float [3][128][6]
enum Bar { kFull0 = 0, kEmpty0 = 2, kBStaged = 4, kBFree = 5, kBetaIn0 = 6, kPairDone0 = 8, kDFull0 = 10, kDEmpty0 = 12,
           kNBar = 14 };
constexpr int kOffBar = kOffXchg + (kGroupsEpi - 1) * kStrip * 6 * 4;
constexpr int kOffMisc = kOffBar + kNBar * 8;
constexpr int kSmemBytes = kOffMisc + 16 + 1024;
static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");

struct Item {
    uint32_t offset, bytes, n, k;
};

struct Frame {
    const float *xw;
    float *y;
    const uint4 *beta16;  // [H][14][W] 16-byte groups ([H][16][W], hi then lo, in FP8 contexts)
    int H, W, tiles_x, tiles_y, tile_base;
};
constexpr int kMaxFrames = 256;

struct Params {
    Frame fr[kMaxFrames];
    int n_frames, tiles_total;
    const uint8_t *stream;  // basis chunk images
    Item item[kChunks];
    int ab_fmt;
    float inv_c;  // FP8: the tensor core's G is 2^c G, so the tap sums are multiplied by 2^-c
    int *status;
};
static_assert(sizeof(Params) <= 32000, "kernel parameter block");

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

// Tap rows of group g in a main chunk: [8 g, 8 g + 8); in the last chunk
// (tap row 32) tap columns [9 g, 9 g + 9) below 33.  One code path serves all
// groups (distinct unrolled bodies per group thrash the instruction cache).
constexpr int kNT = 8;

// x pixel as FP16: (R, G) and (B, 0)
__device__ __forceinline__ uint2 encode_px(float r, float g, float b) {
    const __half2 rg = __floats2half2_rn(r, g), b0 = __floats2half2_rn(b, 0.f);
    return make_uint2(*reinterpret_cast<const uint32_t *>(&rg), *reinterpret_cast<const uint32_t *>(&b0));
}

template <int C>
__device__ __forceinline__ void accumulate_pair(const Params &p, const uint4 *xp, uint32_t lane_base, int col, int rp,
                                                int grp, uint32_t bar0, uint32_t &uses, bool &ok, const Ctl &ctl,
                                                int lane, float (&acc)[2][3]) {
    constexpr int NT = kNT, NW = NT + 1;
    auto BAR = [&](int i) { return bar0 + 8u * (uint32_t)i; };
    const int R0 = NT * grp;
    // Window rows r_s .. r_s + 8 with r_s = 2 rp + 25 - R0 (odd) = pixel pairs j_s .. j_s + 4,
    // j_s = (r_s + 1) / 2; tap row R0 + t reads window row 7 - t (output row 0) and 8 - t (row 1).
    const int xw0 = (rp + 13 - 4 * grp) * kTC + col + 32;  // tap column txx: xw0 - txx
    for (int c = 0; c < kChunks; ++c) {
        const int b = c & 1;
        const uint32_t buf = lane_base + colDB(b);
        const bool got = __all_sync(0xffffffffu, wait_bar(BAR(kDFull0 + b), (uses >> b) & 1, ctl, 128));
        uses ^= (1u << b);
        ok = ok && got;
        ptx::fence_after();
        if (!got) {
        } else if (c < kMainChunks) {
#pragma unroll 1
            for (int u3 = 0; u3 < 3; ++u3) {
                const uint32_t c0 = buf + 32 * u3 + R0;
                uint32_t g0[8], g1[8];
                ptx::tmem_ld8(c0, g0);
                ptx::tmem_ld8(c0 + kMainN, g1);
                const int txx = 3 * c + u3;
                uint4 v[(NW + 1) / 2];  // window rows 2 k, 2 k + 1: (R, G), (B, 0) of each
#pragma unroll
                for (int k = 0; k < (NW + 1) / 2; ++k) v[k] = xp[xw0 + k * kTC - txx];
                ptx::tmem_wait_ld_dep(g0);
                ptx::tmem_wait_ld_dep(g1);
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    // G of both output rows as one FP16 pair; window rows 7 - t (row 0), 8 - t (row 1)
                    const uint32_t gp = tcc::pack_f16x2(__uint_as_float(g0[t]), __uint_as_float(g1[t]));
                    const int w0 = NT - 1 - t, w1 = NT - t;
                    const uint32_t rg0 = (w0 & 1) ? v[w0 >> 1].z : v[w0 >> 1].x;
                    const uint32_t b0 = (w0 & 1) ? v[w0 >> 1].w : v[w0 >> 1].y;
                    const uint32_t rg1 = (w1 & 1) ? v[w1 >> 1].z : v[w1 >> 1].x;
                    const uint32_t b1 = (w1 & 1) ? v[w1 >> 1].w : v[w1 >> 1].y;
                    if (C == 3) {
                        tcc::fma_mix_x2<false>(rg0, gp, acc[0][0], acc[0][1]);
                        tcc::fma_mix_x2<true>(rg1, gp, acc[1][0], acc[1][1]);
                        tcc::fma_mix_x1<false>(b0, gp, acc[0][2]);
                        tcc::fma_mix_x1<true>(b1, gp, acc[1][2]);
                    } else {
                        tcc::fma_mix_x1<false>(rg0, gp, acc[0][0]);
                        tcc::fma_mix_x1<true>(rg1, gp, acc[1][0]);
                    }
                }
            }
        } else {
            // last tap row (tap row 32): tap columns [9 grp, 9 grp + 9) below 33; output row 0
            // reads tile row 2 rp (second pixel of pair rp), row 1 tile row 2 rp + 1 (first of rp + 1)
            uint32_t g0[9], g1[9];
            ptx::tmem_ld9(buf + 9 * grp, g0);
            ptx::tmem_ld9(buf + kMainN + 9 * grp, g1);
            ptx::tmem_wait_ld_dep(g0);
            ptx::tmem_wait_ld_dep(g1);
            const uint2 *xh = reinterpret_cast<const uint2 *>(xp);
            const int xr0 = 2 * (rp * kTC + col + 32 - 9 * grp) + 1, xr1 = xr0 + 2 * kTC - 1;
            const int nq = min(9, 33 - 9 * grp);
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                if (q < nq) {
                    const uint32_t gp = tcc::pack_f16x2(__uint_as_float(g0[q]), __uint_as_float(g1[q]));
                    const uint2 v0 = xh[xr0 - 2 * q], v1 = xh[xr1 - 2 * q];
                    if (C == 3) {
                        tcc::fma_mix_x2<false>(v0.x, gp, acc[0][0], acc[0][1]);
                        tcc::fma_mix_x2<true>(v1.x, gp, acc[1][0], acc[1][1]);
                        tcc::fma_mix_x1<false>(v0.y, gp, acc[0][2]);
                        tcc::fma_mix_x1<true>(v1.y, gp, acc[1][2]);
                    } else {
                        tcc::fma_mix_x1<false>(v0.x, gp, acc[0][0]);
                        tcc::fma_mix_x1<true>(v1.x, gp, acc[1][0]);
                    }
                }
            }
        }
        ptx::fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(BAR(kDEmpty0 + b));
    }
}

template <int C, bool F8>
__global__ void __launch_bounds__(kThreads, 1) gather_kernel(const __grid_constant__ Params p) {
    constexpr int NG = F8 ? kGroups8 : kGroups;  // beta groups staged per row
    extern __shared__ uint8_t smem_raw[];
    // aligned by pointer arithmetic on the __shared__ array, so that the compiler still
    // knows every access through `sm` is to shared memory (ld/st.shared, not generic)
    uint8_t *sm = smem_raw + ((1024u - (uint32_t)((uintptr_t)smem_raw & 1023u)) & 1023u);
    const uint32_t sbase = ptx::smem_u32(sm);
    uint4 *xp = (uint4 *)(sm + kOffX);
    float *xchg = (float *)(sm + kOffXchg);
    const uint32_t bar0 = sbase + kOffBar;
    uint32_t *tmem_holder = (uint32_t *)(sm + kOffMisc);
    volatile int *abort_flag = (volatile int *)(sm + kOffMisc + 4);
    auto BAR = [&](int i) { return bar0 + 8u * (uint32_t)i; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Ctl ctl{abort_flag, p.status};

    if (threadIdx.x == 0) {
        *abort_flag = 0;
        for (int i = 0; i < kSlots; ++i) {
            ptx::mbar_init(BAR(kFull0 + i), 1);
            ptx::mbar_init(BAR(kEmpty0 + i), 2);  // one commit per MMA thread
        }
        ptx::mbar_init(BAR(kBStaged), 1);
        ptx::mbar_init(BAR(kBFree), 2);  // one commit per MMA thread
        for (int r = 0; r < 2; ++r) {
            ptx::mbar_init(BAR(kBetaIn0 + r), 1);
            ptx::mbar_init(BAR(kPairDone0 + r), 1);
        }
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(BAR(kDFull0 + i), 2);  // one commit per MMA thread
            ptx::mbar_init(BAR(kDEmpty0 + i), 4 * kGroupsEpi);
        }
        ptx::mbar_fence_init();
    }
    if (warp == 0) ptx::tmem_alloc(ptx::smem_u32(tmem_holder), 512);
    ptx::fence_before();
    __syncthreads();
    ptx::fence_after();
    const uint32_t tmem = *tmem_holder;
    const uint32_t idesc_n96 = ptx::idesc_f16(p.ab_fmt, kMainN);
    const uint32_t idesc_n48 = ptx::idesc_f16(p.ab_fmt, 48);

    auto n_pairs_of = [&](int tile) {
        const Frame &F = p.fr[frame_of(p, tile)];
        const int ty = (tile - F.tile_base) / F.tiles_x;
        return (min(kBand, F.H - ty * kBand) + 1) >> 1;
    };

    if (warp == 1) {
        // ---------------- producer: beta rows, basis chunks ----------------
        if (lane == 0) {
            uint32_t it = 0, pairs = 0;
            for (int tile = blockIdx.x; tile < p.tiles_total; tile += gridDim.x) {
                const int f = frame_of(p, tile);
                const Frame &F = p.fr[f];
                const int lt = tile - F.tile_base;
                const int tyy = lt / F.tiles_x, c0 = (lt - tyy * F.tiles_x) * kStrip;
                const int npair = n_pairs_of(tile);
                const uint32_t cols = (uint32_t)min(kStrip, F.W - c0);
                for (int rp = 0; rp < npair; ++rp, ++pairs) {
                    // beta of the pair's rows; the staging buffer is free once both rows are in TMEM
                    if (wait_bar(BAR(kBFree), (pairs & 1) ^ 1, ctl, 1)) {
                        const int r0 = tyy * kBand + 2 * rp;
                        const int nrow = min(2, F.H - r0);
                        ptx::mbar_arrive_tx(BAR(kBStaged), (uint32_t)nrow * NG * cols * 16);
                        for (int i = 0; i < nrow; ++i)
                            for (int g = 0; g < NG; ++g)
                                ptx::bulk_g2s(sbase + kOffBeta + i * kBetaRow + g * kStrip * 16,
                                              F.beta16 + ((size_t)(r0 + i) * NG + g) * F.W + c0, cols * 16,
                                              BAR(kBStaged));
                    }
                    for (int c = 0; c < kChunks; ++c, ++it) {
                        const Item itm = p.item[c];
                        const uint32_t slot = it % kSlots;
                        if (!wait_bar(BAR(kEmpty0 + slot), ((it / kSlots) & 1) ^ 1, ctl, 2)) continue;
                        ptx::mbar_arrive_tx(BAR(kFull0 + slot), itm.bytes);
                        ptx::bulk_g2s(sbase + kOffRing + slot * kSlot, p.stream + itm.offset, itm.bytes, BAR(kFull0 + slot));
                    }
                }
            }
            for (uint32_t k = (it > (uint32_t)kSlots ? it - kSlots : 0); k < it; ++k)
                drain_bar(BAR(kFull0 + k % kSlots), (k / kSlots) & 1);
            if (pairs > 0) drain_bar(BAR(kBStaged), (pairs - 1) & 1);
        }
    } else if (warp == 0 || warp == kMmaWarp1) {
        // ---------------- MMA issuers: warp 0 row 0, warp 18 row 1 ----------------
        // One thread issues an MMA about every 76-100 cycles whatever its size; two
        // threads in two warps, each on its own accumulator, keep the tensor core busy.
        if (lane == 0) {
            const int row = warp == 0 ? 0 : 1;
            uint32_t it = 0, pairs = 0, uses[2] = {0, 0};
            for (int tile = blockIdx.x; tile < p.tiles_total; tile += gridDim.x) {
                const int npair = n_pairs_of(tile);
                for (int rp = 0; rp < npair; ++rp, ++pairs) {
                    // this row's beta into TMEM by tcgen05.cp, once the row's MMAs of the
                    // previous pair are done with it: no accumulating warp is involved, so
                    // the pair's first MMAs need not wait for the previous pair's tap sums
                    if (pairs > 0) wait_bar(BAR(kPairDone0 + row), (pairs - 1) & 1, ctl, 8);
                    const bool staged = wait_bar(BAR(kBStaged), pairs & 1, ctl, 8);
                    ptx::fence_after();
                    if (staged) {
#pragma unroll
                        for (int g = 0; g < NG; ++g)
                            ptx::tmem_cp_128x128b(tmem + colBeta<F8>(row) + 4 * g,
                                                  ptx::smem_desc(sbase + kOffBeta + row * kBetaRow + g * kStrip * 16, 16, 128));
                    }
                    ptx::mma_commit(BAR(kBFree));
                    ptx::mma_commit(BAR(kBetaIn0 + row));
                    const bool brdy = staged && wait_bar(BAR(kBetaIn0 + row), pairs & 1, ctl, 8);
                    ptx::fence_after();
                    for (int c = 0; c < kChunks; ++c, ++it) {
                        const int h = c & 1;
                        const uint32_t slot = it % kSlots;
                        const bool full = wait_bar(BAR(kFull0 + slot), (it / kSlots) & 1, ctl, 2);
                        const bool free_buf = wait_bar(BAR(kDEmpty0 + h), (uses[h] & 1) ^ 1, ctl, 16);
                        ptx::fence_after();
                        if (brdy && full && free_buf) {
                            const uint32_t n = p.item[c].n;
                            const uint32_t idesc = (n == (uint32_t)kMainN) ? idesc_n96 : idesc_n48;
                            const uint64_t bd = ptx::smem_desc(sbase + kOffRing + slot * kSlot, n * 16, 128);
                            const uint64_t bstep = (uint64_t)(2 * n);
                            const uint32_t d = tmem + colDB(h) + row * kMainN, a = tmem + colBeta<F8>(row);
                            if (F8) {
                                // G = b_hi H_hi + b_lo H_hi + b_hi H_lo: 3 products x 4 K-steps of 32;
                                // the lo basis image follows the hi one (n rows x 128 bytes)
                                const uint64_t bd_lo = ptx::smem_desc(sbase + kOffRing + slot * kSlot + n * 128, n * 16, 128);
#pragma unroll
                                for (int pr = 0; pr < 3; ++pr)
#pragma unroll
                                    for (int ks = 0; ks < 4; ++ks)
                                        ptx::mma_ts_f8(d, a + (pr == 1 ? 32 : 0) + ks * 8, (pr == 2 ? bd_lo : bd) + ks * bstep,
                                                       idesc, (pr > 0 || ks > 0) ? 1u : 0u);
                            } else {
#pragma unroll
                                for (int ks = 0; ks < kKSteps; ++ks)
                                    ptx::mma_ts(d, a + ks * 8, bd + ks * bstep, idesc, ks > 0 ? 1u : 0u);
                            }
                        }
                        ptx::mma_commit(BAR(kEmpty0 + slot));
                        ptx::mma_commit(BAR(kDFull0 + h));
                        ++uses[h];
                    }
                    ptx::mma_commit(BAR(kPairDone0 + row));
                }
            }
        }
    } else {
        // ---------------- 16 accumulating warps: four per TMEM lane quadrant ----------------
        const int e = warp - 2;
        const int grp = e >> 2;
        const int quad = warp & 3;
        const int col = quad * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
        const int tid_e = threadIdx.x - 64;
        uint32_t pairs = 0, uses = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < p.tiles_total; tile += gridDim.x) {
            const int f = frame_of(p, tile);
            const Frame &F = p.fr[f];
            const int lt = tile - F.tile_base;
            const int tyy = lt / F.tiles_x, txx = lt - tyy * F.tiles_x;
            const int r_band = tyy * kBand, c0 = txx * kStrip;
            const int npair = n_pairs_of(tile);
            ptx::named_bar(1, kEpi);  // previous tile fully consumed
            for (int i = tid_e; i < kXPairs * kTC; i += kEpi) {
                // pair j: tile rows 2 j - 1 and 2 j (rows outside the tile or the frame are 0)
                const int j = i / kTC, tcol = i - j * kTC;
                const int gc = c0 - kHalo + tcol;
                uint2 px2[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int tr = 2 * j - 1 + h, gr = r_band - kHalo + tr;
                    float r = 0.f, g = 0.f, b = 0.f;
                    if (tr >= 0 && tr < kTR && gr >= 0 && gr < F.H && gc >= 0 && gc < F.W) {
                        const float *px = F.xw + ((size_t)gr * F.W + gc) * C;
                        r = __ldg(px);
                        if (C == 3) {
                            g = __ldg(px + 1);
                            b = __ldg(px + 2);
                        }
                    }
                    px2[h] = encode_px(r, g, b);
                }
                xp[i] = make_uint4(px2[0].x, px2[0].y, px2[1].x, px2[1].y);
            }
            ptx::named_bar(1, kEpi);
            for (int rp = 0; rp < npair; ++rp, ++pairs) {
                float acc[2][3];
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) acc[i][ch] = 0.f;
                accumulate_pair<C>(p, xp, lane_base, col, rp, grp, bar0, uses, ok, ctl, lane, acc);
                // ---- add the four groups' partial sums, write the row pair ----
                if (grp > 0) {
                    float *xc = xchg + (grp - 1) * kStrip * 6;
#pragma unroll
                    for (int i = 0; i < 2; ++i)
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) xc[col * 6 + i * 3 + ch] = acc[i][ch];
                }
                ptx::named_bar(2, kEpi);
                if (grp == 0 && ok) {
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const int orow = r_band + 2 * rp + i;
                        if (orow < F.H && c0 + col < F.W) {
                            float *o = F.y + ((size_t)orow * F.W + c0 + col) * C;
#pragma unroll
                            for (int ch = 0; ch < C; ++ch) {
                                const float v = acc[i][ch] + xchg[col * 6 + i * 3 + ch] +
                                                xchg[kStrip * 6 + col * 6 + i * 3 + ch] +
                                                xchg[2 * kStrip * 6 + col * 6 + i * 3 + ch];
                                o[ch] = F8 ? v * p.inv_c : v;
                            }
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

}  // namespace gs

using namespace gs;

p2s_status launch_gather_split(p2s_ctx *ctx, const TcFrame *frames, const void *const *beta16, int n, int C,
                               int *status, cudaStream_t st) {
    if (n <= 0) return P2S_OK;
    p2s_status s0 = tc_prepare(ctx);
    if (s0 != P2S_OK) return s0;
    for (int i0 = 0; i0 < n; i0 += kMaxFrames) {
        const int nb = n - i0 < kMaxFrames ? n - i0 : kMaxFrames;
        thread_local Params p;
        std::memset(&p, 0, sizeof p);
        int tiles = 0;
        double npx = 0.0;
        for (int i = 0; i < nb; ++i) {
            const TcFrame &t = frames[i0 + i];
            Frame &f = p.fr[i];
            f.xw = t.xw;
            f.y = t.y;
            f.beta16 = (const uint4 *)beta16[i0 + i];
            f.H = t.H;
            f.W = t.W;
            f.tiles_x = (t.W + kStrip - 1) / kStrip;
            f.tiles_y = (t.H + kBand - 1) / kBand;
            f.tile_base = tiles;
            tiles += f.tiles_x * f.tiles_y;
            npx += (double)t.H * t.W;
        }
        p.n_frames = nb;
        p.tiles_total = tiles;
        const bool f8 = ctx->prec == P2S_FP8E4M3;
        if (f8) {
            // E4M3 hi/lo basis images (one item per chunk: hi image then lo image)
            p.stream = (const uint8_t *)ctx->tc.d_H8;
            for (int c = 0; c < kChunks; ++c)
                p.item[c] = Item{ctx->tc.item8_off[c], ctx->tc.item8_bytes[c], ctx->tc.item8_n[c], 128};
            p.inv_c = ctx->tc.inv_c8;
        } else {
            p.stream = (const uint8_t *)ctx->tc.d_H;
            const Item16 *items = (const Item16 *)ctx->tc_items.data();
            for (int c = 0; c < kChunks; ++c) {
                const Item16 &it = items[6 + c];
                p.item[c] = Item{it.offset, it.bytes, it.n, it.k};
            }
            p.inv_c = 1.f;
        }
        p.ab_fmt = f8 ? 0 : ctx->tc.fmt;  // E4M3 is type 0 of .kind::f8f6f4, FP16 type 0 of .kind::f16
        p.status = status;
        int sms = 148;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
        const int grid = tiles < sms ? tiles : sms;
        ProfScope pr(ctx, st, f8 ? "blur_tc_gather8" : "blur_tc_gather16", 2.0 * ctx->K * ctx->T * npx,
                     npx * (C * 8.0 + (f8 ? kGroups8 : kGroups) * 16.0));
        auto run = [&](auto kern) -> p2s_status {
            P2S_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
            kern<<<grid, kThreads, kSmemBytes, st>>>(p);
            return P2S_OK;
        };
        p2s_status rs = C == 3 ? (f8 ? run(gather_kernel<3, true>) : run(gather_kernel<3, false>))
                               : (f8 ? run(gather_kernel<1, true>) : run(gather_kernel<1, false>));
        if (rs != P2S_OK) return rs;
        P2S_CUDA(cudaGetLastError());
    }
    return P2S_OK;
}

}  // namespace p2s
