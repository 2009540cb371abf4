// Blur-only tensor-core gather (Sec. 3.1, Eq. 5) reading beta from the
// network kernel's 16-bit operand layout, third variant (P2S_OPT_GATHER_SPLIT
// = 3): the 16x256b-fragment scheme of the second variant (4 adjacent output
// columns per accumulating thread), with x staged in FP32 and every tap
// product of the R and G channels one lane of a packed FP32 FMA
// (fma.rn.f32x2, G broadcast), G taken from TMEM in FP32 as the tensor core
// summed it.  No operand of the tap accumulation is rounded: this kernel's
// only rounding points are beta and H in the 16-bit operand type.  Tiles are
// 128 x 16 so that the FP32 x tile fits beside the basis ring.
//
// Per row pair of a 128 x 32 tile:
//   producer  beta rows (2 x 14 runs of 16-byte groups) into a staging buffer
//             with 1-D bulk copies, basis chunks into a 2-slot ring;
//   MMA       two threads, one per output row: the row's beta into TMEM
//             (tcgen05.cp), then G = beta H chunk by chunk (N = 96: 3 tap
//             columns x 32 tap rows, then N = 48 for the last tap row), two
//             TMEM accumulator buffers;
//   gather    y_c[q] += G[q, t] x_c[q - o(t)] by 8 accumulating warps, two per
//             TMEM lane quadrant.  Each thread reads G through 16x256b
//             fragments: four TMEM lanes, which the network kernel's permuted
//             beta layout makes 4 adjacent output columns, and per chunk 12
//             taps (4 tap rows x 3 tap columns, the basis chunk's columns
//             ordered to match), for both output rows.  Its x window is then
//             5 rows x 6 columns for 96 tap products, half the shared-memory
//             bytes per product of one column per thread.  x is staged as FP16
//             RGB and G rounded to FP16, so each product is one fma.rn.f32.f16
//             (FP16 operands, FP32 accumulation).  The partial sums of the 4
//             threads sharing a pixel meet by shuffles, those of the two warps
//             of a quadrant in shared memory.
// Every wait is bounded.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstring>

#include "p2s_internal.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace p2s {
namespace gx {

using tcc::Ctl;
using tcc::drain_bar;
using tcc::wait_bar;

constexpr int kStrip = 128;
constexpr int kBand = 16;
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
constexpr int kAccWarps = 8;                      // two per TMEM lane quadrant
constexpr int kEpi = 32 * kAccWarps;              // 256
constexpr int kThreads = 64 + kEpi + 32;          // 352: + the second MMA warp (row 1)
constexpr int kMmaWarp1 = (64 + kEpi) / 32;       // 10
constexpr int kXPairs = kTR / 2 + 1;              // x tile rows (2 j - 1, 2 j), j = 0 .. 24
constexpr int kBetaRow = kGroups * kStrip * 16;   // 28,672 B per staged row
constexpr int kItemBase = 6 + kChunks;            // this kernel's basis images in the item table

__host__ __device__ constexpr uint32_t colBeta(int r) { return r ? 56u : 0u; }
__host__ __device__ constexpr uint32_t colDB(int h) { return h ? 320u : 128u; }

constexpr int kOffRing = 0;
constexpr int kOffRG = kOffRing + kSlots * kSlot;          // float4 [kXPairs][kTC]: (R, G) of rows 2 j - 1, 2 j
constexpr int kOffB = kOffRG + kXPairs * kTC * 16;         // float2 [kXPairs][kTC]: B of rows 2 j - 1, 2 j
constexpr int kOffBeta = kOffB + kXPairs * kTC * 8;        // [2 rows][14][128][16 B]
constexpr int kOffXchg = kOffBeta + 2 * kBetaRow;          // float [2 pair parities][128 threads][6]
enum Bar { kFull0 = 0, kEmpty0 = 2, kBStaged = 4, kBFree = 5, kBetaIn0 = 6, kPairDone0 = 8, kDFull0 = 10, kDEmpty0 = 12,
           kNBar = 14 };
constexpr int kOffBar = kOffXchg + 2 * 128 * 6 * 4;
constexpr int kOffMisc = kOffBar + kNBar * 8;
constexpr int kSmemBytes = kOffMisc + 16 + 1024;
static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");

struct Item {
    uint32_t offset, bytes, n, k;
};

struct Frame {
    const float *xw;
    float *y;
    const uint4 *beta16;  // [H][14][pitch] 16-byte groups, columns permuted within 32-column blocks
    int H, W, pitch, tiles_x, tiles_y, tile_base;
};
constexpr int kMaxFrames = 256;

struct Params {
    Frame fr[kMaxFrames];
    int n_frames, tiles_total;
    const uint8_t *stream;  // basis chunk images
    Item item[kChunks];
    int ab_fmt;
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

// Column c of x tile pair row `pair` sits at index pair * kTC + (c ^ swz(pair)) of both
// the RG and the B array.  The threads of a quarter warp (16-byte RG loads) or half warp
// (8-byte B loads) read 2 columns 4 apart in 4 pair rows 2 apart; the swizzle puts them in
// distinct bank groups.
__device__ __forceinline__ int swz(int pair) { return (pair >> 1) & 3; }

// One window column of a main chunk, FP32: rows 0, 1 (pair P0), 2, 3 (pair P0 + 1) and 4
// (the first row of pair P0 + 2).
struct XCol {
    float4 rg0, rg1;  // (R, G) of both rows of a pair
    float2 rg2;       // (R, G) of row 4
    float2 b0, b1;    // B of both rows of a pair
    float b2;         // B of row 4
};

__device__ __forceinline__ void load_col(const float4 *rg, const float2 *bv, int P0, int col, XCol &x) {
    const int i0 = P0 * kTC + (col ^ swz(P0)), i1 = (P0 + 1) * kTC + (col ^ swz(P0 + 1)),
              i2 = (P0 + 2) * kTC + (col ^ swz(P0 + 2));
    x.rg0 = rg[i0];
    x.rg1 = rg[i1];
    x.rg2 = reinterpret_cast<const float2 *>(rg)[2 * i2];
    x.b0 = bv[i0];
    x.b1 = bv[i1];
    x.b2 = reinterpret_cast<const float *>(bv)[2 * i2];
}

// acc += g x for one output pixel and tap: (R, G) as one packed FMA with g broadcast.
template <int C>
__device__ __forceinline__ void tap(float g, float r, float gg, float b, float (&acc)[3]) {
    if (C == 3) {
        tcc::fma2_bcast(g, r, gg, acc[0], acc[1]);
        acc[2] = fmaf(g, b, acc[2]);
    } else {
        acc[0] = fmaf(g, r, acc[0]);
    }
}

// The products of output pixel s of a main chunk's tap column: 2 output rows (r) x 4 tap
// rows (k); x is the window column the pixel reads, row 3 + r - k of it.  G of (s, r, k)
// is register 4 (k / 2) + 2 (s % 2) + k % 2 of the (lane half s / 2, row r) fragment.
template <int C, int S>
__device__ __forceinline__ void tap_pixel(const XCol &x, const uint32_t (&g)[2][2][8], float (&acc)[2][3]) {
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int wi = 3 + r - k;
            float xr, xg, xb;
            if (wi == 4) {
                xr = x.rg2.x;
                xg = x.rg2.y;
                xb = x.b2;
            } else {
                const float4 &v = wi < 2 ? x.rg0 : x.rg1;
                const float2 &b = wi < 2 ? x.b0 : x.b1;
                xr = (wi & 1) ? v.z : v.x;
                xg = (wi & 1) ? v.w : v.y;
                xb = (wi & 1) ? b.y : b.x;
            }
            const float gv = __uint_as_float(g[S >> 1][r][4 * (k >> 1) + 2 * (S & 1) + (k & 1)]);
            tap<C>(gv, xr, xg, xb, acc[r]);
        }
}

template <int C>
__device__ __forceinline__ void tap_column(const XCol &x0, const XCol &x1, const XCol &x2, const XCol &x3,
                                           const uint32_t (&g)[2][2][8], float (&acc)[4][2][3]) {
    tap_pixel<C, 0>(x0, g, acc[0]);
    tap_pixel<C, 1>(x1, g, acc[1]);
    tap_pixel<C, 2>(x2, g, acc[2]);
    tap_pixel<C, 3>(x3, g, acc[3]);
}

// G of tap column u of a main chunk (4 x 16x256b.x2: lane half h, output row r).
__device__ __forceinline__ void load_g(uint32_t tq, uint32_t dcol, int m, int u, uint32_t (&raw)[2][2][8]) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int r = 0; r < 2; ++r)
            ptx::tmem_ld_16x256b_x2(tq + ((uint32_t)(16 * h) << 16) + dcol + r * kMainN + 8 * (6 * m + 2 * u), raw[h][r]);
}

// The last chunk: tap row 32, tap columns 24 m + 6 j + t (t = 2 b + e < nvalid) for this
// thread.  Output row r reads x tile row 2 rp + r (row 0: the second row of pair rp, row 1:
// the first of pair rp + 1), column cl + 5 + s - t; x read per product (1/33 of the taps).
template <int C>
__device__ __forceinline__ void chunk_last(const float4 *rg, const float2 *bv, uint32_t tq, uint32_t dcol, int m,
                                           int rp, int cl, int nvalid, float (&acc)[4][2][3]) {
    const float2 *rg2 = reinterpret_cast<const float2 *>(rg);
    const float *b1 = reinterpret_cast<const float *>(bv);
#pragma unroll 1
    for (int b = 0; b < 3; ++b) {
        // every lane issues the TMEM loads (.sync.aligned: the whole warp, converged)
        uint32_t g[2][2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int r = 0; r < 2; ++r)
                ptx::tmem_ld_16x256b_x1(tq + ((uint32_t)(16 * h) << 16) + dcol + r * kMainN + 24 * m + 8 * b, g[h][r]);
        ptx::tmem_wait_ld_dep(*reinterpret_cast<uint32_t(*)[16]>(&g[0][0][0]));
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int i = s & 1, h = s >> 1, pr = rp + r;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int t = 2 * b + e;
                    if (t < nvalid) {
                        const int idx = pr * kTC + ((cl + 5 + s - t) ^ swz(pr));
                        const int half = r ? 0 : 1;
                        const float2 v = rg2[2 * idx + half];
                        tap<C>(__uint_as_float(g[h][r][2 * i + e]), v.x, v.y, b1[2 * idx + half], acc[s][r]);
                    }
                }
            }
    }
}

// All chunks of one row pair for an accumulating thread (quadrant q, warp team m, lane
// group a = lane / 4, tap-row group j = lane % 4).  Main chunk c covers tap columns
// 3 c .. 3 c + 2 and, for this thread, tap rows 16 m + 4 j .. + 3.
template <int C>
__device__ __forceinline__ void accumulate_pair(const float4 *rg, const float2 *bv, uint32_t tq, int q, int m, int a,
                                                int j, int rp, uint32_t bar0, uint32_t &uses, bool &ok,
                                                const Ctl &ctl, int lane, float (&acc)[4][2][3]) {
    auto BAR = [&](int i) { return bar0 + 8u * (uint32_t)i; };
    // main chunks: window rows 2 rp + 29 - 16 m - 4 j .. + 4 (the first one odd, so it starts a
    // pixel pair), window columns 32 q + 4 a + 30 - 3 c .. + 5
    const int P0 = rp + 15 - 8 * m - 2 * j;
    const int cb0 = 32 * q + 4 * a + 30;
    const int nvalid = min(6, 33 - 24 * m - 6 * j);
    const int cl = 32 * q + 4 * a + 27 - 24 * m - 6 * j;
    auto wait_full = [&](int c) {
        const int b = c & 1;
        const bool got = __all_sync(0xffffffffu, wait_bar(BAR(kDFull0 + b), (uses >> b) & 1, ctl, 128));
        uses ^= (1u << b);
        ok = ok && got;
        ptx::fence_after();
        return got;
    };
    auto release = [&](int c) {
        ptx::fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(BAR(kDEmpty0 + (c & 1)));
    };
#pragma unroll 1
    for (int c = 0; c < kMainChunks; ++c) {
        if (wait_full(c)) {
            // window columns cb .. cb + 5: tap column u reads columns 2 - u .. 5 - u
            const int cb = cb0 - 3 * c;
            const uint32_t dcol = colDB(c & 1);
            uint32_t g[2][2][8];
            XCol x0, x1, x2, x3, x4, x5;
            load_g(tq, dcol, m, 0, g);
            load_col(rg, bv, P0, cb + 2, x2);
            load_col(rg, bv, P0, cb + 3, x3);
            load_col(rg, bv, P0, cb + 4, x4);
            load_col(rg, bv, P0, cb + 5, x5);
            ptx::tmem_wait_ld_dep(*reinterpret_cast<uint32_t(*)[32]>(&g[0][0][0]));
            tap_column<C>(x2, x3, x4, x5, g, acc);
            load_g(tq, dcol, m, 1, g);
            load_col(rg, bv, P0, cb + 1, x1);
            ptx::tmem_wait_ld_dep(*reinterpret_cast<uint32_t(*)[32]>(&g[0][0][0]));
            tap_column<C>(x1, x2, x3, x4, g, acc);
            load_g(tq, dcol, m, 2, g);
            load_col(rg, bv, P0, cb, x0);
            ptx::tmem_wait_ld_dep(*reinterpret_cast<uint32_t(*)[32]>(&g[0][0][0]));
            release(c);  // this chunk's G is in registers
            tap_column<C>(x0, x1, x2, x3, g, acc);
        } else {
            release(c);
        }
    }
    const int cL = kMainChunks;
    if (wait_full(cL)) chunk_last<C>(rg, bv, tq, colDB(cL & 1), m, rp, cl, nvalid, acc);
    release(cL);
}

// Sum the partial sums of the 4 threads of a lane group (lanes 4 a .. 4 a + 3): afterwards
// thread j holds pixels s = 2 (j >> 1) + s2 (s2 = 0, 1) of output row j & 1, all channels.
__device__ __forceinline__ void reduce_quad(const float (&acc)[4][2][3], int j, float (&out)[2][3]) {
    float r1[2][2][3];
    const bool hi2 = j & 2, hi1 = j & 1;
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float keep = hi2 ? acc[s2 + 2][r][ch] : acc[s2][r][ch];
                const float send = hi2 ? acc[s2][r][ch] : acc[s2 + 2][r][ch];
                r1[s2][r][ch] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
            }
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float keep = hi1 ? r1[s2][1][ch] : r1[s2][0][ch];
            const float send = hi1 ? r1[s2][0][ch] : r1[s2][1][ch];
            out[s2][ch] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
        }
}

template <int C>
__global__ void __launch_bounds__(kThreads, 1) gather_kernel(const __grid_constant__ Params p) {
    extern __shared__ uint8_t smem_raw[];
    // aligned by pointer arithmetic on the __shared__ array, so that the compiler still
    // knows every access through `sm` is to shared memory (ld/st.shared, not generic)
    uint8_t *sm = smem_raw + ((1024u - (uint32_t)((uintptr_t)smem_raw & 1023u)) & 1023u);
    const uint32_t sbase = ptx::smem_u32(sm);
    float4 *rg = (float4 *)(sm + kOffRG);
    float2 *bv = (float2 *)(sm + kOffB);
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
            ptx::mbar_init(BAR(kDEmpty0 + i), kAccWarps);
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
                // positions c0 .. c0 + cols - 1 of the permuted rows (pitch a multiple of 32)
                const uint32_t cols = (uint32_t)min(kStrip, F.pitch - c0);
                for (int rp = 0; rp < npair; ++rp, ++pairs) {
                    // beta of the pair's rows; the staging buffer is free once both rows are in TMEM
                    if (wait_bar(BAR(kBFree), (pairs & 1) ^ 1, ctl, 1)) {
                        const int r0 = tyy * kBand + 2 * rp;
                        const int nrow = min(2, F.H - r0);
                        ptx::mbar_arrive_tx(BAR(kBStaged), (uint32_t)nrow * kGroups * cols * 16);
                        for (int i = 0; i < nrow; ++i)
                            for (int g = 0; g < kGroups; ++g)
                                ptx::bulk_g2s(sbase + kOffBeta + i * kBetaRow + g * kStrip * 16,
                                              F.beta16 + ((size_t)(r0 + i) * kGroups + g) * F.pitch + c0, cols * 16,
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
        // ---------------- MMA issuers: warp 0 row 0, warp 10 row 1 ----------------
        // One thread issues an MMA about every 76-100 cycles whatever its size; two
        // threads in two warps, each on its own accumulator, keep the tensor core busy.
        if (lane == 0) {
            const int row = warp == 0 ? 0 : 1;
            uint32_t it = 0, pairs = 0, uses[2] = {0, 0};
            for (int tile = blockIdx.x; tile < p.tiles_total; tile += gridDim.x) {
                const int npair = n_pairs_of(tile);
                for (int rp = 0; rp < npair; ++rp, ++pairs) {
                    // this row's beta into TMEM by tcgen05.cp, once the row's MMAs of the
                    // previous pair are done with it
                    if (pairs > 0) wait_bar(BAR(kPairDone0 + row), (pairs - 1) & 1, ctl, 8);
                    const bool staged = wait_bar(BAR(kBStaged), pairs & 1, ctl, 8);
                    ptx::fence_after();
                    if (staged) {
#pragma unroll
                        for (int g = 0; g < kGroups; ++g)
                            ptx::tmem_cp_128x128b(tmem + colBeta(row) + 4 * g,
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
                            const uint32_t d = tmem + colDB(h) + row * kMainN, a = tmem + colBeta(row);
#pragma unroll
                            for (int ks = 0; ks < kKSteps; ++ks)
                                ptx::mma_ts(d, a + ks * 8, bd + ks * bstep, idesc, ks > 0 ? 1u : 0u);
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
        // ---------------- 8 accumulating warps: two per TMEM lane quadrant ----------------
        const int q = warp & 3;          // the lane quadrant this warp may access
        const int m = (warp - 2) >> 2;   // team: tap rows 16 m .. 16 m + 15 of every chunk
        const int a = lane >> 2, j = lane & 3;
        const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
        const int tid_e = threadIdx.x - 64;
        const int slot = q * 32 + lane;  // this thread's partner in the other team has the same slot
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
                // pair jj: tile rows 2 jj - 1 and 2 jj (rows outside the tile or the frame are 0), FP32
                const int jj = i / kTC, tcol = i - jj * kTC;
                const int gc = c0 - kHalo + tcol;
                float px[2][3];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int tr = 2 * jj - 1 + h, gr = r_band - kHalo + tr;
                    px[h][0] = px[h][1] = px[h][2] = 0.f;
                    if (tr >= 0 && tr < kTR && gr >= 0 && gr < F.H && gc >= 0 && gc < F.W) {
                        const float *p = F.xw + ((size_t)gr * F.W + gc) * C;
                        px[h][0] = __ldg(p);
                        if (C == 3) {
                            px[h][1] = __ldg(p + 1);
                            px[h][2] = __ldg(p + 2);
                        }
                    }
                }
                const int k = jj * kTC + (tcol ^ swz(jj));
                rg[k] = make_float4(px[0][0], px[0][1], px[1][0], px[1][1]);
                bv[k] = make_float2(px[0][2], px[1][2]);
            }
            ptx::named_bar(1, kEpi);
            for (int rp = 0; rp < npair; ++rp, ++pairs) {
                float acc[4][2][3];
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int r = 0; r < 2; ++r)
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) acc[s][r][ch] = 0.f;
                accumulate_pair<C>(rg, bv, tq, q, m, a, j, rp, bar0, uses, ok, ctl, lane, acc);
                float sum[2][3];
                reduce_quad(acc, j, sum);
                // the two teams meet in shared memory (double-buffered by pair parity)
                float *xc = xchg + ((pairs & 1) * 128 + slot) * 6;
                if (m == 1) {
#pragma unroll
                    for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) xc[s2 * 3 + ch] = sum[s2][ch];
                }
                ptx::named_bar(2, kEpi);
                if (m == 0 && ok) {
                    const int orow = r_band + 2 * rp + (j & 1);
#pragma unroll
                    for (int s2 = 0; s2 < 2; ++s2) {
                        const int oc = c0 + 32 * q + 4 * a + 2 * (j >> 1) + s2;
                        if (orow < F.H && oc < F.W) {
                            float *o = F.y + ((size_t)orow * F.W + oc) * C;
#pragma unroll
                            for (int ch = 0; ch < C; ++ch) o[ch] = sum[s2][ch] + xc[s2 * 3 + ch];
                        }
                    }
                }
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

}  // namespace gx

using namespace gx;

p2s_status launch_gather_x32(p2s_ctx *ctx, const TcFrame *frames, const void *const *beta16, int n, int C,
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
            f.pitch = beta16_pitch(t.W, 1);
            f.tiles_x = (t.W + kStrip - 1) / kStrip;
            f.tiles_y = (t.H + kBand - 1) / kBand;
            f.tile_base = tiles;
            tiles += f.tiles_x * f.tiles_y;
            npx += (double)t.H * t.W;
        }
        p.n_frames = nb;
        p.tiles_total = tiles;
        p.stream = (const uint8_t *)ctx->tc.d_H;
        const Item16 *items = (const Item16 *)ctx->tc_items.data();
        if (ctx->tc_items.size() < (size_t)(kItemBase + kChunks) * sizeof(Item16)) {
            set_error("tensor-core operand stream lacks the split gather's basis images");
            return P2S_EUNSUPPORTED;
        }
        for (int c = 0; c < kChunks; ++c) {
            const Item16 &it = items[kItemBase + c];
            p.item[c] = Item{it.offset, it.bytes, it.n, it.k};
        }
        p.ab_fmt = ctx->tc.fmt;
        p.status = status;
        int sms = 148;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
        const int grid = tiles < sms ? tiles : sms;
        ProfScope pr(ctx, st, "blur_tc_gather_x32", 2.0 * ctx->K * ctx->T * npx, npx * (C * 8.0 + kGroups * 16.0));
        if (C == 3) {
            P2S_CUDA(cudaFuncSetAttribute(gather_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
            gather_kernel<3><<<grid, kThreads, kSmemBytes, st>>>(p);
        } else {
            P2S_CUDA(cudaFuncSetAttribute(gather_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
            gather_kernel<1><<<grid, kThreads, kSmemBytes, st>>>(p);
        }
        P2S_CUDA(cudaGetLastError());
    }
    return P2S_OK;
}

}  // namespace p2s
