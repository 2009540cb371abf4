// Blur-only tensor-core gather (Sec. 3.1, Eq. 5) with the tap products as packed
// FP16 FMAs: P2S_OPT_GATHER_SPLIT = 4.  Same roles, tiles and beta layout as the
// split kernel 1 (k_gather.cu); what changes is how a thread's two output rows
// share work.
//
// Output rows r and r + 1 of a pair read the same x_w pixel at tap rows ty and
// ty + 1 of the same tap column: (r - (ty - 16)) = (r + 1 - (ty + 1 - 16)).  So
// one fma.rn.f16x2 with G packed as (G_r[ty, tx], G_r+1[ty + 1, tx]) and x_w
// broadcast to both halves does one tap product for each row: one conversion
// and C packed FMAs per tap pair.  The MMA of row
// r + 1 reads the same basis chunk one tap row (32 N-rows) further in:
//   main chunk c (0 .. 10): extended tap rows e in [3 c, 3 c + 4) x tap columns
//     [0, 32), N-row (e - 3 c) * 32 + tx, tap row ty = e - 1 (rows -1 and 33 zero);
//     row r takes N-rows [0, 96), row r + 1 N-rows [32, 128): tap pair
//     p = 3 c + j (j < 3) is (row r, ty = p - 1) with (row r + 1, ty = p).
//   last chunk (11): N-rows [0, 32) tap row 32 of tap columns 0 .. 31 (row r only),
//     N-rows [32, 65) tap column 32 of tap rows 0 .. 32, then zeros to 80; row r
//     takes [0, 80), row r + 1 [32, 80).
// Tap column 32 is the one place the rows read different pixels for the same
// tap: there the products are mixed FMAs (FP16 operands, FP32 sums), as in
// kernel 1.  The packed sums are FP16 within a chunk (two per channel and row, by
// tap-column parity, 12 products each) and flushed into FP32 at its end; the
// four groups of warps split the tap columns
// (8 each) and add their FP32 partial sums through shared memory.
// Every wait is bounded.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstring>

#include "p2s_internal.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace p2s {
namespace gh {

using tcc::Ctl;
using tcc::drain_bar;
using tcc::wait_bar;

constexpr int kStrip = 128;
constexpr int kBand = 32;
constexpr int kHalo = 16;
constexpr int kTC = kStrip + 2 * kHalo;           // 160 tile columns (tile rows: kBand + 2 kHalo = 64)
constexpr int kXRing = 2 * kHalo + 4;             // 36 x_w rows held: a pair's 34 and the next pair's 2
constexpr int kKSteps = 7;
constexpr int kMainChunks = 11;
constexpr int kChunks = kMainChunks + 1;
constexpr int kImgMain = 128;                     // N-rows of a main chunk image
constexpr int kImgLast = 80;
constexpr int kSlot = 28672;                      // one main chunk image: 128 N-rows x 112 x 2 B
constexpr int kSlots = 3;
constexpr int kGroups = 14;                       // beta16 k-groups
constexpr int kGroupsEpi = 4;                     // accumulating groups of 4 warps
constexpr int kEpi = 128 * kGroupsEpi;            // 512
constexpr int kThreads = 64 + kEpi + 64;          // 640: + the second MMA warp and the beta producer
constexpr int kMmaWarp1 = (64 + kEpi) / 32;       // 18
constexpr int kBetaWarp = kMmaWarp1 + 1;          // 19
constexpr int kBetaRow = kGroups * kStrip * 16;   // 28,672 B per staged row
constexpr int kItemBase = 6 + 2 * kChunks;        // this kernel's basis images in the item table
static_assert(kImgMain * kKSteps * 32 <= kSlot, "basis chunk image fits a ring slot");

__host__ __device__ constexpr uint32_t colBeta(int r) { return r ? 56u : 0u; }
__host__ __device__ constexpr uint32_t colDB(int h) { return h ? 320u : 128u; }

constexpr int kOffRing = 0;
constexpr int kOffX = kOffRing + kSlots * kSlot;           // [kXRing][kTC] pixels (8 B for RGB, 4 B for one channel)
constexpr int kOffBeta = kOffX + kXRing * kTC * 8;         // [2 rows][14][128][16 B]
constexpr int kOffXchg = kOffBeta + 2 * kBetaRow;          // float [3][128][6]
enum Bar { kFull0 = 0, kEmpty0 = 3, kBStaged = 6, kBFree = 7, kBetaIn0 = 8, kPairDone0 = 10, kDFull0 = 12, kDEmpty0 = 14,
           kNBar = 16 };
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
    const uint4 *beta16;  // [H][14][W] 16-byte groups
    int H, W, tiles_x, tiles_y, tile_base;
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

// x_w in shared memory, one entry per tile pixel: three channels as 8 bytes of FP16,
// (R, G) and (B, 0); one channel as one 32-bit word (R, 0), half the shared-memory
// traffic of the 8-byte form (a warp's 8-byte loads take two wavefronts, its 4-byte
// loads one).
template <int C>
struct XPix {
    using T = uint2;
};
template <>
struct XPix<1> {
    using T = uint32_t;
};
__device__ __forceinline__ uint32_t half_pair(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}
template <int C>
__device__ __forceinline__ typename XPix<C>::T encode_px(float r, float g, float b) {
    if constexpr (C == 3)
        return make_uint2(half_pair(r, g), half_pair(b, 0.f));
    else
        return half_pair(r, 0.f);
}
__device__ __forceinline__ uint32_t rg_of(uint2 v) { return v.x; }
__device__ __forceinline__ uint32_t rg_of(uint32_t v) { return v; }

// The packed tap products of 8 tap pairs: G of row r in g0, of row r + 1 in g1, x_w in v;
// a[u & 1][ch] = (channel ch of row r, of row r + 1), x_w broadcast to both halves (the
// broadcast is an operand selector of the packed FMA, not an instruction).  Two sums per
// channel, by the parity of the tap column, halve the dependent chains.  One conversion
// per pair.
template <int C>
__device__ __forceinline__ void tap_pairs8(const uint32_t (&g0)[8], const uint32_t (&g1)[8],
                                           const typename XPix<C>::T (&v)[8], uint32_t (&a)[2][3]) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const uint32_t g2 = tcc::pack_f16x2(__uint_as_float(g0[u]), __uint_as_float(g1[u]));
        tcc::hfma2_bcast<false>(a[u & 1][0], g2, rg_of(v[u]));
        if constexpr (C == 3) {
            tcc::hfma2_bcast<true>(a[u & 1][1], g2, v[u].x);
            tcc::hfma2_bcast<false>(a[u & 1][2], g2, v[u].y);
        }
    }
}

// x_w ring row of tile row tr, given s0 = (2 rp) mod kXRing and tr - 2 rp = d in [0, 36)
__device__ __forceinline__ int xring_row(int s0, int d) {
    const int r = s0 + d;
    return r >= kXRing ? r - kXRing : r;
}

// One row pair: tile row of output row r is 2 rp + 16; tap (ty, tx) of row r reads
// tile row 2 rp + 32 - ty, tile column col + 32 - tx; tile row tr sits in ring row
// tr mod kXRing.
template <int C>
__device__ __forceinline__ void accumulate_pair(const typename XPix<C>::T *xs, uint32_t lane_base, int col, int rp,
                                                int grp,
                                                uint32_t bar0, uint32_t &uses, bool &ok, const Ctl &ctl, int lane,
                                                float (&acc)[2][3]) {
    auto BAR = [&](int i) { return bar0 + 8u * (uint32_t)i; };
    const int T0 = 8 * grp;  // this group's tap columns [T0, T0 + 8)
    const int s0 = (2 * rp) % kXRing;
    for (int c = 0; c < kChunks; ++c) {
        const int b = c & 1;
        const uint32_t buf = lane_base + colDB(b);
        const bool got = __all_sync(0xffffffffu, wait_bar(BAR(kDFull0 + b), (uses >> b) & 1, ctl, 128));
        uses ^= (1u << b);
        ok = ok && got;
        ptx::fence_after();
        uint32_t a[2][3] = {{0u, 0u, 0u}, {0u, 0u, 0u}};
        if (!got) {
        } else if (c < kMainChunks) {
#pragma unroll 1
            for (int j = 0; j < 3; ++j) {
                uint32_t g0[8], g1[8];
                ptx::tmem_ld8(buf + 32 * j + T0, g0);
                ptx::tmem_ld8(buf + 96 + 32 * j + T0, g1);
                // tap pair p = 3 c + j: row r at ty = p - 1, row r + 1 at ty = p
                const int base = xring_row(s0, 33 - (3 * c + j)) * kTC + col + 32 - T0;
                typename XPix<C>::T v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = xs[base - u];
                ptx::tmem_wait_ld_dep(g0);
                ptx::tmem_wait_ld_dep(g1);
                tap_pairs8<C>(g0, g1, v, a);
            }
        } else {
            // tap row 32 of tap columns [T0, T0 + 8), row r only (the high halves add 0)
            uint32_t g0[8], g1[8];
            ptx::tmem_ld8(buf + T0, g0);
            uint32_t h0[9], h1[9];
            // tap column 32, tap rows [9 grp, 9 grp + 9) below 33: both rows
            ptx::tmem_ld9(buf + 32 + 9 * grp, h0);
            ptx::tmem_ld9(buf + 96 + 9 * grp, h1);
            const int base = s0 * kTC + col + 32 - T0;
            typename XPix<C>::T v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                v[u] = xs[base - u];
                g1[u] = 0u;
            }
            ptx::tmem_wait_ld_dep(g0);
            ptx::tmem_wait_ld_dep(h0);
            ptx::tmem_wait_ld_dep(h1);
            tap_pairs8<C>(g0, g1, v, a);
            const int nq = min(9, 33 - 9 * grp);
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                if (q < nq) {
                    const int ty = 9 * grp + q;
                    const uint32_t gp = tcc::pack_f16x2(__uint_as_float(h0[q]), __uint_as_float(h1[q]));
                    const typename XPix<C>::T x0 = xs[xring_row(s0, 32 - ty) * kTC + col],
                                              x1 = xs[xring_row(s0, 33 - ty) * kTC + col];
                    if constexpr (C == 3) {
                        tcc::fma_mix_x2<false>(x0.x, gp, acc[0][0], acc[0][1]);
                        tcc::fma_mix_x1<false>(x0.y, gp, acc[0][2]);
                        tcc::fma_mix_x2<true>(x1.x, gp, acc[1][0], acc[1][1]);
                        tcc::fma_mix_x1<true>(x1.y, gp, acc[1][2]);
                    } else {
                        tcc::fma_mix_x1<false>(x0, gp, acc[0][0]);
                        tcc::fma_mix_x1<true>(x1, gp, acc[1][0]);
                    }
                }
            }
        }
        ptx::fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(BAR(kDEmpty0 + b));
        // the chunk's FP16 sums into the FP32 ones, even tap columns first (the column-32
        // products went there directly)
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int ch = 0; ch < C; ++ch) tcc::flush_f16x2(a[e][ch], acc[0][ch], acc[1][ch]);
    }
}

template <int C>
__global__ void __launch_bounds__(kThreads, 1) gather_h2_kernel(const __grid_constant__ Params p) {
    extern __shared__ uint8_t smem_raw[];
    // aligned by pointer arithmetic on the __shared__ array (accesses stay ld/st.shared)
    uint8_t *sm = smem_raw + ((1024u - (uint32_t)((uintptr_t)smem_raw & 1023u)) & 1023u);
    const uint32_t sbase = ptx::smem_u32(sm);
    using XT = typename XPix<C>::T;
    XT *xs = (XT *)(sm + kOffX);
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
        ptx::mbar_init(BAR(kBFree), 2);
        for (int r = 0; r < 2; ++r) {
            ptx::mbar_init(BAR(kBetaIn0 + r), 1);
            ptx::mbar_init(BAR(kPairDone0 + r), 1);
        }
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(BAR(kDFull0 + i), 2);
            ptx::mbar_init(BAR(kDEmpty0 + i), 4 * kGroupsEpi);
        }
        ptx::mbar_fence_init();
    }
    if (warp == 0) ptx::tmem_alloc(ptx::smem_u32(tmem_holder), 512);
    ptx::fence_before();
    __syncthreads();
    ptx::fence_after();
    const uint32_t tmem = *tmem_holder;

    auto n_pairs_of = [&](int tile) {
        const Frame &F = p.fr[frame_of(p, tile)];
        const int ty = (tile - F.tile_base) / F.tiles_x;
        return (min(kBand, F.H - ty * kBand) + 1) >> 1;
    };

    if (warp == 1) {
        // ---------------- basis producer: chunk images into the ring ----------------
        if (lane == 0) {
            uint32_t it = 0;
            for (int tile = blockIdx.x; tile < p.tiles_total; tile += gridDim.x) {
                const int npair = n_pairs_of(tile);
                for (int rp = 0; rp < npair; ++rp) {
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
        }
    } else if (warp == kBetaWarp) {
        // ---------------- beta producer: the next pair's rows as soon as the buffer frees ----------------
        if (lane == 0) {
            uint32_t pairs = 0;
            for (int tile = blockIdx.x; tile < p.tiles_total; tile += gridDim.x) {
                const int f = frame_of(p, tile);
                const Frame &F = p.fr[f];
                const int lt = tile - F.tile_base;
                const int tyy = lt / F.tiles_x, c0 = (lt - tyy * F.tiles_x) * kStrip;
                const int npair = n_pairs_of(tile);
                const uint32_t cols = (uint32_t)min(kStrip, F.W - c0);
                for (int rp = 0; rp < npair; ++rp, ++pairs) {
                    if (!wait_bar(BAR(kBFree), (pairs & 1) ^ 1, ctl, 1)) continue;
                    const int r0 = tyy * kBand + 2 * rp;
                    const int nrow = min(2, F.H - r0);
                    ptx::mbar_arrive_tx(BAR(kBStaged), (uint32_t)nrow * kGroups * cols * 16);
                    for (int i = 0; i < nrow; ++i)
                        for (int g = 0; g < kGroups; ++g)
                            ptx::bulk_g2s(sbase + kOffBeta + i * kBetaRow + g * kStrip * 16,
                                          F.beta16 + ((size_t)(r0 + i) * kGroups + g) * F.W + c0, cols * 16,
                                          BAR(kBStaged));
                }
            }
            if (pairs > 0) drain_bar(BAR(kBStaged), (pairs - 1) & 1);
        }
    } else if (warp == 0 || warp == kMmaWarp1) {
        // ---------------- MMA issuers: warp 0 row r, warp 18 row r + 1 ----------------
        if (lane == 0) {
            const int row = warp == 0 ? 0 : 1;
            uint32_t it = 0, pairs = 0, uses[2] = {0, 0};
            for (int tile = blockIdx.x; tile < p.tiles_total; tile += gridDim.x) {
                const int npair = n_pairs_of(tile);
                for (int rp = 0; rp < npair; ++rp, ++pairs) {
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
                            const bool last = c == kMainChunks;
                            const uint32_t nimg = p.item[c].n;
                            const uint32_t nr = row == 0 ? (last ? 80u : 96u) : (last ? 48u : 96u);
                            const uint32_t idesc = ptx::idesc_f16(p.ab_fmt, (int)nr);
                            // row r + 1 starts 32 N-rows (4 core matrices of 128 B) into the image
                            const uint64_t bd = ptx::smem_desc(sbase + kOffRing + slot * kSlot + (row ? 512u : 0u),
                                                               nimg * 16, 128);
                            const uint64_t bstep = (uint64_t)(2 * nimg);
                            const uint32_t d = tmem + colDB(h) + row * 96, a = tmem + colBeta(row);
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
        // ---------------- 16 accumulating warps: four per TMEM lane quadrant ----------------
        const int e = warp - 2;
        const int grp = e >> 2;
        const int quad = warp & 3;
        const int col = quad * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
        const int tid_e = threadIdx.x - 64;
        uint32_t uses = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < p.tiles_total; tile += gridDim.x) {
            const int f = frame_of(p, tile);
            const Frame &F = p.fr[f];
            const int lt = tile - F.tile_base;
            const int tyy = lt / F.tiles_x, txx = lt - tyy * F.tiles_x;
            const int r_band = tyy * kBand, c0 = txx * kStrip;
            const int npair = n_pairs_of(tile);
            // x_w at tile row tr, column tcol (0 outside the frame)
            auto load_px = [&](int tr, int tcol, float &r, float &g, float &b) {
                const int gr = r_band - kHalo + tr, gc = c0 - kHalo + tcol;
                r = g = b = 0.f;
                if (gr >= 0 && gr < F.H && gc >= 0 && gc < F.W) {
                    const float *px = F.xw + ((size_t)gr * F.W + gc) * C;
                    r = __ldg(px);
                    if (C == 3) {
                        g = __ldg(px + 1);
                        b = __ldg(px + 2);
                    }
                }
            };
            ptx::named_bar(1, kEpi);  // previous tile fully consumed
            for (int i = tid_e; i < kXRing * kTC; i += kEpi) {
                // ring row tr holds tile row tr for the first pair
                const int tr = i / kTC, tcol = i - tr * kTC;
                float r, g, b;
                load_px(tr, tcol, r, g, b);
                xs[i] = encode_px<C>(r, g, b);
            }
            ptx::named_bar(1, kEpi);
            for (int rp = 0; rp < npair; ++rp) {
                // the next pair's new tile rows 2 rp + 34, 2 rp + 35 (pair 1's came with the first
                // 36): loaded now, stored after this pair's taps into the ring rows of tile rows
                // 2 rp - 2, 2 rp - 1 (free since the last pair's closing barrier, read by no tap
                // of this pair)
                const bool stage = rp >= 1 && rp + 1 < npair && tid_e < 2 * kTC;
                const int ntr = 2 * rp + 34 + (tid_e >= kTC ? 1 : 0), ncol = tid_e >= kTC ? tid_e - kTC : tid_e;
                float nr = 0.f, ng = 0.f, nb = 0.f;
                if (stage) load_px(ntr, ncol, nr, ng, nb);
                float acc[2][3];
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) acc[i][ch] = 0.f;
                accumulate_pair<C>(xs, lane_base, col, rp, grp, bar0, uses, ok, ctl, lane, acc);
                if (stage) xs[(ntr % kXRing) * kTC + ncol] = encode_px<C>(nr, ng, nb);
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
                            for (int ch = 0; ch < C; ++ch)
                                o[ch] = acc[i][ch] + xchg[col * 6 + i * 3 + ch] + xchg[kStrip * 6 + col * 6 + i * 3 + ch] +
                                        xchg[2 * kStrip * 6 + col * 6 + i * 3 + ch];
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

}  // namespace gh

using namespace gh;

p2s_status launch_gather_h2(p2s_ctx *ctx, const TcFrame *frames, const void *const *beta16, int n, int C,
                            int *status, cudaStream_t st) {
    if (n <= 0) return P2S_OK;
    if (ctx->prec != P2S_FP16 && ctx->prec != P2S_BF16) {
        set_error("the packed-FP16 gather kernel takes FP16 or BF16 operands");
        return P2S_EUNSUPPORTED;
    }
    p2s_status s0 = tc_prepare(ctx);
    if (s0 != P2S_OK) return s0;
    if (ctx->tc_items.size() < (size_t)(kItemBase + kChunks) * sizeof(Item16)) {
        set_error("basis images of the packed-FP16 gather kernel are missing");
        return P2S_EINVAL;
    }
    const Item16 *items = (const Item16 *)ctx->tc_items.data();
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
        p.stream = (const uint8_t *)ctx->tc.d_H;
        for (int c = 0; c < kChunks; ++c) {
            const Item16 &it = items[kItemBase + c];
            if (it.n != (uint32_t)(c < kMainChunks ? kImgMain : kImgLast) || it.bytes > (uint32_t)kSlot) {
                set_error("basis image %d of the packed-FP16 gather kernel has the wrong shape", c);
                return P2S_EINVAL;
            }
            p.item[c] = Item{it.offset, it.bytes, it.n, it.k};
        }
        p.ab_fmt = ctx->tc.fmt;
        p.status = status;
        int sms = 148;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
        const int grid = tiles < sms ? tiles : sms;
        ProfScope pr(ctx, st, "blur_tc_gather_h2", 2.0 * ctx->K * ctx->T * npx, npx * (C * 8.0 + kGroups * 16.0));
        auto run = [&](auto kern) -> p2s_status {
            P2S_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
            kern<<<grid, kThreads, kSmemBytes, st>>>(p);
            return P2S_OK;
        };
        p2s_status rs = C == 3 ? run(gather_h2_kernel<3>) : run(gather_h2_kernel<1>);
        if (rs != P2S_OK) return rs;
        P2S_CUDA(cudaGetLastError());
    }
    return P2S_OK;
}

}  // namespace p2s
