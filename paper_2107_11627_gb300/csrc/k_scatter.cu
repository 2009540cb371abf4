// Tensor-core scatter blur (Sec. 3.1): y = sum_k h_k * (beta_k . x_w), each
// source pixel spreading its light with its own PSF G[p, .] = beta[p] H.
//
// Output-stationary on the tensor-core side: TMEM lane l owns TARGET column
// c0 + l of a 128-column strip.  For source row s and tap column tx (offset
// ox = tx - 16) the MMA
//     D[l, ty] = sum_k beta[(s, c0 + l - ox), k] H[k, (ty, tx)],  ty = 0..32,
// takes its A operand from shared memory at a row offset of -ox: beta rows
// sit 16 bytes apart in the no-swizzle K-major layout, so the shift is only
// the descriptor's start address.  N = 48 covers the 33 tap rows of one tap
// column (the basis is stored tap-column-major, so columns 33..47 of D are
// the next tap column's rows and are ignored).  Lane l then holds, for every
// tap row, the light of source (s, c0 + l - ox) that lands in its own target
// column, at target row s + ty - 16; one x value per (s, tx) serves all 33
// tap rows, and the target rows accumulate in registers:
//   warps of half 0 take tap rows 0..15, a 17-row window of target rows;
//   warps of half 1 take tap rows 16..32, an 18-row window;
// both slide down two source rows (one row pair) at a time.  A target row is
// finished by half 1 first (sources T-16..T), handed to half 0 through shared
// memory, finished by half 0 (sources T+1..T+16) and written out.
//
// Work unit: (frame, 128-column strip, segment of source rows).  Target rows
// that also receive light from another segment are added with red.add (the
// output is zeroed first); all other rows are stored.
//
// Operands: beta in the 16-bit layout written by the network kernel,
// [frame][row][k/8][col][8], loaded one source row at a time by a 5-D TMA
// tensor copy of box (8, 160, 14, 1, 1) whose out-of-image columns and rows
// are zero-filled; the basis, tap-column-major [k/8][tap][8] with the folded
// bias rows, streamed in chunks of three tap columns by a 3-D tensor copy.
// Roles: warp 0 issues the MMAs (one thread), warp 1 issues the copies,
// warps 2..9 (two per TMEM lane quadrant) accumulate.  Every wait is bounded.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "half_bits.h"
#include "p2s_internal.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace p2s {
namespace sc {

using tcc::Ctl;
using tcc::drain_bar;
using tcc::wait_bar;

constexpr int kStrip = 128;                       // target columns per unit
constexpr int kHalo = 16;                         // 33 x 33 taps
constexpr int kTaps = 2 * kHalo + 1;
constexpr int kPos = kStrip + 2 * kHalo;          // source positions per row: c0 - 16 .. c0 + 143
constexpr int kGroups = 14;                       // K padded to 112, groups of 8
constexpr int kKSteps = kGroups / 2;
constexpr int kBetaRow = kGroups * kPos * 16;     // 35,840 B per source row
constexpr int kTxPerChunk = 3;
constexpr int kChunks = kTaps / kTxPerChunk;      // 11
constexpr int kHRows = kTxPerChunk * kTaps + 15;  // 114 B rows per chunk
constexpr int kHAll = kTaps * kTaps + 15;         // 1104 packed basis rows
constexpr int kHSlot = 25600;                     // >= 14 * 114 * 16, 1024-aligned
constexpr int kN = 48;
constexpr int kDSlots = 10;
constexpr int kThreads = 416;  // + MMA warps 10, 11, 12
constexpr int kMmaWarp1 = 10;
constexpr int kIssuers = 4;    // (row, tap-column parity)
constexpr int kEpi = 256;

constexpr int kOffBeta = 0;                            // 4 rows (two pairs)
constexpr int kOffH = kOffBeta + 4 * kBetaRow;         // 2 chunks
constexpr int kOffX = kOffH + 2 * kHSlot;              // float [2 buf][2 row][3 ch][160]
constexpr int kOffHb = kOffX + 2 * 2 * 3 * kPos * 4;   // float [2 buf][2 row][3 ch][128]
constexpr int kOffBar = kOffHb + 2 * 2 * 3 * kStrip * 4;
enum Bar { kBFull = 0, kBEmpty = 2, kHFull = 4, kHEmpty = 6, kDFull = 8, kDEmpty = kDFull + kDSlots,
           kDone = kDEmpty + kDSlots, kNBar };
constexpr int kOffMisc = kOffBar + kNBar * 8;
constexpr int kSmemBytes = kOffMisc + 16 + 1024;
static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");
static_assert(kHSlot >= kGroups * kHRows * 16 && kHSlot % 1024 == 0, "basis slot");
static_assert(kBetaRow % 1024 == 0, "beta slot alignment");

// One frame of a launch: its beta (tensor map (8, W, 14, H, 1), 16-bit), x_w and
// output, size, segment rows, and the index of its first unit.  Frames of one
// launch may differ in size.
struct Frame {
    CUtensorMap tmap_beta;
    const float *xw;
    float *y;
    int H, W, seg, nseg, tiles_x, u0;
};

struct Params {
    CUtensorMap tmap_h;  // (8, 1104, 14) 16-bit
    Frame fr[kMaxBatch];
    int *status;
    int nf, ab_fmt, units;
};

static_assert(sizeof(Params) <= 32764, "kernel parameter limit");

struct Unit {
    int f, c0, s0, s1, npair, H, W;
};

// Units run frame by frame; within a frame segment by segment, strip by strip.
__device__ __forceinline__ Unit unit_of(const Params &p, int u) {
    int lo = 0, hi = p.nf - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (u >= p.fr[mid].u0) lo = mid;
        else hi = mid - 1;
    }
    const Frame &F = p.fr[lo];
    Unit r;
    r.f = lo;
    r.H = F.H;
    r.W = F.W;
    const int rem = u - F.u0;
    const int sg = rem / F.tiles_x;
    r.c0 = (rem - sg * F.tiles_x) * kStrip;
    r.s0 = sg * F.seg;
    r.s1 = min(F.H, r.s0 + F.seg);
    r.npair = (r.s1 - r.s0 + 1) >> 1;
    return r;
}

// Write or add one finished (or partial) target row of this lane.
template <int C>
__device__ __forceinline__ void emit_row(const Params &p, const Unit &u, int col, int T, const float *v) {
    if (T < 0 || T >= u.H || col >= u.W || T >= u.s1 + kHalo || T < u.s0 - kHalo) return;
    const bool complete = (u.s0 == 0 || T - kHalo >= u.s0) && (u.s1 == u.H || T + kHalo < u.s1);
    float *o = p.fr[u.f].y + ((size_t)T * u.W + col) * C;
    if (complete) {
#pragma unroll
        for (int ch = 0; ch < C; ++ch) o[ch] = v[ch];
    } else {
#pragma unroll
        for (int ch = 0; ch < C; ++ch) atomicAdd(o + ch, v[ch]);
    }
}

// x_w rows s, s+1 of positions c0-16 .. c0+143, channel-planar; zero outside
template <int C>
__device__ __forceinline__ void x_fetch(const Params &p, const Unit &u, int s, int tid_e, float (&r)[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int e = tid_e + kEpi * k;
        float v = 0.f;
        if (e < 2 * C * kPos) {
            const int i = e / (C * kPos), rem = e - i * (C * kPos);
            const int ch = rem / kPos, pos = rem - ch * kPos;
            const int row = s + i, col = u.c0 - kHalo + pos;
            if (row < u.H && col >= 0 && col < u.W) v = __ldg(p.fr[u.f].xw + ((size_t)row * u.W + col) * C + ch);
        }
        r[k] = v;
    }
}
template <int C>
__device__ __forceinline__ void x_store(float *xs, int tid_e, const float (&r)[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int e = tid_e + kEpi * k;
        if (e < 2 * C * kPos) {
            const int i = e / (C * kPos), rem = e - i * (C * kPos);
            xs[i * 3 * kPos + rem] = r[k];  // [row][ch][pos]
        }
    }
}

template <int C, int HALF>
__device__ void accumulate(const Params &p, uint8_t *sm, uint32_t bar0, uint32_t lane_base, int quad, int lane,
                           const Ctl &ctl) {
    constexpr int NT = HALF ? 17 : 16;  // tap rows of this half
    constexpr int TY0 = HALF ? 16 : 0;
    constexpr int NW = NT + 1;          // target-row window
    auto BAR = [&](int i) { return bar0 + 8u * (uint32_t)i; };
    const int m = quad * 32 + lane;
    const int tid_e = (int)threadIdx.x - 64;
    float *xs = (float *)(sm + kOffX);
    float *hb = (float *)(sm + kOffHb);
    uint32_t dc = 0;
    bool ok = true;
    for (int un = blockIdx.x; un < p.units; un += gridDim.x) {
        const Unit u = unit_of(p, un);
        const int col = u.c0 + m;
        float acc[NW][C];
#pragma unroll
        for (int w = 0; w < NW; ++w)
#pragma unroll
            for (int ch = 0; ch < C; ++ch) acc[w][ch] = 0.f;
        {
            float r[4];
            x_fetch<C>(p, u, u.s0, tid_e, r);
            x_store<C>(xs, tid_e, r);
        }
        ptx::named_bar(1, kEpi);
        int xb = 0;
        for (int pr = 0; pr < u.npair; ++pr) {
            const int s = u.s0 + 2 * pr;
            float nx[4];
            const bool more = pr + 1 < u.npair;
            if (more) x_fetch<C>(p, u, s + 2, tid_e, nx);
            const float *x0 = xs + xb * (2 * 3 * kPos);
            const float *x1 = x0 + 3 * kPos;
#pragma unroll 1
            for (int tx = 0; tx < kTaps; ++tx) {
                const uint32_t d0 = dc % kDSlots, d1 = (dc + 1) % kDSlots;
                const bool g0 = wait_bar(BAR(kDFull + d0), (dc / kDSlots) & 1, ctl, 16);
                const bool g1 = wait_bar(BAR(kDFull + d1), ((dc + 1) / kDSlots) & 1, ctl, 16);
                ok = __all_sync(0xffffffffu, g0 && g1 && ok);
                ptx::fence_after();
                uint32_t a[NT], b[NT];
                if (ok) {
                    ptx::tmem_ld16(lane_base + d0 * kN + TY0, *reinterpret_cast<uint32_t(*)[16]>(&a[0]));
                    ptx::tmem_ld16(lane_base + d1 * kN + TY0, *reinterpret_cast<uint32_t(*)[16]>(&b[0]));
                    if (NT == 17) {
                        ptx::tmem_ld1(lane_base + d0 * kN + TY0 + 16, a[NT - 1]);
                        ptx::tmem_ld1(lane_base + d1 * kN + TY0 + 16, b[NT - 1]);
                    }
                }
                const int pos = m + 2 * kHalo - tx;
                float xv0[C], xv1[C];
#pragma unroll
                for (int ch = 0; ch < C; ++ch) {
                    xv0[ch] = x0[ch * kPos + pos];
                    xv1[ch] = x1[ch * kPos + pos];
                }
                if (ok) ptx::tmem_wait_ld();
                ptx::fence_before();
                __syncwarp();
                if (lane == 0) {
                    ptx::mbar_arrive(BAR(kDEmpty + d0));
                    ptx::mbar_arrive(BAR(kDEmpty + d1));
                }
                dc += 2;
                if (ok) {
#pragma unroll
                    for (int t = 0; t < NT; ++t) {
                        const float ga = __uint_as_float(a[t]), gb = __uint_as_float(b[t]);
                        if (C == 3) {  // (R, G) as one packed FMA per source row
                            tcc::fma2_bcast(ga, xv0[0], xv0[1], acc[t][0], acc[t][1]);
                            tcc::fma2_bcast(gb, xv1[0], xv1[1], acc[t + 1][0], acc[t + 1][1]);
                            acc[t][C - 1] = fmaf(ga, xv0[C - 1], acc[t][C - 1]);
                            acc[t + 1][C - 1] = fmaf(gb, xv1[C - 1], acc[t + 1][C - 1]);
                        } else {
#pragma unroll
                            for (int ch = 0; ch < C; ++ch) {
                                acc[t][ch] = fmaf(ga, xv0[ch], acc[t][ch]);
                                acc[t + 1][ch] = fmaf(gb, xv1[ch], acc[t + 1][ch]);
                            }
                        }
                    }
                }
            }
            // ---- end of the row pair: next x rows, hand-off, emit, slide ----
            if (more) x_store<C>(xs + (xb ^ 1) * (2 * 3 * kPos), tid_e, nx);
            float *hbuf = hb + (pr & 1) * (2 * 3 * kStrip);
            if (HALF) {
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int ch = 0; ch < C; ++ch) hbuf[(j * 3 + ch) * kStrip + m] = acc[j][ch];
#pragma unroll
                for (int w = 0; w < NW; ++w)
#pragma unroll
                    for (int ch = 0; ch < C; ++ch) acc[w][ch] = (w + 2 < NW) ? acc[w + 2][ch] : 0.f;
            }
            ptx::named_bar(1, kEpi);
            if (!HALF) {
#pragma unroll
                for (int ch = 0; ch < C; ++ch) acc[NW - 1][ch] += hbuf[(0 * 3 + ch) * kStrip + m];  // T = s
                if (ok) {
                    emit_row<C>(p, u, col, s - kHalo, acc[0]);
                    emit_row<C>(p, u, col, s - kHalo + 1, acc[1]);
                }
#pragma unroll
                for (int w = 0; w < NW; ++w)
#pragma unroll
                    for (int ch = 0; ch < C; ++ch) acc[w][ch] = (w + 2 < NW) ? acc[w + 2][ch] : 0.f;
#pragma unroll
                for (int ch = 0; ch < C; ++ch) acc[NW - 2][ch] += hbuf[(1 * 3 + ch) * kStrip + m];  // T = s + 1
            }
            xb ^= 1;
        }
        // ---- end of the unit: what is left in the windows ----
        const int s_next = u.s0 + 2 * u.npair;  // window bases after the last slide
        if (ok) {
#pragma unroll
            for (int w = 0; w < NW; ++w) emit_row<C>(p, u, col, (HALF ? s_next : s_next - kHalo) + w, acc[w]);
        }
        // every thread is done with the x and hand-off buffers before the next unit
        ptx::named_bar(1, kEpi);
    }
}

template <int C>
__global__ void __launch_bounds__(kThreads, 1) scatter_kernel(const __grid_constant__ Params p) {
    extern __shared__ uint8_t smem_raw[];
    // aligned by pointer arithmetic on the __shared__ array, so that the compiler still
    // knows every access through `sm` is to shared memory (ld/st.shared, not generic)
    uint8_t *sm = smem_raw + ((1024u - (uint32_t)((uintptr_t)smem_raw & 1023u)) & 1023u);
    const uint32_t sbase = ptx::smem_u32(sm);
    const uint32_t bar0 = sbase + kOffBar;
    uint32_t *tmem_holder = (uint32_t *)(sm + kOffMisc);
    volatile int *abort_flag = (volatile int *)(sm + kOffMisc + 4);
    auto BAR = [&](int i) { return bar0 + 8u * (uint32_t)i; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Ctl ctl{abort_flag, p.status};

    if (threadIdx.x == 0) {
        *abort_flag = 0;
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(BAR(kBFull + i), 1);
            ptx::mbar_init(BAR(kBEmpty + i), kIssuers);  // one commit per MMA thread
            ptx::mbar_init(BAR(kHFull + i), 1);
            ptx::mbar_init(BAR(kHEmpty + i), kIssuers);
        }
        for (int i = 0; i < kDSlots; ++i) {
            ptx::mbar_init(BAR(kDFull + i), 1);
            ptx::mbar_init(BAR(kDEmpty + i), 8);
        }
        ptx::mbar_init(BAR(kDone), kIssuers);
        ptx::mbar_fence_init();
    }
    if (warp == 0) ptx::tmem_alloc(ptx::smem_u32(tmem_holder), 512);
    ptx::fence_before();
    __syncthreads();
    ptx::fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 1) {
        // ---------------- copies: beta row pairs and basis chunks ----------------
        if (lane == 0) {
            uint32_t pc = 0, hc = 0;
            auto load_beta = [&](const Unit &u, int pr) {
                const uint32_t slot = pc & 1;
                if (wait_bar(BAR(kBEmpty + slot), ((pc >> 1) & 1) ^ 1, ctl, 1)) {
                    ptx::mbar_arrive_tx(BAR(kBFull + slot), 2 * kBetaRow);
                    for (int i = 0; i < 2; ++i)
                        ptx::tma_load_5d(sbase + kOffBeta + (2 * slot + i) * kBetaRow, &p.fr[u.f].tmap_beta, 0,
                                         u.c0 - kHalo, 0, u.s0 + 2 * pr + i, 0, BAR(kBFull + slot));
                }
                ++pc;
            };
            auto load_h = [&](int j) {
                const uint32_t slot = hc & 1;
                if (wait_bar(BAR(kHEmpty + slot), ((hc >> 1) & 1) ^ 1, ctl, 2)) {
                    ptx::mbar_arrive_tx(BAR(kHFull + slot), kGroups * kHRows * 16);
                    ptx::tma_load_3d(sbase + kOffH + slot * kHSlot, &p.tmap_h, 0, j * kTxPerChunk * kTaps, 0,
                                     BAR(kHFull + slot));
                }
                ++hc;
            };
            // pair sequence of this CTA; the next pair's beta goes out after the first chunk
            int un = blockIdx.x, pr = 0;
            if (un < p.units) load_beta(unit_of(p, un), 0);
            while (un < p.units) {
                const Unit u = unit_of(p, un);
                int nun = un, npr = pr + 1;
                if (npr >= u.npair) {
                    nun = un + gridDim.x;
                    npr = 0;
                }
                load_h(0);
                if (nun < p.units) load_beta(unit_of(p, nun), npr);
                for (int j = 1; j < kChunks; ++j) load_h(j);
                un = nun;
                pr = npr;
            }
            // issued copies land before shared memory is released
            for (uint32_t k = pc > 2 ? pc - 2 : 0; k < pc; ++k) drain_bar(BAR(kBFull + (k & 1)), (k >> 1) & 1);
            for (uint32_t k = hc > 2 ? hc - 2 : 0; k < hc; ++k) drain_bar(BAR(kHFull + (k & 1)), (k >> 1) & 1);
        }
    } else if (warp == 0 || warp >= kMmaWarp1) {
        // ---------------- MMA issuers: warps 0, 10, 11, 12 ----------------
        // One thread issues an MMA about every 76-100 cycles whatever its size; four
        // threads, each on its own accumulators (row 0 / 1 x even / odd tap column),
        // keep the tensor core busy.  13 warps leave 128 registers per thread (a few
        // bytes of spills in the RGB accumulators), still faster than two issuers.
        if (lane == 0) {
            const int who = warp == 0 ? 0 : warp - kMmaWarp1 + 1;  // 0..3
            const int row = who & 1, par = who >> 1;
            const uint32_t idesc = ptx::idesc_f16(p.ab_fmt, kN);
            uint32_t pc = 0, hc = 0, dc = 0;
            for (int un = blockIdx.x; un < p.units; un += gridDim.x) {
                const Unit u = unit_of(p, un);
                for (int pr = 0; pr < u.npair; ++pr, ++pc) {
                    const uint32_t bslot = pc & 1;
                    const bool bok = wait_bar(BAR(kBFull + bslot), (pc >> 1) & 1, ctl, 4);
                    for (int j = 0; j < kChunks; ++j, ++hc) {
                        const uint32_t hslot = hc & 1;
                        const bool hok = wait_bar(BAR(kHFull + hslot), (hc >> 1) & 1, ctl, 8);
                        // per tap column, this row's accumulator (accumulator slots alternate
                        // between the rows: row 0 even, row 1 odd)
                        for (int uu = 0; uu < kTxPerChunk; ++uu, dc += 2) {
                            const int tx = j * kTxPerChunk + uu;
                            if ((tx & 1) != par) continue;
                            const uint32_t dd = (dc + row) % kDSlots;
                            const bool e = wait_bar(BAR(kDEmpty + dd), (((dc + row) / kDSlots) & 1) ^ 1, ctl, 32);
                            ptx::fence_after();
                            if (bok && hok && e) {
                                const uint64_t bd =
                                    ptx::smem_desc(sbase + kOffH + hslot * kHSlot + uu * kTaps * 16, kHRows * 16, 128);
                                const uint32_t a0 = sbase + kOffBeta + (2 * bslot + row) * kBetaRow + (2 * kHalo - tx) * 16;
                                const uint64_t ad = ptx::smem_desc(a0, kPos * 16, 128);
#pragma unroll
                                for (int ks = 0; ks < kKSteps; ++ks)
                                    ptx::mma_ss(tmem + dd * kN, ad + (uint64_t)(ks * 2 * kPos), bd + (uint64_t)(ks * 2 * kHRows),
                                                idesc, ks > 0 ? 1u : 0u);
                            }
                            ptx::mma_commit(BAR(kDFull + dd));
                        }
                        ptx::mma_commit(BAR(kHEmpty + hslot));
                    }
                    ptx::mma_commit(BAR(kBEmpty + bslot));
                }
            }
            ptx::mma_commit(BAR(kDone));
            drain_bar(BAR(kDone), 0);
        }
    } else {
        const int half = (warp - 2) >> 2;
        const int quad = warp & 3;
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
        if (half)
            accumulate<C, 1>(p, sm, bar0, lane_base, quad, lane, ctl);
        else
            accumulate<C, 0>(p, sm, bar0, lane_base, quad, lane, ctl);
    }
    // ---------------- teardown ----------------
    ptx::fence_before();
    __syncthreads();
    if (warp == 0) {
        ptx::fence_after();
        ptx::tmem_dealloc(tmem, 512);
    }
}


typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encoder() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)ptr;
    }
    return fn;
}

static p2s_status encode(CUtensorMap *m, void *base, int rank, const cuuint64_t *dims, const cuuint64_t *strides,
                         const cuuint32_t *box) {
    EncodeTiledFn fn = encoder();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return P2S_ECUDA;
    }
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, (cuuint32_t)rank, base, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("tensor map encoding failed (CUresult %d)", (int)r);
        return P2S_ECUDA;
    }
    return P2S_OK;
}

}  // namespace sc

using namespace sc;

// The basis, tap-column-major: row r = tx * 33 + ty (r < 1089, then 15 zero
// rows), 16-bit groups of 8 along k: [14][1104][8]; rows K and K + 1 carry the
// folded bias PSF h_b = sum_k b3_k H_k as an exact hi/lo pair.
p2s_status scatter_prepare(p2s_ctx *ctx) {
    if (ctx->tc.d_Hs) return P2S_OK;
    p2s_status s0 = tc_prepare(ctx);
    if (s0 != P2S_OK) return s0;
    const int fmt = ctx->tc.fmt, K = ctx->K, T = ctx->T;
    std::vector<double> hb(T, 0.0);
    for (int k = 0; k < K; ++k)
        for (int t = 0; t < T; ++t) hb[t] += ctx->b[2][k] * ctx->H[(size_t)k * T + t];
    std::vector<uint16_t> img((size_t)kGroups * kHAll * 8, 0);
    for (int r = 0; r < kTaps * kTaps; ++r) {
        const int tx = r / kTaps, ty = r % kTaps, t = ty * kTaps + tx;
        for (int k = 0; k < kGroups * 8; ++k) {
            uint16_t v = 0;
            if (k < K) {
                v = to_half_bits(ctx->H[(size_t)k * T + t], fmt);
            } else if (k == K || k == K + 1) {
                const uint16_t hi = to_half_bits(hb[t], fmt);
                v = k == K ? hi : to_half_bits(hb[t] - from_half_bits(hi, fmt), fmt);
            }
            img[((size_t)(k / 8) * kHAll + r) * 8 + (k % 8)] = v;
        }
    }
    void *d = nullptr;
    if (cudaMalloc(&d, img.size() * 2) != cudaSuccess) {
        set_error("device allocation failed for the scatter basis");
        return P2S_ENOMEM;
    }
    P2S_CUDA(cudaMemcpy(d, img.data(), img.size() * 2, cudaMemcpyHostToDevice));
    ctx->tc.d_Hs = d;
    return P2S_OK;
}

int scatter_segment_rows(const p2s_ctx *ctx, int H) {
    int seg = ctx->tc.seg_rows > 0 ? ctx->tc.seg_rows : 128;
    seg = (seg + 1) & ~1;
    return seg >= H ? ((H + 1) & ~1) : seg;
}

p2s_status launch_scatter_frames(p2s_ctx *ctx, const ScatterFrame *frames, int n, int C, int *status,
                                 cudaStream_t st) {
    if (n <= 0) return P2S_OK;
    if (n > kMaxBatch) {
        set_error("scatter batch larger than %d frames", kMaxBatch);
        return P2S_EINVAL;
    }
    if (C != 1 && C != 3) {
        set_error("C must be 1 or 3");
        return P2S_EINVAL;
    }
    if (ctx->th != kTaps || ctx->tw != kTaps || ctx->K > kGroups * 8 - 2) {
        set_error("tensor-core scatter needs 33x33 taps and K <= %d", kGroups * 8 - 2);
        return P2S_EUNSUPPORTED;
    }
    p2s_status s0 = scatter_prepare(ctx);
    if (s0 != P2S_OK) return s0;
    Params p;
    std::memset(&p, 0, sizeof p);
    {
        const cuuint64_t dims[3] = {8, (cuuint64_t)kHAll, (cuuint64_t)kGroups};
        const cuuint64_t strides[2] = {16, (cuuint64_t)kHAll * 16};
        const cuuint32_t box[3] = {8, kHRows, kGroups};
        s0 = encode(&p.tmap_h, ctx->tc.d_Hs, 3, dims, strides, box);
        if (s0 != P2S_OK) return s0;
    }
    int units = 0;
    double npx = 0.0;
    for (int i = 0; i < n; ++i) {
        const ScatterFrame &q = frames[i];
        if (q.H <= 0 || q.W <= 0) {
            set_error("frame %d of the scatter batch is empty", i);
            return P2S_EINVAL;
        }
        Frame &F = p.fr[i];
        const cuuint64_t dims[5] = {8, (cuuint64_t)q.W, (cuuint64_t)kGroups, (cuuint64_t)q.H, 1};
        const cuuint64_t strides[4] = {16, (cuuint64_t)q.W * 16, (cuuint64_t)q.W * 16 * kGroups,
                                       (cuuint64_t)q.W * 16 * kGroups * q.H};
        const cuuint32_t box[5] = {8, kPos, kGroups, 1, 1};
        s0 = encode(&F.tmap_beta, const_cast<void *>(q.beta), 5, dims, strides, box);
        if (s0 != P2S_OK) return s0;
        F.xw = q.xw;
        F.y = q.y;
        F.H = q.H;
        F.W = q.W;
        F.seg = scatter_segment_rows(ctx, q.H);
        F.nseg = (q.H + F.seg - 1) / F.seg;
        F.tiles_x = (q.W + kStrip - 1) / kStrip;
        F.u0 = units;
        units += F.tiles_x * F.nseg;
        npx += (double)q.H * q.W;
        // rows that receive light from two segments are added into a zeroed output
        if (F.nseg > 1) P2S_CUDA(cudaMemsetAsync(q.y, 0, (size_t)q.H * q.W * C * sizeof(float), st));
    }
    p.status = status;
    p.nf = n;
    p.ab_fmt = ctx->tc.fmt;
    p.units = units;
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const int grid = p.units < sms ? p.units : sms;
    ProfScope pr(ctx, st, "blur_tc_scatter", 2.0 * ctx->K * ctx->T * npx, npx * (C * 8.0 + kGroups * 16.0));
    if (C == 3) {
        P2S_CUDA(cudaFuncSetAttribute(scatter_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
        scatter_kernel<3><<<grid, kThreads, kSmemBytes, st>>>(p);
    } else {
        P2S_CUDA(cudaFuncSetAttribute(scatter_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
        scatter_kernel<1><<<grid, kThreads, kSmemBytes, st>>>(p);
    }
    P2S_CUDA(cudaGetLastError());
    return P2S_OK;
}

p2s_status launch_scatter_tc(p2s_ctx *ctx, int H, int W, int C, int n, const float *const *xw, float *const *y,
                             const void *beta16, int *status, cudaStream_t st) {
    if (n <= 0 || H <= 0 || W <= 0) return P2S_OK;
    const size_t fbytes = beta16_bytes(H, W, 1, 0);
    ScatterFrame fr[kMaxBatch];
    for (int i0 = 0; i0 < n; i0 += kMaxBatch) {
        const int nb = n - i0 < kMaxBatch ? n - i0 : kMaxBatch;
        for (int k = 0; k < nb; ++k)
            fr[k] = ScatterFrame{xw[i0 + k], y[i0 + k], (const char *)beta16 + (size_t)(i0 + k) * fbytes, H, W};
        p2s_status s0 = launch_scatter_frames(ctx, fr, nb, C, status, st);
        if (s0 != P2S_OK) return s0;
    }
    return P2S_OK;
}

}  // namespace p2s
