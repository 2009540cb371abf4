// Internal declarations shared by the translation units of libp2s.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "p2s.h"

namespace p2s {

constexpr int kModes = 35;        // Noll J = 2..36 on the anchor grid
constexpr int kAlphaStride = 36;  // floats per anchor: slot 0 piston, slot j-1 mode j
constexpr int kHiModes = 33;      // J = 4..36, the network input
constexpr int kMaxBatch = 64;     // frames per launch (kernel parameters by value)

void set_error(const char *fmt, ...);

#define P2S_CUDA(call)                                                              \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            ::p2s::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                             __FILE__, __LINE__);                                   \
            return P2S_ECUDA;                                                       \
        }                                                                           \
    } while (0)

// Shape of the anchor grid and the filter torus for an H x W frame.
struct FieldGeom {
    int H, W, s;
    int Ah, Aw;  // anchors
    int Fh, Fw;  // torus (powers of two)
};

// Wavelength-dependent colour: copy one channel of n frames of npx pixels between
// interleaved and planar layouts (strides and offsets in floats).
p2s_status launch_channel_copy(const float *const *src, float *const *dst, int n, long long npx, int src_stride,
                               int src_off, int dst_stride, int dst_off, cudaStream_t st);

// Precisions that run the network and the contraction on the tensor cores.
inline bool tc_precision(p2s_precision p) { return p == P2S_BF16 || p == P2S_FP16 || p == P2S_FP8E4M3; }

// Per-launch frame parameters, passed by value.
struct FrameBatch {
    int n;
    unsigned long long seed[kMaxBatch];
    float scale[kMaxBatch];  // (D/r0)^(5/6), computed in FP64 on the host
};

// Per-frame anchor grids and output blocks of one field launch (frames of one torus):
// f[k] is frame k's [kModes][ah][aw] filtered fields, alpha[k] its [ah][aw][kAlphaStride].
struct FieldFrames {
    int ah[kMaxBatch], aw[kMaxBatch];
    float *f[kMaxBatch];
    float *alpha[kMaxBatch];
};

// Device tables of the separable field filter for one torus length F.
struct FilterTable {
    int F = 0;
    float2 *twiddle = nullptr;  // [F/2]  exp(-2 pi i m / F)
    float *gain = nullptr;      // [n_kernels][F]  sqrt(C1[u]) / F  (IDFT 1/F folded in)
};

// Tensor-core operand packs (filled by the tcgen05 translation unit).
struct TcPack {
    void *d_W = nullptr;      // unused (weights live in the stream below)
    void *d_H = nullptr;      // stream of B images: network weights, then basis chunks
    float *d_bias = nullptr;  // FP32 b1, b2, b3
    size_t W_bytes = 0, H_bytes = 0;
    int n_mlp = 0, h1p = 0, h2p = 0, n3 = 0, fmt = 0, split = 0;
    int ready = 0;
    void *d_Hs = nullptr;  // basis for the scatter kernel, tap-column-major [14][1104][8] 16-bit
    int seg_rows = 0;      // source rows per scatter work unit (0: default)
    int band_rows = 0;     // output rows per fused gather tile: 16 or 32 (0: default 32)
    // FP8 E4M3 contraction (P2S_FP8E4M3): basis chunk images as E4M3 hi/lo pairs, rows
    // scaled by per-basis powers of two, in the split gather's column order (hi image
    // then lo image per chunk); the network writes beta scaled by scale8[k] as hi/lo
    // pairs; G comes out of the tensor core multiplied by 2^c8, undone by inv_c8.
    void *d_H8 = nullptr;
    float *d_scale8 = nullptr;  // [128] beta multipliers (0 beyond the bias columns)
    float inv_c8 = 1.f;
    uint32_t item8_off[12] = {}, item8_bytes[12] = {}, item8_n[12] = {};
};

// One B image of the tensor-core weight stream: byte offset and size in the
// stream, N rows, K depth (canonical no-swizzle K-major layout).
struct Item16 {
    uint32_t offset, bytes, n, k;
};

}  // namespace p2s

namespace p2s {
struct ProfRecord {
    const char *name;
    cudaEvent_t start, stop;
    double flops, bytes;
};
}  // namespace p2s

struct p2s_ctx {
    int device = 0;
    p2s_precision prec = P2S_FP32;
    p2s_blur_form form = P2S_SCATTER;
    // basis
    int K = 0, th = 0, tw = 0, T = 0;
    std::vector<double> H;  // host FP64 [K][T]
    float *d_H32 = nullptr; // device FP32 [K][T]
    float *d_Ht32 = nullptr;// device FP32 [T][K] (tap-major)
    // network
    int n_layers = 0;
    std::vector<int> dims;
    std::vector<std::vector<double>> W, b;
    std::vector<float *> d_Wt32;  // FP32 [in][out] per layer
    std::vector<float *> d_b32;   // FP32 [out] per layer
    // field correlation
    int s = 8, n_kernels = 1, guard = 0;
    std::vector<double> ell;
    double kappa = 0.0;
    float *d_L = nullptr;          // FP32 lower Cholesky factor [35][35]
    std::vector<double> L64;       // the same factor in FP64 (lower triangle used)
    int kernel_of_mode[p2s::kModes];
    int *d_kernel_of_mode = nullptr;
    std::map<int, p2s::FilterTable> tables;
    p2s::TcPack tc;
    std::vector<uint8_t> tc_items;  // item table of the tensor-core stream (opaque here)
    int *d_status = nullptr;        // device status word of bounded waits
    // staging for p2s_simulate_host
    void *stage = nullptr;
    size_t stage_bytes = 0;
    // FFT blur variant: twiddles by length, basis spectra by (Fh << 16 | Fw)
    std::map<int, void *> fft_tw;
    std::map<long long, void *> fft_basis;
    // CUDA graphs of p2s_simulate (P2S_OPT_GRAPHS): scratch arena, internal
    // capture stream, instantiated graphs by batch signature
    int use_graphs = 0;
    int blur_then_warp = 0;  // P2S_OPT_BLUR_THEN_WARP
    int field_method = 0;    // P2S_OPT_FIELD_METHOD: 0 Fourier filtering, 1 dense draw
    int gather_split = 1;    // P2S_OPT_GATHER_SPLIT
    std::map<int, void *> dense_L;  // dense draw: FP32 Cholesky factors [n_kernels][n][n] by n
    void *arena = nullptr;
    size_t arena_bytes = 0;
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t cap_ev[2] = {nullptr, nullptr};
    // p2s_simulate_host: copy streams (host->device, device->host) and per-chunk events
    cudaStream_t copy_stream[2] = {nullptr, nullptr};
    cudaStream_t aux_stream = nullptr;  // second compute stream of p2s_simulate_host
    std::vector<cudaEvent_t> host_ev;
    std::map<std::string, cudaGraphExec_t> graphs;
    long long graph_updates = 0, graph_instantiations = 0;
    // kernel timing
    bool profiling = false;
    std::vector<p2s::ProfRecord> prof;
    std::vector<cudaEvent_t> event_pool;
};

namespace p2s {

// Brackets one kernel launch with CUDA events on its stream while the
// context is profiling; flops/bytes are the launch's algorithmic work.
class ProfScope {
  public:
    ProfScope(const p2s_ctx *ctx, cudaStream_t st, const char *name, double flops, double bytes);
    ~ProfScope();

  private:
    p2s_ctx *ctx_;
    cudaStream_t st_;
    int idx_ = -1;
};

// host setup (p2s_host.cu)
p2s_status geometry(const p2s_ctx *ctx, int H, int W, FieldGeom *g);
p2s_status filter_table(p2s_ctx *ctx, int F, const FilterTable **out);

// fields (k_fields.cu)
p2s_status launch_noise(unsigned long long seed, int mode, int Fh, int Fw, float *out, cudaStream_t st);
size_t fields_scratch_bytes(const FieldGeom &g, int n);
// Fields of frames that share a torus (Fh, Fw) but not an anchor grid, in one launch of the
// one-kernel Fourier filter and one of the colouring; fields_group_ok says whether that
// filter serves the torus and the largest grids (else launch_fields per grid).
bool fields_group_ok(const p2s_ctx *ctx, int Fh, int Fw, int Ah_max, int Aw_max);
p2s_status launch_fields_group(p2s_ctx *ctx, int Fh, int Fw, const FrameBatch &fb, const FieldFrames &geo,
                               cudaStream_t st);
p2s_status launch_fields(p2s_ctx *ctx, const FieldGeom &g, const FrameBatch &fb, float *alpha, void *scratch,
                         cudaStream_t st);

// warp (k_warp.cu)
p2s_status launch_warp(const p2s_ctx *ctx, const FieldGeom &g, int n, const float *const *in, const float *alpha,
                       float *const *out, int C, cudaStream_t st);
// The same over up to kMaxBatch frames of any sizes with C channels, in one launch.
struct WarpFrame {
    const float *in;
    float *out;
    const float *alpha;  // the frame's anchors, [Ah][Aw][36]
    int H, W;
};
p2s_status launch_warp_frames(const p2s_ctx *ctx, const WarpFrame *frames, int n, int C, cudaStream_t st);

// plain FP32 network and blur (k_simt.cu)
p2s_status launch_mlp_simt(const p2s_ctx *ctx, const FieldGeom &g, int n, const float *alpha, float *beta,
                           cudaStream_t st);
p2s_status launch_blur_simt(const p2s_ctx *ctx, int H, int W, int C, int n, const float *const *xw,
                            const float *beta, float *const *y, p2s_blur_form form, cudaStream_t st);

// tensor-core path (k_tc.cu)
p2s_status tc_prepare(p2s_ctx *ctx);
// One frame of a tensor-core launch: warped input, output, anchors of the
// frame ([Ah][Aw][36]), its size; tiles_* and tile_base are filled by the launcher.
struct TcFrame {
    const float *xw;
    float *y;
    const float *alpha;
    int H, W, Ah, Aw, tiles_x, tiles_y, tile_base;
};
constexpr int kMaxTcFrames = 256;  // frames per persistent launch (the table is a kernel parameter)
// Blur-only tensor-core gather over frames whose beta the network kernel
// wrote (launch_net16 with the bias-fold ones); beta16[i] is frame i's.
p2s_status launch_gather_split(p2s_ctx *ctx, const TcFrame *frames, const void *const *beta16, int n, int C,
                               int *status, cudaStream_t st);
// The fragment variant (P2S_OPT_GATHER_SPLIT = 2): beta16 in the permuted layout (perm = 1).
p2s_status launch_gather_frag(p2s_ctx *ctx, const TcFrame *frames, const void *const *beta16, int n, int C,
                              int *status, cudaStream_t st);
// The FP32-x variant (P2S_OPT_GATHER_SPLIT = 3): same beta layout, 128 x 16 tiles.
p2s_status launch_gather_x32(p2s_ctx *ctx, const TcFrame *frames, const void *const *beta16, int n, int C,
                             int *status, cudaStream_t st);
// The packed-FP16 variant (P2S_OPT_GATHER_SPLIT = 4): kernel 1's beta layout (perm = 0).
p2s_status launch_gather_h2(p2s_ctx *ctx, const TcFrame *frames, const void *const *beta16, int n, int C,
                            int *status, cudaStream_t st);
// beta16 layout of the blur-only gather kernel `split` selects: the fragment kernels
// (2, 3) read the permuted layout, kernels 1 and 4 the plain one
inline int gather_perm(int split) { return (split == 2 || split == 3) ? 1 : 0; }
// the blur-only gather kernel `split` (1 .. 4) over n frames
inline p2s_status launch_gather_blur(p2s_ctx *ctx, int split, const TcFrame *frames, const void *const *beta16,
                                     int n, int C, int *status, cudaStream_t st) {
    switch (split) {
        case 2: return launch_gather_frag(ctx, frames, beta16, n, C, status, st);
        case 3: return launch_gather_x32(ctx, frames, beta16, n, C, status, st);
        case 4: return launch_gather_h2(ctx, frames, beta16, n, C, status, st);
        default: return launch_gather_split(ctx, frames, beta16, n, C, status, st);
    }
}
p2s_status launch_tc(p2s_ctx *ctx, int mode, const TcFrame *frames, int n, int C, const float *beta_in,
                     float *beta_out, int *status, cudaStream_t st);
constexpr int kTcFull = 0, kTcMlpOnly = 1, kTcBlurOnly = 2;

// Network kernel: beta of n frames into the 16-bit operand layout
// [frame][row][14][pos][8]; `ones` sets entries K, K + 1 (folded bias).
// perm = 0: pos = column, row pitch W (the layout the scatter kernel and
// p2s_stage_mlp16 use).  perm = 1 (the split gather kernel's): row pitch W
// rounded up to 32, and within each 32-column block column c sits at
// position 8 (c % 4) + (c % 32) / 4, so that TMEM lane L of a 32-lane
// quadrant holds column 4 (L % 8) + L / 8 and the lanes a, a + 8, a + 16,
// a + 24 that one thread reads through 16x256b fragments are 4 adjacent columns.
inline int beta16_pitch(int W, int perm) { return perm ? (W + 31) & ~31 : W; }
size_t beta16_bytes(int H, int W, int n, int perm);
p2s_status launch_net16(p2s_ctx *ctx, const FieldGeom &g, int n, const float *alpha, void *beta16, int ones, int perm,
                        int *status, cudaStream_t st);
// The same over up to kMaxBatch frames of any sizes in one launch: frame i's anchors
// ([Ah][Aw][36]) and its beta block (beta16_bytes or beta8_bytes of one frame).
struct NetFrame {
    const float *alpha;
    void *beta;
    int H, W;
};
p2s_status launch_net16_frames(p2s_ctx *ctx, const NetFrame *frames, int n, int ones, int perm, int *status,
                               cudaStream_t st);
// FP8 contexts: the network kernel writes beta as E4M3 hi/lo pairs in
// [frame][row][16][col][16 B] (groups 0..7 the hi bytes of k = 16 g .. 16 g + 15,
// groups 8..15 the lo bytes), column order natural (perm = 0).
size_t beta8_bytes(int H, int W, int n);
p2s_status launch_pack8(p2s_ctx *ctx, int H, int W, int n, const float *beta, void *beta8, cudaStream_t st);
// FP32 beta [n][H][W][K] -> the 16-bit layout (entries k >= K zero).
p2s_status launch_pack16(p2s_ctx *ctx, int H, int W, int n, const float *beta, void *beta16, int perm,
                         cudaStream_t st);
// Tensor-core scatter blur of n frames of one size from the 16-bit beta.
p2s_status launch_scatter_tc(p2s_ctx *ctx, int H, int W, int C, int n, const float *const *xw, float *const *y,
                             const void *beta16, int *status, cudaStream_t st);
// The same over up to kMaxBatch frames of any sizes with C channels in one launch: frame i's
// x_w, output, and beta block (beta16_bytes of one frame, perm 0).
struct ScatterFrame {
    const float *xw;
    float *y;
    const void *beta;
    int H, W;
};
p2s_status launch_scatter_frames(p2s_ctx *ctx, const ScatterFrame *frames, int n, int C, int *status,
                                 cudaStream_t st);
int scatter_segment_rows(const p2s_ctx *ctx, int H);
// FFT evaluation of the scatter blur (FP32) from FP32 beta [n][H][W][K].
p2s_status launch_blur_fft(p2s_ctx *ctx, int H, int W, int C, int n, const float *const *xw, const float *beta,
                           float *const *y, cudaStream_t st);
p2s_status scatter_prepare(p2s_ctx *ctx);
p2s_status dense_prepare(p2s_ctx *ctx, const FieldGeom &g);

}  // namespace p2s
