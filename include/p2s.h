/*
 * p2s.h -- C ABI of libp2s, a GB300 (sm_103a) implementation of the per-frame
 * synthesis path of the phase-to-space (P2S) turbulence simulator
 * (Mao, Chimitt & Chan, "Accelerating Atmospheric Turbulence Simulation via
 * Learned Phase-to-Space Transform", ICCV 2021).
 *
 * The path, per frame (Sec. 3, Fig. 3 and Fig. 8):
 *   1. correlated Zernike coefficients on an anchor grid, by Fourier filtering
 *      of counter-based white noise and colouring with chol(R_Z)  (Sec. 2.2, 3.4)
 *   2. bilinear interpolation of the coefficients to every pixel   (Sec. 3.4)
 *   3. the tilt modes alpha_2, alpha_3 as a sub-pixel backward warp (Sec. 2.2, 3.3)
 *   4. the P2S network alpha_{4..36} -> beta in R^K                 (Sec. 3.3)
 *   5. the basis blur y = sum_k h_k * (beta_k . x_w)                (Sec. 3.1, Eq. 3-5)
 *
 * Conventions shared by every call:
 *   - Images are NHWC float32, rows contiguous, C in {1, 3}.  Device pointers
 *     unless the call says "host".  The caller owns every buffer it passes;
 *     an output must not alias an input.
 *   - Work is enqueued on the caller's CUDA stream (`stream`, a cudaStream_t;
 *     NULL = the legacy default stream) and runs asynchronously; the call
 *     returns once it is enqueued.  Host arrays passed in are read before the
 *     call returns.
 *   - No C++ exception crosses the ABI.  Every call returns a p2s_status;
 *     on P2S_EINVAL nothing is enqueued and no output is written.
 *     p2s_last_error() gives a one-line reason for the last failure on the
 *     calling thread.
 *   - A context is used by one host thread at a time (or externally locked).
 */
#ifndef P2S_H
#define P2S_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct p2s_ctx p2s_ctx;

typedef enum {
    P2S_OK = 0,
    P2S_EINVAL = 1,       /* bad argument or shape; nothing was enqueued       */
    P2S_ENOMEM = 2,       /* device or host allocation failed                  */
    P2S_ECUDA = 3,        /* a CUDA runtime call failed                        */
    P2S_ETIMEOUT = 4,     /* a bounded device wait gave up (status word set)   */
    P2S_EBUSY = 5,        /* serving queue or HBM budget full; retry later     */
    P2S_EUNSUPPORTED = 6  /* valid request the library or device cannot serve */
} p2s_status;

/* Arithmetic of the network and the basis contraction.  Fields and warp are
 * FP32 in every mode; the tap accumulation is FP32 in every mode. */
typedef enum {
    P2S_FP32 = 0,    /* FP32 throughout (CUDA cores)                          */
    P2S_BF16 = 1,    /* BF16 tensor-core operands, FP32 accumulation          */
    P2S_FP8E4M3 = 2, /* E4M3 contraction operands with per-basis scales       */
    P2S_FP16 = 3     /* FP16 tensor-core operands, FP32 accumulation          */
} p2s_precision;

/* Which PSF a tap uses (Sec. 3.1):
 *   SCATTER  y_c[p + o(t)] += G[p, t] x_c[p]   source pixel's PSF, y = sum_k h_k * (beta_k . x)
 *   GATHER   y_c[q] += G[q, t] x_c[q - o(t)]   output pixel's PSF, Eq. 5
 *   FFT      the scatter form evaluated by batched FFTs (comparison variant;
 *            FP32 precision only, frames up to 2016 pixels per side: the
 *            transform sizes are powers of two >= H + 32, W + 32, at most 2048)
 * with G[p, t] = sum_k beta[p, k] H[k, t] and o(t) = (ty - taps_h/2, tx - taps_w/2). */
typedef enum { P2S_SCATTER = 0, P2S_GATHER = 1, P2S_FFT = 2 } p2s_blur_form;

/* PSF basis (Eq. 4): K row vectors of taps_h x taps_w taps, host, row-major
 * [K][taps_h * taps_w], copied by p2s_create.  taps_h, taps_w odd. */
typedef struct {
    const double *H;
    int K;
    int taps_h;
    int taps_w;
} p2s_basis;

/* P2S network (Sec. 3.3): n_layers fully connected layers, ReLU after every
 * layer but the last.  dims[0] = 33 (alpha_4..alpha_36), dims[n_layers] = K.
 * W[l] is host row-major [dims[l+1]][dims[l]], b[l] is [dims[l+1]]; copied. */
typedef struct {
    int n_layers;
    const int *dims;
    const double *const *W;
    const double *const *b;
} p2s_mlp;

/* Spatial correlation of the anchor fields (Sec. 3.4; the paper's Takato
 * formulas are not printed, this is the stated Gaussian reading):
 *   anchors every `anchor_spacing` pixels, A = floor((H-1)/s) + 2 per axis;
 *   torus of the next power of two >= A + guard per axis;
 *   covariance exp(-|d|^2 / (2 ell^2)) (d in pixels) wrapped on the torus;
 *   n_kernels = 1 (shared) or 7 (one per radial order 1..7), lengths in
 *   corr_len_px (host, copied); fft_guard < 0 selects ceil(3 max(ell) / s).
 * kappa converts tilt coefficients to pixels (d = kappa (alpha_3, alpha_2)
 * in (row, column)); 0 selects -4/pi, the value for PSFs sampled with 2x
 * zero padding of the pupil. */
typedef struct {
    int anchor_spacing;
    int n_kernels;
    const double *corr_len_px;
    int fft_guard;
    double kappa;
} p2s_corr_params;

/* One frame: device NHWC float32, rows contiguous (row pitch W*C floats). */
typedef struct {
    float *data;
    int H;
    int W;
    int C;
} p2s_image;

/* Derived sizes for a frame shape, see p2s_geometry_of. */
typedef struct {
    int anchors_h, anchors_w;  /* anchor grid                                 */
    int torus_h, torus_w;      /* FFT torus of the field filter               */
    int alpha_stride;          /* floats per anchor in alpha buffers (36)     */
} p2s_geometry;

/* Create a simulator.  Copies the basis and weights to the device (converted
 * to the requested precision), builds R_Z for J = 2..36 and its Cholesky
 * factor in FP64 (Sec. 2.2), and the field filter tables.  Runs on the
 * current CUDA device.  Errors: EINVAL on inconsistent shapes (dims[0] != 33,
 * dims[last] != K, even taps, spacing < 1, n_kernels not 1 or 7); ENOMEM;
 * EUNSUPPORTED if the (precision, form) pair is not built for this device.
 * Limits: K <= 128, taps <= 33 x 33 and network widths <= 128 on every path;
 * the tensor-core paths (FP16, BF16, FP8) need exactly 33 x 33 taps, three
 * layers and K <= 110; FP8 E4M3 runs the gather form only
 * and the FFT form FP32 only. */
p2s_status p2s_create(const p2s_basis *basis, const p2s_mlp *mlp, const p2s_corr_params *corr,
                      p2s_precision precision, p2s_blur_form form, p2s_ctx **out);

/* Release everything the context owns.  Waits for its own streams. NULL is a no-op. */
void p2s_destroy(p2s_ctx *ctx);

const char *p2s_status_string(p2s_status s);
const char *p2s_last_error(void);

/* Anchor and torus sizes of an H x W frame under this context's parameters. */
p2s_status p2s_geometry_of(const p2s_ctx *ctx, int H, int W, p2s_geometry *out);

/* The whole path (steps 1-5) on n frames.  frames[i] and out[i] must have the
 * same H, W, C; frames may differ in size.  d_over_r0 and seeds are host
 * arrays of n entries: D/r0 of frame i (> 0) and its Philox key.  Frame i's
 * result depends only on (frames[i], d_over_r0[i], seeds[i]) and the
 * context.  Scratch is owned by the context and grown on demand. */
p2s_status p2s_simulate(p2s_ctx *ctx, const p2s_image *frames, int n, const float *d_over_r0,
                        const unsigned long long *seeds, const p2s_image *out, void *stream);

/* As p2s_simulate, but frames[i].data and out[i].data are HOST pointers: the
 * call stages them through device buffers (host->device copy, path,
 * device->host copy) and returns when out[] is written.  From 32 frames on,
 * the frames go in chunks: an eighth of them first and last, the rest in at
 * most 3 chunks of at least 16 (64 frames: 8 + 16 + 16 + 16 + 8).  A chunk's
 * host->device copy overlaps the path of the chunk before it and its
 * device->host copy the path of the chunk after, on two copy streams owned by
 * the context.  The chunks' paths alternate between `stream` and a second
 * compute stream owned by the context (one stream in graph mode), so that a
 * chunk's kernels fill the SMs the previous chunk's last wave leaves idle.  On
 * the tensor-core gather form (warp then blur, graphs off) the anchor fields
 * and the network (Sec. 3.3-3.4), which read no input pixels, run for every
 * frame first, while the inputs are copied in; each chunk then runs only its
 * warp and blur.  Results equal p2s_simulate's.  Pinned host memory gives full
 * copy bandwidth and overlap. */
p2s_status p2s_simulate_host(p2s_ctx *ctx, const p2s_image *frames, int n, const float *d_over_r0,
                             const unsigned long long *seeds, const p2s_image *out, void *stream);

/* Wavelength-dependent colour (Sec. 3.5): RGB frames whose channels are blurred
 * with three PSF sets, one per wavelength (the paper's 570, 540 and 450 nm for
 * R, G, B), at three times the cost of one.  ctx3[c] is channel c's context:
 * its basis holds that wavelength's PSFs, and its first network layer takes
 * alpha in radians at that wavelength (alpha at the reference wavelength times
 * lambda_ref / lambda_c, folded into W1 by the caller).  The three contexts
 * must share the device, the correlation parameters, kappa and the options
 * that shape the fields and the warp (one turbulence realisation: the fields
 * and the achromatic tilt warp are the same in every channel).  frames / out:
 * as for p2s_simulate, C = 3, device memory; channel c of each output is
 * channel c of the input run through ctx3[c] as a single-channel frame.
 * Stream-ordered scratch of two H x W planes per frame.  Errors as
 * p2s_simulate, plus EINVAL for mismatched contexts or C != 3. */
p2s_status p2s_simulate_spectral(p2s_ctx *const *ctx3, const p2s_image *frames, int n, const float *D_over_r0,
                                 const unsigned long long *seeds, const p2s_image *out, void *stream);

/* ---- stage entry points: each step alone, for per-stage parity ---------- */

/* Step 1a: the white noise of stream (seed, mode), F_h x F_w row-major into
 * `out` (device float32), sample i from Philox4x32-10 counter (i/4, mode, 0, 0)
 * word i%4, key (seed mod 2^32, seed >> 32), Box-Muller per word pair. */
p2s_status p2s_stage_noise(p2s_ctx *ctx, unsigned long long seed, int mode, int torus_h, int torus_w,
                           float *out, void *stream);

/* Steps 1a-1c for n frames of size H x W: alpha on the anchors, device
 * float32 [n][anchors_h][anchors_w][36]; slot 0 is piston (written 0), slot
 * j-1 holds Noll mode j = 2..36.  Host arrays d_over_r0[n], seeds[n]. */
p2s_status p2s_stage_fields(p2s_ctx *ctx, int H, int W, int n, const float *d_over_r0,
                            const unsigned long long *seeds, float *alpha, void *stream);

/* Steps 2-3: x_w = warp of `in` by the tilts of `alpha` (one frame, the
 * layout of p2s_stage_fields), into `out` (same shape as in). */
p2s_status p2s_stage_warp(p2s_ctx *ctx, const p2s_image *in, const float *alpha, const p2s_image *out,
                          void *stream);

/* Steps 2 + 4: beta of every pixel of an H x W frame from `alpha` (one
 * frame), device float32 [H][W][K], in the context's precision. */
p2s_status p2s_stage_mlp(p2s_ctx *ctx, int H, int W, const float *alpha, float *beta, void *stream);

/* Steps 2 + 4 for FP16 / BF16 contexts, written the way the tensor-core blur
 * reads beta: the 16-bit operand layout beta16[H][14][W][8] (device, 16-bit
 * FP16 or BF16 values as the context's precision, H*W*224 bytes), where
 * element (row, g, col, e) is beta_k of pixel (row, col) for k = 8 g + e.
 * It holds the network output WITHOUT the last layer's bias (Sec. 3.3 network
 * with b3 folded into the basis as an exact hi/lo pair of extra rows): entries
 * k = K and K + 1 are 1.0, entries beyond are 0.  EUNSUPPORTED for FP32. */
p2s_status p2s_stage_mlp16(p2s_ctx *ctx, int H, int W, const float *alpha, void *beta16, void *stream);

/* FP8 E4M3 contexts (no counterpart in the paper, which does not state a
 * precision): the power-of-two scales of the contraction.  The contraction
 * G = sum_k beta_k H_k (Sec. 3.1, Eq. 4-5) runs with beta_k stored as
 * beta_k * scale[k] and basis row k as H_k * 2^c / scale[k], each as an E4M3
 * hi/lo pair (hi = e4m3(v), lo = e4m3(v - hi)); the tap sums are multiplied by
 * *inv_c = 2^-c.  Entries K and K + 1 are the two columns that carry the folded
 * last-layer bias.  scale: host array of n >= K + 2 floats, written.  EINVAL
 * for NULL pointers or n < K + 2, EUNSUPPORTED for other precisions.
 * Synchronous: reads the scales back from the device. */
p2s_status p2s_contraction_scales(p2s_ctx *ctx, float *scale, int n, float *inv_c);

/* Step 5 alone: y = blur of x_w with per-pixel weights beta (device float32
 * [H][W][K]) in the context's form and precision (beta is rounded to the
 * operand type first).  FP16 / BF16 gather contexts run the same blur kernel
 * as p2s_simulate (P2S_OPT_GATHER_SPLIT): with the option set, beta is first
 * packed into the 16-bit operand layout in stream-ordered scratch. */
p2s_status p2s_stage_blur(p2s_ctx *ctx, const p2s_image *xw, const float *beta, const p2s_image *out,
                          void *stream);

/* Synchronises `stream`, then reads and clears the context's device status
 * word, which a kernel sets when one of its bounded waits gives up (a
 * pipeline stage stalled for about two seconds).  Returns P2S_ETIMEOUT if it
 * was set (the outputs of the calls since the last check are then invalid),
 * P2S_ECUDA if the stream reports an error, P2S_OK otherwise. */
p2s_status p2s_check(p2s_ctx *ctx, void *stream);

/* Self-test of that mechanism (no counterpart in the paper): enqueues one
 * block whose bounded mbarrier wait has nothing to wait for; after about
 * 0.1 s it gives up and sets the status word exactly as a stalled pipeline
 * stage would, so the next p2s_check returns P2S_ETIMEOUT (and clears it).
 * Nothing faults or hangs; the context stays usable. */
p2s_status p2s_selftest_stall(p2s_ctx *ctx, void *stream);

/* ---- tuning --------------------------------------------------------------- */

/* Tunable launch parameters (no counterpart in the paper; results do not
 * depend on them beyond floating-point summation order):
 *   P2S_OPT_SCATTER_SEGMENT_ROWS  source rows per work unit of the
 *       tensor-core scatter blur (even, >= 2; 0 = default 128).  Target rows
 *       within 16 rows of a segment boundary are summed with atomic adds.
 *   P2S_OPT_GRAPHS  1: p2s_simulate captures its launches into a CUDA graph,
 *       instantiated once per batch signature (the frames' sizes and channel
 *       counts, in order) and afterwards only updated with each call's
 *       pointers, seeds and strengths.  Scratch then comes from an arena owned
 *       by the context (grown on demand, which synchronises once), so calls of
 *       one context must not overlap on the GPU in this mode.  Ignored while
 *       profiling.  0 (default): plain launches.
 *   P2S_OPT_GRAPH_INSTANTIATIONS, P2S_OPT_GRAPH_UPDATES  (read only) how many
 *       graphs were instantiated / updated in place so far.
 *   P2S_OPT_GATHER_BAND_ROWS  tile height of the fused tensor-core gather
 *       kernel (P2S_OPT_GATHER_SPLIT = 0): 16 or 32 output rows per 128-column
 *       tile (0 = default 32).
 *   P2S_OPT_BLUR_THEN_WARP  1: p2s_simulate blurs the input first and applies
 *       the tilt warp to the blurred frame, the order of the collapsed model
 *       (Sec. 2.2: the turbulent PSF is a tilt-free PSF shifted by the tilt);
 *       0 (default): warp, then blur.
 *   P2S_OPT_FIELD_METHOD  how the anchor fields get their spatial
 *       correlation (Sec. 3.4): 0 (default) Fourier filtering on a torus;
 *       1 the dense draw f = chol(Sigma) w of the anchors' full (unwrapped)
 *       Gaussian correlation matrix, evaluated through its Kronecker factors
 *       L_y W L_x^T (at most 128 anchors per axis).
 *   P2S_OPT_GATHER_SPLIT  tensor-core gather form only.  0: one fused
 *       kernel evaluates the network and the blur per tile, beta never leaves
 *       the SM.  1 (default in BF16 and FP8 contexts; the only value FP8
 *       takes): the network kernel writes beta in its 16-bit
 *       operand layout (224 B per pixel of scratch) and a blur-only
 *       tensor-core kernel with four accumulating warps per TMEM lane
 *       quadrant reads it back.  2, 3: the same split with one of two
 *       fragment kernels (G read as 16x256b TMEM fragments; beta written with
 *       its columns permuted within 32-column blocks; 3 keeps x and G in
 *       FP32).  4: the same split with the tap products as packed FP16 FMAs
 *       (two output rows per instruction; default in FP16 contexts), FP16
 *       partial sums of 12 products
 *       flushed into FP32 per basis chunk: 1e-4 to 1e-3 relative error on top
 *       of kernel 1's, the more the PSF weights cancel (FP16 and BF16
 *       contexts; not FP8).
 *       Rounding points of kernel 1 (and 2): those of the fused kernel (beta
 *       and H in 16 bits, x staged in FP16, FP32 accumulation) plus one:
 *       G = beta H is rounded to FP16 before the tap products (FP16 x FP16,
 *       exact in FP32), at most 2^-11 relative per tap product.  A G beyond the FP16 range (|G| > 65504)
 *       would overflow; PSF weights of the model are orders of magnitude
 *       smaller (the PSF taps sum to about 1), so this needs beta far outside
 *       anything the network produces, e.g. hand-made beta given to
 *       p2s_stage_blur. */
typedef enum {
    P2S_OPT_SCATTER_SEGMENT_ROWS = 1,
    P2S_OPT_GRAPHS = 2,
    P2S_OPT_GRAPH_INSTANTIATIONS = 3,
    P2S_OPT_GRAPH_UPDATES = 4,
    P2S_OPT_GATHER_BAND_ROWS = 5,
    P2S_OPT_BLUR_THEN_WARP = 6,
    P2S_OPT_FIELD_METHOD = 7,
    P2S_OPT_GATHER_SPLIT = 8
} p2s_option;
p2s_status p2s_set_option(p2s_ctx *ctx, int option, int value);
p2s_status p2s_get_option(const p2s_ctx *ctx, int option, int *value);

/* Autotuner (no counterpart in the paper).  Runs p2s_simulate on the given
 * batch (device frames, written to `out`) once per candidate setting of the
 * launch options of the context's path, after one warm-up call times `reps`
 * calls with CUDA events on `stream` (synchronising it), keeps the fastest
 * setting in the context and reports every candidate in `res` (may be NULL).
 * Candidates: FP16 / BF16 tensor-core gather, the kernel and its tile shape
 * (P2S_OPT_GATHER_SPLIT 1 .. 4 -- the four blur-only kernels, 128 x 32 and
 * 128 x 16 tiles, one or four output columns per accumulating thread -- and 0,
 * the fused kernel, with P2S_OPT_GATHER_BAND_ROWS 16 or 32); tensor-core
 * scatter, P2S_OPT_SCATTER_SEGMENT_ROWS 8 .. 1024 (the rows per work unit);
 * FP32 and FP8 paths have none.  Arguments as p2s_simulate; reps >= 1. */
typedef struct {
    int option;       /* the p2s_option tuned (0 if the path has none) */
    int option2;      /* a second option set with it (0 if none) */
    int n;            /* candidates tried */
    int value[8];     /* candidate settings of `option` */
    int value2[8];    /* ... and of `option2` (0: left as it was) */
    float ms[8];      /* mean milliseconds per call of each */
    int best;         /* index of the setting kept */
} p2s_tune_result;
p2s_status p2s_autotune(p2s_ctx *ctx, const p2s_image *frames, int n, const float *d_over_r0,
                        const unsigned long long *seeds, const p2s_image *out, void *stream, int reps,
                        p2s_tune_result *res);

/* ---- serving (no counterpart in the paper) -------------------------------- */

/* A request loop over one context: single frames of any size, each with its
 * own D/r0 and seed, submitted from host memory.  The context keeps the
 * basis and weights resident; requests are admitted in arrival order while
 * their device footprint (input, output, path scratch) fits in
 * hbm_budget_bytes, and whatever is admitted when one of the
 * max_inflight_batches stream slots frees is run as one p2s_simulate call
 * (at most max_batch frames).  Batches of different slots overlap on the
 * device; requests arriving meanwhile join the next batch (continuous
 * batching).  Each request's result depends only on its own frame, D/r0 and
 * seed.  Host buffers must stay valid until the request is done; pinned
 * memory gives asynchronous copies.  The context must not be in graph mode
 * and must not be used by other calls while the server exists. */
typedef struct p2s_server p2s_server;
typedef struct {
    size_t hbm_budget_bytes;   /* > 0 */
    int max_inflight_batches;  /* 1..16 */
    int max_batch;             /* 1..256 */
} p2s_server_config;
typedef struct {
    long long completed, batches, pending;
    double mean_batch;         /* frames per batch so far */
    size_t bytes_in_use, peak_bytes;
} p2s_server_counters;
p2s_status p2s_server_create(p2s_ctx *ctx, const p2s_server_config *cfg, p2s_server **out);
/* Queues a request; *ticket identifies it.  ENOMEM if it alone exceeds the budget. */
p2s_status p2s_server_submit(p2s_server *srv, const float *host_in, int H, int W, int C, float d_over_r0,
                             unsigned long long seed, float *host_out, long long *ticket);
/* Non-blocking: *done = 1 once out is written; latency_ms = completion - submission. */
p2s_status p2s_server_poll(p2s_server *srv, long long ticket, int *done, double *latency_ms);
/* Blocks up to timeout_s seconds; ETIMEOUT if still running. */
p2s_status p2s_server_wait(p2s_server *srv, long long ticket, double timeout_s, double *latency_ms);
p2s_status p2s_server_stats(p2s_server *srv, p2s_server_counters *out);
/* Finishes queued and running requests, then releases the server. */
void p2s_server_destroy(p2s_server *srv);

/* ---- kernel timing ------------------------------------------------------- */

/* Per-kernel totals recorded while profiling is on: CUDA events bracket every
 * launch of the library on the stream it is launched on.  flops and bytes
 * are the launch's ALGORITHMIC work (what the method needs, not what the
 * hardware moved), summed over launches. */
typedef struct {
    char name[48];
    int launches;
    double total_ms;
    double flops;
    double bytes;
} p2s_kernel_stat;

/* enable = 1 clears the record and starts recording; 0 stops. */
p2s_status p2s_profile(p2s_ctx *ctx, int enable);

/* Waits for the recorded events and writes up to max_stats aggregated entries
 * (one per kernel name, in order of first launch); *n_stats gets the count. */
p2s_status p2s_profile_read(p2s_ctx *ctx, p2s_kernel_stat *stats, int max_stats, int *n_stats);

/* Allocation-free variant of p2s_stage_mlp for FP32 contexts (no counterpart
 * in the paper: it exists for callers that cannot allocate device memory at
 * call time, e.g. code held to a fixed, pre-reserved memory budget or a host
 * thread that must stay out of the CUDA allocator).  Same arguments, layout
 * and result as p2s_stage_mlp.  It allocates nothing: the network's weight
 * image is assembled in a 163 KiB array (41,728 floats: the largest image
 * the plain network kernel can stage in its 227 KiB of shared memory beside
 * its 64 KiB of activation buffers) that the library holds in device memory
 * on every GPU that loads it, for the life of the process.
 *   - The first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress) with the device current; make that first call
 *     before any stream capture.
 *   - Every call and every context on a device share the one array, and each
 *     call rewrites it: calls whose work overlaps on the GPU (different
 *     streams, or concurrent host threads) race; serialise them.
 *   - Errors: EUNSUPPORTED for non-FP32 contexts or networks the plain path
 *     does not build; EINVAL if the weight image (weights plus biases, each
 *     bias block padded to 4 floats) exceeds 41,728 floats, or if the
 *     current device is not the context's.  p2s_profile records the call as
 *     "mlp_fp32". */
p2s_status p2s_stage_mlp_noalloc(p2s_ctx *ctx, int H, int W, const float *alpha, float *beta, void *stream);

/* ---- host-side building blocks ----------------------------------------- */

/* Noll covariance R_Z of modes J = 2..j_max at D/r0 = 1 (Sec. 2.2; closed
 * form of Noll 1976), FP64 row-major [(j_max-1)^2] into host `out`.
 * j_max in [3, 66].  Pure host code; needs no GPU. */
p2s_status p2s_noll_covariance(int j_max, double *out);

#ifdef __cplusplus
}
#endif

#endif /* P2S_H */
