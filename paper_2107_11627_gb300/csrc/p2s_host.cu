// Host side of libp2s: the C ABI, context set-up in FP64, validation, dispatch.
#include <algorithm>
#include <functional>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "p2s_internal.h"

namespace p2s {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

static p2s_status einval(const char *msg) {
    set_error("%s", msg);
    return P2S_EINVAL;
}

// ---- Noll modes and covariance (Sec. 2.2; closed form of Noll 1976) --------

// Radial order n and |m| of Noll mode j (j >= 1): modes of order n occupy
// j in (n(n+1)/2, (n+1)(n+2)/2]; |m| grows along the order, each m > 0 twice.
static void noll_nm(int j, int *n, int *m) {
    int order = 0;
    while ((order + 1) * (order + 2) / 2 < j) ++order;
    int pos = j - order * (order + 1) / 2 - 1;
    *n = order;
    *m = (order % 2 == 0) ? 2 * ((pos + 1) / 2) : 2 * (pos / 2) + 1;
}

static double noll_entry(int i, int j) {
    int ni, mi, nj, mj;
    noll_nm(i, &ni, &mi);
    noll_nm(j, &nj, &mj);
    if (mi != mj) return 0.0;
    if (mi != 0 && ((i - j) % 2) != 0) return 0.0;
    const double kc = std::tgamma(14.0 / 3.0) * std::pow(24.0 / 5.0 * std::tgamma(6.0 / 5.0), 5.0 / 6.0) *
                      std::tgamma(11.0 / 6.0) * std::tgamma(11.0 / 6.0) / (2.0 * M_PI * M_PI);
    const int e = (ni + nj - 2 * mi) / 2;
    const double sign = (e % 2 == 0) ? 1.0 : -1.0;
    const double num = std::tgamma((ni + nj - 5.0 / 3.0) / 2.0);
    const double den = std::tgamma((ni - nj + 17.0 / 3.0) / 2.0) * std::tgamma((nj - ni + 17.0 / 3.0) / 2.0) *
                       std::tgamma((ni + nj + 23.0 / 3.0) / 2.0);
    return kc * sign * std::sqrt((ni + 1.0) * (nj + 1.0)) * num / den;
}

// In-place lower Cholesky factor of an n x n SPD matrix (row-major).
static bool cholesky(double *a, int n) {
    for (int j = 0; j < n; ++j) {
        double d = a[j * n + j];
        for (int k = 0; k < j; ++k) d -= a[j * n + k] * a[j * n + k];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        a[j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double v = a[i * n + j];
            for (int k = 0; k < j; ++k) v -= a[i * n + k] * a[j * n + k];
            a[i * n + j] = v / d;
        }
        for (int k = j + 1; k < n; ++k) a[j * n + k] = 0.0;
    }
    return true;
}

static int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

p2s_status geometry(const p2s_ctx *ctx, int H, int W, FieldGeom *g) {
    if (H < 1 || W < 1) return einval("frame must be at least 1 x 1");
    g->H = H;
    g->W = W;
    g->s = ctx->s;
    g->Ah = (H - 1) / ctx->s + 2;
    g->Aw = (W - 1) / ctx->s + 2;
    g->Fh = next_pow2(g->Ah + ctx->guard);
    g->Fw = next_pow2(g->Aw + ctx->guard);
    if (g->Fh > 4096 || g->Fw > 4096) {
        set_error("filter torus %dx%d exceeds 4096 (raise anchor_spacing)", g->Fh, g->Fw);
        return P2S_EUNSUPPORTED;
    }
    return P2S_OK;
}

// Separable filter of the wrapped Gaussian covariance on a torus of length F:
// c1[d] = sum_m exp(-(d + mF)^2 s^2 / (2 ell^2)), C1 = DFT(c1) (real, > 0 by
// Poisson summation), gain = sqrt(C1) / F.  sqrt(C2) = gain_h (x) gain_w.
p2s_status filter_table(p2s_ctx *ctx, int F, const FilterTable **out) {
    auto it = ctx->tables.find(F);
    if (it != ctx->tables.end()) {
        *out = &it->second;
        return P2S_OK;
    }
    FilterTable t;
    t.F = F;
    std::vector<float2> tw(F / 2 > 0 ? F / 2 : 1);
    for (int m = 0; m < F / 2; ++m) {
        double a = 2.0 * M_PI * m / F;
        tw[m] = make_float2((float)std::cos(a), (float)-std::sin(a));
    }
    std::vector<float> gain((size_t)ctx->n_kernels * F);
    std::vector<double> c1(F);
    for (int kk = 0; kk < ctx->n_kernels; ++kk) {
        const double ell = ctx->ell[kk], s = ctx->s;
        const int M = (int)std::ceil(40.0 * ell / (s * F)) + 1;
        for (int d = 0; d < F; ++d) {
            double acc = 0.0;
            for (int m = -M; m <= M; ++m) {
                double x = (d + (double)m * F) * s;
                acc += std::exp(-x * x / (2.0 * ell * ell));
            }
            c1[d] = acc;
        }
        for (int u = 0; u < F; ++u) {
            double acc = 0.0;
            for (int d = 0; d < F; ++d) acc += c1[d] * std::cos(2.0 * M_PI * (double)((long long)u * d % F) / F);
            gain[(size_t)kk * F + u] = (float)(std::sqrt(acc > 0.0 ? acc : 0.0) / F);
        }
    }
    P2S_CUDA(cudaMalloc(&t.twiddle, tw.size() * sizeof(float2)));
    P2S_CUDA(cudaMalloc(&t.gain, gain.size() * sizeof(float)));
    P2S_CUDA(cudaMemcpy(t.twiddle, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
    P2S_CUDA(cudaMemcpy(t.gain, gain.data(), gain.size() * sizeof(float), cudaMemcpyHostToDevice));
    auto res = ctx->tables.emplace(F, t);
    *out = &res.first->second;
    return P2S_OK;
}

static cudaEvent_t pool_event(p2s_ctx *ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

ProfScope::ProfScope(const p2s_ctx *ctx, cudaStream_t st, const char *name, double flops, double bytes)
    : ctx_(const_cast<p2s_ctx *>(ctx)), st_(st) {
    if (!ctx_ || !ctx_->profiling) return;
    ProfRecord r{name, pool_event(ctx_), pool_event(ctx_), flops, bytes};
    if (!r.start || !r.stop) return;
    cudaEventRecord(r.start, st_);
    ctx_->prof.push_back(r);
    idx_ = (int)ctx_->prof.size() - 1;
}

ProfScope::~ProfScope() {
    if (idx_ >= 0) cudaEventRecord(ctx_->prof[idx_].stop, st_);
}

static int radial_order(int j) {
    int n, m;
    noll_nm(j, &n, &m);
    return n;
}

}  // namespace p2s

using namespace p2s;

extern "C" {

const char *p2s_status_string(p2s_status s) {
    switch (s) {
        case P2S_OK: return "ok";
        case P2S_EINVAL: return "invalid argument";
        case P2S_ENOMEM: return "out of memory";
        case P2S_ECUDA: return "CUDA error";
        case P2S_ETIMEOUT: return "device wait timed out";
        case P2S_EBUSY: return "busy";
        case P2S_EUNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *p2s_last_error(void) { return g_err; }

p2s_status p2s_noll_covariance(int j_max, double *out) {
    if (!out || j_max < 3 || j_max > 66) return einval("j_max must be in [3, 66] and out non-NULL");
    const int n = j_max - 1;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) out[a * n + b] = noll_entry(a + 2, b + 2);
    return P2S_OK;
}

p2s_status p2s_create(const p2s_basis *basis, const p2s_mlp *mlp, const p2s_corr_params *corr,
                      p2s_precision precision, p2s_blur_form form, p2s_ctx **out) {
    if (!out) return einval("out is NULL");
    *out = nullptr;
    if (!basis || !mlp || !corr) return einval("basis, mlp and corr must be non-NULL");
    if (!basis->H || basis->K < 1 || basis->K > 128) return einval("basis: need H and 1 <= K <= 128");
    if (basis->taps_h < 1 || basis->taps_w < 1 || basis->taps_h % 2 == 0 || basis->taps_w % 2 == 0)
        return einval("basis taps must be odd and positive");
    if (basis->taps_h > 33 || basis->taps_w > 33) {
        set_error("taps larger than 33 x 33 are not built");
        return P2S_EUNSUPPORTED;
    }
    if (mlp->n_layers < 1 || !mlp->dims || !mlp->W || !mlp->b) return einval("mlp: need n_layers >= 1, dims, W, b");
    if (mlp->dims[0] != kHiModes) return einval("mlp: dims[0] must be 33 (alpha_4..alpha_36)");
    if (mlp->dims[mlp->n_layers] != basis->K) return einval("mlp: last width must equal K");
    for (int l = 0; l < mlp->n_layers; ++l) {
        if (mlp->dims[l + 1] < 1 || !mlp->W[l] || !mlp->b[l]) return einval("mlp: bad layer");
        if (mlp->dims[l + 1] > 128) {
            set_error("network widths above 128 are not built");
            return P2S_EUNSUPPORTED;
        }
    }
    if (corr->anchor_spacing < 1) return einval("anchor_spacing must be >= 1");
    if (corr->n_kernels != 1 && corr->n_kernels != 7) return einval("n_kernels must be 1 or 7");
    if (!corr->corr_len_px) return einval("corr_len_px is NULL");
    for (int k = 0; k < corr->n_kernels; ++k)
        if (!(corr->corr_len_px[k] > 0.0) || !std::isfinite(corr->corr_len_px[k])) return einval("corr_len_px must be > 0");
    if (!(form == P2S_SCATTER || form == P2S_GATHER || form == P2S_FFT)) return einval("unknown blur form");
    if (!(precision == P2S_FP32 || precision == P2S_BF16 || precision == P2S_FP16 || precision == P2S_FP8E4M3))
        return einval("unknown precision");
    const bool tc_prec = tc_precision(precision);
    if ((precision == P2S_FP8E4M3 && form != P2S_GATHER) || (form == P2S_FFT && precision != P2S_FP32)) {
        set_error("precision/form pair not built (FP8 E4M3: gather form only; FFT: FP32 only)");
        return P2S_EUNSUPPORTED;
    }

    p2s_ctx *ctx = new (std::nothrow) p2s_ctx();
    if (!ctx) return P2S_ENOMEM;
    auto fail = [&](p2s_status st) {
        p2s_destroy(ctx);
        return st;
    };
    if (cudaGetDevice(&ctx->device) != cudaSuccess) {
        set_error("no CUDA device");
        return fail(P2S_ECUDA);
    }
    ctx->prec = precision;
    ctx->form = form;
    // default blur-only gather kernel: packed FP16 products for FP16 operands, kernel 1 otherwise
    ctx->gather_split = precision == P2S_FP16 ? 4 : 1;
    ctx->K = basis->K;
    ctx->th = basis->taps_h;
    ctx->tw = basis->taps_w;
    ctx->T = ctx->th * ctx->tw;
    ctx->H.assign(basis->H, basis->H + (size_t)ctx->K * ctx->T);
    ctx->n_layers = mlp->n_layers;
    ctx->dims.assign(mlp->dims, mlp->dims + mlp->n_layers + 1);
    for (int l = 0; l < mlp->n_layers; ++l) {
        const int fi = ctx->dims[l], fo = ctx->dims[l + 1];
        ctx->W.emplace_back(mlp->W[l], mlp->W[l] + (size_t)fi * fo);
        ctx->b.emplace_back(mlp->b[l], mlp->b[l] + fo);
    }
    ctx->s = corr->anchor_spacing;
    ctx->n_kernels = corr->n_kernels;
    ctx->ell.assign(corr->corr_len_px, corr->corr_len_px + corr->n_kernels);
    double ell_max = 0.0;
    for (double e : ctx->ell) ell_max = e > ell_max ? e : ell_max;
    ctx->guard = corr->fft_guard >= 0 ? corr->fft_guard : (int)std::ceil(3.0 * ell_max / ctx->s);
    ctx->kappa = corr->kappa != 0.0 ? corr->kappa : -4.0 / M_PI;
    for (int l = 0; l < kModes; ++l) ctx->kernel_of_mode[l] = ctx->n_kernels == 1 ? 0 : radial_order(l + 2) - 1;

    // R_Z (J = 2..36) and its Cholesky factor, FP64.
    std::vector<double> R(kModes * kModes);
    for (int a = 0; a < kModes; ++a)
        for (int c = 0; c < kModes; ++c) R[a * kModes + c] = noll_entry(a + 2, c + 2);
    if (!cholesky(R.data(), kModes)) {
        set_error("R_Z is not positive definite");
        return fail(P2S_EINVAL);
    }
    std::vector<float> Lf(kModes * kModes);
    for (int i = 0; i < kModes * kModes; ++i) Lf[i] = (float)R[i];
    ctx->L64.assign(R.begin(), R.end());

    // FP32 device copies used by the plain path.
    std::vector<float> H32(ctx->H.begin(), ctx->H.end()), Ht32((size_t)ctx->T * ctx->K);
    for (int k = 0; k < ctx->K; ++k)
        for (int t = 0; t < ctx->T; ++t) Ht32[(size_t)t * ctx->K + k] = (float)ctx->H[(size_t)k * ctx->T + t];
    if (cudaMalloc(&ctx->d_L, Lf.size() * 4) != cudaSuccess || cudaMalloc(&ctx->d_H32, H32.size() * 4) != cudaSuccess ||
        cudaMalloc(&ctx->d_Ht32, Ht32.size() * 4) != cudaSuccess ||
        cudaMalloc(&ctx->d_kernel_of_mode, sizeof ctx->kernel_of_mode) != cudaSuccess) {
        set_error("device allocation failed in p2s_create");
        return fail(P2S_ENOMEM);
    }
    if (cudaMemcpy(ctx->d_L, Lf.data(), Lf.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctx->d_H32, H32.data(), H32.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctx->d_Ht32, Ht32.data(), Ht32.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctx->d_kernel_of_mode, ctx->kernel_of_mode, sizeof ctx->kernel_of_mode, cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        set_error("upload failed in p2s_create");
        return fail(P2S_ECUDA);
    }
    for (int l = 0; l < ctx->n_layers; ++l) {
        const int fi = ctx->dims[l], fo = ctx->dims[l + 1];
        std::vector<float> wt((size_t)fi * fo), bb(fo);
        for (int o = 0; o < fo; ++o) {
            for (int i = 0; i < fi; ++i) wt[(size_t)i * fo + o] = (float)ctx->W[l][(size_t)o * fi + i];
            bb[o] = (float)ctx->b[l][o];
        }
        float *dw = nullptr, *db = nullptr;
        if (cudaMalloc(&dw, wt.size() * 4) != cudaSuccess || cudaMalloc(&db, bb.size() * 4) != cudaSuccess) {
            cudaFree(dw);
            set_error("device allocation failed in p2s_create");
            return fail(P2S_ENOMEM);
        }
        ctx->d_Wt32.push_back(dw);
        ctx->d_b32.push_back(db);
        if (cudaMemcpy(dw, wt.data(), wt.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(db, bb.data(), bb.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
            set_error("upload failed in p2s_create");
            return fail(P2S_ECUDA);
        }
    }
    if (cudaMalloc(&ctx->d_status, sizeof(int)) != cudaSuccess || cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess) {
        set_error("device allocation failed in p2s_create");
        return fail(P2S_ENOMEM);
    }
    if (tc_prec) {
        p2s_status st = tc_prepare(ctx);
        if (st != P2S_OK) return fail(st);
    }
    // Keep stream-ordered scratch cached between calls.
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
        unsigned long long thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    *out = ctx;
    return P2S_OK;
}

void p2s_destroy(p2s_ctx *ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    for (auto &r : ctx->prof) {
        cudaEventDestroy(r.start);
        cudaEventDestroy(r.stop);
    }
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    cudaFree(ctx->d_L);
    cudaFree(ctx->d_H32);
    cudaFree(ctx->d_Ht32);
    cudaFree(ctx->d_kernel_of_mode);
    for (float *p : ctx->d_Wt32) cudaFree(p);
    for (float *p : ctx->d_b32) cudaFree(p);
    for (auto &kv : ctx->tables) {
        cudaFree(kv.second.twiddle);
        cudaFree(kv.second.gain);
    }
    cudaFree(ctx->d_status);
    cudaFree(ctx->tc.d_W);
    cudaFree(ctx->tc.d_H);
    cudaFree(ctx->tc.d_bias);
    cudaFree(ctx->tc.d_Hs);
    cudaFree(ctx->tc.d_H8);
    cudaFree(ctx->tc.d_scale8);
    for (auto &kv : ctx->fft_tw) cudaFree(kv.second);
    for (auto &kv : ctx->dense_L) cudaFree(kv.second);
    for (auto &kv : ctx->fft_basis) cudaFree(kv.second);
    for (auto &kv : ctx->graphs)
        if (kv.second) cudaGraphExecDestroy(kv.second);
    cudaFree(ctx->arena);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
    for (cudaStream_t cs : ctx->copy_stream)
        if (cs) cudaStreamDestroy(cs);
    for (cudaEvent_t e : ctx->host_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->cap_ev)
        if (e) cudaEventDestroy(e);
    delete ctx;
}

p2s_status p2s_check(p2s_ctx *ctx, void *stream) {
    if (!ctx) return einval("ctx is NULL");
    P2S_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int word = 0;
    P2S_CUDA(cudaMemcpy(&word, ctx->d_status, sizeof word, cudaMemcpyDeviceToHost));
    if (word != 0) {
        P2S_CUDA(cudaMemset(ctx->d_status, 0, sizeof(int)));
        set_error("a bounded device wait gave up (status word 0x%x)", word);
        return P2S_ETIMEOUT;
    }
    return P2S_OK;
}

p2s_status p2s_profile(p2s_ctx *ctx, int enable) {
    if (!ctx) return einval("ctx is NULL");
    if (enable) {
        for (auto &r : ctx->prof) {
            ctx->event_pool.push_back(r.start);
            ctx->event_pool.push_back(r.stop);
        }
        ctx->prof.clear();
    }
    ctx->profiling = enable != 0;
    return P2S_OK;
}

p2s_status p2s_profile_read(p2s_ctx *ctx, p2s_kernel_stat *stats, int max_stats, int *n_stats) {
    if (!ctx || !n_stats || (max_stats > 0 && !stats)) return einval("bad profile_read arguments");
    std::vector<p2s_kernel_stat> agg;
    for (auto &r : ctx->prof) {
        P2S_CUDA(cudaEventSynchronize(r.stop));
        float ms = 0.0f;
        P2S_CUDA(cudaEventElapsedTime(&ms, r.start, r.stop));
        size_t i = 0;
        for (; i < agg.size(); ++i)
            if (std::strncmp(agg[i].name, r.name, sizeof agg[i].name) == 0) break;
        if (i == agg.size()) {
            p2s_kernel_stat z;
            std::memset(&z, 0, sizeof z);
            std::snprintf(z.name, sizeof z.name, "%s", r.name);
            agg.push_back(z);
        }
        agg[i].launches += 1;
        agg[i].total_ms += ms;
        agg[i].flops += r.flops;
        agg[i].bytes += r.bytes;
    }
    *n_stats = (int)agg.size();
    for (int i = 0; i < (int)agg.size() && i < max_stats; ++i) stats[i] = agg[i];
    return P2S_OK;
}

p2s_status p2s_geometry_of(const p2s_ctx *ctx, int H, int W, p2s_geometry *out) {
    if (!ctx || !out) return einval("ctx and out must be non-NULL");
    FieldGeom g;
    p2s_status st = geometry(ctx, H, W, &g);
    if (st != P2S_OK) return st;
    out->anchors_h = g.Ah;
    out->anchors_w = g.Aw;
    out->torus_h = g.Fh;
    out->torus_w = g.Fw;
    out->alpha_stride = kAlphaStride;
    return P2S_OK;
}

// ---- stage entry points ----------------------------------------------------

p2s_status p2s_stage_noise(p2s_ctx *ctx, unsigned long long seed, int mode, int torus_h, int torus_w, float *out,
                           void *stream) {
    if (!ctx || !out) return einval("ctx and out must be non-NULL");
    if (mode < 0 || torus_h < 1 || torus_w < 1 || (long long)torus_h * torus_w > (1ll << 30))
        return einval("bad noise shape or mode");
    return launch_noise(seed, mode, torus_h, torus_w, out, (cudaStream_t)stream);
}

static p2s_status check_frames_meta(int n, const float *d_over_r0, const unsigned long long *seeds) {
    if (n < 0) return einval("n must be >= 0");
    if (n > 0 && (!d_over_r0 || !seeds)) return einval("d_over_r0 and seeds must be non-NULL");
    for (int i = 0; i < n; ++i)
        if (!(d_over_r0[i] > 0.0f) || !std::isfinite(d_over_r0[i])) return einval("D/r0 must be finite and > 0");
    return P2S_OK;
}

static void fill_batch(FrameBatch *fb, int n, const float *d_over_r0, const unsigned long long *seeds) {
    fb->n = n;
    for (int i = 0; i < n; ++i) {
        fb->seed[i] = seeds[i];
        fb->scale[i] = (float)std::pow((double)d_over_r0[i], 5.0 / 6.0);
    }
}

p2s_status p2s_stage_fields(p2s_ctx *ctx, int H, int W, int n, const float *d_over_r0,
                            const unsigned long long *seeds, float *alpha, void *stream) {
    if (!ctx || (!alpha && n > 0)) return einval("ctx and alpha must be non-NULL");
    p2s_status st = check_frames_meta(n, d_over_r0, seeds);
    if (st != P2S_OK) return st;
    FieldGeom g;
    if ((st = geometry(ctx, H, W, &g)) != P2S_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    for (int i0 = 0; i0 < n; i0 += kMaxBatch) {
        const int nb = n - i0 < kMaxBatch ? n - i0 : kMaxBatch;
        FrameBatch fb;
        fill_batch(&fb, nb, d_over_r0 + i0, seeds + i0);
        void *scratch = nullptr;
        P2S_CUDA(cudaMallocAsync(&scratch, fields_scratch_bytes(g, nb), s));
        st = launch_fields(ctx, g, fb, alpha + (size_t)i0 * g.Ah * g.Aw * kAlphaStride, scratch, s);
        cudaFreeAsync(scratch, s);
        if (st != P2S_OK) return st;
    }
    return P2S_OK;
}

static p2s_status check_image(const p2s_image *im, const char *what) {
    if (!im || !im->data) {
        set_error("%s: NULL image or data", what);
        return P2S_EINVAL;
    }
    if (im->H < 1 || im->W < 1 || !(im->C == 1 || im->C == 3)) {
        set_error("%s: need H, W >= 1 and C in {1, 3}", what);
        return P2S_EINVAL;
    }
    return P2S_OK;
}

static bool same_shape(const p2s_image *a, const p2s_image *b) { return a->H == b->H && a->W == b->W && a->C == b->C; }

p2s_status p2s_stage_warp(p2s_ctx *ctx, const p2s_image *in, const float *alpha, const p2s_image *out, void *stream) {
    if (!ctx || !alpha) return einval("ctx and alpha must be non-NULL");
    p2s_status st;
    if ((st = check_image(in, "in")) != P2S_OK || (st = check_image(out, "out")) != P2S_OK) return st;
    if (!same_shape(in, out)) return einval("in and out shapes differ");
    if (in->data == out->data) return einval("out must not alias in");
    FieldGeom g;
    if ((st = geometry(ctx, in->H, in->W, &g)) != P2S_OK) return st;
    const float *ip[1] = {in->data};
    float *op[1] = {out->data};
    return launch_warp(ctx, g, 1, ip, alpha, op, in->C, (cudaStream_t)stream);
}

p2s_status p2s_stage_mlp(p2s_ctx *ctx, int H, int W, const float *alpha, float *beta, void *stream) {
    if (!ctx || !alpha || !beta) return einval("ctx, alpha and beta must be non-NULL");
    FieldGeom g;
    p2s_status st = geometry(ctx, H, W, &g);
    if (st != P2S_OK) return st;
    if (tc_precision(ctx->prec)) {
        const TcFrame f{nullptr, nullptr, alpha, H, W, g.Ah, g.Aw, 0, 0, 0};
        return launch_tc(ctx, kTcMlpOnly, &f, 1, 1, nullptr, beta, ctx->d_status, (cudaStream_t)stream);
    }
    return launch_mlp_simt(ctx, g, 1, alpha, beta, (cudaStream_t)stream);
}
p2s_status p2s_set_option(p2s_ctx *ctx, int option, int value) {
    if (!ctx) return einval("ctx must be non-NULL");
    if (option == P2S_OPT_SCATTER_SEGMENT_ROWS) {
        if (value != 0 && (value < 2 || (value & 1))) return einval("segment rows must be 0 or an even number >= 2");
        ctx->tc.seg_rows = value;
        return P2S_OK;
    }
    if (option == P2S_OPT_GRAPHS) {
        if (value != 0 && value != 1) return einval("graphs option is 0 or 1");
        ctx->use_graphs = value;
        return P2S_OK;
    }
    if (option == P2S_OPT_GATHER_BAND_ROWS) {
        if (value != 0 && value != 16 && value != 32) return einval("band rows must be 0, 16 or 32");
        ctx->tc.band_rows = value;
        return P2S_OK;
    }
    if (option == P2S_OPT_BLUR_THEN_WARP) {
        if (value != 0 && value != 1) return einval("blur-then-warp option is 0 or 1");
        ctx->blur_then_warp = value;
        return P2S_OK;
    }
    if (option == P2S_OPT_FIELD_METHOD) {
        if (value != 0 && value != 1) return einval("field method is 0 (Fourier filtering) or 1 (dense draw)");
        ctx->field_method = value;
        return P2S_OK;
    }
    if (option == P2S_OPT_GATHER_SPLIT) {
        if (value < 0 || value > 4)
            return einval("gather split is 0 (fused) or 1 .. 4 (network, then one of four blur kernels)");
        if (ctx->prec == P2S_FP8E4M3 && value != 1) {
            set_error("the FP8 E4M3 contraction runs in the split gather kernel 1 only");
            return P2S_EUNSUPPORTED;
        }
        ctx->gather_split = value;
        return P2S_OK;
    }
    return einval("unknown option");
}
p2s_status p2s_get_option(const p2s_ctx *ctx, int option, int *value) {
    if (!ctx || !value) return einval("ctx and value must be non-NULL");
    if (option == P2S_OPT_SCATTER_SEGMENT_ROWS) {
        *value = ctx->tc.seg_rows;
        return P2S_OK;
    }
    if (option == P2S_OPT_GRAPHS) {
        *value = ctx->use_graphs;
        return P2S_OK;
    }
    if (option == P2S_OPT_GRAPH_INSTANTIATIONS) {
        *value = (int)ctx->graph_instantiations;
        return P2S_OK;
    }
    if (option == P2S_OPT_GRAPH_UPDATES) {
        *value = (int)ctx->graph_updates;
        return P2S_OK;
    }
    if (option == P2S_OPT_GATHER_BAND_ROWS) {
        *value = ctx->tc.band_rows;
        return P2S_OK;
    }
    if (option == P2S_OPT_BLUR_THEN_WARP) {
        *value = ctx->blur_then_warp;
        return P2S_OK;
    }
    if (option == P2S_OPT_FIELD_METHOD) {
        *value = ctx->field_method;
        return P2S_OK;
    }
    if (option == P2S_OPT_GATHER_SPLIT) {
        *value = ctx->gather_split;
        return P2S_OK;
    }
    return einval("unknown option");
}
p2s_status p2s_stage_mlp16(p2s_ctx *ctx, int H, int W, const float *alpha, void *beta16, void *stream) {
    if (!ctx || !alpha || !beta16) return einval("ctx, alpha and beta16 must be non-NULL");
    if (!(ctx->prec == P2S_BF16 || ctx->prec == P2S_FP16)) {
        set_error("the 16-bit operand layout exists for FP16 and BF16 contexts only");
        return P2S_EUNSUPPORTED;
    }
    FieldGeom g;
    p2s_status st = geometry(ctx, H, W, &g);
    if (st != P2S_OK) return st;
    return launch_net16(ctx, g, 1, alpha, beta16, 1, 0, ctx->d_status, (cudaStream_t)stream);
}

p2s_status p2s_contraction_scales(p2s_ctx *ctx, float *scale, int n, float *inv_c) {
    if (!ctx || !scale || !inv_c) return einval("ctx, scale and inv_c must be non-NULL");
    if (ctx->prec != P2S_FP8E4M3) {
        set_error("contraction scales exist for FP8 E4M3 contexts only");
        return P2S_EUNSUPPORTED;
    }
    if (n < ctx->K + 2) return einval("scale needs K + 2 entries");
    p2s_status st = tc_prepare(ctx);
    if (st != P2S_OK) return st;
    P2S_CUDA(cudaMemcpy(scale, ctx->tc.d_scale8, (size_t)(ctx->K + 2) * sizeof(float), cudaMemcpyDeviceToHost));
    *inv_c = ctx->tc.inv_c8;
    return P2S_OK;
}

p2s_status p2s_stage_blur(p2s_ctx *ctx, const p2s_image *xw, const float *beta, const p2s_image *out, void *stream) {
    if (!ctx || !beta) return einval("ctx and beta must be non-NULL");
    p2s_status st;
    if ((st = check_image(xw, "xw")) != P2S_OK || (st = check_image(out, "out")) != P2S_OK) return st;
    if (!same_shape(xw, out)) return einval("xw and out shapes differ");
    if (xw->data == out->data) return einval("out must not alias xw");
    const float *ip[1] = {xw->data};
    float *op[1] = {out->data};
    if (ctx->prec == P2S_FP8E4M3) {
        // the FP8 layout (beta times the per-basis scales, E4M3 hi/lo), then the split gather
        FieldGeom g;
        if ((st = geometry(ctx, xw->H, xw->W, &g)) != P2S_OK) return st;
        const TcFrame f{xw->data, out->data, nullptr, xw->H, xw->W, g.Ah, g.Aw, 0, 0, 0};
        cudaStream_t s = (cudaStream_t)stream;
        void *b8 = nullptr;
        P2S_CUDA(cudaMallocAsync(&b8, beta8_bytes(xw->H, xw->W, 1), s));
        st = launch_pack8(ctx, xw->H, xw->W, 1, beta, b8, s);
        const void *bp[1] = {b8};
        if (st == P2S_OK) st = launch_gather_split(ctx, &f, bp, 1, xw->C, ctx->d_status, s);
        cudaFreeAsync(b8, s);
        return st;
    }
    if ((ctx->prec == P2S_BF16 || ctx->prec == P2S_FP16) && ctx->form == P2S_SCATTER) {
        cudaStream_t s = (cudaStream_t)stream;
        void *b16 = nullptr;
        P2S_CUDA(cudaMallocAsync(&b16, beta16_bytes(xw->H, xw->W, 1, 0), s));
        st = launch_pack16(ctx, xw->H, xw->W, 1, beta, b16, 0, s);
        if (st == P2S_OK) st = launch_scatter_tc(ctx, xw->H, xw->W, xw->C, 1, ip, op, b16, ctx->d_status, s);
        cudaFreeAsync(b16, s);
        return st;
    }
    if (ctx->prec == P2S_BF16 || ctx->prec == P2S_FP16) {
        FieldGeom g;
        if ((st = geometry(ctx, xw->H, xw->W, &g)) != P2S_OK) return st;
        const TcFrame f{xw->data, out->data, nullptr, xw->H, xw->W, g.Ah, g.Aw, 0, 0, 0};
        if (ctx->gather_split) {
            // the kernel p2s_simulate runs: beta in the 16-bit operand layout (its k >= K
            // entries 0, so the folded bias rows add nothing: beta here includes the bias)
            cudaStream_t s = (cudaStream_t)stream;
            void *b16 = nullptr;
            const int perm = gather_perm(ctx->gather_split);
            P2S_CUDA(cudaMallocAsync(&b16, beta16_bytes(xw->H, xw->W, 1, perm), s));
            st = launch_pack16(ctx, xw->H, xw->W, 1, beta, b16, perm, s);
            const void *bp[1] = {b16};
            if (st == P2S_OK) st = launch_gather_blur(ctx, ctx->gather_split, &f, bp, 1, xw->C, ctx->d_status, s);
            cudaFreeAsync(b16, s);
            return st;
        }
        return launch_tc(ctx, kTcBlurOnly, &f, 1, xw->C, beta, nullptr, ctx->d_status, (cudaStream_t)stream);
    }
    if (ctx->form == P2S_FFT) return launch_blur_fft(ctx, xw->H, xw->W, xw->C, 1, ip, beta, op, (cudaStream_t)stream);
    return launch_blur_simt(ctx, xw->H, xw->W, xw->C, 1, ip, beta, op, ctx->form, (cudaStream_t)stream);
}

// ---- the whole path --------------------------------------------------------

// Per-call device scratch: stream-ordered allocations, or (graph capture)
// slices of the context's arena.  In arena mode a request that does not fit
// is counted in `needed` and served from the arena base so that the capture
// can finish; the caller then grows the arena and captures again.
struct Scratch {
    p2s_ctx *ctx;
    cudaStream_t s;
    bool arena;
    size_t used = 0, needed = 0;
    bool overflow = false;
    std::vector<void *> blocks;
    void *get(size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        if (arena) {
            needed = std::max(needed, used + bytes);
            if (used + bytes > ctx->arena_bytes) {
                // sizing pass: the capture that gets this address is discarded, never launched
                overflow = true;
                used += bytes;
                return ctx->arena ? ctx->arena : (void *)(uintptr_t)4096;
            }
            void *p = (char *)ctx->arena + used;
            used += bytes;
            return p;
        }
        void *p = nullptr;
        if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) return nullptr;
        blocks.push_back(p);
        return p;
    }
    size_t mark() const { return used; }
    // everything obtained after `m` is dead once the stream reaches this point
    void rewind(size_t m) {
        if (arena) {
            used = m;
        } else {
            for (void *b : blocks) cudaFreeAsync(b, s);
            blocks.clear();
        }
    }
    void release() { rewind(0); }
};


static p2s_status simulate_group(p2s_ctx *ctx, const p2s_image *frames, const p2s_image *out, const int *idx, int n,
                                 const float *d_over_r0, const unsigned long long *seeds, cudaStream_t s,
                                 Scratch &sc) {
    const int H = frames[idx[0]].H, W = frames[idx[0]].W, C = frames[idx[0]].C;
    FieldGeom g;
    p2s_status st = geometry(ctx, H, W, &g);
    if (st != P2S_OK) return st;
    const size_t npx = (size_t)H * W;
    const bool tc = ctx->prec == P2S_BF16 || ctx->prec == P2S_FP16;
    // bound the FP32 path's beta scratch to ~1 GiB per launch group
    int chunk = kMaxBatch;
    const bool tc_scatter = tc && ctx->form == P2S_SCATTER;
    const size_t beta_px = tc_scatter ? beta16_bytes(H, W, 1, 0) : tc ? 0 : npx * ctx->K * sizeof(float);
    const size_t beta_cap = tc_scatter ? (4ull << 30) : (1ull << 30);
    while (chunk > 1 && (size_t)chunk * beta_px > beta_cap) chunk /= 2;
    for (int i0 = 0; i0 < n; i0 += chunk) {
        const int nb = n - i0 < chunk ? n - i0 : chunk;
        FrameBatch fb;
        float dr[kMaxBatch];
        unsigned long long sd[kMaxBatch];
        const float *ip[kMaxBatch];
        float *op[kMaxBatch];
        for (int i = 0; i < nb; ++i) {
            const int f = idx[i0 + i];
            dr[i] = d_over_r0[f];
            sd[i] = seeds[f];
            ip[i] = frames[f].data;
            op[i] = out[f].data;
        }
        fill_batch(&fb, nb, dr, sd);
        const size_t a_bytes = (size_t)nb * g.Ah * g.Aw * kAlphaStride * sizeof(float);
        const size_t f_bytes = fields_scratch_bytes(g, nb);
        const size_t xw_bytes = (size_t)nb * npx * C * sizeof(float);
        const size_t b_bytes = (size_t)nb * beta_px;
        const size_t m0 = sc.mark();
        char *scratch = (char *)sc.get(a_bytes + f_bytes + xw_bytes + b_bytes + 1024);
        if (!scratch) {
            set_error("device allocation failed for per-call scratch");
            return P2S_ENOMEM;
        }
        float *alpha = (float *)scratch;
        void *fscr = scratch + ((a_bytes + 255) & ~(size_t)255);
        float *xw = (float *)((char *)fscr + ((f_bytes + 255) & ~(size_t)255));
        float *beta = (float *)((char *)xw + ((xw_bytes + 255) & ~(size_t)255));
        const float *xwp[kMaxBatch];
        float *xwm[kMaxBatch];
        for (int i = 0; i < nb; ++i) {
            xwm[i] = xw + (size_t)i * npx * C;
            xwp[i] = xwm[i];
        }
        st = launch_fields(ctx, g, fb, alpha, fscr, s);
        // warp then blur (default), or blur the input then warp the result (Sec. 2.2 order);
        // in the second case the x_w buffer holds the blurred, not yet warped frames
        const bool bw = ctx->blur_then_warp;
        float *blur_out[kMaxBatch];
        for (int i = 0; i < nb; ++i) {
            blur_out[i] = bw ? xwm[i] : op[i];
            if (bw) xwp[i] = ip[i];
        }
        if (st == P2S_OK && !bw) st = launch_warp(ctx, g, nb, ip, alpha, xwm, C, s);
        float *const *bop = blur_out;
        if (tc && ctx->form == P2S_SCATTER) {
            if (st == P2S_OK) st = launch_net16(ctx, g, nb, alpha, beta, 1, 0, ctx->d_status, s);
            if (st == P2S_OK) st = launch_scatter_tc(ctx, H, W, C, nb, xwp, bop, beta, ctx->d_status, s);
        } else {
            if (st == P2S_OK) st = launch_mlp_simt(ctx, g, nb, alpha, beta, s);
            if (st == P2S_OK)
                st = ctx->form == P2S_FFT ? launch_blur_fft(ctx, H, W, C, nb, xwp, beta, bop, s)
                                          : launch_blur_simt(ctx, H, W, C, nb, xwp, beta, bop, ctx->form, s);
        }
        if (st == P2S_OK && bw) {
            const float *bin[kMaxBatch];
            for (int i = 0; i < nb; ++i) bin[i] = xwm[i];
            st = launch_warp(ctx, g, nb, bin, alpha, op, C, s);
        }
        sc.rewind(m0);
        if (st != P2S_OK) return st;
    }
    return P2S_OK;
}

// The host entry point's schedule for the gather form (warp then blur): frames
// [bounds[k], bounds[k + 1]) form chunk k, whose inputs are on the device once
// in_ready[k] completes; out_done[k] is recorded once its outputs are written.
// The fields and the network, which read no input pixels, run first over all
// frames; then each chunk's warp and blur, alternating between the call's stream
// and `aux` (if set).
// issue_inputs (if set) queues the input copies and records in_ready[]; it is called once
// the fields and the network are queued, so that their launches do not wait behind the
// copies' host-side submission.
struct Pipeline {
    int nch;
    const int *bounds;
    const cudaEvent_t *in_ready;
    const cudaEvent_t *out_done;
    cudaStream_t aux;
    cudaEvent_t prefix_done, aux_done;
    std::function<p2s_status()> issue_inputs;
};

// Tensor-core path: the fields once per filter torus, the warp and the network
// over frames of any sizes (up to kMaxBatch per launch), then the blur: for the
// gather form ONE persistent launch over every frame of the call (per channel
// count), work ordered frame by frame, tile by tile; for the scatter form one
// launch per channel count and kMaxBatch frames of any sizes.  With a Pipeline
// (gather form, warp then blur) the warp and the blur go chunk by chunk instead.
static p2s_status simulate_tc(p2s_ctx *ctx, const p2s_image *frames, const p2s_image *out, int n,
                              const float *d_over_r0, const unsigned long long *seeds, cudaStream_t s, Scratch &sc,
                              const Pipeline *pl = nullptr) {
    std::vector<TcFrame> tf[2];      // C = 1, C = 3
    std::vector<const void *> b16[2];  // split form: each frame's beta16
    std::vector<int> tf_idx[2];        // each entry's frame index in the call
    const bool scat = ctx->form == P2S_SCATTER;
    const bool split = scat || ctx->gather_split != 0;
    const int perm = scat ? 0 : gather_perm(ctx->gather_split);  // the fragment kernels' beta layout
    const bool f8 = ctx->prec == P2S_FP8E4M3;          // split kernel 1 with the FP8 layout
    struct PostWarp {
        FieldGeom g;
        int C;
        const float *in;
        const float *alpha;
        float *out;
    };
    std::vector<PostWarp> post_warp;
    // one launch batch of frames of one shape: its buffers, for the stages after the fields
    struct ShapeBatch {
        FieldGeom g;
        int C, nb;
        FrameBatch fb;
        float *alpha;
        void *fscratch;
        const float *ip[kMaxBatch];
        float *xwm[kMaxBatch];
        float *op[kMaxBatch];
        int fidx[kMaxBatch];
        char *b16buf;
        bool fields_done;
    };
    std::vector<ShapeBatch> batches;
    std::vector<char> done(n, 0);
    std::vector<int> idx;
    p2s_status st = P2S_OK;
    for (int i = 0; i < n && st == P2S_OK; ++i) {
        if (done[i]) continue;
        idx.clear();
        for (int j = i; j < n; ++j)
            if (!done[j] && same_shape(&frames[i], &frames[j])) {
                idx.push_back(j);
                done[j] = 1;
            }
        const int H = frames[i].H, W = frames[i].W, C = frames[i].C;
        FieldGeom g;
        if ((st = geometry(ctx, H, W, &g)) != P2S_OK) break;
        const size_t npx = (size_t)H * W;
        for (size_t i0 = 0; i0 < idx.size() && st == P2S_OK; i0 += kMaxBatch) {
            const int nb = (int)std::min<size_t>(kMaxBatch, idx.size() - i0);
            FrameBatch fb;
            float dr[kMaxBatch];
            unsigned long long sd[kMaxBatch];
            const float *ip[kMaxBatch];
            float *xwm[kMaxBatch];
            for (int k = 0; k < nb; ++k) {
                dr[k] = d_over_r0[idx[i0 + k]];
                sd[k] = seeds[idx[i0 + k]];
                ip[k] = frames[idx[i0 + k]].data;
            }
            fill_batch(&fb, nb, dr, sd);
            const size_t a_bytes = ((size_t)nb * g.Ah * g.Aw * kAlphaStride * sizeof(float) + 255) & ~(size_t)255;
            const size_t f_bytes = (fields_scratch_bytes(g, nb) + 255) & ~(size_t)255;
            const size_t xw_bytes = ((size_t)nb * npx * C * sizeof(float) + 255) & ~(size_t)255;
            const size_t b_bytes = f8 ? beta8_bytes(H, W, nb) : split ? beta16_bytes(H, W, nb, perm) : 0;
            char *buf = (char *)sc.get(a_bytes + f_bytes + xw_bytes + b_bytes);
            if (!buf) {
                set_error("device allocation failed for per-call scratch");
                st = P2S_ENOMEM;
                break;
            }
            float *alpha = (float *)buf;
            float *xw = (float *)(buf + a_bytes + f_bytes);
            for (int k = 0; k < nb; ++k) xwm[k] = xw + (size_t)k * npx * C;
            const bool bw = ctx->blur_then_warp;
            char *b16buf = buf + a_bytes + f_bytes + xw_bytes;
            ShapeBatch sbt;
            sbt.g = g;
            sbt.C = C;
            sbt.nb = nb;
            sbt.fb = fb;
            sbt.alpha = alpha;
            sbt.fscratch = buf + a_bytes;
            sbt.b16buf = b16buf;
            sbt.fields_done = false;
            for (int k = 0; k < nb; ++k) {
                sbt.ip[k] = ip[k];
                sbt.xwm[k] = xwm[k];
                sbt.op[k] = out[idx[i0 + k]].data;
                sbt.fidx[k] = idx[i0 + k];
            }
            batches.push_back(sbt);
            for (int k = 0; k < nb; ++k) {
                const int f = idx[i0 + k];
                const float *a_k = alpha + (size_t)k * g.Ah * g.Aw * kAlphaStride;
                // blur-then-warp: the fused launch blurs the input into x_w, a warp follows
                tf[C == 3 ? 1 : 0].push_back(
                    TcFrame{bw ? ip[k] : xwm[k], bw ? xwm[k] : out[f].data, a_k, H, W, g.Ah, g.Aw, 0, 0, 0});
                tf_idx[C == 3 ? 1 : 0].push_back(f);
                if (bw) post_warp.push_back(PostWarp{g, C, xwm[k], a_k, out[f].data});
                if (split) b16[C == 3 ? 1 : 0].push_back(b16buf + (size_t)k * (f8 ? beta8_bytes(H, W, 1) : beta16_bytes(H, W, 1, perm)));
            }
        }
    }
    // ---- fields: frames of one torus in one launch, whatever their anchor grids ----
    for (size_t b0 = 0; b0 < batches.size() && st == P2S_OK; ++b0) {
        if (batches[b0].fields_done) continue;
        const int Fh = batches[b0].g.Fh, Fw = batches[b0].g.Fw;
        int ah_max = 0, aw_max = 0;
        std::vector<size_t> same;
        for (size_t b = b0; b < batches.size(); ++b)
            if (!batches[b].fields_done && batches[b].g.Fh == Fh && batches[b].g.Fw == Fw) {
                same.push_back(b);
                ah_max = std::max(ah_max, batches[b].g.Ah);
                aw_max = std::max(aw_max, batches[b].g.Aw);
            }
        if (same.size() > 1 && fields_group_ok(ctx, Fh, Fw, ah_max, aw_max)) {
            FrameBatch fb;
            FieldFrames geo;
            fb.n = 0;
            for (size_t b : same) {
                ShapeBatch &sb = batches[b];
                const FieldGeom &g = sb.g;
                // the field block follows the row-pass scratch, as launch_fields lays it out
                const size_t t_bytes = (size_t)sb.nb * kModes * g.Fh * g.Aw * sizeof(float);
                float *f = (float *)((char *)sb.fscratch + ((t_bytes + 255) & ~(size_t)255));
                for (int k = 0; k < sb.nb && st == P2S_OK; ++k) {
                    fb.seed[fb.n] = sb.fb.seed[k];
                    fb.scale[fb.n] = sb.fb.scale[k];
                    geo.ah[fb.n] = g.Ah;
                    geo.aw[fb.n] = g.Aw;
                    geo.f[fb.n] = f + (size_t)k * kModes * g.Ah * g.Aw;
                    geo.alpha[fb.n] = sb.alpha + (size_t)k * g.Ah * g.Aw * kAlphaStride;
                    if (++fb.n == kMaxBatch) {
                        st = launch_fields_group(ctx, Fh, Fw, fb, geo, s);
                        fb.n = 0;
                    }
                }
                sb.fields_done = true;
            }
            if (st == P2S_OK && fb.n > 0) st = launch_fields_group(ctx, Fh, Fw, fb, geo, s);
        } else {
            ShapeBatch &sb = batches[b0];
            st = launch_fields(ctx, sb.g, sb.fb, sb.alpha, sb.fscratch, s);
            sb.fields_done = true;
        }
    }
    // ---- warp (per channel count) and network: up to kMaxBatch frames of any shapes per launch ----
    {
        std::vector<WarpFrame> wf[2];
        std::vector<NetFrame> nf;
        for (const ShapeBatch &sb : batches) {
            const FieldGeom &g = sb.g;
            const size_t fbytes = f8 ? beta8_bytes(g.H, g.W, 1) : beta16_bytes(g.H, g.W, 1, perm);
            for (int k = 0; k < sb.nb; ++k) {
                const float *a_k = sb.alpha + (size_t)k * g.Ah * g.Aw * kAlphaStride;
                wf[sb.C == 3 ? 1 : 0].push_back(WarpFrame{sb.ip[k], sb.xwm[k], a_k, g.H, g.W});
                nf.push_back(NetFrame{a_k, sb.b16buf + (size_t)k * fbytes, g.H, g.W});
            }
        }
        for (int ci = 1; ci >= 0 && !ctx->blur_then_warp && !pl; --ci)
            for (size_t i0 = 0; i0 < wf[ci].size() && st == P2S_OK; i0 += kMaxBatch)
                st = launch_warp_frames(ctx, wf[ci].data() + i0, (int)std::min<size_t>(kMaxBatch, wf[ci].size() - i0),
                                        ci ? 3 : 1, s);
        for (size_t i0 = 0; split && i0 < nf.size() && st == P2S_OK; i0 += kMaxBatch)
            st = launch_net16_frames(ctx, nf.data() + i0, (int)std::min<size_t>(kMaxBatch, nf.size() - i0), 1, perm,
                                     ctx->d_status, s);
    }
    if (pl && st == P2S_OK) {
        // chunk by chunk: the chunk's inputs, its warp, its blur (the fields and the network
        // of every frame are queued above on s)
        P2S_CUDA(cudaEventRecord(pl->prefix_done, s));
        if (pl->issue_inputs) st = pl->issue_inputs();
        bool used_aux = false;
        for (int k = 0; k < pl->nch && st == P2S_OK; ++k) {
            const int i0 = pl->bounds[k], i1 = pl->bounds[k + 1];
            cudaStream_t cs = (pl->aux && (k & 1)) ? pl->aux : s;
            if (cs != s) {
                P2S_CUDA(cudaStreamWaitEvent(cs, pl->prefix_done, 0));
                used_aux = true;
            }
            P2S_CUDA(cudaStreamWaitEvent(cs, pl->in_ready[k], 0));
            std::vector<WarpFrame> wk;
            for (int ci = 1; ci >= 0 && st == P2S_OK; --ci) {
                wk.clear();
                for (const ShapeBatch &sb : batches) {
                    if (sb.C != (ci ? 3 : 1)) continue;
                    for (int j = 0; j < sb.nb; ++j)
                        if (sb.fidx[j] >= i0 && sb.fidx[j] < i1)
                            wk.push_back(WarpFrame{sb.ip[j], sb.xwm[j],
                                                   sb.alpha + (size_t)j * sb.g.Ah * sb.g.Aw * kAlphaStride, sb.g.H,
                                                   sb.g.W});
                }
                for (size_t w0 = 0; w0 < wk.size() && st == P2S_OK; w0 += kMaxBatch)
                    st = launch_warp_frames(ctx, wk.data() + w0, (int)std::min<size_t>(kMaxBatch, wk.size() - w0),
                                            ci ? 3 : 1, cs);
            }
            for (int ci = 1; ci >= 0 && st == P2S_OK; --ci) {
                std::vector<TcFrame> tk;
                std::vector<const void *> bk;
                for (size_t q = 0; q < tf[ci].size(); ++q)
                    if (tf_idx[ci][q] >= i0 && tf_idx[ci][q] < i1) {
                        tk.push_back(tf[ci][q]);
                        if (split) bk.push_back(b16[ci][q]);
                    }
                if (tk.empty()) continue;
                const int C = ci ? 3 : 1;
                st = split ? launch_gather_blur(ctx, ctx->gather_split, tk.data(), bk.data(), (int)tk.size(), C,
                                                ctx->d_status, cs)
                           : launch_tc(ctx, kTcFull, tk.data(), (int)tk.size(), C, nullptr, nullptr, ctx->d_status, cs);
            }
            if (st == P2S_OK) P2S_CUDA(cudaEventRecord(pl->out_done[k], cs));
        }
        // scratch is released on s: after the other stream's chunks
        if (used_aux) {
            cudaEventRecord(pl->aux_done, pl->aux);
            cudaStreamWaitEvent(s, pl->aux_done, 0);
        }
        sc.release();
        return st;
    }
    // scatter: one launch per channel count and kMaxBatch frames of any sizes (blur-then-warp:
    // the input blurred into x_w)
    if (scat) {
        std::vector<ScatterFrame> sf[2];
        for (const ShapeBatch &sb : batches) {
            const size_t fbytes = beta16_bytes(sb.g.H, sb.g.W, 1, 0);
            for (int k = 0; k < sb.nb; ++k)
                sf[sb.C == 3 ? 1 : 0].push_back(ScatterFrame{ctx->blur_then_warp ? sb.ip[k] : sb.xwm[k],
                                                             ctx->blur_then_warp ? sb.xwm[k] : sb.op[k],
                                                             sb.b16buf + (size_t)k * fbytes, sb.g.H, sb.g.W});
        }
        for (int ci = 1; ci >= 0; --ci)
            for (size_t i0 = 0; i0 < sf[ci].size() && st == P2S_OK; i0 += kMaxBatch)
                st = launch_scatter_frames(ctx, sf[ci].data() + i0, (int)std::min<size_t>(kMaxBatch, sf[ci].size() - i0),
                                           ci ? 3 : 1, ctx->d_status, s);
    }
    for (int ci = 1; ci >= 0 && st == P2S_OK && !scat; --ci) {
        if (tf[ci].empty()) continue;
        const int C = ci ? 3 : 1;
        st = split ? launch_gather_blur(ctx, ctx->gather_split, tf[ci].data(), b16[ci].data(), (int)tf[ci].size(), C,
                                        ctx->d_status, s)
                   : launch_tc(ctx, kTcFull, tf[ci].data(), (int)tf[ci].size(), C, nullptr, nullptr, ctx->d_status, s);
    }
    // blur-then-warp: the blurred frames warped into the outputs, kMaxBatch frames of any
    // sizes per launch and channel count
    {
        std::vector<WarpFrame> pw[2];
        for (const PostWarp &w : post_warp) pw[w.C == 3 ? 1 : 0].push_back(WarpFrame{w.in, w.out, w.alpha, w.g.H, w.g.W});
        for (int ci = 1; ci >= 0; --ci)
            for (size_t i0 = 0; i0 < pw[ci].size() && st == P2S_OK; i0 += kMaxBatch)
                st = launch_warp_frames(ctx, pw[ci].data() + i0, (int)std::min<size_t>(kMaxBatch, pw[ci].size() - i0),
                                        ci ? 3 : 1, s);
    }
    sc.release();
    return st;
}

static p2s_status validate_simulate(p2s_ctx *ctx, const p2s_image *frames, int n, const float *d_over_r0,
                                    const unsigned long long *seeds, const p2s_image *out) {
    if (!ctx) return einval("ctx is NULL");
    p2s_status st = check_frames_meta(n, d_over_r0, seeds);
    if (st != P2S_OK) return st;
    if (n > 0 && (!frames || !out)) return einval("frames and out must be non-NULL");
    for (int i = 0; i < n; ++i) {
        if ((st = check_image(&frames[i], "frames[i]")) != P2S_OK || (st = check_image(&out[i], "out[i]")) != P2S_OK)
            return st;
        if (!same_shape(&frames[i], &out[i])) return einval("frames[i] and out[i] shapes differ");
        if (frames[i].data == out[i].data) return einval("out[i] must not alias frames[i]");
        FieldGeom g;
        if ((st = geometry(ctx, frames[i].H, frames[i].W, &g)) != P2S_OK) return st;
    }
    return P2S_OK;
}

static p2s_status simulate_impl(p2s_ctx *ctx, const p2s_image *frames, int n, const float *d_over_r0,
                                const unsigned long long *seeds, const p2s_image *out, cudaStream_t s, Scratch &sc) {
    if (tc_precision(ctx->prec) && ctx->form == P2S_GATHER) return simulate_tc(ctx, frames, out, n, d_over_r0, seeds, s, sc);
    if (tc_precision(ctx->prec) && ctx->form == P2S_SCATTER) {
        // the path holds every frame's 16-bit beta at once: runs of frames with at most
        // 4 GiB of it (at least one frame each)
        const size_t cap = 4ull << 30;
        for (int i0 = 0; i0 < n;) {
            size_t bytes = 0;
            int i1 = i0;
            while (i1 < n) {
                const size_t b = beta16_bytes(frames[i1].H, frames[i1].W, 1, 0);
                if (i1 > i0 && bytes + b > cap) break;
                bytes += b;
                ++i1;
            }
            p2s_status st = simulate_tc(ctx, frames + i0, out + i0, i1 - i0, d_over_r0 + i0, seeds + i0, s, sc);
            if (st != P2S_OK) return st;
            i0 = i1;
        }
        return P2S_OK;
    }
    // group frames of one shape, in order of first appearance
    std::vector<char> done(n, 0);
    std::vector<int> idx;
    for (int i = 0; i < n; ++i) {
        if (done[i]) continue;
        idx.clear();
        for (int j = i; j < n; ++j)
            if (!done[j] && same_shape(&frames[i], &frames[j])) {
                idx.push_back(j);
                done[j] = 1;
            }
        p2s_status st = simulate_group(ctx, frames, out, idx.data(), (int)idx.size(), d_over_r0, seeds, s, sc);
        if (st != P2S_OK) return st;
    }
    return P2S_OK;
}

// One-time device preparation that must not happen inside a stream capture.
static p2s_status prepare_for_capture(p2s_ctx *ctx) {
    if (tc_precision(ctx->prec)) {
        p2s_status st = tc_prepare(ctx);
        if (st != P2S_OK) return st;
        if (ctx->form == P2S_SCATTER && (st = scatter_prepare(ctx)) != P2S_OK) return st;
    }
    if (!ctx->cap_stream) {
        P2S_CUDA(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        P2S_CUDA(cudaEventCreateWithFlags(&ctx->cap_ev[0], cudaEventDisableTiming));
        P2S_CUDA(cudaEventCreateWithFlags(&ctx->cap_ev[1], cudaEventDisableTiming));
    }
    return P2S_OK;
}

// p2s_simulate as a CUDA graph: the call's launches are captured on the
// context's stream (ordered after the caller's stream by an event), the
// graph is instantiated once per batch signature and later only updated
// with the new arguments (pointers, seeds, strengths), then launched.
static p2s_status simulate_graph(p2s_ctx *ctx, const p2s_image *frames, int n, const float *d_over_r0,
                                 const unsigned long long *seeds, const p2s_image *out, cudaStream_t user) {
    p2s_status st = prepare_for_capture(ctx);
    if (st != P2S_OK) return st;
    // field filter tables of every torus size in the call (built with synchronous copies)
    for (int i = 0; i < n; ++i) {
        FieldGeom g;
        const FilterTable *t;
        if ((st = geometry(ctx, frames[i].H, frames[i].W, &g)) != P2S_OK) return st;
        if ((st = filter_table(ctx, g.Fh, &t)) != P2S_OK || (st = filter_table(ctx, g.Fw, &t)) != P2S_OK) return st;
        if (ctx->field_method == 1 && (st = dense_prepare(ctx, g)) != P2S_OK) return st;
    }
    std::string key;
    for (int i = 0; i < n; ++i) {
        char b[48];
        std::snprintf(b, sizeof b, "%dx%dx%d;", frames[i].H, frames[i].W, frames[i].C);
        key += b;
    }
    cudaStream_t s = ctx->cap_stream;
    for (int attempt = 0; attempt < 2; ++attempt) {
        Scratch sc{ctx, s, true};
        P2S_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        st = simulate_impl(ctx, frames, n, d_over_r0, seeds, out, s, sc);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (st == P2S_OK && ce != cudaSuccess) {
            set_error("stream capture failed: %s", cudaGetErrorString(ce));
            st = P2S_ECUDA;
        }
        if (st == P2S_OK && sc.overflow) {
            cudaGraphDestroy(graph);
            P2S_CUDA(cudaStreamSynchronize(s));
            cudaFree(ctx->arena);
            ctx->arena = nullptr;
            ctx->arena_bytes = 0;
            const size_t want = sc.needed + sc.needed / 8;
            if (cudaMalloc(&ctx->arena, want) != cudaSuccess) {
                set_error("device allocation of %zu bytes failed for the graph arena", want);
                return P2S_ENOMEM;
            }
            ctx->arena_bytes = want;
            continue;
        }
        if (st != P2S_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        cudaGraphExec_t &exec = ctx->graphs[key];
        bool ok = false;
        if (exec) {
            cudaGraphExecUpdateResultInfo info;
            ok = cudaGraphExecUpdate(exec, graph, &info) == cudaSuccess;
            if (ok) {
                ++ctx->graph_updates;
            } else {
                cudaGetLastError();
                cudaGraphExecDestroy(exec);
                exec = nullptr;
            }
        }
        if (!ok) {
            const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
            if (ie != cudaSuccess) {
                cudaGraphDestroy(graph);
                exec = nullptr;
                set_error("graph instantiation failed: %s", cudaGetErrorString(ie));
                return P2S_ECUDA;
            }
            ++ctx->graph_instantiations;
        }
        cudaGraphDestroy(graph);
        P2S_CUDA(cudaEventRecord(ctx->cap_ev[0], user));
        P2S_CUDA(cudaStreamWaitEvent(s, ctx->cap_ev[0], 0));
        P2S_CUDA(cudaGraphLaunch(exec, s));
        P2S_CUDA(cudaEventRecord(ctx->cap_ev[1], s));
        P2S_CUDA(cudaStreamWaitEvent(user, ctx->cap_ev[1], 0));
        return P2S_OK;
    }
    set_error("graph arena could not be sized");
    return P2S_ENOMEM;
}

p2s_status p2s_simulate(p2s_ctx *ctx, const p2s_image *frames, int n, const float *d_over_r0,
                        const unsigned long long *seeds, const p2s_image *out, void *stream) {
    p2s_status st = validate_simulate(ctx, frames, n, d_over_r0, seeds, out);
    if (st != P2S_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx->use_graphs && !ctx->profiling && n > 0 && ctx->form != P2S_FFT)
        return simulate_graph(ctx, frames, n, d_over_r0, seeds, out, s);
    Scratch sc{ctx, s, false};
    st = simulate_impl(ctx, frames, n, d_over_r0, seeds, out, s, sc);
    sc.release();
    return st;
}

p2s_status p2s_simulate_spectral(p2s_ctx *const *ctx3, const p2s_image *frames, int n, const float *d_over_r0,
                                 const unsigned long long *seeds, const p2s_image *out, void *stream) {
    if (!ctx3 || !ctx3[0] || !ctx3[1] || !ctx3[2]) return einval("ctx3 must hold three contexts");
    const p2s_ctx *a = ctx3[0];
    for (int c = 1; c < 3; ++c) {
        const p2s_ctx *b = ctx3[c];
        // one turbulence realisation: identical fields and warps in every channel
        if (b->device != a->device || b->s != a->s || b->n_kernels != a->n_kernels || b->ell != a->ell ||
            b->guard != a->guard || b->kappa != a->kappa || b->field_method != a->field_method ||
            b->blur_then_warp != a->blur_then_warp)
            return einval("the three contexts must share device, correlation parameters, kappa and options");
    }
    p2s_status st = validate_simulate(ctx3[0], frames, n, d_over_r0, seeds, out);
    if (st != P2S_OK) return st;
    for (int i = 0; i < n; ++i)
        if (frames[i].C != 3) return einval("spectral frames are RGB (C = 3)");
    if (n == 0) return P2S_OK;
    cudaStream_t s = (cudaStream_t)stream;
    // per frame: an input plane and an output plane of H x W floats
    size_t total = 0;
    std::vector<size_t> off(n);
    for (int i = 0; i < n; ++i) {
        off[i] = total;
        total += (((size_t)frames[i].H * frames[i].W * sizeof(float)) + 255) & ~(size_t)255;
    }
    char *buf = nullptr;
    P2S_CUDA(cudaMallocAsync((void **)&buf, 2 * total, s));
    std::vector<p2s_image> pin(n), pout(n);
    for (int i = 0; i < n; ++i) {
        pin[i] = p2s_image{(float *)(buf + off[i]), frames[i].H, frames[i].W, 1};
        pout[i] = p2s_image{(float *)(buf + total + off[i]), frames[i].H, frames[i].W, 1};
    }
    // channel copies in one launch per run of consecutive frames of one size
    std::vector<const float *> rgb_in(n), plane_out(n);
    std::vector<float *> plane_in(n), rgb_out(n);
    for (int i = 0; i < n; ++i) {
        rgb_in[i] = frames[i].data;
        plane_in[i] = pin[i].data;
        plane_out[i] = pout[i].data;
        rgb_out[i] = out[i].data;
    }
    auto copy_runs = [&](const std::vector<const float *> &src, const std::vector<float *> &dst, int ss, int so, int ds,
                         int dof) -> p2s_status {
        for (int i0 = 0; i0 < n;) {
            int i1 = i0 + 1;
            while (i1 < n && frames[i1].H == frames[i0].H && frames[i1].W == frames[i0].W) ++i1;
            const p2s_status r = launch_channel_copy(src.data() + i0, dst.data() + i0, i1 - i0,
                                                     (long long)frames[i0].H * frames[i0].W, ss, so, ds, dof, s);
            if (r != P2S_OK) return r;
            i0 = i1;
        }
        return P2S_OK;
    };
    for (int c = 0; c < 3 && st == P2S_OK; ++c) {
        st = copy_runs(rgb_in, plane_in, 3, c, 1, 0);
        if (st == P2S_OK) st = p2s_simulate(ctx3[c], pin.data(), n, d_over_r0, seeds, pout.data(), stream);
        if (st == P2S_OK) st = copy_runs(plane_out, rgb_out, 1, 0, 3, c);
    }
    cudaFreeAsync(buf, s);
    return st;
}

p2s_status p2s_autotune(p2s_ctx *ctx, const p2s_image *frames, int n, const float *d_over_r0,
                        const unsigned long long *seeds, const p2s_image *out, void *stream, int reps,
                        p2s_tune_result *res) {
    p2s_status st = validate_simulate(ctx, frames, n, d_over_r0, seeds, out);
    if (st != P2S_OK) return st;
    if (reps < 1) return einval("reps must be >= 1");
    const bool tc = ctx->prec == P2S_BF16 || ctx->prec == P2S_FP16;  // FP8: one kernel, nothing to tune
    int option = 0, option2 = 0;
    std::vector<int> cand, cand2;
    if (tc && ctx->form == P2S_GATHER) {
        option = P2S_OPT_GATHER_SPLIT;
        option2 = P2S_OPT_GATHER_BAND_ROWS;  // the fused kernel's tile height
        cand = {1, 2, 3, 4, 0, 0};
        cand2 = {0, 0, 0, 0, 32, 16};
    } else if (tc && ctx->form == P2S_SCATTER) {
        option = P2S_OPT_SCATTER_SEGMENT_ROWS;
        cand = {8, 16, 32, 64, 128, 1024};
        cand2.assign(cand.size(), 0);
    }
    p2s_tune_result r;
    std::memset(&r, 0, sizeof r);
    r.option = option;
    r.option2 = option2;
    if (cand.empty()) {
        if (res) *res = r;
        return P2S_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    P2S_CUDA(cudaEventCreate(&e0));
    P2S_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (size_t c = 0; c < cand.size() && c < 8; ++c) {
        if ((st = p2s_set_option(ctx, option, cand[c])) != P2S_OK) break;
        if (cand2[c] && (st = p2s_set_option(ctx, option2, cand2[c])) != P2S_OK) break;
        if ((st = p2s_simulate(ctx, frames, n, d_over_r0, seeds, out, stream)) != P2S_OK) break;
        cudaEventRecord(e0, s);
        for (int k = 0; k < reps && st == P2S_OK; ++k) st = p2s_simulate(ctx, frames, n, d_over_r0, seeds, out, stream);
        cudaEventRecord(e1, s);
        if (st != P2S_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = P2S_ECUDA;
            set_error("autotune: stream failed");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        r.value[r.n] = cand[c];
        r.value2[r.n] = cand2[c];
        r.ms[r.n] = ms / reps;
        if (r.ms[r.n] < best) {
            best = r.ms[r.n];
            r.best = r.n;
        }
        ++r.n;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != P2S_OK) return st;
    st = p2s_set_option(ctx, option, r.value[r.best]);
    if (st == P2S_OK && r.value2[r.best]) st = p2s_set_option(ctx, option2, r.value2[r.best]);
    if (res) *res = r;
    return st;
}

p2s_status p2s_simulate_host(p2s_ctx *ctx, const p2s_image *frames, int n, const float *d_over_r0,
                             const unsigned long long *seeds, const p2s_image *out, void *stream) {
    p2s_status st = validate_simulate(ctx, frames, n, d_over_r0, seeds, out);
    if (st != P2S_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // The frames go in chunks: chunk k's host->device copy (copy stream 0) overlaps the
    // path of chunk k - 1 (the caller's stream), whose device->host copy (copy stream 1)
    // overlaps the path of chunk k + 1.  Only the first chunk's copy in and the last
    // chunk's copy out are exposed, so those two chunks take an eighth of the frames each
    // and the rest go in chunks of at least 16 frames (full persistent launches), at most
    // 3 of them: 64 frames as 8 + 16 + 16 + 16 + 8.
    std::vector<int> bounds{0};
    if (n >= 32) {
        const int edge = n / 8, mid = n - 2 * edge, nmid = std::max(1, std::min(3, mid / 16));
        bounds.push_back(edge);
        for (int k = 1; k <= nmid; ++k) bounds.push_back(edge + (int)((long long)mid * k / nmid));
    }
    bounds.push_back(n);
    bounds.erase(std::unique(bounds.begin(), bounds.end()), bounds.end());
    const int nch = (int)bounds.size() - 1;
    for (int i = 0; i < 2; ++i)
        if (!ctx->copy_stream[i]) P2S_CUDA(cudaStreamCreateWithFlags(&ctx->copy_stream[i], cudaStreamNonBlocking));
    // Chunks alternate between the caller's stream and a second compute stream, so that the
    // next chunk's kernels take the SMs the current chunk's last wave leaves idle.  Graph
    // mode keeps one stream: its captured launches share the context's scratch arena.
    const bool two = nch > 1 && !ctx->use_graphs;
    if (two && !ctx->aux_stream) P2S_CUDA(cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking));
    while ((int)ctx->host_ev.size() < 2 * nch + 5) {
        cudaEvent_t e;
        P2S_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->host_ev.push_back(e);
    }
    cudaEvent_t ev_alloc = ctx->host_ev[0], ev_done = ctx->host_ev[1];
    cudaStream_t cin = ctx->copy_stream[0], cout = ctx->copy_stream[1];
    size_t total = 0;
    for (int i = 0; i < n; ++i) total += 2 * (((size_t)frames[i].H * frames[i].W * frames[i].C * 4 + 255) & ~(size_t)255);
    char *buf = nullptr;
    P2S_CUDA(cudaMallocAsync((void **)&buf, total + 256, s));
    P2S_CUDA(cudaEventRecord(ev_alloc, s));
    P2S_CUDA(cudaStreamWaitEvent(cin, ev_alloc, 0));
    if (two) P2S_CUDA(cudaStreamWaitEvent(ctx->aux_stream, ev_alloc, 0));
    std::vector<p2s_image> din(n), dout(n);
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        const size_t bytes = (size_t)frames[i].H * frames[i].W * frames[i].C * 4;
        din[i] = frames[i];
        din[i].data = (float *)(buf + off);
        off += (bytes + 255) & ~(size_t)255;
        dout[i] = out[i];
        dout[i].data = (float *)(buf + off);
        off += (bytes + 255) & ~(size_t)255;
    }
    auto chunk_begin = [&](int k) { return bounds[k]; };
    // all host->device copies, chunk by chunk, each chunk's end marked
    auto copy_in = [&]() -> p2s_status {
        for (int k = 0; k < nch; ++k) {
            for (int i = chunk_begin(k); i < chunk_begin(k + 1); ++i) {
                const size_t bytes = (size_t)frames[i].H * frames[i].W * frames[i].C * 4;
                if (cudaMemcpyAsync(din[i].data, frames[i].data, bytes, cudaMemcpyHostToDevice, cin) != cudaSuccess) {
                    set_error("host->device copy failed");
                    return P2S_ECUDA;
                }
            }
            if (cudaEventRecord(ctx->host_ev[2 + 2 * k], cin) != cudaSuccess) return P2S_ECUDA;
        }
        return P2S_OK;
    };
    // The tensor-core gather (warp then blur, no graphs): the fields and the network of every
    // frame first, the input copies queued right after them (they read no input pixels), then
    // each chunk's warp and blur once its inputs are in.  Otherwise the copies first and the
    // whole path per chunk.
    const bool piped = !ctx->use_graphs && tc_precision(ctx->prec) && ctx->form == P2S_GATHER && !ctx->blur_then_warp;
    if (!piped) st = copy_in();
    if (piped && st == P2S_OK) {
        std::vector<cudaEvent_t> in_ready(nch), out_done(nch);
        for (int k = 0; k < nch; ++k) {
            in_ready[k] = ctx->host_ev[2 + 2 * k];
            out_done[k] = ctx->host_ev[3 + 2 * k];
        }
        const Pipeline pl{nch,
                          bounds.data(),
                          in_ready.data(),
                          out_done.data(),
                          two ? ctx->aux_stream : nullptr,
                          ctx->host_ev[3 + 2 * nch],
                          ctx->host_ev[4 + 2 * nch],
                          copy_in};
        Scratch sc{ctx, s, false};
        st = simulate_tc(ctx, din.data(), dout.data(), n, d_over_r0, seeds, s, sc, &pl);
        sc.release();
    }
    // the path per chunk (or, piped, only the copies back), each chunk's results copied back
    for (int k = 0; k < nch && st == P2S_OK; ++k) {
        const int i0 = chunk_begin(k), i1 = chunk_begin(k + 1);
        if (!piped) {
            cudaStream_t cs = (two && (k & 1)) ? ctx->aux_stream : s;
            P2S_CUDA(cudaStreamWaitEvent(cs, ctx->host_ev[2 + 2 * k], 0));
            st = p2s_simulate(ctx, din.data() + i0, i1 - i0, d_over_r0 + i0, seeds + i0, dout.data() + i0, (void *)cs);
            if (st != P2S_OK) break;
            P2S_CUDA(cudaEventRecord(ctx->host_ev[3 + 2 * k], cs));
        }
        P2S_CUDA(cudaStreamWaitEvent(cout, ctx->host_ev[3 + 2 * k], 0));
        for (int i = i0; i < i1; ++i) {
            const size_t bytes = (size_t)out[i].H * out[i].W * out[i].C * 4;
            if (cudaMemcpyAsync(out[i].data, dout[i].data, bytes, cudaMemcpyDeviceToHost, cout) != cudaSuccess) {
                set_error("device->host copy failed");
                st = P2S_ECUDA;
                break;
            }
        }
    }
    // the buffers are released on the caller's stream once every copy and chunk is done
    if (two) {
        cudaEventRecord(ctx->host_ev[2 + 2 * nch], ctx->aux_stream);
        cudaStreamWaitEvent(s, ctx->host_ev[2 + 2 * nch], 0);
    }
    cudaEventRecord(ev_done, cout);
    cudaStreamWaitEvent(s, ev_done, 0);
    cudaEventRecord(ev_done, cin);
    cudaStreamWaitEvent(s, ev_done, 0);
    cudaFreeAsync(buf, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && st == P2S_OK) {
        set_error("stream synchronize failed: %s", cudaGetErrorString(cudaGetLastError()));
        st = P2S_ECUDA;
    }
    return st;
}

}  // extern "C"
