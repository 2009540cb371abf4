// Serving loop: single-frame requests of mixed size and strength, admitted
// by HBM footprint and batched continuously onto a few CUDA streams.
//
// A scheduler thread takes requests in arrival order.  A request is admitted
// when its device footprint (input, output and the path's scratch) fits in
// what is left of the budget; admitted requests wait for a free stream slot,
// and whatever is admitted when a slot frees is launched together as ONE
// p2s_simulate call (frames of different sizes share one persistent
// tensor-core launch).  Per batch, on its slot's stream: host->device copies,
// the path, device->host copies, then a host callback that stamps the
// completion time of every request of the batch and returns its memory to
// the budget.  Requests that arrive while batches run are admitted as soon
// as a slot and memory are free (continuous batching); work of different
// slots overlaps on the device.  Only the scheduler thread calls into the
// context, so the context's one-thread rule holds.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "p2s_internal.h"

using Clock = std::chrono::steady_clock;

namespace {

p2s_status bad(const char *msg) {
    p2s::set_error("%s", msg);
    return P2S_EINVAL;
}

struct Request {
    long long ticket;
    const float *in;
    float *out;
    int H, W, C;
    float dr;
    unsigned long long seed;
    size_t bytes;  // admitted device footprint
    Clock::time_point t_submit;
};

struct Batch {
    p2s_server *srv;
    int slot;
    std::vector<Request> req;
    std::vector<float *> d_in, d_out;
    size_t bytes;
};

}  // namespace

struct p2s_server {
    p2s_ctx *ctx;
    p2s_server_config cfg;
    std::vector<cudaStream_t> streams;
    std::vector<int> slot_busy;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> pending;
    std::unordered_map<long long, double> done_ms;  // ticket -> latency (ms), or < 0 on error
    std::unordered_map<long long, p2s_status> failed;
    long long next_ticket = 1;
    size_t in_use = 0, peak = 0;
    long long n_batches = 0, n_done = 0, n_frames_batched = 0;
    int running = 1;
    p2s_status last_error = P2S_OK;
    std::thread worker;
};

namespace {

// device bytes one request holds while its batch runs
size_t footprint(const p2s_ctx *ctx, const p2s::FieldGeom &g, int C) {
    const size_t px = (size_t)g.H * g.W;
    size_t b = 2 * px * C * sizeof(float);                                      // input + output
    b += px * C * sizeof(float);                                                // warped frame
    b += (size_t)g.Ah * g.Aw * p2s::kAlphaStride * sizeof(float);               // anchors
    b += p2s::fields_scratch_bytes(g, 1);                                       // field torus
    if (ctx->prec == P2S_FP8E4M3)
        b += p2s::beta8_bytes(g.H, g.W, 1);
    else if ((ctx->prec == P2S_BF16 || ctx->prec == P2S_FP16) && (ctx->form == P2S_SCATTER || ctx->gather_split))
        b += p2s::beta16_bytes(g.H, g.W, 1, (ctx->form != P2S_SCATTER) ? p2s::gather_perm(ctx->gather_split) : 0);
    else if (!p2s::tc_precision(ctx->prec))
        b += px * ctx->K * sizeof(float);
    return b + 4 * 1024;
}

void CUDART_CB batch_done(void *arg) {
    Batch *b = (Batch *)arg;
    p2s_server *s = b->srv;
    const Clock::time_point now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (const Request &r : b->req) {
            s->done_ms[r.ticket] = std::chrono::duration<double, std::milli>(now - r.t_submit).count();
            ++s->n_done;
        }
        s->in_use -= b->bytes;
        s->slot_busy[b->slot] = 0;
    }
    s->cv.notify_all();
    // device buffers were released with stream-ordered frees before this callback
    delete b;
}

void launch_batch(p2s_server *s, Batch *b) {
    cudaStream_t st = s->streams[b->slot];
    const size_t n = b->req.size();
    std::vector<p2s_image> fi(n), fo(n);
    std::vector<float> dr(n);
    std::vector<unsigned long long> sd(n);
    p2s_status err = P2S_OK;
    for (size_t i = 0; i < n && err == P2S_OK; ++i) {
        const Request &r = b->req[i];
        const size_t bytes = (size_t)r.H * r.W * r.C * sizeof(float);
        float *di = nullptr, *dout = nullptr;
        if (cudaMallocAsync((void **)&di, bytes, st) != cudaSuccess ||
            cudaMallocAsync((void **)&dout, bytes, st) != cudaSuccess) {
            err = P2S_ENOMEM;
            break;
        }
        b->d_in.push_back(di);
        b->d_out.push_back(dout);
        cudaMemcpyAsync(di, r.in, bytes, cudaMemcpyHostToDevice, st);
        fi[i] = p2s_image{di, r.H, r.W, r.C};
        fo[i] = p2s_image{dout, r.H, r.W, r.C};
        dr[i] = r.dr;
        sd[i] = r.seed;
    }
    if (err == P2S_OK) err = p2s_simulate(s->ctx, fi.data(), (int)n, dr.data(), sd.data(), fo.data(), st);
    if (err == P2S_OK)
        for (size_t i = 0; i < n; ++i)
            cudaMemcpyAsync(b->req[i].out, b->d_out[i], (size_t)b->req[i].H * b->req[i].W * b->req[i].C * sizeof(float),
                            cudaMemcpyDeviceToHost, st);
    for (float *p : b->d_in) cudaFreeAsync(p, st);
    for (float *p : b->d_out) cudaFreeAsync(p, st);
    if (err != P2S_OK) {
        std::lock_guard<std::mutex> lk(s->mu);
        for (const Request &r : b->req) s->failed[r.ticket] = err;
        s->last_error = err;
    }
    if (cudaLaunchHostFunc(st, batch_done, b) != cudaSuccess) {
        // the stream is broken: finish the batch here so waiters do not hang
        cudaStreamSynchronize(st);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (const Request &r : b->req) s->failed[r.ticket] = P2S_ECUDA;
            s->last_error = P2S_ECUDA;
        }
        batch_done(b);
    }
}

void scheduler(p2s_server *s) {
    cudaSetDevice(s->ctx->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        if (!s->running && s->pending.empty()) break;
        int slot = -1;
        for (size_t k = 0; k < s->slot_busy.size(); ++k)
            if (!s->slot_busy[k]) {
                slot = (int)k;
                break;
            }
        Batch *b = nullptr;
        if (slot >= 0 && !s->pending.empty()) {
            // admit in arrival order while the budget holds
            size_t add = 0;
            std::vector<Request> take;
            while (!s->pending.empty() && (int)take.size() < s->cfg.max_batch) {
                const Request &r = s->pending.front();
                if (s->in_use + add + r.bytes > s->cfg.hbm_budget_bytes) break;
                add += r.bytes;
                take.push_back(r);
                s->pending.pop_front();
            }
            if (!take.empty()) {
                b = new Batch{s, slot, std::move(take), {}, {}, add};
                s->slot_busy[slot] = 1;
                s->in_use += add;
                if (s->in_use > s->peak) s->peak = s->in_use;
                ++s->n_batches;
                s->n_frames_batched += (long long)b->req.size();
            }
        }
        if (b) {
            lk.unlock();
            launch_batch(s, b);
            lk.lock();
            continue;
        }
        s->cv.wait_for(lk, std::chrono::milliseconds(5));
    }
}

}  // namespace

extern "C" {

p2s_status p2s_server_create(p2s_ctx *ctx, const p2s_server_config *cfg, p2s_server **out) {
    if (!ctx || !cfg || !out) return bad("ctx, cfg and out must be non-NULL");
    if (cfg->max_inflight_batches < 1 || cfg->max_inflight_batches > 16 || cfg->max_batch < 1 ||
        cfg->max_batch > p2s::kMaxTcFrames || cfg->hbm_budget_bytes == 0)
        return bad("server config: 1..16 slots, 1..256 requests per batch, budget > 0");
    if (ctx->use_graphs) return bad("the server needs a context without graph mode (calls overlap on its streams)");
    p2s_server *s = new (std::nothrow) p2s_server();
    if (!s) return P2S_ENOMEM;
    s->ctx = ctx;
    s->cfg = *cfg;
    cudaSetDevice(ctx->device);
    for (int k = 0; k < cfg->max_inflight_batches; ++k) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t t : s->streams) cudaStreamDestroy(t);
            delete s;
            p2s::set_error("stream creation failed");
            return P2S_ECUDA;
        }
        s->streams.push_back(st);
        s->slot_busy.push_back(0);
    }
    s->worker = std::thread(scheduler, s);
    *out = s;
    return P2S_OK;
}

p2s_status p2s_server_submit(p2s_server *s, const float *host_in, int H, int W, int C, float d_over_r0,
                             unsigned long long seed, float *host_out, long long *ticket) {
    if (!s || !host_in || !host_out || !ticket) return bad("server, buffers and ticket must be non-NULL");
    if (H < 1 || W < 1 || !(C == 1 || C == 3) || !(d_over_r0 > 0.f)) return bad("bad frame request");
    p2s::FieldGeom g;
    p2s_status st = p2s::geometry(s->ctx, H, W, &g);
    if (st != P2S_OK) return st;
    const size_t bytes = footprint(s->ctx, g, C);
    if (bytes > s->cfg.hbm_budget_bytes) {
        p2s::set_error("request needs %zu bytes, more than the whole budget", bytes);
        return P2S_ENOMEM;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (!s->running) return bad("server is shutting down");
        *ticket = s->next_ticket++;
        s->pending.push_back(Request{*ticket, host_in, host_out, H, W, C, d_over_r0, seed, bytes, Clock::now()});
    }
    s->cv.notify_all();
    return P2S_OK;
}

p2s_status p2s_server_poll(p2s_server *s, long long ticket, int *done, double *latency_ms) {
    if (!s || !done) return bad("server and done must be non-NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->done_ms.find(ticket);
    *done = it != s->done_ms.end();
    if (*done) {
        if (latency_ms) *latency_ms = it->second;
        auto f = s->failed.find(ticket);
        if (f != s->failed.end()) return f->second;
    }
    return P2S_OK;
}

p2s_status p2s_server_wait(p2s_server *s, long long ticket, double timeout_s, double *latency_ms) {
    if (!s) return bad("server must be non-NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto limit = Clock::now() + std::chrono::duration<double>(timeout_s);
    while (s->done_ms.find(ticket) == s->done_ms.end()) {
        if (s->cv.wait_until(lk, limit) == std::cv_status::timeout && s->done_ms.find(ticket) == s->done_ms.end()) {
            p2s::set_error("request %lld not done within %.3f s", ticket, timeout_s);
            return P2S_ETIMEOUT;
        }
    }
    if (latency_ms) *latency_ms = s->done_ms[ticket];
    auto f = s->failed.find(ticket);
    return f != s->failed.end() ? f->second : P2S_OK;
}

p2s_status p2s_server_stats(p2s_server *s, p2s_server_counters *out) {
    if (!s || !out) return bad("server and out must be non-NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    out->completed = s->n_done;
    out->batches = s->n_batches;
    out->pending = (long long)s->pending.size();
    out->mean_batch = s->n_batches ? (double)s->n_frames_batched / (double)s->n_batches : 0.0;
    out->bytes_in_use = s->in_use;
    out->peak_bytes = s->peak;
    return P2S_OK;
}

void p2s_server_destroy(p2s_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->running = 0;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    delete s;
}

}  // extern "C"
