// ih_server.cu -- the request loop: continuous batching of frames and their
// queries from many tracker streams under an HBM budget.
//
// One scheduler thread owns the device work.  Each pass it
//   1. retires the ticks whose completion event has fired (a tick is the set
//      of requests launched together): their completions are queued for
//      ih_server_poll, and each tracker's previous resident frame is
//      released once the tracker's newer frame is done;
//   2. admits pending requests in arrival order into new ticks while a slot
//      is free: a request is admitted if its tensors fit the context's
//      budget, after evicting resident frames of completed requests (least
//      recently completed first) if needed; a request larger than the whole
//      budget completes with IH_EBUDGET; a cancelled request leaves the
//      queue (ih_server_cancel), or, once on the device, is released when
//      its tick retires instead of staying resident;
//   3. launches each new tick on the next of its CUDA streams: one upload of
//      the tick's descriptor tables, one batched feature pre-pass, the five
//      batched build kernels and the batched rectangle and weighted queries,
//      then a completion event.
// Requests that arrive while ticks are running join the next tick; ticks on
// different streams overlap on the device.  The arithmetic of a request does
// not depend on which other requests share its tick (every work item reads
// only its own frame's data), so results are identical alone and in a mix.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/ih.h"
#include "ih_ctx.h"
#include "ih_internal.cuh"
#include "ih_plan.h"

using namespace ih;

namespace {

struct Req {
    ih_request r;
    double t_submit = 0;
    FrameRec fr;
    int handle = -1;
    bool cancelled = false;  // set by ih_server_cancel while the request is on the device
};

struct Slot {
    bool busy = false;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    char *h_tab = nullptr;  // pinned staging of the descriptor tables
    char *d_tab = nullptr;
    size_t cap = 0;
    std::vector<Req *> reqs;
    double t_admit = 0;
};

constexpr int kMaxBatch = 256;

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

size_t table_bytes(int n)
{
    return a256(sizeof(PlaneSet) * n) + a256(sizeof(CountView) * n) + a256(sizeof(QueryJob) * n) +
           a256(sizeof(FeatJob) * n) + a256(sizeof(int64_t) * (8 * (n + 1)));
}

}  // namespace

struct ih_server {
    ih_ctx *ctx = nullptr;
    ih_server_config cfg{};
    std::vector<cudaStream_t> streams;
    int next_stream = 0;
    std::vector<Slot> slots;
    std::deque<Req *> pending;
    std::deque<ih_completion> done;
    std::map<int, int> resident;           // tracker -> handle of its latest completed frame
    std::list<std::pair<int, int>> lru;    // (tracker, handle), oldest completion first
    std::thread thr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    int64_t submitted = 0, completed = 0;
    cudaEvent_t ref = nullptr;
    double t_ref = 0;
    std::chrono::steady_clock::time_point t0;

    double clock() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

void complete(ih_server *s, Req *q, int status, double t_admit, double t_done)
{
    ih_completion c;
    c.user = q->r.user;
    c.status = status;
    c.handle = q->handle;
    c.t_submit = q->t_submit;
    c.t_admit = t_admit;
    c.t_done = t_done;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->done.push_back(c);
        ++s->completed;
    }
    s->cv_done.notify_all();
}

void release_handle(ih_ctx *ctx, int h)
{
    FrameRec *fr = get_frame(ctx, h);
    if (!fr) return;
    cudaFreeAsync(fr->d_ih, 0);
    if (fr->d_mom) cudaFreeAsync(fr->d_mom, 0);
    ctx->used -= fr->count_bytes + fr->moment_bytes;
    *fr = FrameRec();
}

// ctx lock held.
void retire(ih_server *s)
{
    for (Slot &sl : s->slots) {
        if (!sl.busy || cudaEventQuery(sl.done) != cudaSuccess) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, s->ref, sl.done);
        const double t_done = s->t_ref + ms / 1e3;
        for (Req *q : sl.reqs) {
            if (q->cancelled) {  // its result is dropped: release the frame now
                release_handle(s->ctx, q->handle);
                q->handle = -1;
                complete(s, q, IH_ECANCELLED, sl.t_admit, t_done);
                delete q;
                continue;
            }
            const int tr = q->r.tracker;
            auto it = s->resident.find(tr);
            if (it != s->resident.end()) {
                s->lru.remove(std::make_pair(tr, it->second));
                release_handle(s->ctx, it->second);
            }
            s->resident[tr] = q->handle;
            s->lru.emplace_back(tr, q->handle);
            complete(s, q, IH_OK, sl.t_admit, t_done);
            delete q;
        }
        sl.reqs.clear();
        sl.busy = false;
    }
}

// Enqueue one tick (ctx lock held).  Returns false if a CUDA call failed.
bool launch_tick(ih_server *s, Slot &sl, std::vector<Req *> &reqs)
{
    ih_ctx *ctx = s->ctx;
    const int n = (int)reqs.size();
    cudaStream_t st = sl.st;
    std::vector<PlaneSet> sets(n);
    std::vector<FeatJob> feats;
    std::vector<void *> transient;
    std::vector<size_t> cb(n);
    size_t carry_total = 0;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        const ih_frame &f = reqs[k]->r.frame;
        FrameRec &fr = reqs[k]->fr;
        e = pool_alloc(ctx, &fr.d_ih, fr.count_bytes, st);
        if (e == cudaSuccess && fr.Bw) e = pool_alloc(ctx, &fr.d_mom, fr.moment_bytes, st);
        uint8_t *feat = nullptr;
        const int64_t fp = (f.width + 15) & ~15;
        const int64_t ps3 = (int64_t)f.height * f.pitch_bytes;
        const uint8_t *planes[kMaxChannels];
        int64_t cpitch[kMaxChannels];
        if (e == cudaSuccess && f.input == IH_INPUT_RGB_FEATURES) {
            e = pool_alloc(ctx, &feat, (size_t)4 * fp * f.height, st);
            transient.push_back(feat);
            feats.push_back({f.d_pixels, f.d_pixels + ps3, f.d_pixels + 2 * ps3, f.pitch_bytes, f.height, f.width,
                             feat, feat + fp * f.height, fp});
            for (int c = 0; c < 3; ++c) {
                planes[c] = f.d_pixels + c * ps3;
                cpitch[c] = f.pitch_bytes;
            }
            for (int c = 3; c < 7; ++c) {
                planes[c] = feat + (c - 3) * fp * f.height;
                cpitch[c] = fp;
            }
        } else {
            for (int c = 0; c < f.channels; ++c) {
                planes[c] = f.d_pixels + c * ps3;
                cpitch[c] = f.pitch_bytes;
            }
        }
        if (e == cudaSuccess) make_planeset(ctx, f, fr, planes, cpitch, sets[k]);
    }
    if (e == cudaSuccess) {
        // (a tick keeps each frame's own grid: batch_grids' large tiles
        // measured a higher p50 frame-to-answer latency here)
        for (int k = 0; k < n; ++k) {
            cb[k] = a256(carry_bytes(sets[k]));
            carry_total += cb[k];
        }
    }
    char *carries = nullptr;
    if (e == cudaSuccess && carry_total) {
        e = pool_alloc(ctx, &carries, carry_total, st);
        transient.push_back(carries);
    }
    if (e != cudaSuccess) return false;
    // tables
    char *h = sl.h_tab;
    const size_t oS = 0, oV = oS + a256(sizeof(PlaneSet) * n), oQ = oV + a256(sizeof(CountView) * n);
    const size_t oF = oQ + a256(sizeof(QueryJob) * n), oP = oF + a256(sizeof(FeatJob) * n);
    PlaneSet *d_sets = reinterpret_cast<PlaneSet *>(sl.d_tab + oS);
    CountView *d_views = reinterpret_cast<CountView *>(sl.d_tab + oV);
    QueryJob *d_q = reinterpret_cast<QueryJob *>(sl.d_tab + oQ);
    FeatJob *d_feat = reinterpret_cast<FeatJob *>(sl.d_tab + oF);
    int64_t *d_pre = reinterpret_cast<int64_t *>(sl.d_tab + oP);
    int64_t *pre = reinterpret_cast<int64_t *>(h + oP);
    memset(pre, 0, sizeof(int64_t) * 8 * (n + 1));
    int64_t *pre_r = pre + 5 * (n + 1), *pre_w = pre + 6 * (n + 1), *pre_f = pre + 7 * (n + 1);
    size_t off = 0;
    int nf = 0;
    for (int k = 0; k < n; ++k) {
        Req *q = reqs[k];
        carve_carries(sets[k], cb[k] ? carries + off : nullptr);
        off += cb[k];
        make_view(sets[k], q->fr.d_ih, q->fr.view);
        q->fr.R = sets[k].g.R;
        q->fr.Wc = sets[k].g.Wc;
        int64_t c[5];
        batch_counts(sets[k], c);
        for (int j = 0; j < 5; ++j) pre[j * (n + 1) + k + 1] = pre[j * (n + 1) + k] + c[j];
        QueryJob jb;
        memset(&jb, 0, sizeof jb);
        jb.v = d_views + k;
        jb.m = MomentView{q->fr.wch >= 0 ? q->fr.bin_off[q->fr.wch] : 0, q->fr.d_mom, q->fr.Bw, q->fr.mbits == 32};
        const int64_t nr = q->r.d_rects ? q->r.n_rects : 0, nw = q->r.d_windows ? q->r.n_windows : 0;
        jb.rects = q->r.d_rects;
        jb.rect_out = q->r.d_rect_out;
        jb.wins = q->r.d_windows;
        jb.wout = q->r.d_weighted_out;
        jb.normalize = (q->r.weighted_flags & IH_NORMALIZE) ? 1 : 0;
        jb.kernel = IH_KERNEL_EPANECHNIKOV;
        jb.layers = 0;
        pre_r[k + 1] = pre_r[k] + nr * rect_items(q->fr.view);
        pre_w[k + 1] = pre_w[k] + nw * q->fr.Bw;
        memcpy(h + oS + sizeof(PlaneSet) * k, &sets[k], sizeof(PlaneSet));
        memcpy(h + oV + sizeof(CountView) * k, &q->fr.view, sizeof(CountView));
        memcpy(h + oQ + sizeof(QueryJob) * k, &jb, sizeof(QueryJob));
    }
    for (size_t k = 0; k < feats.size(); ++k) {
        memcpy(h + oF + sizeof(FeatJob) * k, &feats[k], sizeof(FeatJob));
        pre_f[k + 1] = pre_f[k] + feature_tiles(feats[k].H, feats[k].W);
        ++nf;
    }
    if ((e = cudaMemcpyAsync(sl.d_tab, sl.h_tab, oP + sizeof(int64_t) * 8 * (n + 1), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return false;
    BatchDev bd;
    bd.sets = d_sets;
    bd.n = n;
    bd.pre_sums0 = d_pre;
    bd.pre_sums1 = d_pre + (n + 1);
    bd.pre_scan = d_pre + 2 * (n + 1);
    bd.pre_tiles = d_pre + 3 * (n + 1);
    bd.pre_mom = d_pre + 4 * (n + 1);
    bd.max_R = 1;
    for (int k = 0; k < n; ++k) bd.max_R = std::max(bd.max_R, sets[k].g.R);
    int64_t totals[5];
    for (int j = 0; j < 5; ++j) totals[j] = pre[j * (n + 1) + n];
    const Prof *prof = prof_of(ctx);
    int nl = 0, k = 0;
    if (pre_f[nf]) {
        k = launch_features_batch(d_feat, d_pre + 7 * (n + 1), nf, pre_f[nf], st, prof);
        nl += k < 0 ? 0 : k;
    }
    if (k >= 0) {
        k = launch_build_batch(bd, totals, st, prof);
        nl += k < 0 ? 0 : k;
    }
    if (k >= 0 && (pre_r[n] || pre_w[n])) {
        k = launch_queries_batch(d_q, d_pre + 5 * (n + 1), d_pre + 6 * (n + 1), n, pre_r[n], pre_w[n], ctx->d_err, st,
                                 prof);
        nl += k < 0 ? 0 : k;
    }
    for (void *p : transient) cudaFreeAsync(p, st);
    if (k < 0) return false;
    ctx->launches += nl;
    cudaEventRecord(sl.done, st);
    for (Req *q : reqs) q->handle = publish_frame(ctx, q->fr);
    sl.reqs = reqs;
    sl.busy = true;
    sl.t_admit = s->clock();
    return true;
}

// ctx lock held.  Returns the number of ticks launched.
int admit(ih_server *s)
{
    ih_ctx *ctx = s->ctx;
    int launched = 0;
    for (Slot &sl : s->slots) {
        if (sl.busy) continue;
        std::vector<Req *> tick;
        uint64_t need = 0;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            while (!s->pending.empty() && (int)tick.size() < s->cfg.max_batch) {
                Req *q = s->pending.front();
                const uint64_t b = q->fr.count_bytes + q->fr.moment_bytes;
                if (ctx->budget && ctx->used + need + b > ctx->budget) {
                    // evict resident frames of completed requests, oldest first
                    while (!s->lru.empty() && ctx->used + need + b > ctx->budget) {
                        const auto v = s->lru.front();
                        s->lru.pop_front();
                        s->resident.erase(v.first);
                        release_handle(ctx, v.second);
                    }
                    if (ctx->used + need + b > ctx->budget) {
                        bool busy = !tick.empty();
                        for (const Slot &o : s->slots) busy = busy || o.busy;
                        if (!busy) {  // can never fit
                            s->pending.pop_front();
                            s->mu.unlock();
                            complete(s, q, IH_EBUDGET, s->clock(), s->clock());
                            s->mu.lock();
                            delete q;
                            continue;
                        }
                        break;
                    }
                }
                s->pending.pop_front();
                need += b;
                tick.push_back(q);
            }
        }
        if (tick.empty()) break;
        sl.st = s->streams[s->next_stream++ % s->streams.size()];
        if (!launch_tick(s, sl, tick)) {
            for (Req *q : tick) {
                complete(s, q, IH_ECUDA, s->clock(), s->clock());
                delete q;
            }
            cudaGetLastError();
            continue;
        }
        ++launched;
    }
    return launched;
}

void run(ih_server *s)
{
    cudaSetDevice(s->ctx->device);
    for (;;) {
        bool any_busy = false;
        {
            std::lock_guard<std::recursive_mutex> lk(s->ctx->mu);
            retire(s);
            admit(s);
            for (const Slot &sl : s->slots) any_busy = any_busy || sl.busy;
        }
        std::unique_lock<std::mutex> lk(s->mu);
        if (s->stop && s->pending.empty() && !any_busy) break;
        if (any_busy)
            s->cv_work.wait_for(lk, std::chrono::microseconds(20));
        else if (s->pending.empty())
            s->cv_work.wait_for(lk, std::chrono::milliseconds(5), [&] { return s->stop || !s->pending.empty(); });
    }
}

}  // namespace

extern "C" {

ih_status ih_server_create(ih_ctx *ctx, const ih_server_config *cfg, ih_server **out)
{
    if (!ctx || !cfg || !out) return IH_EINVAL;
    if (cfg->streams < 1 || cfg->streams > 64 || cfg->max_inflight < 1 || cfg->max_inflight > 64 ||
        cfg->max_batch < 1 || cfg->max_batch > kMaxBatch || cfg->flags)
        return fail(ctx, IH_EINVAL, "server config");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    DevGuard dg(ctx->device);
    ih_server *s = new ih_server();
    s->ctx = ctx;
    s->cfg = *cfg;
    s->t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < cfg->streams && e == cudaSuccess; ++k) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) s->streams.push_back(st);
    }
    s->slots.resize(cfg->max_inflight);
    const size_t cap = table_bytes(cfg->max_batch);
    for (Slot &sl : s->slots) {
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDefault);
        if (e == cudaSuccess) e = cudaHostAlloc(&sl.h_tab, cap, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_tab, cap);
        sl.cap = cap;
    }
    if (e == cudaSuccess) e = cudaEventCreate(&s->ref);
    if (e == cudaSuccess) e = cudaEventRecord(s->ref, s->streams[0]);
    if (e == cudaSuccess) e = cudaEventSynchronize(s->ref);
    if (e != cudaSuccess) {
        ih_server_destroy(s);
        return cuda_fail(ctx, e, "server creation");
    }
    s->t_ref = s->clock();
    s->thr = std::thread(run, s);
    *out = s;
    return IH_OK;
}

ih_status ih_server_submit(ih_server *s, const ih_request *req)
{
    if (!s || !req) return IH_EINVAL;
    ih_ctx *ctx = s->ctx;
    Req *q = new Req();
    q->r = *req;
    if (req->frame.channels > 16 || req->frame.channels < 1 || !req->frame.chan) {
        delete q;
        return IH_EINVAL;
    }
    memcpy(q->r.chan, req->frame.chan, sizeof(ih_channel) * req->frame.channels);
    q->r.frame.chan = q->r.chan;
    {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        ih_status st = validate(ctx, q->r.frame);
        if (st == IH_OK && req->tracker < 0) st = fail(ctx, IH_EINVAL, "tracker id %d", req->tracker);
        if (st == IH_OK && req->d_windows && req->n_windows > 0 && req->frame.weighted_channel < 0)
            st = fail(ctx, IH_EINVAL, "weighted windows without a weighted channel");
        if (st == IH_OK && ((req->d_rects && !req->d_rect_out) || (req->d_windows && !req->d_weighted_out) ||
                            req->n_rects < 0 || req->n_windows < 0 || (req->weighted_flags & ~(uint32_t)IH_NORMALIZE)))
            st = fail(ctx, IH_EINVAL, "request queries");
        if (st != IH_OK) {
            delete q;
            return st;
        }
        frame_record(q->r.frame, q->fr);
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        q->t_submit = s->clock();
        s->pending.push_back(q);
        ++s->submitted;
    }
    s->cv_work.notify_all();
    return IH_OK;
}

int32_t ih_server_poll(ih_server *s, ih_completion *out, int32_t max, int32_t wait_ms)
{
    if (!s || !out || max < 1) return 0;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && wait_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
    int32_t n = 0;
    while (n < max && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    return n;
}

ih_status ih_server_cancel(ih_server *s, uint64_t user)
{
    if (!s) return IH_EINVAL;
    Req *gone = nullptr;
    {
        // the scheduler holds ctx->mu while it moves requests into ticks
        std::lock_guard<std::recursive_mutex> lc(s->ctx->mu);
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto it = s->pending.begin(); it != s->pending.end(); ++it)
            if ((*it)->r.user == user) {
                gone = *it;
                s->pending.erase(it);
                break;
            }
        if (!gone) {
            for (Slot &sl : s->slots)
                if (sl.busy)
                    for (Req *q : sl.reqs)
                        if (q->r.user == user && !q->cancelled) {
                            q->cancelled = true;
                            return IH_OK;
                        }
            return IH_EINVAL;
        }
    }
    const double t = s->clock();
    complete(s, gone, IH_ECANCELLED, t, t);
    delete gone;
    return IH_OK;
}

ih_status ih_server_drain(ih_server *s)
{
    if (!s) return IH_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->completed >= s->submitted; });
    return IH_OK;
}

double ih_server_clock(ih_server *s) { return s ? s->clock() : 0.0; }

ih_status ih_server_destroy(ih_server *s)
{
    if (!s) return IH_OK;
    if (s->thr.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        s->thr.join();
    }
    {
        std::lock_guard<std::recursive_mutex> lk(s->ctx->mu);
        DevGuard dg(s->ctx->device);
        cudaDeviceSynchronize();
        for (auto &v : s->resident) release_handle(s->ctx, v.second);
        cudaDeviceSynchronize();
        for (Slot &sl : s->slots) {
            if (sl.done) cudaEventDestroy(sl.done);
            if (sl.h_tab) cudaFreeHost(sl.h_tab);
            if (sl.d_tab) cudaFree(sl.d_tab);
        }
        for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
        if (s->ref) cudaEventDestroy(s->ref);
    }
    delete s;
    return IH_OK;
}

}  // extern "C"
