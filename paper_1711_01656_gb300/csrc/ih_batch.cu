// ih_batch.cu -- batched builds: many frames of uneven size in one launch
// per kernel, optionally captured in a CUDA graph, with tile grids chosen by
// measurement (ih_autotune).
//
// A batch is planned once: every frame's tensors, feature scratch and tile
// carries are allocated, each frame's plane set is made (its tile grid taken
// from the context's tuned grids when present), and the descriptor tables
// the batched kernels read (plane sets, prefix sums of each kernel's work
// per frame, feature jobs, query jobs) are uploaded.  A run then enqueues a
// fixed sequence of launches -- the feature pre-pass of all RGB frames, the
// five build kernels over all frames, and the rectangle and weighted queries
// of all frames -- or replays the CUDA graph captured from that sequence.
#include <algorithm>
#include <array>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ih.h"
#include "ih_ctx.h"
#include "ih_internal.cuh"
#include "ih_plan.h"

using namespace ih;

struct ih_batch {
    ih_ctx *ctx = nullptr;
    int n = 0;
    std::vector<void *> allocs;  // device memory owned by the batch
    BatchDev bd{};
    int64_t totals[5] = {0, 0, 0, 0, 0};
    FeatJob *d_feat = nullptr;
    int64_t *d_feat_pre = nullptr;
    int nfeat = 0;
    int64_t feat_total = 0;
    QueryJob *d_q = nullptr;
    int64_t *d_pre_r = nullptr, *d_pre_w = nullptr;
    int64_t q_rects = 0, q_wins = 0;
    // IH_BATCH_PERSISTENT: the build as one launch of k_build_persistent
    bool persistent = false;
    PersistDev pdev{};
    int persist_layout = -1;  // the layout of every frame, or -1
    int32_t *d_counters = nullptr;  // [3 n] done counters, then the ticket
    size_t counter_bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches_per_run = 0;
    // a batch of one frame runs the single-frame kernels (no per-item frame
    // search, tables in kernel parameters) with these host copies
    bool single = false;
    bool single_feat = false;
    FeatJob feat0{};
    PlaneSet set0{};
    CountView view0{};
    QueryJob q0{};
};

namespace {

template <typename T>
cudaError_t batch_alloc(ih_batch *b, T **p, size_t bytes, cudaStream_t st)
{
    cudaError_t e = pool_alloc(b->ctx, p, bytes, st);
    if (e == cudaSuccess) b->allocs.push_back(*p);
    return e;
}

// The batch's launches, in order, on `st` (prof may be null).
int enqueue_run(ih_batch *b, cudaStream_t st, const Prof *prof)
{
    int n = 0, k = 0;
    if (b->single) {
        if (b->single_feat) {
            const FeatJob &f = b->feat0;
            k = launch_features(f.r, f.g, f.b, f.pitch, f.H, f.W, nullptr, f.out_i, f.out_hog, f.opitch, st, prof);
            if (k < 0) return -1;
            n += k;
        }
        const QueryJob &q = b->q0;
        const int64_t nr = q.rects ? b->q_rects / rect_items(b->view0) : 0, nw = q.wins ? b->q_wins / q.m.Bw : 0;
        if (b->set0.small && b->set0.sm_bar && nr && !nw) {
            // a small frame and its rectangles in one launch
            const SmallQuery sq{q.rects, nr, q.rect_out};
            k = launch_build_small(b->set0, st, prof, &sq);
            return k < 0 ? -1 : n + k;
        }
        k = launch_build(b->set0, st, prof);
        if (k < 0) return -1;
        n += k;
        if (nr || nw) {
            k = launch_query_both(b->view0, q.m, q.rects, nr, q.rect_out, q.wins, nw, q.kernel, q.layers, q.normalize,
                                  q.wout, b->ctx->d_err, st, prof);
            if (k < 0) return -1;
            n += k;
        }
        return n;
    }
    if (b->feat_total) {
        k = launch_features_batch(b->d_feat, b->d_feat_pre, b->nfeat, b->feat_total, st, prof);
        if (k < 0) return -1;
        n += k;
    }
    if (b->persistent) {
        if (cudaMemsetAsync(b->d_counters, 0, b->counter_bytes, st) != cudaSuccess) return -1;
        k = launch_build_persistent(b->pdev, b->persist_layout, b->bd.max_R, st, prof);
    } else {
        k = launch_build_batch(b->bd, b->totals, st, prof);
    }
    if (k < 0) return -1;
    n += k;
    if (b->q_rects || b->q_wins) {
        k = launch_queries_batch(b->d_q, b->d_pre_r, b->d_pre_w, b->n, b->q_rects, b->q_wins, b->ctx->d_err, st, prof);
        if (k < 0) return -1;
        n += k;
    }
    return n;
}

void free_batch(ih_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (void *p : b->allocs) cudaFreeAsync(p, 0);
    cudaStreamSynchronize(0);
    b->allocs.clear();
}

// Channel planes of a frame (feature scratch for RGB input: 4 planes of fp x H).
void frame_planes(const ih_frame &f, uint8_t *feat, int64_t fp, const uint8_t **planes, int64_t *cpitch)
{
    const int64_t plane_stride = (int64_t)f.height * f.pitch_bytes;
    if (f.input == IH_INPUT_RGB_FEATURES) {
        for (int c = 0; c < 3; ++c) {
            planes[c] = f.d_pixels + c * plane_stride;
            cpitch[c] = f.pitch_bytes;
        }
        for (int c = 3; c < 7; ++c) {
            planes[c] = feat + (c - 3) * fp * f.height;
            cpitch[c] = fp;
        }
    } else {
        for (int c = 0; c < f.channels; ++c) {
            planes[c] = f.d_pixels + c * plane_stride;
            cpitch[c] = f.pitch_bytes;
        }
    }
}

// Time one build of `f` with each candidate tile grid; keep the fastest.
ih_status tune_frame(ih_ctx *ctx, const ih_frame &f, cudaStream_t st)
{
    FrameRec fr;
    frame_record(f, fr);
    cudaError_t e = pool_alloc(ctx, &fr.d_ih, fr.count_bytes, st);
    if (e == cudaSuccess && fr.Bw) e = pool_alloc(ctx, &fr.d_mom, fr.moment_bytes, st);
    uint8_t *feat = nullptr;
    const int64_t fp = (f.width + 15) & ~15;
    if (e == cudaSuccess && f.input == IH_INPUT_RGB_FEATURES) e = pool_alloc(ctx, &feat, (size_t)4 * fp * f.height, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune allocation");
    const uint8_t *planes[kMaxChannels];
    int64_t cpitch[kMaxChannels];
    frame_planes(f, feat, fp, planes, cpitch);
    if (feat) {
        const int64_t ps3 = (int64_t)f.height * f.pitch_bytes;
        launch_features(f.d_pixels, f.d_pixels + ps3, f.d_pixels + 2 * ps3, f.pitch_bytes, f.height, f.width, nullptr,
                        feat, feat + fp * f.height, fp, st, nullptr);
    }
    PlaneSet ps;
    if (!make_planeset(ctx, f, fr, planes, cpitch, ps)) return fail(ctx, IH_EINVAL, "too many bins for one build");
    static const int kR[] = {8, 16, 32, 64, 128};
    static const int kWc[] = {128, 256, 512, 1024};
    std::vector<std::pair<int, int>> cands;
    size_t max_carry = 0;
    for (int R : kR)
        for (int Wc : kWc) {
            const TileGrid g = make_grid(fr.H, fr.W, R, Wc);
            if (std::find(cands.begin(), cands.end(), std::make_pair(g.R, g.Wc)) != cands.end()) continue;
            cands.push_back({g.R, g.Wc});
            PlaneSet t = ps;
            t.g = g;
            t.g.P = fr.P;
            max_carry = std::max(max_carry, carry_bytes(t));
        }
    void *scratch = nullptr;
    if (max_carry) e = pool_alloc(ctx, &scratch, max_carry, st);
    cudaEvent_t a, z;
    cudaEventCreate(&a);
    cudaEventCreate(&z);
    float best = 1e30f;
    std::pair<int, int> pick = cands.front();
    for (const auto &c : cands) {
        PlaneSet t = ps;
        t.g = make_grid(fr.H, fr.W, c.first, c.second);
        t.g.P = fr.P;
        carve_carries(t, scratch);
        if (launch_build(t, st, nullptr) < 0) break;  // warm-up
        float ms[3];
        for (float &m : ms) {
            cudaEventRecord(a, st);
            launch_build(t, st, nullptr);
            cudaEventRecord(z, st);
            cudaEventSynchronize(z);
            cudaEventElapsedTime(&m, a, z);
        }
        std::sort(ms, ms + 3);
        if (ms[1] < best) {
            best = ms[1];
            pick = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    if (scratch) cudaFreeAsync(scratch, st);
    if (feat) cudaFreeAsync(feat, st);
    cudaFreeAsync(fr.d_ih, st);
    if (fr.d_mom) cudaFreeAsync(fr.d_mom, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune");
    ctx->tuned[shape_key(f)] = pick;
    return IH_OK;
}

}  // namespace

extern "C" {

ih_status ih_autotune(ih_ctx *ctx, const ih_frame *frame, void *stream)
{
    if (!ctx || !frame) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    DevGuard dg(ctx->device);
    ih_status s = validate(ctx, *frame);
    if (s != IH_OK) return s;
    return tune_frame(ctx, *frame, static_cast<cudaStream_t>(stream));
}

ih_status ih_tune_set(ih_ctx *ctx, const ih_frame *frame, int32_t band_rows, int32_t strip_cols)
{
    if (!ctx || !frame) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    ih_status s = validate(ctx, *frame);
    if (s != IH_OK) return s;
    if (band_rows < 1 || band_rows > kMaxBandRows || strip_cols < kChunk || strip_cols % kChunk)
        return fail(ctx, IH_EINVAL, "tile grid %d x %d (band rows 1..%d, strip columns a multiple of %d)", band_rows,
                    strip_cols, kMaxBandRows, kChunk);
    ctx->tuned[shape_key(*frame)] = std::make_pair((int)band_rows, (int)strip_cols);
    return IH_OK;
}

ih_status ih_batch_create(ih_ctx *ctx, const ih_frame *frames, int32_t n, const ih_batch_queries *q, uint32_t flags,
                          ih_batch **out, int32_t *out_handles)
{
    if (!ctx) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (!frames || n < 1 || !out || !out_handles) return fail(ctx, IH_EINVAL, "ih_batch_create: bad arguments");
    if (flags & ~(uint32_t)(IH_BATCH_GRAPH | IH_BATCH_AUTOTUNE | IH_BATCH_PERSISTENT))
        return fail(ctx, IH_EINVAL, "batch flags %u", flags);
    if (q && ((q->d_rects && (!q->rects || !q->d_rect_out)) || (q->d_windows && (!q->windows || !q->d_weighted_out)) ||
              q->kernel > IH_K_WEDDING_CAKE || (q->flags & ~((uint32_t)IH_NORMALIZE | IH_LAYERS(0xff))) ||
              weighted_layers(q->flags) > 64))
        return fail(ctx, IH_EINVAL, "ih_batch_create: bad query description");
    DevGuard dg(ctx->device);
    std::vector<FrameRec> recs(n);
    uint64_t need = 0;
    for (int k = 0; k < n; ++k) {
        ih_status s = validate(ctx, frames[k]);
        if (s != IH_OK) return s;
        if (q && q->d_windows && q->windows[k] > 0 && frames[k].weighted_channel < 0)
            return fail(ctx, IH_EINVAL, "frame %d has weighted windows but no weighted channel", k);
        frame_record(frames[k], recs[k]);
        need += recs[k].count_bytes + recs[k].moment_bytes;
    }
    if (ctx->budget && ctx->used + need > ctx->budget)
        return fail(ctx, IH_EBUDGET, "ih_batch_create: %llu bytes live + %llu needed > budget %llu",
                    (unsigned long long)ctx->used, (unsigned long long)need, (unsigned long long)ctx->budget);
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        return fail(ctx, IH_ECUDA, "stream creation");
    if (flags & IH_BATCH_AUTOTUNE) {
        std::vector<std::string> done;
        for (int k = 0; k < n; ++k) {
            const std::string key = shape_key(frames[k]);
            if (std::find(done.begin(), done.end(), key) != done.end()) continue;
            done.push_back(key);
            ih_status s = tune_frame(ctx, frames[k], st);
            if (s != IH_OK) {
                cudaStreamDestroy(st);
                return s;
            }
        }
    }
    ih_batch *b = new ih_batch();
    b->ctx = ctx;
    b->n = n;
    auto bail = [&](ih_status s) {
        for (auto &fr : recs) {
            if (fr.d_ih) cudaFreeAsync(fr.d_ih, st);
            if (fr.d_mom) cudaFreeAsync(fr.d_mom, st);
        }
        cudaStreamSynchronize(st);
        free_batch(b);
        delete b;
        cudaStreamDestroy(st);
        return s;
    };
    // tensors, features, plane sets
    std::vector<PlaneSet> sets(n);
    std::vector<FeatJob> feats;
    std::vector<int64_t> feat_pre(1, 0);
    size_t carry_total = 0;
    for (int k = 0; k < n; ++k) {
        const ih_frame &f = frames[k];
        FrameRec &fr = recs[k];
        cudaError_t e = pool_alloc(ctx, &fr.d_ih, fr.count_bytes, st);
        if (e == cudaSuccess && fr.Bw) e = pool_alloc(ctx, &fr.d_mom, fr.moment_bytes, st);
        if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "tensor allocation"));
        uint8_t *feat = nullptr;
        const int64_t fp = (f.width + 15) & ~15;
        if (f.input == IH_INPUT_RGB_FEATURES) {
            if ((e = batch_alloc(b, &feat, (size_t)4 * fp * f.height, st)) != cudaSuccess)
                return bail(cuda_fail(ctx, e, "feature scratch allocation"));
            const int64_t ps3 = (int64_t)f.height * f.pitch_bytes;
            feats.push_back({f.d_pixels, f.d_pixels + ps3, f.d_pixels + 2 * ps3, f.pitch_bytes, f.height, f.width, feat,
                             feat + fp * f.height, fp});
            feat_pre.push_back(feat_pre.back() + feature_tiles(f.height, f.width));
        }
        const uint8_t *planes[kMaxChannels];
        int64_t cpitch[kMaxChannels];
        frame_planes(f, feat, fp, planes, cpitch);
        // a one-frame batch runs the single-frame kernels, the small-frame build included
        const bool one = n == 1 && !(flags & IH_BATCH_PERSISTENT);
        if (!make_planeset(ctx, f, fr, planes, cpitch, sets[k], one))
            return bail(fail(ctx, IH_EINVAL, "too many bins"));
    }
    batch_grids(sets.data(), n, ctx->nsm);
    for (int k = 0; k < n; ++k) carry_total += (carry_bytes(sets[k]) + 255) & ~size_t(255);
    char *carries = nullptr;
    if (carry_total) {
        cudaError_t e = batch_alloc(b, &carries, carry_total, st);
        if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "carry allocation"));
    }
    std::vector<int64_t> pre(5 * (n + 1), 0);
    size_t off = 0;
    for (int k = 0; k < n; ++k) {
        const size_t cb = carry_bytes(sets[k]);
        carve_carries(sets[k], cb ? carries + off : nullptr);
        off += (cb + 255) & ~size_t(255);
        make_view(sets[k], recs[k].d_ih, recs[k].view);
        recs[k].R = sets[k].g.R;
        recs[k].Wc = sets[k].g.Wc;
        int64_t c[5];
        batch_counts(sets[k], c);
        for (int j = 0; j < 5; ++j) pre[j * (n + 1) + k + 1] = pre[j * (n + 1) + k] + c[j];
    }
    for (int j = 0; j < 5; ++j) b->totals[j] = pre[j * (n + 1) + n];
    // queries
    std::vector<QueryJob> qj(n);
    std::vector<int64_t> pre_r(n + 1, 0), pre_w(n + 1, 0);
    CountView *d_views = nullptr;
    cudaError_t e = batch_alloc(b, &d_views, sizeof(CountView) * n, st);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "table allocation"));
    int64_t roff = 0, woff = 0, rout = 0, wout = 0;
    for (int k = 0; k < n; ++k) {
        const FrameRec &fr = recs[k];
        QueryJob &j = qj[k];
        memset(&j, 0, sizeof j);
        j.v = d_views + k;
        j.m = MomentView{fr.wch >= 0 ? fr.bin_off[fr.wch] : 0, fr.d_mom, fr.Bw, fr.mbits == 32};
        const int64_t nr = (q && q->d_rects) ? q->rects[k] : 0;
        const int64_t nw = (q && q->d_windows) ? q->windows[k] : 0;
        if (nr) {
            j.rects = q->d_rects + 4 * roff;
            j.rect_out = q->d_rect_out + rout;
        }
        if (nw) {
            j.wins = q->d_windows + 4 * woff;
            j.wout = q->d_weighted_out + wout;
            j.normalize = (q->flags & IH_NORMALIZE) ? 1 : 0;
            j.kernel = (int32_t)q->kernel;
            j.layers = weighted_layers(q->flags);
        }
        roff += nr;
        rout += nr * fr.B;
        woff += nw;
        wout += nw * fr.Bw;
        pre_r[k + 1] = pre_r[k] + nr * rect_items(fr.view);
        pre_w[k + 1] = pre_w[k] + nw * fr.Bw;
    }
    b->q_rects = pre_r[n];
    b->q_wins = pre_w[n];
    // upload the tables
    PlaneSet *d_sets = nullptr;
    int64_t *d_pre = nullptr;
    if ((e = batch_alloc(b, &d_sets, sizeof(PlaneSet) * n, st)) != cudaSuccess ||
        (e = batch_alloc(b, &d_pre, sizeof(int64_t) * (7 * (n + 1) + feat_pre.size()), st)) != cudaSuccess ||
        (e = batch_alloc(b, &b->d_q, sizeof(QueryJob) * n, st)) != cudaSuccess ||
        (!feats.empty() && (e = batch_alloc(b, &b->d_feat, sizeof(FeatJob) * feats.size(), st)) != cudaSuccess))
        return bail(cuda_fail(ctx, e, "table allocation"));
    std::vector<int64_t> allpre(pre);
    allpre.insert(allpre.end(), pre_r.begin(), pre_r.end());
    allpre.insert(allpre.end(), pre_w.begin(), pre_w.end());
    allpre.insert(allpre.end(), feat_pre.begin(), feat_pre.end());
    std::vector<CountView> views(n);
    for (int k = 0; k < n; ++k) views[k] = recs[k].view;
    cudaMemcpyAsync(d_sets, sets.data(), sizeof(PlaneSet) * n, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_pre, allpre.data(), sizeof(int64_t) * allpre.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_views, views.data(), sizeof(CountView) * n, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(b->d_q, qj.data(), sizeof(QueryJob) * n, cudaMemcpyHostToDevice, st);
    if (!feats.empty()) cudaMemcpyAsync(b->d_feat, feats.data(), sizeof(FeatJob) * feats.size(), cudaMemcpyHostToDevice, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bail(cuda_fail(ctx, e, "table upload"));
    b->bd.sets = d_sets;
    b->bd.n = n;
    b->bd.pre_sums0 = d_pre;
    b->bd.pre_sums1 = d_pre + (n + 1);
    b->bd.pre_scan = d_pre + 2 * (n + 1);
    b->bd.pre_tiles = d_pre + 3 * (n + 1);
    b->bd.pre_mom = d_pre + 4 * (n + 1);
    b->bd.max_R = 1;
    for (int k = 0; k < n; ++k) b->bd.max_R = std::max(b->bd.max_R, sets[k].g.R);
    b->d_pre_r = d_pre + 5 * (n + 1);
    b->d_pre_w = d_pre + 6 * (n + 1);
    b->d_feat_pre = d_pre + 7 * (n + 1);
    b->nfeat = (int)feats.size();
    b->feat_total = feat_pre.back();
    if (flags & IH_BATCH_PERSISTENT) {
        // segments in phase order: every frame's tile sums (weighted windows
        // first), then every frame's carry scan, then every frame's tiles; a
        // frame's later phase waits only for its own earlier ones
        std::vector<PersistSeg> segs;
        std::vector<int64_t> seg_pre(1, 0);
        std::vector<int32_t> need(3 * n, 0);
        std::vector<std::array<int64_t, kPersistKinds>> cnt(n);
        for (int k = 0; k < n; ++k) {
            persistent_counts(sets[k], cnt[k].data());
            need[3 * k] = (int32_t)(cnt[k][0] + cnt[k][1]);
            need[3 * k + 1] = (int32_t)cnt[k][2];
            need[3 * k + 2] = (int32_t)(cnt[k][3] + cnt[k][4]);
        }
        const int order[3][2] = {{0, 1}, {2, -1}, {3, 4}};
        for (const auto &ph : order)
            for (int k = 0; k < n; ++k)
                for (int kind : ph)
                    if (kind >= 0 && cnt[k][kind] > 0) {
                        segs.push_back(PersistSeg{k, kind, 0, cnt[k][kind]});
                        seg_pre.push_back(seg_pre.back() + cnt[k][kind]);
                    }
        PersistSeg *d_segs = nullptr;
        int64_t *d_seg_pre = nullptr;
        int32_t *d_need = nullptr;
        b->counter_bytes = sizeof(int32_t) * (3 * (size_t)n + 1);
        if ((e = batch_alloc(b, &d_segs, sizeof(PersistSeg) * segs.size(), st)) != cudaSuccess ||
            (e = batch_alloc(b, &d_seg_pre, sizeof(int64_t) * seg_pre.size(), st)) != cudaSuccess ||
            (e = batch_alloc(b, &d_need, sizeof(int32_t) * need.size(), st)) != cudaSuccess ||
            (e = batch_alloc(b, &b->d_counters, b->counter_bytes, st)) != cudaSuccess)
            return bail(cuda_fail(ctx, e, "persistent table allocation"));
        cudaMemcpyAsync(d_segs, segs.data(), sizeof(PersistSeg) * segs.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_seg_pre, seg_pre.data(), sizeof(int64_t) * seg_pre.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_need, need.data(), sizeof(int32_t) * need.size(), cudaMemcpyHostToDevice, st);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bail(cuda_fail(ctx, e, "table upload"));
        b->persistent = true;
        b->persist_layout = sets[0].layout;
        for (int k = 1; k < n; ++k)
            if (sets[k].layout != b->persist_layout) b->persist_layout = -1;
        b->pdev.sets = d_sets;
        b->pdev.segs = d_segs;
        b->pdev.seg_pre = d_seg_pre;
        b->pdev.nsegs = (int32_t)segs.size();
        b->pdev.total = seg_pre.back();
        b->pdev.done = b->d_counters;
        b->pdev.need = d_need;
        b->pdev.ticket = reinterpret_cast<unsigned int *>(b->d_counters + 3 * (size_t)n);
        b->pdev.err = ctx->d_err;
    } else if (n == 1) {
        b->single = true;
        b->single_feat = !feats.empty();
        if (b->single_feat) b->feat0 = feats[0];
        b->set0 = sets[0];
        if (b->set0.small && b->set0.sm_bar) {
            // the small-frame build's barrier counters: zeroed once here, left zero by every run
            if ((e = cudaMemsetAsync(b->set0.sm_bar, 0, 2 * sizeof(unsigned int), st)) != cudaSuccess)
                return bail(cuda_fail(ctx, e, "counter initialisation"));
            b->set0.sm_zeroed = 1;
        }
        b->view0 = recs[0].view;
        b->q0 = qj[0];
    }
    // graph
    if (flags & IH_BATCH_GRAPH) {
        prepare_kernels();
        int nl = 0;
        if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) == cudaSuccess) {
            nl = enqueue_run(b, st, nullptr);
            e = cudaStreamEndCapture(st, &b->graph);
        }
        if (e == cudaSuccess && nl >= 0) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess || nl < 0) return bail(cuda_fail(ctx, e != cudaSuccess ? e : cudaGetLastError(), "graph capture"));
        b->launches_per_run = nl;
    } else {
        b->launches_per_run = -1;
    }
    cudaStreamDestroy(st);
    for (int k = 0; k < n; ++k) out_handles[k] = publish_frame(ctx, recs[k]);
    *out = b;
    return IH_OK;
}

ih_status ih_batch_run(ih_batch *b, void *stream)
{
    if (!b) return IH_EINVAL;
    ih_ctx *ctx = b->ctx;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    DevGuard dg(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (b->exec) {
        const cudaError_t e = cudaGraphLaunch(b->exec, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
        ctx->launches += b->launches_per_run;
        return IH_OK;
    }
    const int nl = enqueue_run(b, st, prof_of(ctx));
    if (nl < 0) return cuda_fail(ctx, cudaGetLastError(), "batch launch");
    ctx->launches += nl;
    return IH_OK;
}

ih_status ih_batch_destroy(ih_batch *b)
{
    if (!b) return IH_OK;
    {
        std::lock_guard<std::recursive_mutex> lk(b->ctx->mu);
        DevGuard dg(b->ctx->device);
        cudaDeviceSynchronize();
        free_batch(b);
    }
    delete b;
    return IH_OK;
}

}  // extern "C"
