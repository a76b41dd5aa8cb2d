// ih_capi.cu -- the C ABI of include/ih.h: contexts, frame table, HBM
// budget, stream-ordered device memory and the launch plan of a build.
//
// Memory: every tensor and every scratch buffer comes from a per-context
// CUDA memory pool through cudaMallocFromPoolAsync / cudaFreeAsync on the
// caller's stream, so a build never synchronises the device and freed
// memory is reused by later builds in stream order.  The pool keeps what it
// has reserved (release threshold = max), which makes steady-state builds
// allocation-free at the driver level.
#include <cstdarg>
#include <mutex>
#include <string>
#include <vector>
#include <cstdio>
#include <cstring>

#include "../../include/ih.h"
#include "ih_ctx.h"
#include "ih_internal.cuh"
#include "ih_plan.h"

using namespace ih;

namespace ih {

ih_status fail(ih_ctx *ctx, ih_status s, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->last_error = buf;
    }
    return s;
}

ih_status cuda_fail(ih_ctx *ctx, cudaError_t e, const char *what)
{
    return fail(ctx, IH_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

cudaEvent_t take_event(ih_ctx *ctx)
{
    if (!ctx->ev_free.empty()) {
        cudaEvent_t e = ctx->ev_free.back();
        ctx->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_mark_cb(void *p, int kid, int phase, cudaStream_t st)
{
    ih_ctx *ctx = static_cast<ih_ctx *>(p);
    if (!((ctx->prof_mask >> kid) & 1u)) return;
    cudaEvent_t e = take_event(ctx);
    cudaEventRecord(e, st);
    if (phase == 0) {
        ctx->prof_open = e;
        ctx->prof_open_kid = kid;
    } else if (ctx->prof_open && ctx->prof_open_kid == kid) {
        ctx->prof_pending.push_back({kid, ctx->prof_open, e});
        ctx->prof_open = nullptr;
        ctx->prof_open_kid = -1;
    } else {
        ctx->ev_free.push_back(e);
    }
}

const Prof *prof_of(ih_ctx *ctx) { return ctx->profiling ? &ctx->prof : nullptr; }

const char *kernel_name(int kid)
{
    static const char *names[KID_COUNT] = {"features",      "tile_sums/count", "tile_sums/weighted",
                                           "carry_scan",    "tiles/count",     "tiles/moments",
                                           "query_rects",   "query_weighted",  "export",
                                           "tiles/count+moments", "match_window", "accumulate",
                                           "local_median", "phog_build",     "phog_query",
                                           "tile_sums", "queries",      "tiles/mma", "persistent_build", "onepass_build",
                                           "small_build"};
    return (kid >= 0 && kid < KID_COUNT) ? names[kid] : "?";
}


ih_status validate(ih_ctx *ctx, const ih_frame &f)
{
    if (f.height < 1 || f.width < 1) return fail(ctx, IH_EINVAL, "frame size %dx%d", f.height, f.width);
    if ((int64_t)f.height * f.width > (int64_t)1 << 31)
        return fail(ctx, IH_EINVAL, "frame of %d x %d pixels is above 2^31", f.height, f.width);
    if (f.channels < 1 || f.channels > kMaxChannels)
        return fail(ctx, IH_EINVAL, "channels = %d (1..%d)", f.channels, kMaxChannels);
    if (!f.chan || !f.d_pixels) return fail(ctx, IH_EINVAL, "NULL chan or pixels");
    if (f.pitch_bytes < f.width) return fail(ctx, IH_EINVAL, "pitch_bytes %lld < width", (long long)f.pitch_bytes);
    if (f.input != IH_INPUT_PLANES && f.input != IH_INPUT_RGB_FEATURES)
        return fail(ctx, IH_EINVAL, "input kind %d", f.input);
    if (f.input == IH_INPUT_RGB_FEATURES && f.channels != 7)
        return fail(ctx, IH_EINVAL, "IH_INPUT_RGB_FEATURES needs 7 channels");
    if (f.layout != IH_LAYOUT_BIN_MAJOR && f.layout != IH_LAYOUT_SLAB && f.layout != IH_LAYOUT_RECORD)
        return fail(ctx, IH_EINVAL, "layout %d", f.layout);
    for (int c = 0; c < f.channels; ++c) {
        if (f.chan[c].bins < 1 || f.chan[c].bins > 256)
            return fail(ctx, IH_EINVAL, "channel %d bins = %d (1..256)", c, f.chan[c].bins);
        if (f.chan[c].mode != IH_BIN_UNIFORM8 && f.chan[c].mode != IH_BIN_INDEX)
            return fail(ctx, IH_EINVAL, "channel %d mode = %d", c, f.chan[c].mode);
    }
    int total = 0;
    for (int c = 0; c < f.channels; ++c) total += f.chan[c].bins;
    if (total > kMaxBins) return fail(ctx, IH_EINVAL, "%d bins in one frame (at most %d)", total, kMaxBins);
    if (f.layout == IH_LAYOUT_RECORD) {
        int bins[kMaxChannels], np = 0, words = 0;
        GroupDev sp[kMaxGroups];
        int16_t rw[kMaxGroups];
        for (int c = 0; c < f.channels; ++c) bins[c] = f.chan[c].bins;
        if (record_plan(bins, f.channels, sp, kMaxGroups, rw, &np, &words) < 0 || words > kMaxBins)
            return fail(ctx, IH_EINVAL, "IH_LAYOUT_RECORD: the channels need more than %d bin groups", kMaxGroups);
    }
    if (f.moment_bits != 0 && f.moment_bits != 32 && f.moment_bits != 64)
        return fail(ctx, IH_EINVAL, "moment_bits = %d (0, 32 or 64)", f.moment_bits);
    if (f.weighted_channel < -1 || f.weighted_channel >= f.channels)
        return fail(ctx, IH_EINVAL, "weighted_channel = %d", f.weighted_channel);
    return IH_OK;
}

// Bin groups: split each channel's bins evenly into groups of <= cap.
int make_groups(const int *bins, int nchan, int cap, GroupDev *out, int max_out)
{
    int n = 0;
    for (int c = 0; c < nchan; ++c) {
        const int ng = (bins[c] + cap - 1) / cap;
        for (int g = 0; g < ng; ++g) {
            if (n >= max_out) return -1;
            const int lo = bins[c] * g / ng, hi = bins[c] * (g + 1) / ng;
            out[n] = GroupDev{};
            out[n].chan = (int16_t)c;
            out[n].b_lo = (int16_t)lo;
            out[n].nb = (int16_t)(hi - lo);
            ++n;
        }
    }
    return n;
}

// LAYOUT_RECORD: the bin order (channel after channel) is cut into groups
// of up to 8 consecutive bins drawn from at most two channels; each group
// takes 8 words (one 32-byte sector) of the pixel record, its padding words
// holding 0, and consecutive groups share a plane while the plane's record
// stays within 16 words.  sp[] receives the groups with their plane and word
// offset, rec_w[] the record width of each plane.  Returns the number of
// groups, or -1 if there are more than max_sp.
int record_plan(const int *bins, int nchan, GroupDev *sp, int max_sp, int16_t *rec_w, int *nplanes, int *words)
{
    int n = 0;
    GroupDev *cur = nullptr;
    for (int c = 0; c < nchan; ++c) {
        int b = 0;
        while (b < bins[c]) {
            const int used = cur ? cur->nb + cur->nb1 : kGroupBins;
            const bool two = cur && cur->nb1 > 0;
            if (!cur || used == kGroupBins || two) {
                if (n >= max_sp) return -1;
                cur = &sp[n++];
                *cur = GroupDev{};
                cur->chan = (int16_t)c;
                cur->b_lo = (int16_t)b;
            } else if (cur->chan != c) {
                cur->chan1 = (int16_t)c;  // the group continues with channel c
                cur->b_lo1 = (int16_t)b;
            }
            const int take = std::min(kGroupBins - (cur->nb + cur->nb1), bins[c] - b);
            if (cur->chan == c)
                cur->nb = (int16_t)(cur->nb + take);
            else
                cur->nb1 = (int16_t)(cur->nb1 + take);
            b += take;
        }
    }
    int p = 0, w = 0, total = 0;
    for (int k = 0; k < n; ++k) {
        const int wk = kGroupBins;
        if (w + wk > 2 * kGroupBins) {
            rec_w[p++] = (int16_t)w;
            total += w;
            w = 0;
        }
        sp[k].plane = (int16_t)p;
        sp[k].off = (int16_t)w;
        w += wk;
    }
    rec_w[p] = (int16_t)w;
    *nplanes = n ? p + 1 : 0;
    *words = total + w;
    return n;
}

// Count groups ordered by size (one tiles launch per size), except in
// LAYOUT_RECORD (record_plan's order); tile-sums windows with the weighted
// channel's windows last.
bool plan_groups(PlaneSet &ps)
{
    int bins[kMaxChannels];
    for (int c = 0; c < ps.nchan; ++c) bins[c] = ps.chan[c].bins;
    GroupDev tmp[kMaxGroups];
    int n = 0;
    if (ps.layout == LAYOUT_RECORD) {
        int words = 0;
        n = record_plan(bins, ps.nchan, ps.grp, kMaxGroups, ps.rec_w, &ps.nplanes, &words);
        if (n < 0) return false;
        ps.seg2 = 0;
        for (int k = 0; k < n; ++k) ps.seg2 |= ps.grp[k].nb1 > 0;
    } else {
        const int ng = make_groups(bins, ps.nchan, kGroupBins, tmp, kMaxGroups);
        if (ng < 0) return false;
        for (int size = kGroupBins; size >= 1; --size)
            for (int k = 0; k < ng; ++k)
                if (tmp[k].nb == size) {
                    ps.grp[n] = tmp[k];
                    ps.grp[n].plane = (int16_t)n;
                    ps.rec_w[n] = tmp[k].nb;
                    ++n;
                }
        ps.nplanes = n;
    }
    ps.ngroups = n;
    const int nw = make_groups(bins, ps.nchan, kWindowBins, tmp, kMaxGroups);
    if (nw < 0) return false;
    n = 0;
    for (int k = 0; k < nw; ++k)
        if (tmp[k].chan != ps.wch) ps.win[n++] = tmp[k];
    ps.nwin_count = n;
    for (int k = 0; k < nw; ++k)
        if (tmp[k].chan == ps.wch) ps.win[n++] = tmp[k];
    ps.nwin = n;
    return true;
}

// Slab offsets of the groups (LAYOUT_SLAB) and the read view of the tensor.
void make_view(const PlaneSet &ps, const int32_t *d, CountView &v)
{
    memset(&v, 0, sizeof v);
    v.d = d;
    v.B = ps.B;
    v.H = ps.g.H;
    v.W = ps.g.W;
    v.P = ps.g.P;
    v.layout = ps.layout;
    v.ngroups = ps.nplanes;
    for (int p = 0; p < ps.nplanes; ++p) {
        v.group_nb[p] = ps.rec_w[p];
        v.slab_off[p] = ps.slab_off[p];
        v.plane_w0[p] = (int16_t)(p ? v.plane_w0[p - 1] + ps.rec_w[p - 1] : 0);
    }
    int words = 0;
    for (int p = 0; p < ps.nplanes; ++p) words += ps.rec_w[p];
    for (int w = 0; w < words && w < kMaxBins; ++w) v.word_bin[w] = -1;
    v.nquarters = words / 4;
    for (int k = 0; k < v.nquarters && k < kMaxBins / 4; ++k) {
        int p = 0;
        while (p + 1 < ps.nplanes && v.plane_w0[p + 1] <= 4 * k) ++p;
        v.quarter_plane[k] = (int16_t)p;
    }
    for (int k = 0; k < ps.ngroups; ++k) {
        const GroupDev &gr = ps.grp[k];
        const int gb0 = ps.chan[gr.chan].bin_off + gr.b_lo;
        if (ps.layout != LAYOUT_RECORD) v.group_bin0[gr.plane] = (int16_t)gb0;
        for (int b = 0; b < gr.nb + gr.nb1; ++b) {
            v.bin_group[gb0 + b] = gr.plane;
            v.bin_local[gb0 + b] = (int16_t)(gr.off + b);
            v.word_bin[v.plane_w0[gr.plane] + gr.off + b] = (int16_t)(gb0 + b);
        }
    }
}

void frame_record(const ih_frame &f, FrameRec &fr)
{
    fr.H = f.height;
    fr.W = f.width;
    fr.nchan = f.channels;
    fr.P = (f.width + 3) & ~3;
    int off = 0;
    for (int c = 0; c < f.channels; ++c) {
        fr.bins[c] = f.chan[c].bins;
        fr.bin_off[c] = off;
        off += f.chan[c].bins;
    }
    fr.B = off;
    fr.wch = f.weighted_channel;
    fr.Bw = fr.wch >= 0 ? fr.bins[fr.wch] : 0;
    fr.mbits = f.moment_bits == 32 ? 32 : 64;
    int words = fr.B;
    if (f.layout == IH_LAYOUT_RECORD) {
        GroupDev sp[kMaxGroups];
        int16_t rw[kMaxGroups];
        int np = 0;
        if (record_plan(fr.bins, fr.nchan, sp, kMaxGroups, rw, &np, &words) < 0) words = fr.B;
    }
    fr.count_bytes = (int64_t)words * fr.H * fr.P * 4;
    fr.moment_bytes = (int64_t)4 * fr.Bw * fr.H * fr.P * (fr.mbits / 8);
}

std::string shape_key(const ih_frame &f)
{
    std::string k = std::to_string(f.height) + "x" + std::to_string(f.width) + ":" + std::to_string(f.input) + ":" +
                    std::to_string(f.weighted_channel) + ":" + std::to_string(f.layout);
    for (int c = 0; c < f.channels; ++c) k += ":" + std::to_string(f.chan[c].bins) + "/" + std::to_string(f.chan[c].mode);
    return k;
}

bool make_planeset(ih_ctx *ctx, const ih_frame &f, const FrameRec &fr, const uint8_t *const *planes,
                   const int64_t *cpitch, PlaneSet &ps, bool small)
{
    memset(&ps, 0, sizeof ps);
    ps.B = fr.B;
    ps.nchan = fr.nchan;
    ps.layout = f.layout;
    ps.wch = fr.wch;
    for (int c = 0; c < fr.nchan; ++c) {
        ps.chan[c].plane = planes[c];
        ps.chan[c].pitch = cpitch[c];
        ps.chan[c].bins = f.chan[c].bins;
        ps.chan[c].mode = f.chan[c].mode;
        ps.chan[c].bin_off = fr.bin_off[c];
    }
    if (!plan_groups(ps)) return false;
    auto it = ctx->tuned.find(shape_key(f));
    ps.g = it != ctx->tuned.end() ? make_grid(fr.H, fr.W, it->second.first, it->second.second)
                                  : choose_grid(fr.H, fr.W, ps.ngroups, ctx->nsm);
    ps.g.P = fr.P;
    int64_t off = 0;
    for (int p = 0; p < ps.nplanes; ++p) {
        ps.slab_off[p] = off;
        off += (int64_t)fr.H * fr.P * ps.rec_w[p];
    }
    ps.out = fr.d_ih;
    ps.mom = fr.d_mom;
    ps.mom32 = fr.mbits == 32;
    ps.err = ctx->d_err;
    if (it == ctx->tuned.end()) {
        // a small frame built in one pass takes 16-row bands: fewer bands to
        // look back over (the tiles of 128 columns stay)
        PlaneSet t = ps;
        t.g = make_grid(fr.H, fr.W, 16, kChunk);
        t.g.P = fr.P;
        if (onepass_ok(t)) ps.g = t.g;
    }
    ps.uni = 1;
    for (int c = 0; c < fr.nchan; ++c)
        if (f.chan[c].mode != 0) ps.uni = 0;
    // a single frame too small to fill the GPU with the three-kernel build
    // is built by one cooperative launch (its own tile grid)
    if (small && it == ctx->tuned.end() && !onepass_ok(ps)) small_plan(ps);
    return true;
}

FrameRec *get_frame(ih_ctx *ctx, int32_t handle)
{
    if (handle < 0 || handle >= (int32_t)ctx->frames.size() || !ctx->frames[handle].live) return nullptr;
    return &ctx->frames[handle];
}

FrameRec *count_frame(ih_ctx *ctx, int32_t handle)
{
    FrameRec *fr = get_frame(ctx, handle);
    return (fr && !fr->phog) ? fr : nullptr;
}

int publish_frame(ih_ctx *ctx, FrameRec &fr)
{
    int h = -1;
    for (size_t i = 0; i < ctx->frames.size(); ++i)
        if (!ctx->frames[i].live) {
            h = (int)i;
            break;
        }
    if (h < 0) {
        h = (int)ctx->frames.size();
        ctx->frames.emplace_back();
    }
    fr.live = true;
    ctx->frames[h] = fr;
    ctx->used += fr.count_bytes + fr.moment_bytes;
    return h;
}

}  // namespace ih

extern "C" {

ih_status ih_create(const ih_config *cfg, ih_ctx **out)
{
    if (!cfg || !out) return IH_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) return IH_EINVAL;
    ih_ctx *ctx = new ih_ctx();
    ctx->device = cfg->device;
    ctx->budget = cfg->hbm_budget_bytes;
    ctx->profiling = (cfg->flags & IH_CFG_PROFILE) != 0;
    ctx->prof.ctx = ctx;
    ctx->prof.mark = prof_mark_cb;
    DevGuard dg(ctx->device);
    cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->device);
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = ctx->device;
    cudaError_t e = cudaMemPoolCreate(&ctx->pool, &props);
    if (e == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &thr);
        e = cudaMalloc(&ctx->d_err, sizeof(int));
    }
    if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(int));
    if (e == cudaSuccess) {
        prepare_kernels();  // one-time tables and kernel attributes, before any launch or capture
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
        delete ctx;
        return IH_ECUDA;
    }
    *out = ctx;
    return IH_OK;
}

ih_status ih_build(ih_ctx *ctx, const ih_frame *frames, int32_t n, int32_t *out_handles, void *stream)
{
    if (!ctx) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (!frames || !out_handles || n < 1) return fail(ctx, IH_EINVAL, "ih_build: bad arguments");
    DevGuard dg(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // host validation and budget of all frames first: all or nothing
    uint64_t need = 0;
    std::vector<FrameRec> recs(n);
    for (int k = 0; k < n; ++k) {
        const ih_frame &f = frames[k];
        ih_status s = validate(ctx, f);
        if (s != IH_OK) return s;
        FrameRec &fr = recs[k];
        frame_record(f, fr);
        need += fr.count_bytes + fr.moment_bytes;
    }
    if (ctx->budget && ctx->used + need > ctx->budget)
        return fail(ctx, IH_EBUDGET, "ih_build: %llu bytes live + %llu needed > budget %llu",
                    (unsigned long long)ctx->used, (unsigned long long)need,
                    (unsigned long long)ctx->budget);
    for (int k = 0; k < n; ++k) {
        const ih_frame &f = frames[k];
        FrameRec &fr = recs[k];
        cudaError_t e = pool_alloc(ctx, &fr.d_ih, fr.count_bytes, st);
        if (e == cudaSuccess && fr.Bw) e = pool_alloc(ctx, &fr.d_mom, fr.moment_bytes, st);
        if (e != cudaSuccess) {
            if (fr.d_ih) cudaFreeAsync(fr.d_ih, st);
            for (int kk = 0; kk < k; ++kk) {
                cudaFreeAsync(recs[kk].d_ih, st);
                if (recs[kk].d_mom) cudaFreeAsync(recs[kk].d_mom, st);
            }
            return cuda_fail(ctx, e, "tensor allocation");
        }
        // channel planes
        const uint8_t *planes[kMaxChannels];
        uint8_t *feat = nullptr;
        int64_t cpitch[kMaxChannels];
        const int64_t plane_stride = (int64_t)f.height * f.pitch_bytes;
        if (f.input == IH_INPUT_RGB_FEATURES) {
            const int64_t fp = (f.width + 15) & ~15;
            e = pool_alloc(ctx, &feat, (size_t)4 * fp * f.height, st);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "feature scratch allocation");
            const uint8_t *R = f.d_pixels, *G = R + plane_stride, *Bp = G + plane_stride;
            if (launch_features(R, G, Bp, f.pitch_bytes, f.height, f.width, nullptr, feat,
                                feat + fp * f.height, fp, st, prof_of(ctx)) < 0)
                return cuda_fail(ctx, cudaGetLastError(), "feature launch");
            ctx->launches += 1;
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
        PlaneSet ps;
        if (!make_planeset(ctx, f, fr, planes, cpitch, ps, true))
            return fail(ctx, IH_EINVAL, "too many bins for one build");
        void *scratch = nullptr;
        const size_t cb = carry_bytes(ps);
        if (cb) {
            e = pool_alloc(ctx, &scratch, cb, st);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "scratch allocation");
        }
        carve_carries(ps, scratch);
        const int nl = launch_build(ps, st, prof_of(ctx));
        if (scratch) cudaFreeAsync(scratch, st);
        ih_status s = IH_OK;
        if (nl < 0)
            s = cuda_fail(ctx, cudaGetLastError(), "build launch");
        else
            ctx->launches += nl;
        make_view(ps, fr.d_ih, fr.view);
        fr.R = ps.g.R;
        fr.Wc = ps.g.Wc;
        if (feat) cudaFreeAsync(feat, st);
        if (s != IH_OK) return s;
    }
    for (int k = 0; k < n; ++k) out_handles[k] = publish_frame(ctx, recs[k]);
    return IH_OK;
}

ih_status ih_build_mma(ih_ctx *ctx, const ih_frame *f, int32_t *out_handle, void *stream)
{
    if (!ctx) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (!f || !out_handle) return fail(ctx, IH_EINVAL, "ih_build_mma: bad arguments");
    ih_status s = validate(ctx, *f);
    if (s != IH_OK) return s;
    if (f->layout != IH_LAYOUT_BIN_MAJOR || f->input != IH_INPUT_PLANES || f->weighted_channel != -1)
        return fail(ctx, IH_EINVAL, "ih_build_mma: bin-major planes without moment planes only");
    DevGuard dg(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    FrameRec fr;
    frame_record(*f, fr);
    if (ctx->budget && ctx->used + fr.count_bytes > ctx->budget)
        return fail(ctx, IH_EBUDGET, "ih_build_mma: %llu bytes over the budget", (unsigned long long)fr.count_bytes);
    cudaError_t e = pool_alloc(ctx, &fr.d_ih, fr.count_bytes, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tensor allocation");
    const uint8_t *planes[kMaxChannels];
    int64_t cpitch[kMaxChannels];
    for (int c = 0; c < f->channels; ++c) {
        planes[c] = f->d_pixels + c * (int64_t)f->height * f->pitch_bytes;
        cpitch[c] = f->pitch_bytes;
    }
    PlaneSet ps;
    if (!make_planeset(ctx, *f, fr, planes, cpitch, ps)) {
        cudaFreeAsync(fr.d_ih, st);
        return fail(ctx, IH_EINVAL, "too many bins for one build");
    }
    ps.g = make_grid(fr.H, fr.W, 128, 128);  // the tensor-core tile
    ps.g.P = fr.P;
    void *scratch = nullptr;
    const size_t cb = carry_bytes(ps);
    if (cb && (e = pool_alloc(ctx, &scratch, cb, st)) != cudaSuccess) {
        cudaFreeAsync(fr.d_ih, st);
        return cuda_fail(ctx, e, "scratch allocation");
    }
    carve_carries(ps, scratch);
    int nl = launch_carries(ps, st, prof_of(ctx));
    const int nm = nl < 0 ? -1 : launch_tiles_mma(ps, ctx->d_err, st, prof_of(ctx));
    if (scratch) cudaFreeAsync(scratch, st);
    if (nm < 0) {
        cudaFreeAsync(fr.d_ih, st);
        return cuda_fail(ctx, cudaGetLastError(), "build launch");
    }
    ctx->launches += nl + nm;
    make_view(ps, fr.d_ih, fr.view);
    fr.R = ps.g.R;
    fr.Wc = ps.g.Wc;
    *out_handle = publish_frame(ctx, fr);
    return IH_OK;
}

ih_status ih_query_rects(ih_ctx *ctx, int32_t handle, const int32_t *d_rects, int64_t n, int32_t *d_out,
                         void *stream)
{
    if (!ctx) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    FrameRec *fr = count_frame(ctx, handle);
    if (!fr) return fail(ctx, IH_ENOTBUILT, "no live frame %d", handle);
    if (n < 0 || (n > 0 && (!d_rects || !d_out))) return fail(ctx, IH_EINVAL, "ih_query_rects: bad arguments");
    DevGuard dg(ctx->device);
    const int k = launch_query_rects(fr->view, d_rects, n, d_out, ctx->d_err, static_cast<cudaStream_t>(stream),
                                     prof_of(ctx));
    if (k < 0) return cuda_fail(ctx, cudaGetLastError(), "query launch");
    ctx->launches += k;
    return IH_OK;
}

ih_status ih_query_weighted(ih_ctx *ctx, int32_t handle, const int32_t *d_windows, int64_t n, uint32_t kernel,
                            uint32_t flags, float *d_out, void *stream)
{
    if (!ctx) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    FrameRec *fr = count_frame(ctx, handle);
    if (!fr) return fail(ctx, IH_ENOTBUILT, "no live frame %d", handle);
    if (!fr->Bw) return fail(ctx, IH_EINVAL, "frame %d has no moment planes", handle);
    const int layers = weighted_layers(flags);
    if (kernel > IH_K_WEDDING_CAKE || (flags & ~((uint32_t)IH_NORMALIZE | IH_LAYERS(0xff))) || layers > 64)
        return fail(ctx, IH_EINVAL, "kernel %u / flags %u", kernel, flags);
    if (n < 0 || (n > 0 && (!d_windows || !d_out))) return fail(ctx, IH_EINVAL, "ih_query_weighted: bad arguments");
    DevGuard dg(ctx->device);
    const MomentView m{fr->bin_off[fr->wch], fr->d_mom, fr->Bw, fr->mbits == 32};
    const int k = launch_query_weighted(fr->view, m, d_windows, n, (int)kernel, layers,
                                        (flags & IH_NORMALIZE) ? 1 : 0, d_out, ctx->d_err,
                                        static_cast<cudaStream_t>(stream), prof_of(ctx));
    if (k < 0) return cuda_fail(ctx, cudaGetLastError(), "query launch");
    ctx->launches += k;
    return IH_OK;
}

ih_status ih_query(ih_ctx *ctx, int32_t handle, const int32_t *d_rects, int64_t n_rects, int32_t *d_rect_out,
                   const int32_t *d_windows, int64_t n_windows, uint32_t kernel, uint32_t flags,
                   float *d_weighted_out, void *stream)
{
    if (!ctx) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    FrameRec *fr = count_frame(ctx, handle);
    if (!fr) return fail(ctx, IH_ENOTBUILT, "no live frame %d", handle);
    if (n_rects < 0 || (n_rects > 0 && (!d_rects || !d_rect_out)) || n_windows < 0 ||
        (n_windows > 0 && (!d_windows || !d_weighted_out)))
        return fail(ctx, IH_EINVAL, "ih_query: bad arguments");
    const int layers = weighted_layers(flags);
    if (n_windows > 0) {
        if (!fr->Bw) return fail(ctx, IH_EINVAL, "frame %d has no moment planes", handle);
        if (kernel > IH_K_WEDDING_CAKE || (flags & ~((uint32_t)IH_NORMALIZE | IH_LAYERS(0xff))) || layers > 64)
            return fail(ctx, IH_EINVAL, "kernel %u / flags %u", kernel, flags);
    }
    DevGuard dg(ctx->device);
    const MomentView m{fr->Bw ? fr->bin_off[fr->wch] : 0, fr->d_mom, fr->Bw, fr->mbits == 32};
    const int k = launch_query_both(fr->view, m, d_rects, n_rects, d_rect_out, d_windows, n_windows, (int)kernel,
                                    layers, (flags & IH_NORMALIZE) ? 1 : 0, d_weighted_out, ctx->d_err,
                                    static_cast<cudaStream_t>(stream), prof_of(ctx));
    if (k < 0) return cuda_fail(ctx, cudaGetLastError(), "query launch");
    ctx->launches += k;
    return IH_OK;
}

ih_status ih_match_window(ih_ctx *ctx, int32_t handle, int32_t bin0, int32_t nbins, const int32_t *d_target,
                          int32_t win_h, int32_t win_w, const int32_t *search, int32_t *d_out, void *stream)
{
    if (!ctx) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    FrameRec *fr = count_frame(ctx, handle);
    if (!fr) return fail(ctx, IH_ENOTBUILT, "no live frame %d", handle);
    if (!search || !d_target || !d_out) return fail(ctx, IH_EINVAL, "ih_match_window: NULL argument");
    const int sr0 = search[0], sc0 = search[1], sr1 = search[2], sc1 = search[3];
    if (nbins < 1 || bin0 < 0 || bin0 + nbins > fr->B || win_h < 1 || win_w < 1 || sr0 < 0 || sc0 < 0 ||
        sr1 < sr0 || sc1 < sc0 || (int64_t)sr1 + win_h > fr->H || (int64_t)sc1 + win_w > fr->W)
        return fail(ctx, IH_EINVAL, "ih_match_window: bins [%d, %d) / window %dx%d / search (%d,%d)-(%d,%d)",
                    bin0, bin0 + nbins, win_h, win_w, sr0, sc0, sr1, sc1);
    DevGuard dg(ctx->device);
    const int k = launch_match_window(fr->view, bin0, nbins, d_target, win_h, win_w, sr0, sc0, sr1, sc1, d_out,
                                      static_cast<cudaStream_t>(stream), prof_of(ctx));
    if (k < 0) return cuda_fail(ctx, cudaGetLastError(), "match launch");
    ctx->launches += k;
    return IH_OK;
}

ih_status ih_accumulate(ih_ctx *ctx, int32_t dst, int32_t add, int32_t sub, void *stream)
{
    if (!ctx) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    FrameRec *d = count_frame(ctx, dst);
    FrameRec *a = add >= 0 ? count_frame(ctx, add) : nullptr;
    FrameRec *b = sub >= 0 ? count_frame(ctx, sub) : nullptr;
    if (!d || (add >= 0 && !a) || (sub >= 0 && !b)) return fail(ctx, IH_ENOTBUILT, "ih_accumulate: no such frame");
    for (const FrameRec *o : {a, b}) {
        if (!o) continue;
        bool same = o->H == d->H && o->W == d->W && o->nchan == d->nchan && o->P == d->P &&
                    o->count_bytes == d->count_bytes && o->view.layout == d->view.layout;
        for (int c = 0; same && c < d->nchan; ++c) same = o->bins[c] == d->bins[c];
        if (!same) return fail(ctx, IH_EINVAL, "ih_accumulate: frames of different shape, bins or layout");
    }
    if (d->d_mom || (a && a->d_mom) || (b && b->d_mom))
        return fail(ctx, IH_EINVAL, "ih_accumulate: frames with moment planes");
    DevGuard dg(ctx->device);
    const int k = launch_accumulate(d->d_ih, a ? a->d_ih : nullptr, b ? b->d_ih : nullptr, d->count_bytes / 4,
                                    static_cast<cudaStream_t>(stream), prof_of(ctx));
    if (k < 0) return cuda_fail(ctx, cudaGetLastError(), "accumulate launch");
    ctx->launches += k;
    return IH_OK;
}

ih_status ih_local_median(ih_ctx *ctx, int32_t handle, int32_t bin0, int32_t nbins, int32_t m, int32_t n,
                          int32_t *d_out, void *stream)
{
    if (!ctx) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    FrameRec *fr = count_frame(ctx, handle);
    if (!fr) return fail(ctx, IH_ENOTBUILT, "no live frame %d", handle);
    if (!d_out || nbins < 1 || bin0 < 0 || bin0 + nbins > fr->B || m < 1 || n < 1)
        return fail(ctx, IH_EINVAL, "ih_local_median: bins [%d, %d) / box %d x %d", bin0, bin0 + nbins, m, n);
    DevGuard dg(ctx->device);
    const int k = launch_local_median(fr->view, bin0, nbins, m, n, d_out, static_cast<cudaStream_t>(stream),
                                      prof_of(ctx));
    if (k < 0) return cuda_fail(ctx, cudaGetLastError(), "median launch");
    ctx->launches += k;
    return IH_OK;
}

ih_status ih_phog_build(ih_ctx *ctx, const uint8_t *d_gray, int32_t height, int32_t width, int64_t pitch_bytes,
                        int32_t tau_low, int32_t tau_high, int32_t *out_handle, void *stream)
{
    if (!ctx) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (!d_gray || !out_handle || height < 1 || width < 1 || pitch_bytes < width || tau_low < 0 ||
        tau_high < tau_low || tau_high > IH_CANNY_MAX_THRESHOLD || (int64_t)height * width > ((int64_t)1 << 30))
        return fail(ctx, IH_EINVAL, "ih_phog_build: bad arguments");
    DevGuard dg(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    FrameRec fr;
    fr.H = height;
    fr.W = width;
    fr.nchan = 1;
    fr.B = kPhogBins;
    fr.bins[0] = kPhogBins;
    fr.P = (width + 3) & ~3;
    fr.phog = true;
    fr.moment_bytes = (int64_t)kPhogBins * height * fr.P * 8;
    if (ctx->budget && ctx->used + (uint64_t)fr.moment_bytes > ctx->budget)
        return fail(ctx, IH_EBUDGET, "pyramid planes of %lld bytes exceed the HBM budget", (long long)fr.moment_bytes);
    const int64_t px = (int64_t)height * width;
    const size_t cbytes = (canny_scratch_bytes(height, width) + 255) & ~size_t(255);
    uint8_t *scratch = nullptr;
    cudaError_t e = pool_alloc(ctx, &fr.d_mom, fr.moment_bytes, st);
    if (e == cudaSuccess) e = pool_alloc(ctx, &scratch, cbytes + (size_t)px * 5 + 16, st);
    if (e != cudaSuccess) {
        if (fr.d_mom) cudaFreeAsync(fr.d_mom, st);
        return cuda_fail(ctx, e, "pyramid allocation");
    }
    const CannyScratch cs = carve_canny(scratch, height, width);
    int32_t *wt = reinterpret_cast<int32_t *>(scratch + cbytes);
    uint8_t *bins = scratch + cbytes + px * 4;
    const int k = launch_phog_build(d_gray, pitch_bytes, height, width, tau_low, tau_high, cs, bins, wt, fr.P,
                                    fr.d_mom, ctx->d_err, st, prof_of(ctx));
    cudaFreeAsync(scratch, st);
    if (k < 0) {
        cudaFreeAsync(fr.d_mom, st);
        return cuda_fail(ctx, cudaGetLastError(), "pyramid launch");
    }
    ctx->launches += k;
    *out_handle = publish_frame(ctx, fr);
    return IH_OK;
}

ih_status ih_canny_edges(ih_ctx *ctx, const uint8_t *d_gray, int32_t height, int32_t width, int64_t pitch_bytes,
                         int32_t tau_low, int32_t tau_high, uint8_t *d_edges, int64_t edges_pitch, void *stream)
{
    if (!ctx) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (!d_gray || !d_edges || height < 1 || width < 1 || pitch_bytes < width || edges_pitch < width ||
        tau_low < 0 || tau_high < tau_low || tau_high > IH_CANNY_MAX_THRESHOLD ||
        (int64_t)height * width > ((int64_t)1 << 30))
        return fail(ctx, IH_EINVAL, "ih_canny_edges: bad arguments");
    DevGuard dg(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *scratch = nullptr;
    cudaError_t e = pool_alloc(ctx, &scratch, canny_scratch_bytes(height, width), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "edge-detector scratch");
    const int k = launch_canny_edges(d_gray, pitch_bytes, height, width, tau_low, tau_high,
                                     carve_canny(scratch, height, width), d_edges, edges_pitch, ctx->d_err, st,
                                     prof_of(ctx));
    cudaFreeAsync(scratch, st);
    if (k < 0) return cuda_fail(ctx, cudaGetLastError(), "edge-detector launch");
    ctx->launches += k;
    return IH_OK;
}

ih_status ih_phog_descriptors(ih_ctx *ctx, int32_t handle, int32_t levels, const int32_t *d_windows, int64_t n,
                              int64_t *d_out, void *stream)
{
    if (!ctx) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    FrameRec *fr = get_frame(ctx, handle);
    if (!fr || !fr->phog) return fail(ctx, IH_ENOTBUILT, "no pyramid frame %d", handle);
    if (levels < 0 || levels > kPhogMaxLevels || n < 0 || (n > 0 && (!d_windows || !d_out)))
        return fail(ctx, IH_EINVAL, "ih_phog_descriptors: levels %d / n %lld", levels, (long long)n);
    if (n == 0) return IH_OK;
    DevGuard dg(ctx->device);
    const int k = launch_phog_descriptors(fr->d_mom, fr->H, fr->W, fr->P, levels, d_windows, n, d_out, ctx->d_err,
                                          static_cast<cudaStream_t>(stream), prof_of(ctx));
    if (k < 0) return cuda_fail(ctx, cudaGetLastError(), "descriptor launch");
    ctx->launches += k;
    return IH_OK;
}

ih_status ih_phog_match(ih_ctx *ctx, int32_t handle, int32_t levels, const int64_t *d_target, int32_t win_h,
                        int32_t win_w, const int32_t *search, float *d_out, void *stream)
{
    if (!ctx) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    FrameRec *fr = get_frame(ctx, handle);
    if (!fr || !fr->phog) return fail(ctx, IH_ENOTBUILT, "no pyramid frame %d", handle);
    if (!search || !d_target || !d_out || levels < 0 || levels > kPhogMaxLevels)
        return fail(ctx, IH_EINVAL, "ih_phog_match: bad arguments");
    const int sr0 = search[0], sc0 = search[1], sr1 = search[2], sc1 = search[3];
    if (win_h < 1 || win_w < 1 || sr0 < 0 || sc0 < 0 || sr1 < sr0 || sc1 < sc0 || (int64_t)sr1 + win_h > fr->H ||
        (int64_t)sc1 + win_w > fr->W)
        return fail(ctx, IH_EINVAL, "ih_phog_match: window %dx%d / search (%d,%d)-(%d,%d)", win_h, win_w, sr0, sc0,
                    sr1, sc1);
    DevGuard dg(ctx->device);
    const int k = launch_phog_match(fr->d_mom, fr->H, fr->P, levels, d_target, win_h, win_w, sr0, sc0, sr1, sc1,
                                    d_out, static_cast<cudaStream_t>(stream), prof_of(ctx));
    if (k < 0) return cuda_fail(ctx, cudaGetLastError(), "pyramid match launch");
    ctx->launches += k;
    return IH_OK;
}

ih_status ih_release(ih_ctx *ctx, int32_t handle, void *stream)
{
    if (!ctx) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    FrameRec *fr = get_frame(ctx, handle);
    if (!fr) return fail(ctx, IH_ENOTBUILT, "no live frame %d", handle);
    DevGuard dg(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaFreeAsync(fr->d_ih, st);
    if (fr->d_mom) cudaFreeAsync(fr->d_mom, st);
    ctx->used -= fr->count_bytes + fr->moment_bytes;
    *fr = FrameRec();
    return IH_OK;
}

ih_status ih_sync(ih_ctx *ctx, void *stream)
{
    if (!ctx) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    DevGuard dg(ctx->device);
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
    int h = 0;
    e = cudaMemcpy(&h, ctx->d_err, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "error word read");
    if (h) {
        cudaMemset(ctx->d_err, 0, sizeof(int));
        if (h & 1) return fail(ctx, IH_EINVAL, "a query named a rectangle outside the frame or empty");
        return fail(ctx, IH_ETIMEOUT, "a device-side wait or pointer walk gave up");
    }
    return IH_OK;
}

ih_status ih_info(ih_ctx *ctx, int32_t handle, ih_frame_info *out)
{
    if (!ctx || !out) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    FrameRec *fr = get_frame(ctx, handle);
    if (!fr) return fail(ctx, IH_ENOTBUILT, "no live frame %d", handle);
    out->height = fr->H;
    out->width = fr->W;
    out->channels = fr->nchan;
    out->total_bins = fr->B;
    out->weighted_channel = fr->wch;
    out->weighted_bins = fr->Bw;
    out->pitch_elems = fr->P;
    out->count_bytes = fr->count_bytes;
    out->moment_bytes = fr->moment_bytes;
    out->tile_rows = fr->R;
    out->tile_cols = fr->Wc;
    return IH_OK;
}

ih_status ih_export(ih_ctx *ctx, int32_t handle, int32_t *d_dst, void *stream)
{
    if (!ctx || !d_dst) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    FrameRec *fr = count_frame(ctx, handle);
    if (!fr) return fail(ctx, IH_ENOTBUILT, "no live frame %d", handle);
    DevGuard dg(ctx->device);
    if (launch_export(fr->view, d_dst, static_cast<cudaStream_t>(stream), prof_of(ctx)) < 0)
        return cuda_fail(ctx, cudaGetLastError(), "export launch");
    ctx->launches += 1;
    return IH_OK;
}

ih_status ih_export_moments(ih_ctx *ctx, int32_t handle, int32_t plane, int64_t *d_dst, void *stream)
{
    if (!ctx || !d_dst) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    FrameRec *fr = count_frame(ctx, handle);
    if (!fr) return fail(ctx, IH_ENOTBUILT, "no live frame %d", handle);
    if (!fr->Bw || plane < 0 || plane > 3) return fail(ctx, IH_EINVAL, "no moment plane %d", plane);
    DevGuard dg(ctx->device);
    if (launch_export_moments(fr->d_mom, fr->mbits == 32, fr->Bw, fr->H, fr->W, fr->P, plane, d_dst,
                              static_cast<cudaStream_t>(stream), prof_of(ctx)) < 0)
        return cuda_fail(ctx, cudaGetLastError(), "export launch");
    ctx->launches += 1;
    return IH_OK;
}

ih_status ih_features(ih_ctx *ctx, const uint8_t *d_rgb, int32_t height, int32_t width, int64_t pitch_bytes,
                      uint8_t *d_out, void *stream)
{
    if (!ctx) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (!d_rgb || !d_out || height < 1 || width < 1 || pitch_bytes < width)
        return fail(ctx, IH_EINVAL, "ih_features: bad arguments");
    DevGuard dg(ctx->device);
    const int64_t ps = (int64_t)height * pitch_bytes, po = (int64_t)height * width;
    if (launch_features(d_rgb, d_rgb + ps, d_rgb + 2 * ps, pitch_bytes, height, width, d_out, d_out + 3 * po,
                        d_out + 4 * po, width, static_cast<cudaStream_t>(stream), prof_of(ctx)) < 0)
        return cuda_fail(ctx, cudaGetLastError(), "feature launch");
    ctx->launches += 1;
    return IH_OK;
}

ih_status ih_destroy(ih_ctx *ctx)
{
    if (!ctx) return IH_OK;
    {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        DevGuard dg(ctx->device);
        cudaDeviceSynchronize();
        for (auto &f : ctx->frames)
            if (f.live) {
                cudaFreeAsync(f.d_ih, 0);
                if (f.d_mom) cudaFreeAsync(f.d_mom, 0);
            }
        cudaDeviceSynchronize();
        if (ctx->d_err) cudaFree(ctx->d_err);
        for (auto &r : ctx->prof_pending) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : ctx->ev_free) cudaEventDestroy(e);
        if (ctx->prof_open) cudaEventDestroy(ctx->prof_open);
        if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    }
    delete ctx;
    return IH_OK;
}

ih_status ih_profile_select(ih_ctx *ctx, const char *const *names, int32_t n)
{
    if (!ctx) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (!ctx->profiling) return fail(ctx, IH_EINVAL, "context was created without IH_CFG_PROFILE");
    if (n < 0 || (n > 0 && !names)) return fail(ctx, IH_EINVAL, "ih_profile_select: bad arguments");
    uint32_t mask = n ? 0u : ~0u;
    for (int32_t i = 0; i < n; ++i) {
        int kid = -1;
        for (int k = 0; k < KID_COUNT; ++k)
            if (names[i] && strcmp(names[i], kernel_name(k)) == 0) kid = k;
        if (kid < 0) return fail(ctx, IH_EINVAL, "ih_profile_select: no kernel named %s", names[i] ? names[i] : "");
        mask |= 1u << kid;
    }
    ctx->prof_mask = mask;
    return IH_OK;
}

ih_status ih_profile_read(ih_ctx *ctx, ih_kernel_stat *out, int32_t max, int32_t *count, int32_t reset)
{
    if (!ctx) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (!ctx->profiling) return fail(ctx, IH_EINVAL, "context was created without IH_CFG_PROFILE");
    if (!count || (max > 0 && !out)) return fail(ctx, IH_EINVAL, "ih_profile_read: bad arguments");
    DevGuard dg(ctx->device);
    for (const ProfRec &r : ctx->prof_pending) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "profile events");
        ctx->prof_launches[r.kid] += 1;
        ctx->prof_ms[r.kid] += ms;
        ctx->ev_free.push_back(r.a);
        ctx->ev_free.push_back(r.b);
    }
    ctx->prof_pending.clear();
    int n = 0;
    for (int k = 0; k < KID_COUNT; ++k) {
        if (!ctx->prof_launches[k]) continue;
        if (n < max) {
            memset(&out[n], 0, sizeof out[n]);
            snprintf(out[n].name, sizeof out[n].name, "%s", kernel_name(k));
            out[n].launches = ctx->prof_launches[k];
            out[n].total_ms = ctx->prof_ms[k];
        }
        ++n;
    }
    *count = n < max ? n : max;
    if (reset)
        for (int k = 0; k < KID_COUNT; ++k) {
            ctx->prof_launches[k] = 0;
            ctx->prof_ms[k] = 0;
        }
    return IH_OK;
}

int64_t ih_launch_count(ih_ctx *ctx)
{
    if (!ctx) return 0;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    return ctx->launches;
}

ih_status ih_wait_selftest(ih_ctx *ctx, int32_t polls, void *stream)
{
    if (!ctx) return IH_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (polls < 1 || polls > (1 << 24)) return fail(ctx, IH_EINVAL, "ih_wait_selftest: polls %d (1..2^24)", polls);
    DevGuard dg(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t *never = nullptr;
    cudaError_t e = pool_alloc(ctx, &never, sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(never, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "self-test counter");
    const int k = launch_wait_selftest(never, polls, ctx->d_err, st);
    cudaFreeAsync(never, st);
    if (k < 0) return cuda_fail(ctx, cudaGetLastError(), "self-test launch");
    ctx->launches += k;
    return IH_OK;
}

uint64_t ih_memory_used(ih_ctx *ctx)
{
    if (!ctx) return 0;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    return ctx->used;
}

const char *ih_last_error(ih_ctx *ctx)
{
    if (!ctx) return "NULL context";
    return ctx->last_error.c_str();
}

}  // extern "C"
